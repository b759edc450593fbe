// hg_gs_run_noalloc: Gerchberg-Saxton for one Fourier hologram without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool or arena it does not own,
// plug-ins whose host application forbids allocation after start-up, and real-time loops where an
// allocation (which may synchronise the device) would break the latency budget.  hg_plan_create
// allocates the field workspace and tables, so those callers cannot use hg_gs_run.  This file gives
// them one entry point whose scratch -- the field, the reduction partials, and the
// twiddle and level tables -- lives in a file-scope device array that the CUDA runtime reserves on
// every device that loads this library, for as long as the process lives.
//
// The kernels are the ones hg_gs_run launches (k_row_init, k_col_gs, k_row_gs); only the memory
// their scratch pointers point at differs.
#include <dlfcn.h>

#include <cstdio>
#include <mutex>

#include "hologen.h"
#include "hg_kernels.cuh"
#include "hg_launch.h"

namespace {

// Scratch capacity: a field of up to 2^20 pixels (e.g. 1024 x 1024, 2048 x 512) plus tables
// (8 MiB + 155 KiB).
constexpr size_t kMaxPixels = size_t(1) << 20;
constexpr size_t kFieldBytes = kMaxPixels * sizeof(float2);  // 8 MiB
constexpr size_t kPartialBytes = 3 * 1024 * sizeof(float2);  // <= 1024 column strips
constexpr int kTwEntries = 8192;                              // per-stage twiddle tables of one length
constexpr size_t kTwBytes = kTwEntries * sizeof(float2);
constexpr size_t kLevBytes = 256 * sizeof(float2);
constexpr size_t kLevPhaseBytes = 256 * sizeof(float);
constexpr size_t kOffPartials = kFieldBytes;
constexpr size_t kOffTwRow = kOffPartials + kPartialBytes;
constexpr size_t kOffTwCol = kOffTwRow + kTwBytes;
constexpr size_t kOffLev = kOffTwCol + kTwBytes;
constexpr size_t kOffLevPhase = kOffLev + kLevBytes;
constexpr size_t kScratchBytes = kOffLevPhase + kLevPhaseBytes;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Entry i of a per-stage twiddle blob: exp(-2 pi i r k / (ns R)) of the table holding i.
__device__ float2 blob_entry(const hg::TwiddleLayout& l, int i) {
  for (int t = 0; t < l.count; ++t) {
    const int ns = l.ns[t], n = ns * l.r[t];
    if (i >= l.off[t] && i < l.off[t] + (l.r[t] - 1) * ns) {
      const int q = (i - l.off[t]) / ns + 1, k = (i - l.off[t]) % ns;
      double s, c;
      sincospi(2.0 * (double)((q * k) % n) / (double)n, &s, &c);
      return make_float2((float)c, (float)-s);
    }
  }
  return make_float2(1.f, 0.f);
}

// Fills the twiddle tables of this call's lengths and the level tables, in float64 then rounded
// (the values hg_plan_create computes on the host).
__global__ void k_noalloc_tables(const hg::TwiddleLayout tw_w, const hg::TwiddleLayout tw_h, int n_levels) {
  float2* tw_row = reinterpret_cast<float2*>(g_scratch + kOffTwRow);
  float2* tw_col = reinterpret_cast<float2*>(g_scratch + kOffTwCol);
  float2* lev = reinterpret_cast<float2*>(g_scratch + kOffLev);
  float* lev_phase = reinterpret_cast<float*>(g_scratch + kOffLevPhase);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double s, c;
  if (i < tw_w.size) tw_row[i] = blob_entry(tw_w, i);
  if (i < tw_h.size) tw_col[i] = blob_entry(tw_h, i);
  const int nl = n_levels > 0 ? n_levels : 1;
  if (i < nl) {
    if ((4 * i) % nl == 0) {
      const int quarter = (4 * i / nl) % 4;
      lev[i] = make_float2(quarter == 0 ? 1.f : (quarter == 2 ? -1.f : 0.f),
                           quarter == 1 ? 1.f : (quarter == 3 ? -1.f : 0.f));
    } else {
      sincospi(2.0 * (double)i / (double)nl, &s, &c);
      lev[i] = make_float2((float)c, (float)s);
    }
    lev_phase[i] = (float)(6.283185307179586476925286766559 * (double)i / (double)nl);
  }
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_base[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};  // driver ID of the context g_base[dev] belongs to

hg_status err(hg_status s, const char* m) {
  hg::set_last_error(m);
  return s;
}

// cuCtxGetCurrent and cuCtxGetId from the driver, looked up at run time (the library does not link
// libcuda).  A context's ID is unique for the life of the process, unlike its handle, which a new
// context may reuse after the old one is destroyed.
typedef int (*ctx_current_fn_t)(void**);
typedef int (*ctx_id_fn_t)(void*, unsigned long long*);
struct CtxFns {
  ctx_current_fn_t current = nullptr;
  ctx_id_fn_t id = nullptr;
};
const CtxFns& ctx_fns() {
  static const CtxFns f = [] {
    CtxFns x;
    if (void* h = dlopen("libcuda.so.1", RTLD_NOW | RTLD_LOCAL)) {
      x.current = (ctx_current_fn_t)dlsym(h, "cuCtxGetCurrent");
      x.id = (ctx_id_fn_t)dlsym(h, "cuCtxGetId");
    }
    return x;
  }();
  return f;
}

// ID of the calling thread's current context, or 0 when it cannot be told.
unsigned long long current_ctx_id() {
  const CtxFns& f = ctx_fns();
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (!f.current || !f.id || f.current(&ctx) != 0 || !ctx || f.id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of g_scratch in the current device's context.  It is looked up with
// cudaGetSymbolAddress the first time and again whenever the current context is not the one the
// cached address belongs to (the module holding g_scratch is loaded anew in a new context, e.g.
// after cudaDeviceReset, and the array may then sit elsewhere); where the driver cannot name the
// context the lookup is made on every call.
hg_status scratch_base(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return err(HG_ERR_CUDA, "no usable current CUDA device");
  }
  std::lock_guard<std::mutex> lock(g_mu);
  const unsigned long long id = current_ctx_id();
  if (!g_base[dev] || id == 0 || id != g_ctx_id[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return err(HG_ERR_CUDA, "cudaGetSymbolAddress(g_scratch) failed");
    }
    g_base[dev] = static_cast<unsigned char*>(ptr);
    // the lookup makes the device's primary context current if nothing was: take its ID now
    g_ctx_id[dev] = current_ctx_id();
  }
  *out = g_base[dev];
  return HG_OK;
}

// cuMemGetAddressRange_v2 from the driver (looked up at run time; the library does not link libcuda)
typedef int (*range_fn_t)(unsigned long long*, size_t*, unsigned long long);
range_fn_t range_fn() {
  static range_fn_t fn = [] {
    void* h = dlopen("libcuda.so.1", RTLD_NOW | RTLD_LOCAL);
    return h ? (range_fn_t)dlsym(h, "cuMemGetAddressRange_v2") : (range_fn_t) nullptr;
  }();
  return fn;
}

// device (or managed) memory of the current device, aligned, and -- where the driver can tell --
// [p, p + bytes) inside one allocation
bool is_device_buffer(const void* p, size_t bytes, size_t align) {
  if ((uintptr_t)p % align) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return false;
  int dev = -1;
  if (at.type == cudaMemoryTypeDevice && (cudaGetDevice(&dev) != cudaSuccess || at.device != dev)) return false;
  if (range_fn_t fn = range_fn()) {
    unsigned long long base = 0;
    size_t size = 0;
    if (fn(&base, &size, (unsigned long long)(uintptr_t)p) == 0 && (unsigned long long)(uintptr_t)p + bytes > base + size)
      return false;
  }
  return true;
}

hg_status run_kernel(const void* fn, dim3 grid, int nt, int smem, const hg::PassArgs& a, cudaStream_t st) {
  void* args[] = {(void*)&a};
  if (cudaLaunchKernel(fn, grid, dim3(nt), args, (size_t)smem, st) != cudaSuccess) {
    cudaGetLastError();
    return err(HG_ERR_CUDA, "kernel launch failed");
  }
  return HG_OK;
}

}  // namespace

extern "C" hg_status hg_gs_run_noalloc(int32_t height, int32_t width, int32_t quant_levels, const float* target_amp,
                                       const float* init_phase, uint64_t seed, int32_t n_iter, float* phase_out,
                                       uint8_t* level_out, float* nmse_out, void* stream) {
  if (height < 1 || width < 1) return err(HG_ERR_INVALID_ARG, "height and width must be >= 1");
  if ((size_t)height * (size_t)width > kMaxPixels)
    return err(HG_ERR_UNSUPPORTED_SIZE, "height * width exceeds the 1048576-pixel static scratch");
  const hg::RowKernels* rk = hg::row_kernels(width);
  const hg::ColKernels* ck = hg::col_kernels(height);
  if (!rk || !ck) return err(HG_ERR_UNSUPPORTED_SIZE, "height / width is not a supported FFT length");
  if (quant_levels < 0 || quant_levels == 1 || quant_levels > 256)
    return err(HG_ERR_INVALID_ARG, "quant_levels must be 0 or 2..256");
  if (n_iter < 0 || n_iter > 1000000) return err(HG_ERR_INVALID_ARG, "n_iter must be 0..1000000");
  const size_t px = (size_t)height * (size_t)width;
  if (!target_amp || !is_device_buffer(target_amp, px * 4, 4))
    return err(HG_ERR_INVALID_ARG, "target_amp is not a device buffer of height * width floats");
  if (init_phase && !is_device_buffer(init_phase, px * 4, 4))
    return err(HG_ERR_INVALID_ARG, "init_phase is not a device buffer of height * width floats");
  if (phase_out && !is_device_buffer(phase_out, px * 4, 4))
    return err(HG_ERR_INVALID_ARG, "phase_out is not a device buffer of height * width floats");
  if (level_out && !is_device_buffer(level_out, px, 1))
    return err(HG_ERR_INVALID_ARG, "level_out is not a device buffer of height * width bytes");
  if (level_out && quant_levels == 0) return err(HG_ERR_INVALID_ARG, "level_out needs quant_levels >= 2");
  if (nmse_out && !is_device_buffer(nmse_out, (size_t)(n_iter + 1) * 4, 4))
    return err(HG_ERR_INVALID_ARG, "nmse_out is not a device buffer of n_iter + 1 floats");
  if (rk->tw.size > kTwEntries || ck->tw.size > kTwEntries) return err(HG_ERR_INTERNAL, "twiddle tables overflow");
  const int col_blocks = (width + ck->cols - 1) / ck->cols;
  if (col_blocks * 3 * (int)sizeof(double) > (int)kPartialBytes) return err(HG_ERR_INTERNAL, "partials overflow");

  unsigned char* base = nullptr;
  hg_status s = scratch_base(&base);
  if (s != HG_OK) return s;
  rk->set_attrs();
  ck->set_attrs();
  cudaStream_t st = (cudaStream_t)stream;

  // one thread per table entry (twiddle blobs <= kTwEntries, levels <= 256)
  k_noalloc_tables<<<kTwEntries / 256, 256, 0, st>>>(rk->tw, ck->tw, quant_levels);
  if (cudaGetLastError() != cudaSuccess) return err(HG_ERR_CUDA, "table kernel launch failed");

  hg::PassArgs a{};
  a.n_items = 1;
  a.H = height;
  a.W = width;
  a.n_levels = quant_levels;
  a.nmse_stride = n_iter + 1;
  a.tw_row = reinterpret_cast<const float2*>(base + kOffTwRow);
  a.tw_col = reinterpret_cast<const float2*>(base + kOffTwCol);
  a.lev = reinterpret_cast<const float2*>(base + kOffLev);
  a.lev_phase = reinterpret_cast<const float*>(base + kOffLevPhase);
  a.field = reinterpret_cast<float2*>(base);
  a.partials = reinterpret_cast<float2*>(base + kOffPartials);
  a.col_blocks = col_blocks;
  if (rk->gen) a.gen_row = *rk->gen;
  if (ck->gen) a.gen_col = *ck->gen;
  a.nmse = nmse_out;
  a.seed = seed;
  a.target[0] = target_amp;
  a.phase_in[0] = init_phase;
  const dim3 grow((height + rk->rows - 1) / rk->rows, 1), gcol(col_blocks, 1);

  hg::PassArgs a0 = a;
  if (n_iter == 0) {
    a0.phase_out[0] = phase_out;
    a0.level_out[0] = level_out;
  }
  if ((s = run_kernel(rk->init[0], grow, rk->nt, rk->smem, a0, st)) != HG_OK) return s;
  hg::PassArgs ao = a;
  ao.phase_out[0] = phase_out;
  ao.level_out[0] = level_out;
  for (int it = 0; it < n_iter; ++it) {
    a.iter = it;
    if ((s = run_kernel(ck->gs[1][0], gcol, ck->nt, ck->smem_gs, a, st)) != HG_OK) return s;
    const bool last = it == n_iter - 1;
    hg::PassArgs ar = last ? ao : a;
    ar.finalize = nmse_out != nullptr;  // the row pass first adds up this column pass's NMSE
    ar.fin_iter = it;
    if ((s = run_kernel(rk->gs[last][0], grow, rk->nt, rk->smem, ar, st)) != HG_OK) return s;
  }
  a.iter = n_iter;
  a.fin_iter = n_iter;
  if ((s = run_kernel(ck->gs[0][0], gcol, ck->nt, ck->smem_gs, a, st)) != HG_OK) return s;
  return nmse_out ? run_kernel((const void*)&hg::k_finalize<0>, dim3(1, 1), 32, 0, a, st) : HG_OK;
}
