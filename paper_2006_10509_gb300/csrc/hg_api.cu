// C ABI of libhologen: plan objects, argument validation and the launch sequences of each call.
//
// Role of the paper's AlgorithmCuda base class (section "Algorithm Libraries": it keeps the target,
// illumination and starting images and common parameters, and handles device transfer): here the
// caller owns the images in device memory and the plan owns everything derived from the parameters
// (twiddle, chirp and level tables; the field workspace; reduction scratch).
#include <dlfcn.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#ifndef HG_PDL
#define HG_PDL 1
#endif

#include "hologen.h"
#include "hg_dbs.h"
#include "hg_kernels.cuh"
#include "hg_launch.h"

namespace hg {

// The compiled instance of a length, else the generic kernels (any n = 2^a 3^b 5^c up to
// kGenMaxLength), else nullptr.
const RowKernels* row_kernels(int n) {
  switch (n) {
#define HG_CASE(N) \
  case N:          \
    return &row_kernels_##N();
    HG_FOR_EACH_LENGTH(HG_CASE)
#undef HG_CASE
    default:
      return gen_row_kernels(n);
  }
}

const ColKernels* col_kernels(int n) {
  switch (n) {
#define HG_CASE(N) \
  case N:          \
    return &col_kernels_##N();
    HG_FOR_EACH_LENGTH(HG_CASE)
#undef HG_CASE
    default:
      return gen_col_kernels(n);
  }
}

}  // namespace hg

namespace {
thread_local std::string g_err;
}  // namespace

void hg::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

namespace {

hg_status fail(hg_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

hg_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return fail(HG_ERR_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
  return fail(HG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define HG_CUDA(call, what)                         \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// cuMemGetAddressRange_v2 from the driver, found at run time (the library does not link libcuda).
typedef int (*range_fn_t)(unsigned long long*, size_t*, unsigned long long);
range_fn_t range_fn() {
  static range_fn_t fn = [] {
    void* h = dlopen("libcuda.so.1", RTLD_NOW | RTLD_LOCAL);
    return h ? (range_fn_t)dlsym(h, "cuMemGetAddressRange_v2") : (range_fn_t) nullptr;
  }();
  return fn;
}

constexpr int kMaxItems = 256;

// Kernel kinds for the timing facility.
enum Kind {
  K_ROW_INIT = 0, K_ROW_GS, K_COL_GS, K_COL_NMSE, K_ROW_FFT, K_COL_FFT, K_ROW_OSPR, K_COL_OSPR,
  K_ROW_MP_INIT, K_ROW_MP, K_ROW_GD_FWD, K_COL_GD_FWD, K_COL_GD_BWD, K_ROW_GD_BWD, K_AMP_ENERGY, K_FINALIZE,
  K_TILE_TARGET, K_GS_CLUSTER, K_DBS, K_NUM_KINDS
};
const char* const kKindNames[K_NUM_KINDS] = {"row_init",   "row_gs",     "col_gs",     "col_nmse",  "row_fft",
                                             "col_fft",    "row_ospr",   "col_ospr",   "row_mp_init", "row_mp",
                                             "row_gd_fwd", "col_gd_fwd", "col_gd_bwd", "row_gd_bwd",
                                             "amp_energy", "finalize", "tile_target", "gs_cluster", "dbs"};
constexpr int kMaxLevels = 256;

struct SizeClass {
  int H = 0, W = 0;
  std::vector<int> items;  // plan item indices, in order; slot = position
  const hg::RowKernels* rk = nullptr;
  const hg::ColKernels* ck = nullptr;
  float2* field = nullptr;       // [slot][plane][H][W]
  float2* partials = nullptr;    // [slot][plane][3 * col_blocks] (hi, lo) pairs
  float* acc = nullptr;          // [slot][H][W] OSPR accumulated intensity (allocated on first use)
  float* ttile = nullptr;        // [slot][plane][strip][H][C] targets re-laid out for the GS column passes
  float2* hio = nullptr;         // [slot][strip][H][C] HIO replay-plane input (allocated on first use)
  double* stats = nullptr;       // [slot][plane][4] gradient-descent loss statistics
  float2* gacc = nullptr;        // [slot][H][W] generic-length multi-plane accumulator (first use)
  std::vector<float2*> cx, cy;   // per plane (Fresnel)
  int row_blocks() const { return (H + rk->rows - 1) / rk->rows; }
  int col_blocks() const { return (W + ck->cols - 1) / ck->cols; }    // strips on a row-major field
  // strip width of the tiled GS field (0: single-plane GS keeps the field row-major; -1: GS runs
  // in the whole-run cluster kernel); the default rule at plan creation, or the autotuner's choice
  int tile = 0;
  // radix plan of the tiled GS passes, per pass: 0 the length's default plan, 1 its alternative
  // (PlanV); the autotuner's choice, or set by hand.  Used where the width's kernels exist with that
  // plan and the run takes the plain kernels (not MRAF / HIO / illumination / a level table).
  int pv_row = 0, pv_col = 0;
  // sizes covering any strip width (the narrowest tiled one is 2): partial sums per strip, and the
  // strips x H x width target copies
  size_t max_strips() const { return (size_t)std::max(col_blocks(), (W + 1) / 2); }
  size_t max_strip_cols() const {
    return std::max((size_t)col_blocks() * ck->cols, (size_t)(W + 15) / 16 * 16);
  }
  // GS with the whole run in one thread-block cluster per item (strip width -1): CTAs per cluster
  // (0: not available for this class), kernel, threads, shared memory
  int cl = 0;
  const void* cl_fn = nullptr;
  int cl_nt = 0, cl_smem = 0;
  // whether the GS field can be tiled in strips of width w here (kernels exist, rows tile evenly);
  // w = -1: the whole-run cluster kernel; several planes (multi-plane GS) take widths 2, 4 and 8
  bool tileable(int w, int planes) const;
};

// index of a column-strip tile width (2 / 4 / 8 / 16) in the kernels' tiled tables
int tile_index(int cols) { return cols == 2 ? 0 : (cols == 4 ? 1 : (cols == 8 ? 2 : 3)); }

bool SizeClass::tileable(int w, int planes) const {
  if (w == -1) return planes == 1 && cl > 0;
  if ((w != 2 && w != 4 && w != 8 && w != 16) || W % w != 0) return false;
  const int ti = tile_index(w);
  if (ck->tiled[ti].gs[0][0] == nullptr) return false;
  return planes == 1 ? rk->init_t[ti][0] != nullptr : (rk->mp_init_t[ti] != nullptr && rk->mp_t[ti][0] != nullptr);
}

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      ok = false;
      return;
    }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

struct hg_plan {
  int device = 0;
  int n_items = 0;
  std::vector<int> H, W;
  int propagation = HG_FOURIER;
  double lambda = 0, pitch = 0;
  int P = 1;
  std::vector<double> z;
  int levels = 0;
  std::vector<SizeClass> classes;
  std::vector<int> item_class, item_slot;
  std::map<int, float2*> tw;
  std::map<int, float2*> tw_alt;  // twiddle tables of the alternative radix plans, per length
  std::map<int, float2*> roots;  // direct binary search: exp(-2 pi i j / N), j < N, per length
  float2* lev = nullptr;
  float* lev_phase = nullptr;
  // the plan's phase-only level set (quant_levels and its tables), kept while a multi-amplitude
  // table is set (levels = -M, lev / lev_phase pointing at the table)
  int levels0 = 0;
  float2* lev0 = nullptr;
  float* lev_phase0 = nullptr;
  std::vector<const float*> illum;  // per item SLM illumination amplitude (nullptr: uniform)
  std::vector<void*> allocs;
  // run order, graphs and latency stamps
  std::vector<size_t> class_order;  // size classes, smallest first
  unsigned long long* stamps = nullptr;  // [1 + classes]: run start, end of each class (%globaltimer)
  bool graph = false;
  bool centred = false;             // HG_TARGET_CENTRED: targets in display order
  bool capturing = false;           // enqueueing into a graph capture
  cudaStream_t cap = nullptr;       // capture stream of graph mode
  // graph mode keeps one executable graph per timing state: [1] also records a pair of events
  // around every kernel (graph nodes); the timing totals take its latest replay
  struct Pending {
    cudaEvent_t a, b;
    int kind;
  };
  struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    std::vector<uintptr_t> key;
    int64_t kernels = 0;
    std::vector<Pending> events;
    bool replayed = false;  // events hold a replay that has not been folded in yet
  };
  GraphSlot gslot[2];
  // timing facility
  bool timing = false;
  int64_t launches = 0;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  double kind_ms[K_NUM_KINDS] = {};
  int64_t kind_count[K_NUM_KINDS] = {};

  ~hg_plan() {
    for (GraphSlot& g : gslot) drop_graph(g);
    if (cap) cudaStreamDestroy(cap);
    for (void* p : allocs) cudaFree(p);
    for (auto& q : pending) {
      cudaEventDestroy(q.a);
      cudaEventDestroy(q.b);
    }
    for (cudaEvent_t e : event_pool) cudaEventDestroy(e);
  }
  cudaEvent_t get_event() {
    if (!event_pool.empty()) {
      cudaEvent_t e = event_pool.back();
      event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }
  void add_time(const Pending& q) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      kind_ms[q.kind] += ms;
      kind_count[q.kind] += 1;
    } else {
      cudaGetLastError();
    }
  }
  // folds completed timing events into the per-kind totals (device must be idle): stream launches,
  // and the latest replay of the timed graph
  void fold() {
    for (auto& q : pending) {
      add_time(q);
      event_pool.push_back(q.a);
      event_pool.push_back(q.b);
    }
    pending.clear();
    for (GraphSlot& g : gslot)
      if (g.replayed) {
        for (auto& q : g.events) add_time(q);
        g.replayed = false;
      }
  }
  void drop_graph(GraphSlot& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.key.clear();
    for (auto& q : g.events) {
      event_pool.push_back(q.a);
      event_pool.push_back(q.b);
    }
    g.events.clear();
    g.replayed = false;
  }
  template <class T>
  hg_status alloc(T** p, size_t count, const char* what) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e != cudaSuccess) return cuda_fail(e, what);
    allocs.push_back(q);
    *p = (T*)q;
    return HG_OK;
  }
};

namespace {

// Device pointer check: device (or managed) memory of the plan's device, aligned, and -- where the
// driver can tell -- [ptr, ptr + bytes) inside one allocation.
hg_status check_ptr(const hg_plan* p, const void* ptr, size_t bytes, size_t align, const char* what, int idx) {
  if (!ptr) return fail(HG_ERR_INVALID_ARG, "%s[%d] is NULL", what, idx);
  if ((uintptr_t)ptr % align) return fail(HG_ERR_INVALID_ARG, "%s[%d] is not %zu-byte aligned", what, idx, align);
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(HG_ERR_INVALID_ARG, "%s[%d] is not a CUDA pointer (%s)", what, idx, cudaGetErrorString(e));
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(HG_ERR_INVALID_ARG, "%s[%d] is not device memory", what, idx);
  if (at.type == cudaMemoryTypeDevice && at.device != p->device)
    return fail(HG_ERR_INVALID_ARG, "%s[%d] lives on device %d, plan is on device %d", what, idx, at.device, p->device);
  if (range_fn_t fn = range_fn()) {
    unsigned long long base = 0;
    size_t size = 0;
    if (fn(&base, &size, (unsigned long long)(uintptr_t)ptr) == 0) {
      if ((unsigned long long)(uintptr_t)ptr + bytes > base + size)
        return fail(HG_ERR_INVALID_ARG, "%s[%d]: %zu bytes do not fit in its allocation", what, idx, bytes);
    }
  }
  return HG_OK;
}

hg_status launch(hg_plan* p, int kind, const void* fn, dim3 grid, int nt, int smem, const hg::PassArgs& a,
                 cudaStream_t s, int extra_int = 0, float* extra_ptr = nullptr, int cluster_x = 0) {
  void* args3[] = {(void*)&a, (void*)&extra_int, (void*)&extra_ptr};
  void** args = args3;  // kernels with one parameter read only the first entry
  cudaEvent_t ea = nullptr, eb = nullptr;
  if (p->timing) {
    ea = p->get_event();
    eb = p->get_event();
    // inside a graph capture the records must be external ones to become event-record nodes
    if (ea && eb) cudaEventRecordWithFlags(ea, s, p->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
  }
  cudaError_t e;
  // GS passes (they wait for their predecessor in-kernel) of at most 2048^2 pixels per launch, on
  // a stream: programmatic stream serialisation hides the launch gap between the passes (measured
  // on GB300: 256^2 +39 %, 1024^2 +11 %, 2048^2 +2 %); larger launches ran slower with it (4096^2:
  // -10 %), and so did replayed graphs (2048^2: 19.7k against 21.1k it/s without), which keep it off.
  const bool pdl = HG_PDL && !p->timing && !p->capturing &&
                   (kind == K_COL_GS || kind == K_ROW_GS || kind == K_COL_NMSE) &&
                   (int64_t)a.H * a.W * a.n_items <= (int64_t)2048 * 2048;
  if (cluster_x > 0) {  // thread-block clusters of cluster_x CTAs along x
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = (unsigned)cluster_x;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelExC(&cfg, fn, args);
  } else if (pdl) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelExC(&cfg, fn, args);
  } else {
    e = cudaLaunchKernel(fn, grid, dim3(nt), args, (size_t)smem, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  p->launches++;
  if (ea && eb) {
    cudaEventRecordWithFlags(eb, s, p->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
    p->pending.push_back({ea, eb, kind});
  } else {
    if (ea) p->event_pool.push_back(ea);
    if (eb) p->event_pool.push_back(eb);
  }
  return HG_OK;
}

// per-stage twiddle tables: entry off + (r-1) ns + k = exp(-2 pi i r k / (ns R)), float64 then rounded
std::vector<float2> twiddles(const hg::TwiddleLayout& l) {
  std::vector<float2> t(l.size > 0 ? l.size : 1, make_float2(1.f, 0.f));
  const double two_pi = 6.283185307179586476925286766559;
  for (int i = 0; i < l.count; ++i) {
    const int ns = l.ns[i], r = l.r[i], n = ns * r;
    for (int q = 1; q < r; ++q)
      for (int k = 0; k < ns; ++k) {
        const double a = two_pi * (double)((q * k) % n) / (double)n;
        t[l.off[i] + (q - 1) * ns + k] = make_float2((float)std::cos(a), (float)-std::sin(a));
      }
  }
  return t;
}

// chirp factor exp(i pi (d p)^2 / (lambda z)), d = index - floor(n/2); the phase is reduced in turns
// (fractional part of (d p)^2 / (2 lambda z)) in float64 before the trig call
std::vector<float2> chirp_axis(int n, double pitch, double lambda, double z) {
  std::vector<float2> c(n);
  const double two_pi = 6.283185307179586476925286766559;
  for (int i = 0; i < n; ++i) {
    const double d = (double)(i - n / 2) * pitch;
    double turns = d * d / (2.0 * lambda * z);
    turns -= std::floor(turns);
    c[i] = make_float2((float)std::cos(two_pi * turns), (float)std::sin(two_pi * turns));
  }
  return c;
}

template <class T>
hg_status upload(hg_plan* p, T** dst, const std::vector<T>& v, const char* what) {
  hg_status s = p->alloc(dst, v.size(), what);
  if (s != HG_OK) return s;
  HG_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), what);
  return HG_OK;
}

// The whole-run cluster kernel of a square class: 16 CTAs per cluster where the device can run such
// a cluster (a non-portable size), else 8; none for other shapes or lengths.
void pick_cluster(SizeClass& c) {
  c.cl = 0;
  if (c.H != c.W) return;
  for (int i = 1; i >= 0; --i) {
    const void* fn = c.rk->gs_cluster[i];
    if (!fn) continue;
    const int cl = i ? 16 : 8;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cl, 1);
    cfg.blockDim = dim3(c.rk->nt_cluster[i]);
    cfg.dynamicSmemBytes = (size_t)c.rk->smem_cluster[i];
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = (unsigned)cl;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess || n < 1) {
      cudaGetLastError();  // not available: clear the error and try the smaller cluster
      continue;
    }
    c.cl = cl;
    c.cl_fn = fn;
    c.cl_nt = c.rk->nt_cluster[i];
    c.cl_smem = c.rk->smem_cluster[i];
    return;
  }
}

void fill_common(const hg_plan* p, const SizeClass& c, int plane, hg::PassArgs& a) {
  a.H = c.H;
  a.W = c.W;
  a.n_levels = p->levels;
  a.tw_row = p->tw.at(c.W);
  a.tw_col = p->tw.at(c.H);
  a.cx = p->propagation == HG_FRESNEL ? c.cx[plane] : nullptr;
  a.cy = p->propagation == HG_FRESNEL ? c.cy[plane] : nullptr;
  a.lev = p->lev;
  a.lev_phase = p->lev_phase;
  a.field = c.field;
  a.partials = c.partials;
  a.col_blocks = c.col_blocks();
  a.n_planes = p->P;
  for (int q = 0; q < p->P; ++q) {
    a.cxp[q] = p->propagation == HG_FRESNEL ? c.cx[q] : nullptr;
    a.cyp[q] = p->propagation == HG_FRESNEL ? c.cy[q] : nullptr;
  }
  a.stats = c.stats;
  a.centred = p->centred ? 1 : 0;
  if (c.rk->gen) a.gen_row = *c.rk->gen;
  if (c.ck->gen) a.gen_col = *c.ck->gen;
}

}  // namespace

// Re-lays the targets out per column strip for the GS column passes: strip t of (item, plane) holds
// [H][C] contiguous (zero past W), so a column pass streams its strip with contiguous copies instead
// of C-float pieces of every row; targets and masks given in display order are ifftshifted on the
// way.  blockIdx.x = strip, blockIdx.y = item * P + plane.
__global__ void k_tile_target(const __grid_constant__ hg::PassArgs a, int C, float* ttile) {
  const int P = a.n_planes > 1 ? a.n_planes : 1;
  const int k = blockIdx.y / P, p = blockIdx.y % P;
  const float* A = a.target[k * P + p];
  const int H = a.H, W = a.W, col0 = blockIdx.x * C;
  float* dst = ttile + (((size_t)a.class_slot[k] * P + p) * gridDim.x + blockIdx.x) * (size_t)H * C;
  const uint8_t* mask = a.mix > 0.f ? a.mask[k] : nullptr;  // MRAF: -1 marks the noise region
  for (int i = threadIdx.x; i < H * C; i += blockDim.x) {
    const int n = i / C, b = i % C;
    if (col0 + b >= W) {
      dst[i] = 0.f;
      continue;
    }
    const size_t px = hg::target_index(a, n, col0 + b);  // display-order targets: ifftshift here
    dst[i] = (mask && !__ldg(&mask[px])) ? -1.f : __ldg(&A[px]);
  }
}

// Per (item, plane) block partials of the target amplitude energy sum A^2 (finalised by
// k_finalize<2> into stats[4 sp + 3] = 1 / sqrt(sum A^2); multi-plane GS weights each plane's
// back-propagated field by it).  blockIdx.y = item * P + plane, gridDim.x = column blocks.
__global__ void k_amp_energy(const __grid_constant__ hg::PassArgs a) {
  const int P = a.n_planes > 1 ? a.n_planes : 1;
  const int k = blockIdx.y / P, p = blockIdx.y % P;
  const int sp = a.class_slot[k] * P + p;
  const float* A = a.target[k * P + p];
  const uint8_t* mask = a.mix > 0.f ? a.mask[k] : nullptr;  // MRAF: the signal region's energy
  const size_t n = (size_t)a.H * a.W;
  float e = 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float x = (mask && !__ldg(&mask[i])) ? 0.f : __ldg(&A[i]);
    e = fmaf(x, x, e);
  }
  hg::block_partials(e, 0.f, 0.f, a.partials + (size_t)sp * 3 * gridDim.x);
}

namespace {

// items per launch: (item, plane) pairs of one launch must fit the argument block
int chunk_items(const hg_plan* p) { return std::max(1, hg::kMaxBatch / p->P); }

// Grid of the generic multi-plane pointwise kernels: a grid-stride loop over one item's field per
// blockIdx.y.
dim3 pointwise_grid(const SizeClass& c, int nb) {
  const int64_t blocks = ((int64_t)c.H * c.W + 255) / 256;
  return dim3((unsigned)std::min<int64_t>(blocks, 4 * 152), (unsigned)nb);
}

// Generic row lengths: the multi-plane accumulator of a class, allocated on first use.
hg_status ensure_plane_acc(hg_plan* p, SizeClass& c) {
  if (!c.rk->gen || c.gacc) return HG_OK;
  return p->alloc(&c.gacc, c.items.size() * (size_t)c.H * c.W, "multi-plane accumulator");
}

// Generic row lengths: every plane's forward row FFTs of the accumulator c_p -> field p.
hg_status plane_forwards(hg_plan* p, const SizeClass& c, int kind, const hg::PassArgs& a, dim3 grow, cudaStream_t st) {
  hg_status s;
  for (int q = 0; q < p->P; ++q)
    if ((s = launch(p, kind, c.rk->plane.fwd, grow, c.rk->nt, c.rk->smem, a, st, q, (float*)c.gacc)) != HG_OK)
      return s;
  return HG_OK;
}

// Generic row lengths: the sum over planes of conj(c_p) (inverse row FFTs of field p) -> accumulator.
hg_status plane_backs(hg_plan* p, const SizeClass& c, int kind, const hg::PassArgs& a, dim3 grow, cudaStream_t st) {
  hg_status s;
  for (int q = 0; q < p->P; ++q)
    if ((s = launch(p, kind, c.rk->plane.back, grow, c.rk->nt, c.rk->smem, a, st, q, (float*)c.gacc)) != HG_OK)
      return s;
  return HG_OK;
}

}  // namespace

extern "C" {

const char* hg_status_string(hg_status s) {
  switch (s) {
    case HG_OK: return "HG_OK";
    case HG_ERR_INVALID_ARG: return "HG_ERR_INVALID_ARG";
    case HG_ERR_UNSUPPORTED_SIZE: return "HG_ERR_UNSUPPORTED_SIZE";
    case HG_ERR_OUT_OF_MEMORY: return "HG_ERR_OUT_OF_MEMORY";
    case HG_ERR_CUDA: return "HG_ERR_CUDA";
    case HG_ERR_TIMEOUT: return "HG_ERR_TIMEOUT";
    case HG_ERR_INTERNAL: return "HG_ERR_INTERNAL";
  }
  return "HG_ERR_UNKNOWN";
}

const char* hg_last_error(void) { return g_err.c_str(); }

hg_status hg_plan_set_timing(hg_plan* p, int32_t enabled) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  p->timing = enabled != 0;
  return HG_OK;
}

hg_status hg_plan_reset_timing(hg_plan* p) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  DeviceGuard g(p->device);
  cudaDeviceSynchronize();
  p->fold();
  for (int k = 0; k < K_NUM_KINDS; ++k) {
    p->kind_ms[k] = 0.0;
    p->kind_count[k] = 0;
  }
  return HG_OK;
}

hg_status hg_plan_kernel_time(hg_plan* p, int32_t kind, double* total_ms, int64_t* launches) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  if (kind < 0 || kind >= K_NUM_KINDS) return fail(HG_ERR_INVALID_ARG, "kind %d out of range", kind);
  if (!total_ms || !launches) return fail(HG_ERR_INVALID_ARG, "output is NULL");
  DeviceGuard g(p->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "device error");
  p->fold();
  *total_ms = p->kind_ms[kind];
  *launches = p->kind_count[kind];
  return HG_OK;
}

hg_status hg_plan_set_graph(hg_plan* p, int32_t enabled) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  p->graph = enabled != 0;
  if (!p->graph) {
    DeviceGuard g(p->device);
    cudaDeviceSynchronize();
    p->fold();
    for (auto& slot : p->gslot) p->drop_graph(slot);
  }
  return HG_OK;
}

hg_status hg_plan_item_latency(hg_plan* p, double* ms_out) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  if (!ms_out) return fail(HG_ERR_INVALID_ARG, "ms_out is NULL");
  DeviceGuard g(p->device);
  std::vector<unsigned long long> st(1 + p->classes.size());
  HG_CUDA(cudaDeviceSynchronize(), "device error");
  HG_CUDA(cudaMemcpy(st.data(), p->stamps, st.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost), "stamps");
  for (int i = 0; i < p->n_items; ++i) {
    const unsigned long long end = st[1 + p->item_class[i]];
    ms_out[i] = end >= st[0] ? (double)(end - st[0]) * 1e-6 : 0.0;
  }
  return HG_OK;
}

const char* hg_kernel_kind_name(int32_t kind) { return kind >= 0 && kind < K_NUM_KINDS ? kKindNames[kind] : nullptr; }

int64_t hg_plan_launch_count(const hg_plan* p) { return p ? p->launches : 0; }

int32_t hg_supported_length(int32_t n) { return hg::row_kernels(n) != nullptr && hg::col_kernels(n) != nullptr; }

hg_status hg_plan_create(const hg_plan_desc* d, hg_plan** out) {
  if (!out) return fail(HG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!d) return fail(HG_ERR_INVALID_ARG, "desc is NULL");
  if (d->n_items < 1 || d->n_items > kMaxItems) return fail(HG_ERR_INVALID_ARG, "n_items must be 1..%d", kMaxItems);
  if (!d->heights || !d->widths) return fail(HG_ERR_INVALID_ARG, "heights / widths is NULL");
  if (d->propagation != HG_FOURIER && d->propagation != HG_FRESNEL)
    return fail(HG_ERR_INVALID_ARG, "unknown propagation %d", d->propagation);
  if (d->n_planes < 1 || d->n_planes > 16) return fail(HG_ERR_INVALID_ARG, "n_planes must be 1..16");
  if (d->propagation == HG_FOURIER && d->n_planes != 1)
    return fail(HG_ERR_INVALID_ARG, "Fourier plans have exactly one plane");
  if (d->quant_levels < 0 || d->quant_levels == 1 || d->quant_levels > kMaxLevels)
    return fail(HG_ERR_INVALID_ARG, "quant_levels must be 0 or 2..%d", kMaxLevels);
  if (d->flags & ~(HG_PLAN_AUTOTUNE | HG_TARGET_CENTRED))
    return fail(HG_ERR_INVALID_ARG, "unknown flags 0x%x", d->flags);
  if (d->propagation == HG_FRESNEL) {
    if (!(d->wavelength_m > 0) || !(d->pitch_m > 0) || !std::isfinite(d->wavelength_m) || !std::isfinite(d->pitch_m))
      return fail(HG_ERR_INVALID_ARG, "Fresnel plans need wavelength_m > 0 and pitch_m > 0");
    if (!d->z_m) return fail(HG_ERR_INVALID_ARG, "z_m is NULL");
    for (int i = 0; i < d->n_planes; ++i)
      if (!(d->z_m[i] > 0) || !std::isfinite(d->z_m[i])) return fail(HG_ERR_INVALID_ARG, "z_m[%d] must be > 0", i);
  }
  for (int i = 0; i < d->n_items; ++i) {
    const int h = d->heights[i], w = d->widths[i];
    if (h < 1 || w < 1) return fail(HG_ERR_INVALID_ARG, "item %d: size %dx%d", i, h, w);
    if (!hg_supported_length(h) || !hg_supported_length(w))
      return fail(HG_ERR_UNSUPPORTED_SIZE, "item %d: %dx%d is not a supported size", i, h, w);
  }

  hg_plan* p = new (std::nothrow) hg_plan();
  if (!p) return fail(HG_ERR_OUT_OF_MEMORY, "host allocation");
  auto bail = [&](hg_status s) {
    delete p;
    return s;
  };
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(HG_ERR_CUDA, "no CUDA device"));
  }
  p->n_items = d->n_items;
  p->H.assign(d->heights, d->heights + d->n_items);
  p->W.assign(d->widths, d->widths + d->n_items);
  p->propagation = d->propagation;
  p->lambda = d->wavelength_m;
  p->pitch = d->pitch_m;
  p->P = d->n_planes;
  if (d->propagation == HG_FRESNEL) p->z.assign(d->z_m, d->z_m + d->n_planes);
  p->levels = d->quant_levels;
  p->centred = (d->flags & HG_TARGET_CENTRED) != 0;

  // size classes
  p->item_class.resize(p->n_items);
  p->item_slot.resize(p->n_items);
  for (int i = 0; i < p->n_items; ++i) {
    int ci = -1;
    for (size_t c = 0; c < p->classes.size(); ++c)
      if (p->classes[c].H == p->H[i] && p->classes[c].W == p->W[i]) ci = (int)c;
    if (ci < 0) {
      SizeClass c;
      c.H = p->H[i];
      c.W = p->W[i];
      c.rk = hg::row_kernels(c.W);
      c.ck = hg::col_kernels(c.H);
      p->classes.push_back(c);
      ci = (int)p->classes.size() - 1;
    }
    p->item_class[i] = ci;
    p->item_slot[i] = (int)p->classes[ci].items.size();
    p->classes[ci].items.push_back(i);
  }

  hg_status s;
  for (SizeClass& c : p->classes) {
    c.rk->set_attrs();
    c.ck->set_attrs();
    const size_t n = c.items.size() * (size_t)p->P;
    if ((s = p->alloc(&c.field, n * c.H * c.W, "field workspace")) != HG_OK) return bail(s);
    pick_cluster(c);
    // default: the whole-run cluster kernel for a class of one item where it exists (measured on
    // GB300, 20 iterations: 64^2 112 against 160 us, 128^2 177 against 207, 256^2 222 against 224;
    // with 16 items of 256^2 it takes twice as long as the two-pass kernels, whose launches then
    // fill the GPU), else the measured strip width
    c.tile = (c.items.size() == 1 && c.tileable(-1, p->P)) ? -1 : (c.tileable(c.ck->tile, p->P) ? c.ck->tile : 0);
    if ((s = p->alloc(&c.partials, n * 3 * c.max_strips(), "reduction scratch")) != HG_OK) return bail(s);
    if ((s = p->alloc(&c.stats, n * 4, "loss statistics")) != HG_OK) return bail(s);
    if ((s = p->alloc(&c.ttile, n * c.max_strip_cols() * c.H, "target tiles")) != HG_OK)
      return bail(s);
    if (cudaMemset(c.stats, 0, n * 4 * sizeof(double)) != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "memset"));
    for (int pl = 0; pl < p->P; ++pl) {
      float2 *cx = nullptr, *cy = nullptr;
      if (p->propagation == HG_FRESNEL) {
        if ((s = upload(p, &cx, chirp_axis(c.W, p->pitch, p->lambda, p->z[pl]), "chirp table")) != HG_OK) return bail(s);
        if ((s = upload(p, &cy, chirp_axis(c.H, p->pitch, p->lambda, p->z[pl]), "chirp table")) != HG_OK) return bail(s);
      }
      c.cx.push_back(cx);
      c.cy.push_back(cy);
    }
    for (int len : {c.H, c.W}) {
      if (p->tw.count(len)) continue;
      float2* t = nullptr;
      if ((s = upload(p, &t, twiddles(hg::row_kernels(len)->tw), "twiddle table")) != HG_OK) return bail(s);
      p->tw[len] = t;
      if (hg::row_kernels(len)->has_alt) {
        if ((s = upload(p, &t, twiddles(hg::row_kernels(len)->tw_alt), "twiddle table")) != HG_OK) return bail(s);
        p->tw_alt[len] = t;
      }
    }
  }
  // level tables exp(2 pi i q / N) and 2 pi q / N, exact on the axes
  {
    const int nl = p->levels > 0 ? p->levels : 1;
    std::vector<float2> lev(nl);
    std::vector<float> ph(nl);
    const double two_pi = 6.283185307179586476925286766559;
    for (int q = 0; q < nl; ++q) {
      const double a = two_pi * (double)q / (double)nl;
      lev[q] = make_float2((float)std::cos(a), (float)std::sin(a));
      if ((4 * q) % nl == 0) {
        const int quarter = (4 * q / nl) % 4;
        const float ax[4][2] = {{1.f, 0.f}, {0.f, 1.f}, {-1.f, 0.f}, {0.f, -1.f}};
        lev[q] = make_float2(ax[quarter][0], ax[quarter][1]);
      }
      ph[q] = (float)a;
    }
    if ((s = upload(p, &p->lev, lev, "level table")) != HG_OK) return bail(s);
    if ((s = upload(p, &p->lev_phase, ph, "level table")) != HG_OK) return bail(s);
    p->levels0 = p->levels;
    p->lev0 = p->lev;
    p->lev_phase0 = p->lev_phase;
  }
  if ((s = p->alloc(&p->stamps, 1 + p->classes.size(), "latency stamps")) != HG_OK) return bail(s);
  if (cudaMemset(p->stamps, 0, (1 + p->classes.size()) * sizeof(unsigned long long)) != cudaSuccess)
    return bail(cuda_fail(cudaGetLastError(), "memset"));
  p->class_order.resize(p->classes.size());
  for (size_t i = 0; i < p->classes.size(); ++i) p->class_order[i] = i;
  std::stable_sort(p->class_order.begin(), p->class_order.end(), [&](size_t x, size_t y) {
    return (size_t)p->classes[x].H * p->classes[x].W < (size_t)p->classes[y].H * p->classes[y].W;
  });
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "plan set-up"));
  if ((d->flags & HG_PLAN_AUTOTUNE) && (s = hg_plan_autotune(p, nullptr)) != HG_OK) return bail(s);
  *out = p;
  return HG_OK;
}

hg_status hg_plan_destroy(hg_plan* p) {
  if (!p) return HG_OK;
  DeviceGuard g(p->device);
  cudaDeviceSynchronize();
  cudaGetLastError();
  delete p;
  return HG_OK;
}

hg_status hg_plan_sync(hg_plan* p) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  DeviceGuard g(p->device);
  if (!g.ok) return fail(HG_ERR_CUDA, "cannot select device %d", p->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "device error");
  return HG_OK;
}

hg_status hg_propagate(hg_plan* p, int32_t plane, int32_t direction, const void* const* in, void* const* out,
                       void* stream) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  if (plane < 0 || plane >= p->P) return fail(HG_ERR_INVALID_ARG, "plane %d out of range", plane);
  if (direction != 1 && direction != -1) return fail(HG_ERR_INVALID_ARG, "direction must be +1 or -1");
  if (!in || !out) return fail(HG_ERR_INVALID_ARG, "in / out is NULL");
  DeviceGuard g(p->device);
  if (!g.ok) return fail(HG_ERR_CUDA, "cannot select device %d", p->device);
  hg_status s;
  for (int i = 0; i < p->n_items; ++i) {
    const size_t bytes = (size_t)p->H[i] * p->W[i] * 8;
    if ((s = check_ptr(p, in[i], bytes, 8, "in", i)) != HG_OK) return s;
    if ((s = check_ptr(p, out[i], bytes, 8, "out", i)) != HG_OK) return s;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool inv = direction < 0;
  const bool fres = p->propagation == HG_FRESNEL;
  for (const SizeClass& c : p->classes) {
    for (size_t c0 = 0; c0 < c.items.size(); c0 += hg::kMaxBatch) {
      const int nb = (int)std::min<size_t>(hg::kMaxBatch, c.items.size() - c0);
      hg::PassArgs a{};
      fill_common(p, c, plane, a);
      a.n_items = nb;
      a.scale = (float)(1.0 / std::sqrt((double)c.H * (double)c.W));
      for (int k = 0; k < nb; ++k) {
        const int item = c.items[c0 + k];
        a.item_index[k] = item;
        a.class_slot[k] = (int)(c0 + k);
        a.in[k] = (const float2*)in[item];
        a.out[k] = (float2*)out[item];
      }
      if ((s = launch(p, K_ROW_FFT, c.rk->fft[inv][fres && !inv], dim3(c.row_blocks(), nb), c.rk->nt, c.rk->smem, a, st)) != HG_OK)
        return s;
      if ((s = launch(p, K_COL_FFT, c.ck->fft[inv][fres && inv], dim3(c.col_blocks(), nb), c.ck->nt, c.ck->smem, a, st)) != HG_OK)
        return s;
    }
  }
  return HG_OK;
}

}  // extern "C"

namespace {

struct GsCall {
  const float* const* target_amp;
  const float* const* init_phase;
  uint64_t seed;
  int32_t n_iter;
  float* const* phase_out;
  uint8_t* const* level_out;
  float* nmse_out;
  const uint8_t* const* mask = nullptr;  // MRAF signal regions (per item, nullable)
  float mix = 0.f;                       // MRAF mixing parameter (0: plain GS; 1 under HIO)
  bool hio = false;                      // HIO: noise-region feedback X' = X - beta Y
  float beta = 0.f;
};

__global__ void k_stamp(unsigned long long* dst) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *dst = t;
}

// Launch sequence of one size class (every chunk of its items) on stream st.
hg_status gs_class(hg_plan* p, const SizeClass& c, const GsCall& g, cudaStream_t st) {
  const float* const* target_amp = g.target_amp;
  const float* const* init_phase = g.init_phase;
  const uint64_t seed = g.seed;
  const int32_t n_iter = g.n_iter;
  float* const* phase_out = g.phase_out;
  uint8_t* const* level_out = g.level_out;
  float* nmse_out = g.nmse_out;
  hg_status s;
  const int P = p->P;
  const int chunk = chunk_items(p);
  for (size_t c0 = 0; c0 < c.items.size(); c0 += chunk) {
    const int nb = (int)std::min<size_t>(chunk, c.items.size() - c0);
    hg::PassArgs a{};
    fill_common(p, c, 0, a);
    a.n_items = nb;
    a.nmse = nmse_out;
    a.nmse_stride = n_iter + 1;
    a.seed = seed;
    for (int k = 0; k < nb; ++k) {
      const int item = c.items[c0 + k];
      a.item_index[k] = item;
      a.class_slot[k] = (int)(c0 + k);
      for (int q = 0; q < P; ++q) a.target[k * P + q] = target_amp[item * P + q];
      a.phase_in[k] = init_phase ? init_phase[item] : nullptr;
      a.mask[k] = g.mask ? g.mask[item] : nullptr;
      a.illum[k] = p->illum.empty() ? nullptr : p->illum[item];
    }
    a.mix = g.mix;
    a.hio = g.hio ? c.hio : nullptr;
    a.beta = g.beta;
    bool lit = false;
    for (int k = 0; k < nb; ++k) lit = lit || a.illum[k] != nullptr;
    if (c.tile == -1 && P == 1 && g.mix == 0.f && !lit && p->levels >= 0) {
      // the whole run in one launch: one cluster per item, the field in the cluster's shared memory
      for (int k = 0; k < nb; ++k) {
        const int item = c.items[c0 + k];
        a.phase_out[k] = phase_out ? phase_out[item] : nullptr;
        a.level_out[k] = level_out ? level_out[item] : nullptr;
      }
      a.n_iter = n_iter;
      if ((s = launch(p, K_GS_CLUSTER, c.cl_fn, dim3(c.cl, nb), c.cl_nt, c.cl_smem, a, st, 0, nullptr, c.cl)) !=
          HG_OK)
        return s;
      continue;
    }
    // field layout: single-plane runs tile the field in column strips when the row length allows
    // (contiguous strips for the column pass), else row-major; MRAF, HIO and illuminated runs of a
    // class set to the cluster kernel take the default strip width
    const int width = c.tile == -1 ? (c.tileable(c.ck->tile, P) ? c.ck->tile : 0) : c.tile;
    const bool tiled = width > 0;
    const int ti = tiled ? tile_index(width) : 0;
    const int strip = tiled ? width : c.ck->cols;
    const int strips = tiled ? (c.W + width - 1) / width : c.col_blocks();
    a.col_blocks = strips;
    // targets re-laid out per column strip once per run (read by every column pass of the run)
    if ((s = launch(p, K_TILE_TARGET, (const void*)&k_tile_target, dim3(strips, nb * P), 256, 0, a, st, strip,
                    c.ttile)) != HG_OK)
      return s;
    a.ttile = c.ttile;
    if (P > 1) {
      // multi-plane GS: averaged projections over the P planes, on the tiled field (strips of
      // width C: the column passes stream contiguous strips) or the row-major one
      const dim3 grow(tiled ? (c.H + c.rk->rows_t[ti] - 1) / c.rk->rows_t[ti] : c.row_blocks(), nb),
          gcol(strips, nb * P);
      const void* k_init = tiled ? c.rk->mp_init_t[ti] : c.rk->mp_init[1];
      const void* k_row[2] = {tiled ? c.rk->mp_t[ti][0] : c.rk->mp[0], tiled ? c.rk->mp_t[ti][1] : c.rk->mp[1]};
      if (tiled && width == 2 && c.H == c.W && c.rk->mp_sq[0] != nullptr) {  // square: compile-time strip height
        k_row[0] = c.rk->mp_sq[0];
        k_row[1] = c.rk->mp_sq[1];
      }
      const void* k_col[2] = {tiled ? c.ck->tiled[ti].gs[0][0] : c.ck->gs[0][0],
                              tiled ? c.ck->tiled[ti].gs[1][0] : c.ck->gs[1][0]};
      const int rnt = tiled ? c.rk->nt_t[ti] : c.rk->nt, rsm = tiled ? c.rk->smem_t[ti] : c.rk->smem;
      const int cnt = tiled ? c.ck->tiled[ti].nt : c.ck->nt, csm = tiled ? c.ck->tiled[ti].smem_gs : c.ck->smem_gs;
      hg::PassArgs a0 = a, ao = a;
      for (int k = 0; k < nb; ++k) {
        const int item = c.items[c0 + k];
        ao.phase_out[k] = phase_out ? phase_out[item] : nullptr;
        ao.level_out[k] = level_out ? level_out[item] : nullptr;
        if (n_iter == 0) {
          a0.phase_out[k] = ao.phase_out[k];
          a0.level_out[k] = ao.level_out[k];
        }
      }
      const dim3 gfin(1, nb);
      const bool gen = c.rk->gen != nullptr;  // generic row length: one launch per plane
      float* acc = (float*)c.gacc;
      if ((s = launch(p, K_AMP_ENERGY, (const void*)&k_amp_energy, gcol, 256, 0, a, st)) != HG_OK) return s;
      if ((s = launch(p, K_FINALIZE, (const void*)&hg::k_finalize<2>, gfin, 32, 0, a, st)) != HG_OK) return s;
      if (gen) {
        if ((s = launch(p, K_ROW_MP_INIT, c.rk->plane.start[1], pointwise_grid(c, nb), 256, 0, a0, st, 0, acc)) !=
                HG_OK ||
            (s = plane_forwards(p, c, K_ROW_MP_INIT, a, grow, st)) != HG_OK)
          return s;
      } else if ((s = launch(p, K_ROW_MP_INIT, k_init, grow, rnt, rsm, a0, st)) != HG_OK) {
        return s;
      }
      for (int it = 0; it < n_iter; ++it) {
        a.iter = it;
        if ((s = launch(p, K_COL_GS, k_col[1], gcol, cnt, csm, a, st)) != HG_OK) return s;
        const bool last = it == n_iter - 1;
        hg::PassArgs ar = last ? ao : a;
        ar.finalize = nmse_out != nullptr;
        ar.fin_iter = it;
        if (gen) {
          if ((s = plane_backs(p, c, K_ROW_MP, ar, grow, st)) != HG_OK ||
              (s = launch(p, K_ROW_MP, c.rk->plane.project, pointwise_grid(c, nb), 256, 0, ar, st, 0, acc)) != HG_OK ||
              (s = plane_forwards(p, c, K_ROW_MP, a, grow, st)) != HG_OK)
            return s;
        } else if ((s = launch(p, K_ROW_MP, k_row[last], grow, rnt, rsm, ar, st)) != HG_OK) {
          return s;
        }
      }
      a.iter = n_iter;
      a.fin_iter = n_iter;
      if ((s = launch(p, K_COL_NMSE, k_col[0], gcol, cnt, csm, a, st)) != HG_OK) return s;
      if (nmse_out && (s = launch(p, K_FINALIZE, (const void*)&hg::k_finalize<0>, gfin, 32, 0, a, st)) != HG_OK)
        return s;
      continue;
    }
    if (g.mix > 0.f || p->levels < 0) {
      // MRAF / HIO: the signal region's target energy, for the absolute scale of m A_s; a
      // multi-amplitude SLM: the target energy, for the unitary scale of the field it projects
      const dim3 genergy(strips, nb), gfin(1, nb);
      if ((s = launch(p, K_AMP_ENERGY, (const void*)&k_amp_energy, genergy, 256, 0, a, st)) != HG_OK) return s;
      if ((s = launch(p, K_FINALIZE, (const void*)&hg::k_finalize<2>, gfin, 32, 0, a, st)) != HG_OK) return s;
    }
    // extended kernels only when the run uses MRAF / HIO, an illumination profile or a
    // multi-amplitude SLM
    const int x = (g.mix > 0.f || lit || p->levels < 0) ? 1 : 0;
    // the alternative radix plan per pass, where chosen and compiled for this width (plain runs)
    const bool prow = tiled && x == 0 && c.pv_row == 1 && c.rk->init_tp[ti] != nullptr;
    const bool pcol = tiled && x == 0 && c.pv_col == 1 && c.ck->tiled[ti].gs_p[0] != nullptr;
    const void* k_init = prow ? c.rk->init_tp[ti] : (tiled ? c.rk->init_t[ti][x] : c.rk->init[x]);
    const void* k_row[2] = {prow ? c.rk->gs_tp[ti][0] : (tiled ? c.rk->gs_t[ti][0][x] : c.rk->gs[0][x]),
                            prow ? c.rk->gs_tp[ti][1] : (tiled ? c.rk->gs_t[ti][1][x] : c.rk->gs[1][x])};
    const void* k_col[2] = {pcol ? c.ck->tiled[ti].gs_p[0] : (tiled ? c.ck->tiled[ti].gs[0][x] : c.ck->gs[0][x]),
                            pcol ? c.ck->tiled[ti].gs_p[1] : (tiled ? c.ck->tiled[ti].gs[1][x] : c.ck->gs[1][x])};
    const int rrows = tiled ? c.rk->rows_t[ti] : c.rk->rows;
    const int rnt = prow ? c.rk->nt_tp[ti] : (tiled ? c.rk->nt_t[ti] : c.rk->nt);
    const int rsm = prow ? c.rk->smem_tp[ti] : (tiled ? c.rk->smem_t[ti] : c.rk->smem);
    const int cnt = pcol ? c.ck->tiled[ti].nt_p : (tiled ? c.ck->tiled[ti].nt : c.ck->nt);
    const int csm = pcol ? c.ck->tiled[ti].smem_gs_p : (tiled ? c.ck->tiled[ti].smem_gs : c.ck->smem_gs);
    if (prow) a.tw_row = p->tw_alt.at(c.W);
    if (pcol) a.tw_col = p->tw_alt.at(c.H);
    // square items on 2-column strips: the row pass instance with the strip height at compile time
    if (tiled && width == 2 && x == 0 && c.H == c.W && c.rk->gs_sq[prow ? 1 : 0][0] != nullptr) {
      k_row[0] = c.rk->gs_sq[prow ? 1 : 0][0];
      k_row[1] = c.rk->gs_sq[prow ? 1 : 0][1];
    }
    const dim3 grow((c.H + rrows - 1) / rrows, nb), gcol(strips, nb);
    // prologue (writes h_0 out when there is no iteration)
    hg::PassArgs a0 = a;
    if (n_iter == 0)
      for (int k = 0; k < nb; ++k) {
        const int item = c.items[c0 + k];
        a0.phase_out[k] = phase_out ? phase_out[item] : nullptr;
        a0.level_out[k] = level_out ? level_out[item] : nullptr;
      }
    if ((s = launch(p, K_ROW_INIT, k_init, grow, rnt, rsm, a0, st)) != HG_OK) return s;
    hg::PassArgs ao = a;
    for (int k = 0; k < nb; ++k) {
      const int item = c.items[c0 + k];
      ao.phase_out[k] = phase_out ? phase_out[item] : nullptr;
      ao.level_out[k] = level_out ? level_out[item] : nullptr;
    }
    for (int it = 0; it < n_iter; ++it) {
      a.iter = it;
      if ((s = launch(p, K_COL_GS, k_col[1], gcol, cnt, csm, a, st)) != HG_OK) return s;
      const bool last = it == n_iter - 1;
      hg::PassArgs ar = last ? ao : a;
      ar.finalize = nmse_out != nullptr;  // the row pass first adds up this column pass's NMSE
      ar.fin_iter = it;
      if ((s = launch(p, K_ROW_GS, k_row[last], grow, rnt, rsm, ar, st)) != HG_OK) return s;
    }
    a.iter = n_iter;
    a.fin_iter = n_iter;
    if ((s = launch(p, K_COL_NMSE, k_col[0], gcol, cnt, csm, a, st)) != HG_OK) return s;
    if (nmse_out && (s = launch(p, K_FINALIZE, (const void*)&hg::k_finalize<0>, dim3(1, nb), 32, 0, a, st)) != HG_OK)
      return s;
  }
  return HG_OK;
}

// Every size class of a GS run, smallest holograms first (shortest job first: batched launches keep
// the GPU full either way, and small holograms then finish early), each followed by a %globaltimer
// stamp for the per-hologram latency.
hg_status gs_enqueue(hg_plan* p, const GsCall& g, cudaStream_t st) {
  hg_status s;
  k_stamp<<<1, 1, 0, st>>>(p->stamps);
  for (size_t i : p->class_order) {
    if ((s = gs_class(p, p->classes[i], g, st)) != HG_OK) return s;
    k_stamp<<<1, 1, 0, st>>>(p->stamps + 1 + i);
  }
  return HG_OK;
}

// Runs enqueue(stream) directly, or -- in graph mode -- replays the CUDA graph captured for this
// argument key (capturing it first when the key is new).  Capture happens on the plan's own stream
// (the caller's may be the legacy default stream, which cannot be captured); capturing executes
// nothing, and the graph is launched on the caller's stream.
hg_status run_maybe_graph(hg_plan* p, const std::vector<uintptr_t>& key,
                          const std::function<hg_status(cudaStream_t)>& enqueue, cudaStream_t st) {
  if (!p->graph) return enqueue(st);
  hg_plan::GraphSlot& g = p->gslot[p->timing ? 1 : 0];
  if (!g.exec || key != g.key) {
    if (g.exec) {
      HG_CUDA(cudaDeviceSynchronize(), "device error");
      p->fold();
      p->drop_graph(g);
    }
    const int64_t launches0 = p->launches;
    const size_t pending0 = p->pending.size();
    if (!p->cap) HG_CUDA(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking), "capture stream");
    HG_CUDA(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal), "graph capture");
    p->capturing = true;
    const hg_status s = enqueue(p->cap);
    p->capturing = false;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(p->cap, &graph);
    g.kernels = p->launches - launches0;
    p->launches = launches0;
    // timing events recorded during the capture are nodes of this graph: they belong to the slot
    g.events.assign(p->pending.begin() + pending0, p->pending.end());
    p->pending.resize(pending0);
    if (s != HG_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      p->drop_graph(g);
      return s != HG_OK ? s : cuda_fail(e, "graph capture");
    }
    const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      g.exec = nullptr;
      p->drop_graph(g);
      return cuda_fail(ei, "graph instantiate");
    }
    g.key = key;
  }
  // a timed graph's events are overwritten by every replay: the totals take the latest one
  HG_CUDA(cudaGraphLaunch(g.exec, st), "graph launch");
  p->launches += g.kernels;
  g.replayed = !g.events.empty();
  return HG_OK;
}

// MRAF and HIO: GS with a signal region (the rest of the replay plane is the noise region).
// Direct binary search for every size class: per chunk of items the start h_0 and its replay
// R_0 = F(h_0 c) (the GS prologue's row pass, then forward column FFTs in place, unnormalised),
// then one cluster launch that runs every sweep.
hg_status dbs_enqueue(hg_plan* p, const float* const* target_amp, const float* const* init_phase, uint64_t seed,
                      int32_t n_sweeps, bool anneal, double t0, double alpha, float* const* phase_out,
                      uint8_t* const* level_out, float* nmse_out, cudaStream_t st) {
  hg_status s;
  for (size_t ci : p->class_order) {
    const SizeClass& c = p->classes[ci];
    const int cl = (c.H * c.W + hg::kDbsPixelsPerCta - 1) / hg::kDbsPixelsPerCta;
    const int chunk = std::min(hg::kMaxBatch, hg::kDbsMaxBatch);
    for (size_t c0 = 0; c0 < c.items.size(); c0 += chunk) {
      const int nb = (int)std::min<size_t>(chunk, c.items.size() - c0);
      hg::PassArgs a{};
      fill_common(p, c, 0, a);
      a.n_items = nb;
      a.seed = seed;
      a.scale = 1.f;
      hg::DbsArgs d{};
      d.H = c.H;
      d.W = c.W;
      d.n_sweeps = n_sweeps;
      d.nmse_stride = n_sweeps + 1;
      d.seed = seed;
      d.wy = p->roots.at(c.H);
      d.wx = p->roots.at(c.W);
      d.cx = a.cx;
      d.cy = a.cy;
      d.centred = p->centred ? 1 : 0;
      d.anneal = anneal ? 1 : 0;
      d.t0 = t0;
      d.alpha = alpha;
      d.nmse = nmse_out;
      for (int k = 0; k < nb; ++k) {
        const int item = c.items[c0 + k];
        a.item_index[k] = item;
        a.class_slot[k] = (int)(c0 + k);
        a.phase_in[k] = init_phase ? init_phase[item] : nullptr;
        a.out[k] = c.field + (c0 + k) * (size_t)c.H * c.W;
        d.field[k] = a.out[k];
        d.target[k] = target_amp[item];
        d.phase_in[k] = a.phase_in[k];
        d.phase_out[k] = phase_out ? phase_out[item] : nullptr;
        d.level_out[k] = level_out ? level_out[item] : nullptr;
        d.item_index[k] = item;
      }
      if ((s = launch(p, K_ROW_INIT, c.rk->init[0], dim3(c.row_blocks(), nb), c.rk->nt, c.rk->smem, a, st)) != HG_OK)
        return s;
      if ((s = launch(p, K_COL_FFT, c.ck->fft[0][0], dim3(c.col_blocks(), nb), c.ck->nt, c.ck->smem, a, st)) !=
          HG_OK)
        return s;
      // the search itself: one cluster of cl CTAs per item
      cudaEvent_t ea = nullptr, eb = nullptr;
      if (p->timing) {
        ea = p->get_event();
        eb = p->get_event();
        if (ea && eb) cudaEventRecordWithFlags(ea, st, p->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
      }
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(cl, nb);
      cfg.blockDim = dim3(hg::kDbsThreads);
      cfg.dynamicSmemBytes = (size_t)hg::dbs_smem(c.H, c.W);
      cfg.stream = st;
      cudaLaunchAttribute attr{};
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = (unsigned)cl;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      void* args[] = {(void*)&d};
      const cudaError_t e = cudaLaunchKernelExC(&cfg, hg::dbs_kernel(), args);
      if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
      p->launches++;
      if (ea && eb) {
        cudaEventRecordWithFlags(eb, st, p->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
        p->pending.push_back({ea, eb, K_DBS});
      } else {
        if (ea) p->event_pool.push_back(ea);
        if (eb) p->event_pool.push_back(eb);
      }
    }
  }
  return HG_OK;
}

hg_status region_run(hg_plan* p, const char* name, const float* const* target_amp,
                     const uint8_t* const* signal_mask, float mix, bool hio, float beta,
                     const float* const* init_phase, uint64_t seed, int32_t n_iter, float* const* phase_out,
                     uint8_t* const* level_out, float* nmse_out, void* stream) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  if (p->P != 1) return fail(HG_ERR_INVALID_ARG, "%s needs a single-plane plan", name);
  if (!p->illum.empty()) return fail(HG_ERR_INVALID_ARG, "%s does not take an illumination profile", name);
  if (n_iter < 0 || n_iter > 1000000) return fail(HG_ERR_INVALID_ARG, "n_iter must be 0..1000000");
  if (!target_amp) return fail(HG_ERR_INVALID_ARG, "target_amp is NULL");
  if (level_out && p->levels == 0) {
    for (int i = 0; i < p->n_items; ++i)
      if (level_out[i]) return fail(HG_ERR_INVALID_ARG, "level_out needs a quantised plan");
  }
  DeviceGuard g(p->device);
  if (!g.ok) return fail(HG_ERR_CUDA, "cannot select device %d", p->device);
  hg_status s;
  for (int i = 0; i < p->n_items; ++i) {
    const size_t px = (size_t)p->H[i] * p->W[i];
    if ((s = check_ptr(p, target_amp[i], px * 4, 4, "target_amp", i)) != HG_OK) return s;
    if (signal_mask && signal_mask[i] && (s = check_ptr(p, signal_mask[i], px, 1, "signal_mask", i)) != HG_OK)
      return s;
    if (init_phase && init_phase[i] && (s = check_ptr(p, init_phase[i], px * 4, 4, "init_phase", i)) != HG_OK)
      return s;
    if (phase_out && phase_out[i] && (s = check_ptr(p, phase_out[i], px * 4, 4, "phase_out", i)) != HG_OK) return s;
    if (level_out && level_out[i] && (s = check_ptr(p, level_out[i], px, 1, "level_out", i)) != HG_OK) return s;
  }
  if (nmse_out && (s = check_ptr(p, nmse_out, (size_t)p->n_items * (n_iter + 1) * 4, 4, "nmse_out", 0)) != HG_OK)
    return s;
  if (hio)
    for (SizeClass& c : p->classes)  // sized for any strip width, like the target tiles
      if (!c.hio && (s = p->alloc(&c.hio, c.items.size() * c.max_strip_cols() * c.H, "HIO input buffer")) != HG_OK)
        return s;
  GsCall call{target_amp, init_phase, seed, n_iter, phase_out, level_out, nmse_out};
  call.mask = signal_mask;
  call.mix = mix;
  call.hio = hio;
  call.beta = beta;
  uint32_t bits[2];
  std::memcpy(&bits[0], &mix, sizeof mix);
  std::memcpy(&bits[1], &beta, sizeof beta);
  std::vector<uintptr_t> key{(uintptr_t)(hio ? 4 : 3), (uintptr_t)n_iter, (uintptr_t)seed, (uintptr_t)nmse_out,
                             (uintptr_t)bits[0], (uintptr_t)bits[1]};
  if (p->graph)
    for (int i = 0; i < p->n_items; ++i) {
      key.push_back((uintptr_t)target_amp[i]);
      key.push_back((uintptr_t)(signal_mask ? signal_mask[i] : nullptr));
      key.push_back((uintptr_t)(init_phase ? init_phase[i] : nullptr));
      key.push_back((uintptr_t)(phase_out ? phase_out[i] : nullptr));
      key.push_back((uintptr_t)(level_out ? level_out[i] : nullptr));
    }
  return run_maybe_graph(p, key, [&](cudaStream_t q) { return gs_enqueue(p, call, q); }, (cudaStream_t)stream);
}

hg_status search_run(hg_plan* p, const char* name, const float* const* target_amp, const float* const* init_phase,
                     uint64_t seed, int32_t n_sweeps, bool anneal, double t0, double alpha,
                     float* const* phase_out, uint8_t* const* level_out, float* nmse_out, void* stream);

}  // namespace

extern "C" {

hg_status hg_gs_run(hg_plan* p, const float* const* target_amp, const float* const* init_phase, uint64_t seed,
                    int32_t n_iter, float* const* phase_out, uint8_t* const* level_out, float* nmse_out,
                    void* stream) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  if (n_iter < 0 || n_iter > 1000000) return fail(HG_ERR_INVALID_ARG, "n_iter must be 0..1000000");
  if (!target_amp) return fail(HG_ERR_INVALID_ARG, "target_amp is NULL");
  if (level_out && p->levels == 0) {
    for (int i = 0; i < p->n_items; ++i)
      if (level_out[i]) return fail(HG_ERR_INVALID_ARG, "level_out needs a quantised plan");
  }
  DeviceGuard g(p->device);
  if (!g.ok) return fail(HG_ERR_CUDA, "cannot select device %d", p->device);
  hg_status s;
  for (int i = 0; i < p->n_items; ++i) {
    const size_t px = (size_t)p->H[i] * p->W[i];
    for (int q = 0; q < p->P; ++q)
      if ((s = check_ptr(p, target_amp[i * p->P + q], px * 4, 4, "target_amp", i * p->P + q)) != HG_OK) return s;
    if (init_phase && init_phase[i] && (s = check_ptr(p, init_phase[i], px * 4, 4, "init_phase", i)) != HG_OK)
      return s;
    if (phase_out && phase_out[i] && (s = check_ptr(p, phase_out[i], px * 4, 4, "phase_out", i)) != HG_OK) return s;
    if (level_out && level_out[i] && (s = check_ptr(p, level_out[i], px, 1, "level_out", i)) != HG_OK) return s;
  }
  if (nmse_out && (s = check_ptr(p, nmse_out, (size_t)p->n_items * (n_iter + 1) * 4, 4, "nmse_out", 0)) != HG_OK)
    return s;

  if (p->P > 1)
    for (SizeClass& c : p->classes)
      if ((s = ensure_plane_acc(p, c)) != HG_OK) return s;
  const GsCall call{target_amp, init_phase, seed, n_iter, phase_out, level_out, nmse_out};
  std::vector<uintptr_t> key{1, (uintptr_t)n_iter, (uintptr_t)seed, (uintptr_t)nmse_out};
  if (p->graph)
    for (int i = 0; i < p->n_items; ++i) {
      key.push_back((uintptr_t)(p->illum.empty() ? nullptr : p->illum[i]));
      for (int q = 0; q < p->P; ++q) key.push_back((uintptr_t)target_amp[i * p->P + q]);
      key.push_back((uintptr_t)(init_phase ? init_phase[i] : nullptr));
      key.push_back((uintptr_t)(phase_out ? phase_out[i] : nullptr));
      key.push_back((uintptr_t)(level_out ? level_out[i] : nullptr));
    }
  return run_maybe_graph(p, key, [&](cudaStream_t q) { return gs_enqueue(p, call, q); }, (cudaStream_t)stream);
}

hg_status hg_plan_set_illumination(hg_plan* p, const float* const* illum_amp) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  if (!illum_amp) {
    p->illum.clear();
    return HG_OK;
  }
  if (p->P != 1) return fail(HG_ERR_INVALID_ARG, "an illumination profile needs a single-plane plan");
  if (p->levels < 0) return fail(HG_ERR_INVALID_ARG, "an illumination profile needs a phase-only SLM");
  DeviceGuard g(p->device);
  if (!g.ok) return fail(HG_ERR_CUDA, "cannot select device %d", p->device);
  hg_status s;
  for (int i = 0; i < p->n_items; ++i)
    if (illum_amp[i] &&
        (s = check_ptr(p, illum_amp[i], (size_t)p->H[i] * p->W[i] * 4, 4, "illum_amp", i)) != HG_OK)
      return s;
  p->illum.assign(illum_amp, illum_amp + p->n_items);
  return HG_OK;
}

hg_status hg_plan_set_slm_levels(hg_plan* p, const float* levels, int32_t n_levels) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  if (!levels || n_levels == 0) {
    p->levels = p->levels0;
    p->lev = p->lev0;
    p->lev_phase = p->lev_phase0;
    for (auto& slot : p->gslot) p->drop_graph(slot);
    return HG_OK;
  }
  if (p->P != 1) return fail(HG_ERR_INVALID_ARG, "a multi-amplitude SLM needs a single-plane plan");
  if (!p->illum.empty()) return fail(HG_ERR_INVALID_ARG, "a multi-amplitude SLM does not take an illumination profile");
  if (n_levels < 2 || n_levels > kMaxLevels)
    return fail(HG_ERR_INVALID_ARG, "n_levels must be 2..%d", kMaxLevels);
  std::vector<float2> lev(n_levels);
  std::vector<float> ph(n_levels);
  const double two_pi = 6.283185307179586476925286766559;
  for (int q = 0; q < n_levels; ++q) {
    const float re = levels[2 * q], im = levels[2 * q + 1];
    if (!std::isfinite(re) || !std::isfinite(im)) return fail(HG_ERR_INVALID_ARG, "level %d is not finite", q);
    lev[q] = make_float2(re, im);
    double a = std::atan2((double)im, (double)re);
    if (a < 0.0) a += two_pi;
    if (a >= two_pi) a = 0.0;
    ph[q] = (float)a;
  }
  DeviceGuard g(p->device);
  if (!g.ok) return fail(HG_ERR_CUDA, "cannot select device %d", p->device);
  HG_CUDA(cudaDeviceSynchronize(), "device error");
  float2* dl = nullptr;
  float* dp = nullptr;
  hg_status s;
  if ((s = upload(p, &dl, lev, "SLM level table")) != HG_OK) return s;
  if ((s = upload(p, &dp, ph, "SLM level table")) != HG_OK) return s;
  p->levels = -n_levels;
  p->lev = dl;
  p->lev_phase = dp;
  for (auto& slot : p->gslot) p->drop_graph(slot);
  return HG_OK;
}

hg_status hg_mraf_run(hg_plan* p, const float* const* target_amp, const uint8_t* const* signal_mask, float mix,
                      const float* const* init_phase, uint64_t seed, int32_t n_iter, float* const* phase_out,
                      uint8_t* const* level_out, float* nmse_out, void* stream) {
  if (!(mix > 0.f && mix <= 1.f)) return fail(HG_ERR_INVALID_ARG, "mix must be in (0, 1]");
  return region_run(p, "MRAF", target_amp, signal_mask, mix, false, 0.f, init_phase, seed, n_iter, phase_out,
                    level_out, nmse_out, stream);
}

hg_status hg_dbs_run(hg_plan* p, const float* const* target_amp, const float* const* init_phase, uint64_t seed,
                     int32_t n_sweeps, float* const* phase_out, uint8_t* const* level_out, float* nmse_out,
                     void* stream) {
  return search_run(p, "DBS", target_amp, init_phase, seed, n_sweeps, false, 0.0, 1.0, phase_out, level_out,
                    nmse_out, stream);
}

hg_status hg_sa_run(hg_plan* p, const float* const* target_amp, const float* const* init_phase, uint64_t seed,
                    int32_t n_sweeps, double t0, double alpha, float* const* phase_out, uint8_t* const* level_out,
                    float* nmse_out, void* stream) {
  if (!(t0 > 0.0) || !std::isfinite(t0)) return fail(HG_ERR_INVALID_ARG, "t0 must be finite and > 0");
  if (!(alpha > 0.0 && alpha <= 1.0)) return fail(HG_ERR_INVALID_ARG, "alpha must be in (0, 1]");
  return search_run(p, "SA", target_amp, init_phase, seed, n_sweeps, true, t0, alpha, phase_out, level_out,
                    nmse_out, stream);
}

}  // extern "C"

namespace {

// Direct binary search and simulated annealing: checks, tables, then the search launches.
hg_status search_run(hg_plan* p, const char* name, const float* const* target_amp, const float* const* init_phase,
                     uint64_t seed, int32_t n_sweeps, bool anneal, double t0, double alpha,
                     float* const* phase_out, uint8_t* const* level_out, float* nmse_out, void* stream) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  if (p->P != 1) return fail(HG_ERR_INVALID_ARG, "%s needs a single-plane plan", name);
  if (p->levels != 2) return fail(HG_ERR_INVALID_ARG, "%s needs a binary plan (quant_levels 2)", name);
  if (!p->illum.empty()) return fail(HG_ERR_INVALID_ARG, "%s does not take an illumination profile", name);
  if (n_sweeps < 0 || n_sweeps > 10000) return fail(HG_ERR_INVALID_ARG, "n_sweeps must be 0..10000");
  if (!target_amp) return fail(HG_ERR_INVALID_ARG, "target_amp is NULL");
  for (int i = 0; i < p->n_items; ++i)
    if ((int64_t)p->H[i] * p->W[i] > (int64_t)hg::kDbsMaxCluster * hg::kDbsPixelsPerCta)
      return fail(HG_ERR_UNSUPPORTED_SIZE, "item %d: %s takes at most %d pixels", i, name,
                  hg::kDbsMaxCluster * hg::kDbsPixelsPerCta);
  DeviceGuard g(p->device);
  if (!g.ok) return fail(HG_ERR_CUDA, "cannot select device %d", p->device);
  hg_status s;
  for (int i = 0; i < p->n_items; ++i) {
    const size_t px = (size_t)p->H[i] * p->W[i];
    if ((s = check_ptr(p, target_amp[i], px * 4, 4, "target_amp", i)) != HG_OK) return s;
    if (init_phase && init_phase[i] && (s = check_ptr(p, init_phase[i], px * 4, 4, "init_phase", i)) != HG_OK)
      return s;
    if (phase_out && phase_out[i] && (s = check_ptr(p, phase_out[i], px * 4, 4, "phase_out", i)) != HG_OK) return s;
    if (level_out && level_out[i] && (s = check_ptr(p, level_out[i], px, 1, "level_out", i)) != HG_OK) return s;
  }
  if (nmse_out && (s = check_ptr(p, nmse_out, (size_t)p->n_items * (n_sweeps + 1) * 4, 4, "nmse_out", 0)) != HG_OK)
    return s;
  hg::dbs_set_attrs();
  for (const SizeClass& c : p->classes) {
    for (int len : {c.H, c.W}) {
      if (p->roots.count(len)) continue;
      std::vector<float2> r(len);
      const double two_pi = 6.283185307179586476925286766559;
      for (int j = 0; j < len; ++j)
        r[j] = make_float2((float)std::cos(two_pi * j / len), (float)-std::sin(two_pi * j / len));
      float2* dptr = nullptr;
      if ((s = upload(p, &dptr, r, "DBS root table")) != HG_OK) return s;
      p->roots[len] = dptr;
    }
    // the class's cluster must fit on the device
    const int cl = (c.H * c.W + hg::kDbsPixelsPerCta - 1) / hg::kDbsPixelsPerCta;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(cl, 1);
    cfg.blockDim = dim3(hg::kDbsThreads);
    cfg.dynamicSmemBytes = (size_t)hg::dbs_smem(c.H, c.W);
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = (unsigned)cl;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, hg::dbs_kernel(), &cfg) != cudaSuccess || n < 1) {
      cudaGetLastError();
      return fail(HG_ERR_UNSUPPORTED_SIZE, "%dx%d: the device cannot run a DBS cluster of %d CTAs", c.H, c.W, cl);
    }
  }
  uint64_t tb[2];
  std::memcpy(&tb[0], &t0, sizeof t0);
  std::memcpy(&tb[1], &alpha, sizeof alpha);
  std::vector<uintptr_t> key{(uintptr_t)(anneal ? 6 : 5), (uintptr_t)n_sweeps, (uintptr_t)seed, (uintptr_t)nmse_out,
                             (uintptr_t)tb[0], (uintptr_t)tb[1]};
  if (p->graph)
    for (int i = 0; i < p->n_items; ++i) {
      key.push_back((uintptr_t)target_amp[i]);
      key.push_back((uintptr_t)(init_phase ? init_phase[i] : nullptr));
      key.push_back((uintptr_t)(phase_out ? phase_out[i] : nullptr));
      key.push_back((uintptr_t)(level_out ? level_out[i] : nullptr));
    }
  return run_maybe_graph(
      p, key,
      [&](cudaStream_t q) {
        return dbs_enqueue(p, target_amp, init_phase, seed, n_sweeps, anneal, t0, alpha, phase_out, level_out,
                           nmse_out, q);
      },
      (cudaStream_t)stream);
}

}  // namespace

extern "C" {

hg_status hg_hio_run(hg_plan* p, const float* const* target_amp, const uint8_t* const* signal_mask, float beta,
                     const float* const* init_phase, uint64_t seed, int32_t n_iter, float* const* phase_out,
                     uint8_t* const* level_out, float* nmse_out, void* stream) {
  if (!(beta > 0.f && beta <= 2.f)) return fail(HG_ERR_INVALID_ARG, "beta must be in (0, 2]");
  return region_run(p, "HIO", target_amp, signal_mask, 1.f, true, beta, init_phase, seed, n_iter, phase_out,
                    level_out, nmse_out, stream);
}

// ---------------------------------------------------------------- autotuner
//
// For every size class of a single-plane plan, times a short GS run (10 iterations, seeded start, a
// zero target in plan-owned scratch: the kernels' work does not depend on the values; the fastest of
// five runs) with each strip width the class allows -- 2 / 4 / 8 / 16 columns on the tiled field,
// the whole-run cluster kernel, or the row-major field -- and, on a tiled field, each radix plan of
// the row and column passes, and keeps the fastest.  Choices are cached per process by (device, H,
// W, items in the class, quantisation, propagation), so plans of the same shape reuse them.

namespace {
std::mutex g_tune_mu;
std::map<std::vector<int64_t>, std::array<int, 3>> g_tune_cache;  // (width, row plan, column plan)
}  // namespace

static hg_status autotune_class(hg_plan* p, SizeClass& c, cudaStream_t st) {
  // candidates (width, row plan, column plan): the cluster kernel and the row-major field take the
  // default plans; a tiled width also takes the alternative plan of either pass where compiled
  struct Cand {
    int w, pr, pc;
  };
  std::vector<Cand> cand;
  if (c.tileable(-1, p->P)) cand.push_back({-1, 0, 0});  // whole run in one cluster per item
  for (int w : {2, 4, 8, 16})
    if (c.tileable(w, p->P)) {
      const int ti = tile_index(w);
      // (the multi-plane kernels have the default plans only)
      const bool ar = p->P == 1 && c.rk->init_tp[ti] != nullptr, ac = p->P == 1 && c.ck->tiled[ti].gs_p[0] != nullptr;
      for (int pr = 0; pr <= (ar ? 1 : 0); ++pr)
        for (int pc = 0; pc <= (ac ? 1 : 0); ++pc) cand.push_back({w, pr, pc});
    }
  cand.push_back({0, 0, 0});  // row-major field
  if (cand.size() == 1) {
    c.tile = 0;
    c.pv_row = c.pv_col = 0;
    return HG_OK;
  }
  const std::vector<int64_t> key{p->device, c.H, c.W, (int64_t)c.items.size(), p->levels, p->propagation};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      c.tile = it->second[0];
      c.pv_row = it->second[1];
      c.pv_col = it->second[2];
      return HG_OK;
    }
  }
  float* zero = nullptr;
  HG_CUDA(cudaMalloc(&zero, (size_t)c.H * c.W * sizeof(float)), "autotune scratch");
  struct Free {
    float* q;
    ~Free() { cudaFree(q); }
  } guard{zero};
  HG_CUDA(cudaMemsetAsync(zero, 0, (size_t)c.H * c.W * sizeof(float), st), "memset");
  std::vector<const float*> targets(p->n_items * p->P, zero);
  const GsCall call{targets.data(), nullptr, 1, 10, nullptr, nullptr, nullptr};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HG_CUDA(cudaEventCreate(&e0), "event");
  HG_CUDA(cudaEventCreate(&e1), "event");
  float best_ms = 0.f;
  Cand best = cand[0];
  hg_status s = HG_OK;
  for (const Cand& cd : cand) {
    c.tile = cd.w;
    c.pv_row = cd.pr;
    c.pv_col = cd.pc;
    if ((s = gs_class(p, c, call, st)) != HG_OK) break;  // warm-up
    // the fastest of five 10-iteration runs (one run of a small class takes tens of microseconds,
    // so single timings are noisy; the minimum is the steadiest estimate)
    float ms = 0.f;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < 5 && s == HG_OK && e == cudaSuccess; ++r) {
      cudaEventRecord(e0, st);
      s = gs_class(p, c, call, st);
      cudaEventRecord(e1, st);
      if (s != HG_OK) break;
      float one = 0.f;
      e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&one, e0, e1);
      if (r == 0 || one < ms) ms = one;
    }
    if (s != HG_OK) break;
    if (e != cudaSuccess) {
      s = cuda_fail(e, "autotune timing");
      break;
    }
    if (&cd == &cand[0] || ms < best_ms) {
      best_ms = ms;
      best = cd;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c.tile = best.w;
  c.pv_row = best.pr;
  c.pv_col = best.pc;
  if (s != HG_OK) return s;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = {best.w, best.pr, best.pc};
  return HG_OK;
}

hg_status hg_plan_autotune(hg_plan* p, void* stream) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  DeviceGuard g(p->device);
  if (!g.ok) return fail(HG_ERR_CUDA, "cannot select device %d", p->device);
  const cudaStream_t st = (cudaStream_t)stream;
  HG_CUDA(cudaStreamSynchronize(st), "device error");
  // the tuning runs are neither timed nor counted, and captured graphs are rebuilt afterwards
  const bool timing = p->timing;
  const int64_t launches = p->launches;
  p->timing = false;
  hg_status s = HG_OK;
  for (SizeClass& c : p->classes)
    if ((s = autotune_class(p, c, st)) != HG_OK) break;
  p->timing = timing;
  p->launches = launches;
  HG_CUDA(cudaStreamSynchronize(st), "device error");
  for (auto& slot : p->gslot) p->drop_graph(slot);
  return s;
}

hg_status hg_plan_set_strip_width(hg_plan* p, int32_t item, int32_t width) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  if (item < 0 || item >= p->n_items) return fail(HG_ERR_INVALID_ARG, "item %d out of range", item);
  SizeClass& c = p->classes[p->item_class[item]];
  if (width != 0 && !c.tileable(width, p->P))
    return fail(HG_ERR_INVALID_ARG, "strip width %d is not available for %dx%d%s", width, c.H, c.W,
                p->P != 1 ? " with several planes" : "");
  DeviceGuard g(p->device);
  if (!g.ok) return fail(HG_ERR_CUDA, "cannot select device %d", p->device);
  HG_CUDA(cudaDeviceSynchronize(), "device error");
  c.tile = width;
  for (auto& slot : p->gslot) p->drop_graph(slot);
  return HG_OK;
}

hg_status hg_plan_strip_width(const hg_plan* p, int32_t item, int32_t* width_out) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  if (item < 0 || item >= p->n_items) return fail(HG_ERR_INVALID_ARG, "item %d out of range", item);
  if (!width_out) return fail(HG_ERR_INVALID_ARG, "width_out is NULL");
  *width_out = p->classes[p->item_class[item]].tile;
  return HG_OK;
}

hg_status hg_plan_set_radix_plan(hg_plan* p, int32_t item, int32_t row_plan, int32_t col_plan) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  if (item < 0 || item >= p->n_items) return fail(HG_ERR_INVALID_ARG, "item %d out of range", item);
  SizeClass& c = p->classes[p->item_class[item]];
  if (row_plan != 0 && row_plan != 1) return fail(HG_ERR_INVALID_ARG, "row_plan must be 0 or 1");
  if (col_plan != 0 && col_plan != 1) return fail(HG_ERR_INVALID_ARG, "col_plan must be 0 or 1");
  if (row_plan == 1 && !c.rk->has_alt)
    return fail(HG_ERR_INVALID_ARG, "row length %d has no alternative radix plan", c.W);
  if (col_plan == 1 && !c.ck->has_alt)
    return fail(HG_ERR_INVALID_ARG, "column length %d has no alternative radix plan", c.H);
  DeviceGuard g(p->device);
  if (!g.ok) return fail(HG_ERR_CUDA, "cannot select device %d", p->device);
  HG_CUDA(cudaDeviceSynchronize(), "device error");
  c.pv_row = row_plan;
  c.pv_col = col_plan;
  for (auto& slot : p->gslot) p->drop_graph(slot);
  return HG_OK;
}

hg_status hg_plan_radix_plan(const hg_plan* p, int32_t item, int32_t* row_plan, int32_t* col_plan) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  if (item < 0 || item >= p->n_items) return fail(HG_ERR_INVALID_ARG, "item %d out of range", item);
  if (!row_plan || !col_plan) return fail(HG_ERR_INVALID_ARG, "output is NULL");
  const SizeClass& c = p->classes[p->item_class[item]];
  *row_plan = c.pv_row;
  *col_plan = c.pv_col;
  return HG_OK;
}

hg_status hg_ospr_run(hg_plan* p, const float* const* target_amp, int32_t n_subframes, int32_t n_iter,
                      uint64_t seed, uint32_t* const* bits_out, float* nmse_out, void* stream) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  if (n_subframes < 1 || n_subframes > 65535) return fail(HG_ERR_INVALID_ARG, "n_subframes must be 1..65535");
  if (n_iter < 0 || n_iter > 10000) return fail(HG_ERR_INVALID_ARG, "n_iter must be 0..10000");
  if (!target_amp) return fail(HG_ERR_INVALID_ARG, "target_amp is NULL");
  if (p->P != 1) return fail(HG_ERR_INVALID_ARG, "OSPR needs a single-plane plan");
  if (!p->illum.empty()) return fail(HG_ERR_INVALID_ARG, "OSPR does not take an illumination profile");
  DeviceGuard g(p->device);
  if (!g.ok) return fail(HG_ERR_CUDA, "cannot select device %d", p->device);
  hg_status s;
  for (int i = 0; i < p->n_items; ++i) {
    const size_t px = (size_t)p->H[i] * p->W[i];
    if ((s = check_ptr(p, target_amp[i], px * 4, 4, "target_amp", i)) != HG_OK) return s;
    const size_t words = (size_t)n_subframes * p->H[i] * ((p->W[i] + 31) / 32);
    if (bits_out && bits_out[i] && (s = check_ptr(p, bits_out[i], words * 4, 4, "bits_out", i)) != HG_OK) return s;
  }
  if (nmse_out && (s = check_ptr(p, nmse_out, (size_t)p->n_items * n_subframes * 4, 4, "nmse_out", 0)) != HG_OK)
    return s;
  for (SizeClass& c : p->classes)  // [slot][strip][H][C]
    if (!c.acc && (s = p->alloc(&c.acc, c.items.size() * (size_t)c.col_blocks() * c.H * c.ck->cols,
                                "OSPR intensity buffer")) != HG_OK)
      return s;

  std::vector<uintptr_t> key{2, (uintptr_t)n_subframes, (uintptr_t)n_iter, (uintptr_t)seed, (uintptr_t)nmse_out};
  if (p->graph)
    for (int i = 0; i < p->n_items; ++i) {
      key.push_back((uintptr_t)target_amp[i]);
      key.push_back((uintptr_t)(bits_out ? bits_out[i] : nullptr));
    }
  auto enqueue = [&](cudaStream_t st) -> hg_status {
    hg_status s;
    for (const SizeClass& c : p->classes) {
      for (size_t c0 = 0; c0 < c.items.size(); c0 += hg::kMaxBatch) {
        const int nb = (int)std::min<size_t>(hg::kMaxBatch, c.items.size() - c0);
        hg::PassArgs a{};
        fill_common(p, c, 0, a);
        a.n_levels = 2;
        a.n_items = nb;
        a.acc = c.acc;
        a.nmse_stride = n_subframes;
        a.seed = seed;
        for (int k = 0; k < nb; ++k) {
          const int item = c.items[c0 + k];
          a.item_index[k] = item;
          a.class_slot[k] = (int)(c0 + k);
          a.target[k] = target_amp[item];
          a.bits[k] = bits_out ? bits_out[item] : nullptr;
        }
        hg::PassArgs ag = a;  // binary GS refinements inside a subframe: no NMSE, no bits
        ag.nmse = nullptr;
        a.nmse = nmse_out;
        const dim3 grow(c.row_blocks(), nb), gcol(c.col_blocks(), nb);
        const int rs = c.rk->smem_ospr;
        // targets re-laid out per column strip (read by every column pass of the run)
        if ((s = launch(p, K_TILE_TARGET, (const void*)&k_tile_target, gcol, 256, 0, a, st, c.ck->cols, c.ttile)) !=
            HG_OK)
          return s;
        a.ttile = c.ttile;
        ag.ttile = c.ttile;
        a.iter = 0;
        if ((s = launch(p, K_COL_OSPR, c.ck->ospr[0], gcol, c.ck->nt, c.ck->smem_ospr, a, st)) != HG_OK) return s;
        for (int sf = 0; sf < n_subframes; ++sf) {
          a.iter = sf;
          hg::PassArgs ar = a;  // the first row pass of subframe sf adds up NMSE[sf - 1]
          ar.finalize = nmse_out != nullptr && sf > 0;
          ar.fin_iter = sf - 1;
          if ((s = launch(p, K_ROW_OSPR, c.rk->ospr[n_iter == 0], grow, c.rk->nt, rs, ar, st)) != HG_OK) return s;
          for (int it = 0; it < n_iter; ++it) {
            if ((s = launch(p, K_COL_GS, c.ck->gs[1][0], gcol, c.ck->nt, c.ck->smem_gs, ag, st)) != HG_OK) return s;
            if ((s = launch(p, K_ROW_OSPR, c.rk->ospr[it == n_iter - 1], grow, c.rk->nt, rs, a, st)) != HG_OK)
              return s;
          }
          a.iter = sf + 1;
          a.acc_read = sf > 0;
          const int variant = sf + 1 < n_subframes ? 1 : 2;
          if ((s = launch(p, K_COL_OSPR, c.ck->ospr[variant], gcol, c.ck->nt, c.ck->smem_ospr, a, st)) != HG_OK)
            return s;
        }
        a.fin_iter = n_subframes - 1;
        if (nmse_out && (s = launch(p, K_FINALIZE, (const void*)&hg::k_finalize<0>, dim3(1, nb), 32, 0, a, st)) != HG_OK)
          return s;
      }
    }
    return HG_OK;
  };
  return run_maybe_graph(p, key, enqueue, (cudaStream_t)stream);
}

// Shared driver of the gradient-descent calls.  FWD: forward row pass (h = e^{i phi}, per-plane row
// FFTs -> checkpoint fields) and forward column pass (loss statistics, loss_out).  BWD: backward
// column pass (adjoint fields) and backward row pass (gradient; Adam when adam).
static hg_status gd_run(hg_plan* p, float* const* phase, const float* const* target_int, float* const* adam_m,
                        float* const* adam_v, bool adam, int32_t step, float lr, float beta1, float beta2, float eps,
                        float* loss_out, float* const* grad_out, const float* grad_scale, bool fwd, bool bwd,
                        void* stream) {
  if (!p) return fail(HG_ERR_INVALID_ARG, "plan is NULL");
  if (!phase || !target_int) return fail(HG_ERR_INVALID_ARG, "phase / target_int is NULL");
  if (p->levels != 0) return fail(HG_ERR_INVALID_ARG, "gradient descent needs a continuous-phase plan");
  if (!p->illum.empty()) return fail(HG_ERR_INVALID_ARG, "gradient descent does not take an illumination profile");
  if (adam) {
    if (!adam_m || !adam_v) return fail(HG_ERR_INVALID_ARG, "adam_m / adam_v is NULL");
    if (step < 1) return fail(HG_ERR_INVALID_ARG, "step must be >= 1");
    if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
      return fail(HG_ERR_INVALID_ARG, "Adam needs lr > 0, 0 <= beta < 1, eps > 0");
  }
  DeviceGuard g(p->device);
  if (!g.ok) return fail(HG_ERR_CUDA, "cannot select device %d", p->device);
  hg_status s;
  const int P = p->P;
  for (int i = 0; i < p->n_items; ++i) {
    const size_t px = (size_t)p->H[i] * p->W[i];
    if ((s = check_ptr(p, phase[i], px * 4, 4, "phase", i)) != HG_OK) return s;
    for (int q = 0; q < P; ++q)
      if ((s = check_ptr(p, target_int[i * P + q], px * 4, 4, "target_int", i * P + q)) != HG_OK) return s;
    if (adam && ((s = check_ptr(p, adam_m[i], px * 4, 4, "adam_m", i)) != HG_OK ||
                 (s = check_ptr(p, adam_v[i], px * 4, 4, "adam_v", i)) != HG_OK))
      return s;
    if (grad_out && grad_out[i] && (s = check_ptr(p, grad_out[i], px * 4, 4, "grad_out", i)) != HG_OK) return s;
  }
  if (loss_out && (s = check_ptr(p, loss_out, (size_t)p->n_items * (P + 1) * 4, 4, "loss_out", 0)) != HG_OK) return s;
  if (grad_scale && (s = check_ptr(p, grad_scale, 4, 4, "grad_scale", 0)) != HG_OK) return s;
  for (SizeClass& c : p->classes)
    if ((s = ensure_plane_acc(p, c)) != HG_OK) return s;

  cudaStream_t st = (cudaStream_t)stream;
  const int chunk = chunk_items(p);
  for (const SizeClass& c : p->classes) {
    for (size_t c0 = 0; c0 < c.items.size(); c0 += chunk) {
      const int nb = (int)std::min<size_t>(chunk, c.items.size() - c0);
      hg::PassArgs a{};
      fill_common(p, c, 0, a);
      a.n_levels = 0;
      a.n_items = nb;
      a.loss = loss_out;
      a.grad_scale = grad_scale;
      a.adam = adam ? 1 : 0;
      if (adam) {
        a.lr = lr;
        a.beta1 = beta1;
        a.beta2 = beta2;
        a.eps = eps;
        a.bc1 = (float)(1.0 - std::pow((double)beta1, (double)step));
        a.bc2 = (float)(1.0 - std::pow((double)beta2, (double)step));
      }
      for (int k = 0; k < nb; ++k) {
        const int item = c.items[c0 + k];
        a.item_index[k] = item;
        a.class_slot[k] = (int)(c0 + k);
        for (int q = 0; q < P; ++q) a.target[k * P + q] = target_int[item * P + q];
        a.phi[k] = phase[item];
        a.adam_m[k] = adam ? adam_m[item] : nullptr;
        a.adam_v[k] = adam ? adam_v[item] : nullptr;
        a.grad[k] = grad_out ? grad_out[item] : nullptr;
      }
      const dim3 grow(c.row_blocks(), nb), gcol(c.col_blocks(), nb * P);
      const bool gen = c.rk->gen != nullptr;  // generic row length: one launch per plane
      // square items: the column passes with the row length at compile time
      const bool sq = c.H == c.W && c.ck->gd_sq[0] != nullptr;
      const void* kgd[2] = {sq ? c.ck->gd_sq[0] : c.ck->gd[0], sq ? c.ck->gd_sq[1] : c.ck->gd[1]};
      if (fwd) {
        if (gen) {
          if ((s = launch(p, K_ROW_GD_FWD, c.rk->plane.start[0], pointwise_grid(c, nb), 256, 0, a, st, 0,
                          (float*)c.gacc)) != HG_OK ||
              (s = plane_forwards(p, c, K_ROW_GD_FWD, a, grow, st)) != HG_OK)
            return s;
        } else if ((s = launch(p, K_ROW_GD_FWD, c.rk->mp_init[0], grow, c.rk->nt, c.rk->smem, a, st)) != HG_OK) {
          return s;
        }
        if ((s = launch(p, K_COL_GD_FWD, kgd[0], gcol, c.ck->nt, c.ck->smem, a, st)) != HG_OK) return s;
        if ((s = launch(p, K_FINALIZE, (const void*)&hg::k_finalize<1>, dim3(1, nb), 32, 0, a, st)) != HG_OK) return s;
      }
      if (bwd) {
        if ((s = launch(p, K_COL_GD_BWD, kgd[1], gcol, c.ck->nt, c.ck->smem, a, st)) != HG_OK) return s;
        if (gen) {
          if ((s = plane_backs(p, c, K_ROW_GD_BWD, a, grow, st)) != HG_OK ||
              (s = launch(p, K_ROW_GD_BWD, c.rk->plane.grad, pointwise_grid(c, nb), 256, 0, a, st, 0,
                          (float*)c.gacc)) != HG_OK)
            return s;
        } else if ((s = launch(p, K_ROW_GD_BWD, c.rk->gd_bwd, grow, c.rk->nt, c.rk->smem, a, st)) != HG_OK) {
          return s;
        }
      }
    }
  }
  return HG_OK;
}

hg_status hg_gd_step(hg_plan* p, float* const* phase, const float* const* target_int, float* const* adam_m,
                     float* const* adam_v, int32_t step, float lr, float beta1, float beta2, float eps, float* loss_out,
                     float* const* grad_out, void* stream) {
  return gd_run(p, phase, target_int, adam_m, adam_v, true, step, lr, beta1, beta2, eps, loss_out, grad_out,
                nullptr, true, true, stream);
}

hg_status hg_gd_forward(hg_plan* p, float* const* phase, const float* const* target_int, float* loss_out,
                        void* stream) {
  return gd_run(p, phase, target_int, nullptr, nullptr, false, 0, 0.f, 0.f, 0.f, 0.f, loss_out, nullptr, nullptr,
                true, false, stream);
}

hg_status hg_gd_backward(hg_plan* p, float* const* phase, const float* const* target_int, const float* grad_scale,
                         float* const* grad_out, void* stream) {
  if (!grad_out) return fail(HG_ERR_INVALID_ARG, "grad_out is NULL");
  return gd_run(p, phase, target_int, nullptr, nullptr, false, 0, 0.f, 0.f, 0.f, 0.f, nullptr, grad_out, grad_scale,
                false, true, stream);
}

}  // extern "C"
