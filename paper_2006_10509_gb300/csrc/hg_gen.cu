// Generic row- and column-pass kernels: every FFT length n = 2^a 3^b 5^c (1 <= n <= 4096) that has
// no compiled instance in hg_len.cu runs on these, so a plan takes any hologram size whose sides
// have no prime factor above 5 (the paper's FFT handler wraps cuFFT, which takes any size: section
// "Algorithm Libraries", FFTHandlerCuda; the hologram size is a user parameter).
//
// The compiled kernels keep the data in registers between stages and fuse the transform's first and
// last stages with global memory; here the length is a run-time value, so the tile (B sequences of
// length n: rows of the field, or the columns of a strip) stays resident in shared memory and each
// Stockham stage moves its butterflies' values through registers:
//   read the R inputs x[j + r n/R] of each butterfly the thread owns, barrier,
//   twiddle by w_{ns R}^{r (j mod ns)}, R-point DFT (the compiled kernels' butterflies, dispatched on
//   the stage's run-time radix), write the outputs to (j / ns) ns R + (j mod ns) + r ns, barrier.
// The pointwise steps run over the tile in shared memory between the transforms; they are those of
// the compiled kernels in hg_kernels.cuh (same projections, replacement, partial sums, Philox draws)
// on a row-major field.
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "hg_kernels.cuh"
#include "hg_launch.h"

namespace hg {

namespace gen {

constexpr int kVmax = 18;  // values a thread holds in one stage (radix R: kVmax / R butterflies)
// Row tiles hold at most 4096 values: at most 288 threads (4096 / 15, rounded up to warps).  Column
// strips (up to 15360 values) take up to 1024 threads.
constexpr int kRowThreads = 512;

// shared-memory slot of tile element i, padded by one float2 per 16
__device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded(int count) { return (count + (count >> 4) + 15) / 16 * 16; }

template <int R, bool INV>
__device__ __forceinline__ void stage(int N, int B, int ns, const float2* __restrict__ tw) {
  extern __shared__ __align__(16) float2 X[];  // the tile, at the start of dynamic shared memory
  constexpr int BPT = kVmax / R;
  // the butterfly indices below do not change between calls; inside the multi-plane kernels' plane
  // loops the compiler hoisted those of every stage out of the loop and spilled them (1-3 KB per
  // thread): an opaque copy of n keeps them here
  N = opaque(N);
  const int nb = N / R, total = B * nb;
  float2 v[BPT][R];
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int u = threadIdx.x + i * blockDim.x;
    if (u < total) {
      const int b = u / nb, j = u - b * nb;
      const int base = b * N + j;
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = X[pidx(base + r * nb)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < BPT; ++i) {
    const int u = threadIdx.x + i * blockDim.x;
    if (u < total) {
      const int b = u / nb, j = u - b * nb;
      const int k = j % ns;
      if (ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const float2 w = __ldg(tw + (r - 1) * ns + k);
          v[i][r] = INV ? c_mulc(v[i][r], w) : c_mul(v[i][r], w);
        }
      }
      dft<R, INV>(v[i]);
      const int base = b * N + (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) X[pidx(base + r * ns)] = v[i][r];
    }
  }
  __syncthreads();
}

// Unnormalised FFT of the B sequences of the tile at the start of dynamic shared memory (sequence b
// at elements [b n, (b + 1) n), slots pidx), in place, natural order.  The tile must be complete on
// entry (after a barrier); it is complete on return.  Each radix has a loop of its own, run from the
// plan's scalar stage counts in the planner's order, with ns and the twiddle-table offset carried
// along: a run-time switch over the radices inside one stage loop, or per-stage arrays read inside
// the multi-plane kernels' plane loops, made ptxas spill (1-3 KB per thread); these loops do not.
template <bool INV>
__device__ __forceinline__ void fft(const GenPlan& pl, int B, const float2* __restrict__ tw) {
  const int N = pl.n;
  int ns = 1, off = 0;
  auto run = [&](auto rc) {
    constexpr int R = decltype(rc)::value;
    stage<R, INV>(N, B, ns, tw + off);
    if (ns > 1) off += (R - 1) * ns;
    ns *= R;
  };
  for (int i = 0; i < pl.n16; ++i) run(std::integral_constant<int, 16>{});
  if (pl.r2 == 8)
    run(std::integral_constant<int, 8>{});
  else if (pl.r2 == 4)
    run(std::integral_constant<int, 4>{});
  else if (pl.r2 == 2)
    run(std::integral_constant<int, 2>{});
  for (int i = 0; i < pl.n9; ++i) run(std::integral_constant<int, 9>{});
  if (pl.n3) run(std::integral_constant<int, 3>{});
  for (int i = 0; i < pl.n5; ++i) run(std::integral_constant<int, 5>{});
}

// ---------------------------------------------------------------- row passes (row-major field)
//
// Tile element e (e < B W) is row row0 + e / W, column e % W; rows past H are zeros.

__device__ __forceinline__ void load_rows(float2* X, const float2* __restrict__ f, int row0, int B, int W, int H) {
  for (int e = threadIdx.x; e < B * W; e += blockDim.x) {
    const int row = row0 + e / W;
    X[pidx(e)] = row < H ? f[(size_t)row0 * W + e] : make_float2(0.f, 0.f);
  }
}

__device__ __forceinline__ void store_rows(const float2* X, float2* __restrict__ f, int row0, int B, int W, int H) {
  for (int e = threadIdx.x; e < B * W; e += blockDim.x)
    if (row0 + e / W < H) f[(size_t)row0 * W + e] = X[pidx(e)];
}

// The SLM pixel's starting value: exp(i phi0) (phi0 given) or the seeded draw.
__device__ __forceinline__ float2 start_value(const PassArgs& a, const float* ph, size_t p, int k) {
  if (ph) {
    float sn, cs;
    sincosf(__ldg(&ph[p]), &sn, &cs);
    return make_float2(cs, sn);
  }
  return init_unit((uint32_t)p, a.seed, a.item_index[k]);
}

// GS prologue: h0 = P_SLM(exp(i phi0)) (+ outputs when the run has no iteration), illumination,
// chirp, forward row FFTs -> field.
__global__ void __launch_bounds__(kRowThreads) kg_row_init(const __grid_constant__ PassArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  const GenPlan& pl = a.gen_row;
  const int W = a.W, H = a.H, B = pl.batch, k = blockIdx.y, row0 = blockIdx.x * B;
  float2* f = a.field + (size_t)a.class_slot[k] * H * W;
  const float* ph = a.phase_in[k];
  float* po = a.phase_out[k];
  uint8_t* lo = a.level_out[k];
  const float* il = a.illum[k];
  for (int e = threadIdx.x; e < B * W; e += blockDim.x) {
    const int row = row0 + e / W, n = e % W;
    float2 h = make_float2(0.f, 0.f);
    if (row < H) {
      const size_t p = (size_t)row * W + n;
      int q;
      h = slm_project_x<true>(start_value(a, ph, p, k), a.n_levels, a.lev, q);
      if (po) po[p] = a.n_levels ? __ldg(&a.lev_phase[q]) : phase_0_2pi(h);
      if (lo) lo[p] = (uint8_t)q;
      if (il) h = c_scale(h, __ldg(&il[p]));
      if (a.cx) h = c_mul(h, c_mul(__ldg(&a.cx[n]), __ldg(&a.cy[row])));
    }
    sm[pidx(e)] = h;
  }
  __syncthreads();
  fft<false>(pl, B, a.tw_row);
  store_rows(sm, f, row0, B, W, H);
}

// GS row pass: inverse row FFTs, conj chirp, SLM projection (outputs when OUT; a multi-amplitude
// table in the loop's unitary scale), illumination, chirp, forward row FFTs.
template <bool OUT>
__global__ void __launch_bounds__(kRowThreads) kg_row_gs(const __grid_constant__ PassArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  const GenPlan& pl = a.gen_row;
  const int W = a.W, H = a.H, B = pl.batch, k = blockIdx.y, row0 = blockIdx.x * B;
  pdl_wait_then_release();
  if (a.finalize && blockIdx.x == 0 && threadIdx.x < 32) finalize_nmse(a, k);
  float2* f = a.field + (size_t)a.class_slot[k] * H * W;
  load_rows(sm, f, row0, B, W, H);
  __syncthreads();
  fft<true>(pl, B, a.tw_row);
  float* po = OUT ? a.phase_out[k] : nullptr;
  uint8_t* lo = OUT ? a.level_out[k] : nullptr;
  const float* il = a.illum[k];
  const bool table = a.n_levels < 0;
  const float gscale = table ? (a.mix > 0.f ? 1.f / ((float)H * (float)W)
                                            : (float)__ldcg(&a.stats[(size_t)a.class_slot[k] * 4 + 3]))
                             : 1.f;
  for (int e = threadIdx.x; e < B * W; e += blockDim.x) {
    const int row = row0 + e / W, n = e % W;
    float2 h = make_float2(0.f, 0.f);
    if (row < H) {
      float2 g = sm[pidx(e)];
      float2 c = make_float2(1.f, 0.f);
      if (a.cx) {
        c = c_mul(__ldg(&a.cx[n]), __ldg(&a.cy[row]));
        g = c_mulc(g, c);
      }
      int q;
      h = table ? table_project(c_scale(g, gscale), -a.n_levels, a.lev, q) : slm_project(g, a.n_levels, a.lev, q);
      const size_t p = (size_t)row * W + n;
      if (po) po[p] = a.n_levels ? __ldg(&a.lev_phase[q]) : phase_0_2pi(h);
      if (lo) lo[p] = (uint8_t)q;
      if (il) h = c_scale(h, __ldg(&il[p]));
      if (a.cx) h = c_mul(h, c);
    }
    sm[pidx(e)] = h;
  }
  __syncthreads();
  fft<false>(pl, B, a.tw_row);
  store_rows(sm, f, row0, B, W, H);
}

// Bare row FFTs (propagation): in (times the chirp when PRE) -> FFT -> out.
template <bool INV, bool PRE>
__global__ void __launch_bounds__(kRowThreads) kg_row_fft(const __grid_constant__ PassArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  const GenPlan& pl = a.gen_row;
  const int W = a.W, H = a.H, B = pl.batch, k = blockIdx.y, row0 = blockIdx.x * B;
  const float2* src = a.in[k];
  for (int e = threadIdx.x; e < B * W; e += blockDim.x) {
    const int row = row0 + e / W, n = e % W;
    float2 x = make_float2(0.f, 0.f);
    if (row < H) {
      x = __ldg(&src[(size_t)row * W + n]);
      if (PRE) x = c_mul(x, c_mul(__ldg(&a.cx[n]), __ldg(&a.cy[row])));
    }
    sm[pidx(e)] = x;
  }
  __syncthreads();
  fft<INV>(pl, B, a.tw_row);
  store_rows(sm, a.out[k], row0, B, W, H);
}

// OSPR row pass: inverse row FFTs, conj chirp, binary projection (bits LSB-first when BITS),
// chirp, forward row FFTs.
template <bool BITS>
__global__ void __launch_bounds__(kRowThreads) kg_row_ospr(const __grid_constant__ PassArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  const GenPlan& pl = a.gen_row;
  const int W = a.W, H = a.H, B = pl.batch, k = blockIdx.y, row0 = blockIdx.x * B;
  const int words = (W + 31) / 32;
  unsigned char* qs = reinterpret_cast<unsigned char*>(sm + padded(B * W));  // [B][W] decisions
  float2* f = a.field + (size_t)a.class_slot[k] * H * W;
  uint32_t* bits = BITS ? a.bits[k] : nullptr;
  if (a.finalize && blockIdx.x == 0 && threadIdx.x < 32) finalize_nmse(a, k);
  load_rows(sm, f, row0, B, W, H);
  __syncthreads();
  fft<true>(pl, B, a.tw_row);
  for (int e = threadIdx.x; e < B * W; e += blockDim.x) {
    const int row = row0 + e / W, n = e % W;
    float2 g = sm[pidx(e)];
    float2 c = make_float2(1.f, 0.f);
    if (a.cx && row < H) {
      c = c_mul(__ldg(&a.cx[n]), __ldg(&a.cy[row]));
      g = c_mulc(g, c);
    }
    const int q = (g.x < 0.f || (g.x == 0.f && g.y > 0.f)) ? 1 : 0;
    if (BITS) qs[e] = (unsigned char)q;
    float2 h = make_float2(q ? -1.f : 1.f, 0.f);
    if (a.cx) h = c_mul(h, c);
    sm[pidx(e)] = row < H ? h : make_float2(0.f, 0.f);
  }
  __syncthreads();
  if (BITS && bits) {
    uint32_t* dst = bits + (size_t)a.iter * H * words;
    for (int w = threadIdx.x; w < B * words; w += blockDim.x) {
      const int b = w / words, word = w % words, row = row0 + b;
      if (row >= H) continue;
      uint32_t x = 0;
      for (int i = 0; i < 32; ++i) {
        const int n = word * 32 + i;
        if (n < W) x |= (uint32_t)qs[b * W + n] << i;
      }
      dst[(size_t)row * words + word] = x;
    }
  }
  fft<false>(pl, B, a.tw_row);
  store_rows(sm, f, row0, B, W, H);
}

// ---------------------------------------------------------------- multi-plane row passes
//
// Multi-plane GS and gradient descent sum the back-propagated fields of all planes before the
// projection.  Here each plane's row FFTs are a launch of their own and the sum goes through a
// plan-owned accumulator acc [slot][H][W] (a loop over the planes around the transform inside one
// kernel made ptxas spill 1-3 KB per thread, whatever the loop's form):
//   start      h_0 into acc (multi-plane GS: P_SLM(exp(i phi)), outputs when set; GD: exp(i phi))
//   plane_fwd  for plane p: acc c_p -> forward row FFTs -> field p
//   plane_back for plane p: conj(c_p) (inverse row FFTs of field p) -> acc (p = 0: written, else added)
//   project    acc -> P_SLM(acc) in place (outputs when set)          (multi-plane GS)
//   gd_grad    dL/dphi = 2 Im(acc conj(e^{i phi})) (times *grad_scale), gradient out, Adam (GD)
// The pointwise launches cover one item's field per blockIdx.y with a grid-stride loop.

// Start value of a multi-plane run into acc.  PROJECT (multi-plane GS): P_SLM(exp(i phi)), outputs
// when phase_out / level_out are set (the run has no iteration); else exp(i phi) (GD, phi from a.phi).
template <bool PROJECT>
__global__ void __launch_bounds__(256) kg_mp_start(const __grid_constant__ PassArgs a, int, float* accf) {
  const int k = blockIdx.y, W = a.W, H = a.H;
  float2* acc = reinterpret_cast<float2*>(accf) + (size_t)a.class_slot[k] * H * W;
  const float* ph = PROJECT ? a.phase_in[k] : a.phi[k];
  float* po = PROJECT ? a.phase_out[k] : nullptr;
  uint8_t* lo = PROJECT ? a.level_out[k] : nullptr;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < (size_t)H * W; p += (size_t)gridDim.x * blockDim.x) {
    float2 h = start_value(a, ph, p, k);
    if (PROJECT) {
      int q;
      h = slm_project(h, a.n_levels, a.lev, q);
      if (po) po[p] = a.n_levels ? __ldg(&a.lev_phase[q]) : phase_0_2pi(h);
      if (lo) lo[p] = (uint8_t)q;
    }
    acc[p] = h;
  }
}

// Plane p's forward row FFTs of acc c_p -> field p.
__global__ void __launch_bounds__(kRowThreads) kg_row_plane_fwd(const __grid_constant__ PassArgs a, int p, float* accf) {
  extern __shared__ __align__(16) float2 sm[];
  const GenPlan& pl = a.gen_row;
  const int W = a.W, H = a.H, B = pl.batch, k = blockIdx.y, row0 = blockIdx.x * B;
  const int P = a.n_planes > 1 ? a.n_planes : 1;
  const int slot = a.class_slot[k];
  const float2* acc = reinterpret_cast<const float2*>(accf) + (size_t)slot * H * W;
  const float2* cx = a.cxp[p];
  const float2* cy = a.cyp[p];
  for (int e = threadIdx.x; e < B * W; e += blockDim.x) {
    const int row = row0 + e / W, n = e % W;
    float2 h = make_float2(0.f, 0.f);
    if (row < H) {
      h = acc[(size_t)row0 * W + e];
      if (cx) h = c_mul(h, c_mul(__ldg(&cx[n]), __ldg(&cy[row])));
    }
    sm[pidx(e)] = h;
  }
  __syncthreads();
  fft<false>(pl, B, a.tw_row);
  store_rows(sm, a.field + ((size_t)slot * P + p) * H * W, row0, B, W, H);
}

// Plane p's inverse row FFTs, times conj(c_p), into acc (written for p = 0, else added).  The first
// plane's launch of a multi-plane GS row pass also finishes the preceding column pass's NMSE.
__global__ void __launch_bounds__(kRowThreads) kg_row_plane_back(const __grid_constant__ PassArgs a, int p, float* accf) {
  extern __shared__ __align__(16) float2 sm[];
  const GenPlan& pl = a.gen_row;
  const int W = a.W, H = a.H, B = pl.batch, k = blockIdx.y, row0 = blockIdx.x * B;
  const int P = a.n_planes > 1 ? a.n_planes : 1;
  const int slot = a.class_slot[k];
  if (p == 0 && a.finalize && blockIdx.x == 0 && threadIdx.x < 32) finalize_nmse(a, k);
  float2* acc = reinterpret_cast<float2*>(accf) + (size_t)slot * H * W;
  load_rows(sm, a.field + ((size_t)slot * P + p) * H * W, row0, B, W, H);
  __syncthreads();
  fft<true>(pl, B, a.tw_row);
  const float2* cx = a.cxp[p];
  const float2* cy = a.cyp[p];
  for (int e = threadIdx.x; e < B * W; e += blockDim.x) {
    const int row = row0 + e / W, n = e % W;
    if (row >= H) continue;
    float2 x = sm[pidx(e)];
    if (cx) x = c_mulc(x, c_mul(__ldg(&cx[n]), __ldg(&cy[row])));
    float2* d = acc + (size_t)row0 * W + e;
    *d = p == 0 ? x : c_add(*d, x);
  }
}

// Multi-plane GS: acc -> P_SLM(acc) in place; phase / levels out when set.
__global__ void __launch_bounds__(256) kg_mp_project(const __grid_constant__ PassArgs a, int, float* accf) {
  const int k = blockIdx.y, W = a.W, H = a.H;
  float2* acc = reinterpret_cast<float2*>(accf) + (size_t)a.class_slot[k] * H * W;
  float* po = a.phase_out[k];
  uint8_t* lo = a.level_out[k];
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < (size_t)H * W; p += (size_t)gridDim.x * blockDim.x) {
    int q;
    const float2 h = slm_project(acc[p], a.n_levels, a.lev, q);
    if (po) po[p] = a.n_levels ? __ldg(&a.lev_phase[q]) : phase_0_2pi(h);
    if (lo) lo[p] = (uint8_t)q;
    acc[p] = h;
  }
}

// Gradient descent: g = acc (the summed back-propagation of the adjoint fields),
// dL/dphi = 2 Im(g conj(e^{i phi})) (times *grad_scale), gradient out, Adam update of phi, m, v.
__global__ void __launch_bounds__(256) kg_gd_grad(const __grid_constant__ PassArgs a, int, float* accf) {
  const int k = blockIdx.y, W = a.W, H = a.H;
  const float2* acc = reinterpret_cast<const float2*>(accf) + (size_t)a.class_slot[k] * H * W;
  const float gs = a.grad_scale ? __ldg(a.grad_scale) : 1.f;
  float* phi = a.phi[k];
  float* gout = a.grad[k];
  float* m = a.adam_m[k];
  float* vv = a.adam_v[k];
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < (size_t)H * W; p += (size_t)gridDim.x * blockDim.x) {
    const float2 g = acc[p];
    const float p0 = phi[p];
    float sn, cs;
    sincosf(p0, &sn, &cs);
    const float gr = 2.f * gs * fmaf(g.y, cs, -g.x * sn);
    if (gout) gout[p] = gr;
    if (a.adam) {
      const float m1 = fmaf(a.beta1, m[p], (1.f - a.beta1) * gr);
      const float v1 = fmaf(a.beta2, vv[p], (1.f - a.beta2) * gr * gr);
      m[p] = m1;
      vv[p] = v1;
      phi[p] = p0 - a.lr * (m1 / a.bc1) / (sqrtf(v1 / a.bc2) + a.eps);
    }
  }
}

// ---------------------------------------------------------------- column passes (row-major field)
//
// A strip is C columns of the field, col0 = blockIdx.x C; sequence b (column col0 + b) sits at tile
// elements [b H, (b + 1) H).  Loops run over i < C H with b = i % C, n = i / C, so consecutive
// threads touch consecutive columns of a row in global memory; columns past W are zeros.

__device__ __forceinline__ void load_strip(float2* X, const float2* __restrict__ f, int col0, int C, int W, int H) {
  for (int i = threadIdx.x; i < C * H; i += blockDim.x) {
    const int b = i % C, n = i / C, col = col0 + b;
    X[pidx(b * H + n)] = col < W ? f[(size_t)n * W + col] : make_float2(0.f, 0.f);
  }
}

__device__ __forceinline__ void store_strip(const float2* X, float2* __restrict__ f, int col0, int C, int W, int H) {
  for (int i = threadIdx.x; i < C * H; i += blockDim.x) {
    const int b = i % C, n = i / C, col = col0 + b;
    if (col < W) f[(size_t)n * W + col] = X[pidx(b * H + n)];
  }
}

// GS column pass: forward column FFTs, NMSE partials of I = |R|^2 against T = A^2 and amplitude
// replacement (MRAF / HIO noise regions where the target copy holds -1; P planes: each plane's
// amplitude at a unit-modulus field's energy), inverse column FFTs (REPLACE).
template <bool REPLACE>
__global__ void __launch_bounds__(1024) kg_col_gs(const __grid_constant__ PassArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  const GenPlan& pl = a.gen_col;
  const int P = a.n_planes > 1 ? a.n_planes : 1;
  const int k = blockIdx.y / P, p = blockIdx.y % P;
  const int W = a.W, H = a.H, C = pl.batch, col0 = blockIdx.x * C;
  const int slot = a.class_slot[k];
  const size_t sp = (size_t)slot * P + p;
  pdl_wait_then_release();
  float2* f = a.field + sp * H * W;
  const float* A = a.target[k * P + p];
  const float* tt = a.ttile ? a.ttile + (sp * gridDim.x + blockIdx.x) * H * C : nullptr;
  load_strip(sm, f, col0, C, W, H);
  __syncthreads();
  fft<false>(pl, C, a.tw_col);
  const bool mraf = a.mix > 0.f;
  const float esc = (P > 1 || mraf) ? (float)__ldcg(&a.stats[sp * 4 + 3]) : 1.f;
  const float amp_scale = mraf ? a.mix * (float)H * (float)W * esc : esc;
  float2* hx = a.hio ? a.hio + (sp * gridDim.x + blockIdx.x) * H * C : nullptr;
  float s_it = 0.f, s_ii = 0.f, s_tt = 0.f;
  for (int i = threadIdx.x; i < C * H; i += blockDim.x) {
    const int b = i % C, n = i / C, col = col0 + b;
    const float2 r = sm[pidx(b * H + n)];
    const float amp = tt ? tt[n * C + b] : (col < W ? __ldg(&A[(size_t)n * W + col]) : 0.f);
    if (mraf && amp < 0.f) {  // noise region, outside the ROI NMSE
      if (REPLACE) {
        if (hx) {  // HIO: X' = X - beta Y, with X_0 = Y_0
          float2* xp = hx + n * C + b;
          const float2 x0 = a.iter == 0 ? r : __ldcg(xp);
          const float2 xn = make_float2(fmaf(-a.beta, r.x, x0.x), fmaf(-a.beta, r.y, x0.y));
          __stcg(xp, xn);
          sm[pidx(b * H + n)] = xn;
        } else {  // MRAF: R' = (1 - m) R
          sm[pidx(b * H + n)] = c_scale(r, 1.f - a.mix);
        }
      }
      continue;
    }
    const float i2 = fmaf(r.x, r.x, r.y * r.y);
    const float t2 = amp * amp;
    s_it = fmaf(i2, t2, s_it);
    s_ii = fmaf(i2, i2, s_ii);
    s_tt = fmaf(t2, t2, s_tt);
    if (REPLACE) {
      const float as = amp * amp_scale;
      sm[pidx(b * H + n)] = i2 > 0.f ? c_scale(r, as * rsqrtf(i2)) : make_float2(as, 0.f);
    }
  }
  if (REPLACE) {
    __syncthreads();
    fft<true>(pl, C, a.tw_col);
    store_strip(sm, f, col0, C, W, H);
  }
  block_partials(s_it, s_ii, s_tt, a.partials + sp * 3 * gridDim.x);
}

// Bare column FFTs (propagation), in place on out: FFT -> scale -> (times conj chirp when POST).
template <bool INV, bool POST>
__global__ void __launch_bounds__(1024) kg_col_fft(const __grid_constant__ PassArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  const GenPlan& pl = a.gen_col;
  const int W = a.W, H = a.H, C = pl.batch, col0 = blockIdx.x * C, k = blockIdx.y;
  float2* f = a.out[k];
  load_strip(sm, f, col0, C, W, H);
  __syncthreads();
  fft<INV>(pl, C, a.tw_col);
  for (int i = threadIdx.x; i < C * H; i += blockDim.x) {
    const int b = i % C, n = i / C, col = col0 + b;
    if (col < W) {
      float2 x = c_scale(sm[pidx(b * H + n)], a.scale);
      if (POST) x = c_mulc(x, c_mul(__ldg(&a.cx[col]), __ldg(&a.cy[n])));
      f[(size_t)n * W + col] = x;
    }
  }
}

// OSPR column pass.  FINISH: the field holds rowFFT(h_{s-1} c): accumulate its replay intensity
// (add to the stored sum when acc_read) and the NMSE partials.  START: the random-phase subframe s
// (Philox counter (pixel, s, 0, 0), key (seed_lo, seed_hi ^ target)), inverse column FFTs -> field.
// Target and accumulated intensity are per strip ([strip][H][C]).
template <bool FINISH, bool START>
__global__ void __launch_bounds__(1024) kg_col_ospr(const __grid_constant__ PassArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  const GenPlan& pl = a.gen_col;
  const int W = a.W, H = a.H, C = pl.batch, col0 = blockIdx.x * C, k = blockIdx.y;
  const int slot = a.class_slot[k];
  float2* f = a.field + (size_t)slot * H * W;
  const size_t strip = ((size_t)slot * gridDim.x + blockIdx.x) * H * C;
  float* acc = a.acc + strip;
  const float* tt = a.ttile + strip;
  float s_it = 0.f, s_ii = 0.f, s_tt = 0.f;
  if (FINISH) {
    load_strip(sm, f, col0, C, W, H);
    __syncthreads();
    fft<false>(pl, C, a.tw_col);
    for (int i = threadIdx.x; i < C * H; i += blockDim.x) {
      const int b = i % C, n = i / C;
      if (col0 + b >= W) continue;
      const int q = n * C + b;
      const float2 r = sm[pidx(b * H + n)];
      float i2 = fmaf(r.x, r.x, r.y * r.y);
      if (a.acc_read) i2 += acc[q];
      acc[q] = i2;
      const float t2 = tt[q] * tt[q];
      s_it = fmaf(i2, t2, s_it);
      s_ii = fmaf(i2, i2, s_ii);
      s_tt = fmaf(t2, t2, s_tt);
    }
  }
  if (START) {
    __syncthreads();  // FINISH's reads of the tile are done
    for (int i = threadIdx.x; i < C * H; i += blockDim.x) {
      const int b = i % C, n = i / C, col = col0 + b;
      float2 e = make_float2(0.f, 0.f);
      if (col < W) e = ospr::random_field((uint32_t)((size_t)n * W + col), a.iter, a.seed, a.item_index[k], tt[n * C + b]);
      sm[pidx(b * H + n)] = e;
    }
    __syncthreads();
    fft<true>(pl, C, a.tw_col);
    store_strip(sm, f, col0, C, W, H);
  }
  if (FINISH) block_partials(s_it, s_ii, s_tt, a.partials + (size_t)slot * 3 * gridDim.x);
}

// Gradient-descent column pass, one (item, plane) per blockIdx.y.  Forward: loss statistics of
// U = F(h c_p) against the target intensity.  Backward: the adjoint field
// (2/P) s_u (s_u I - T) / sum T^2 U, inverse column FFTs -> field p.
template <bool BWD>
__global__ void __launch_bounds__(1024) kg_col_gd(const __grid_constant__ PassArgs a) {
  extern __shared__ __align__(16) float2 sm[];
  const GenPlan& pl = a.gen_col;
  const int P = a.n_planes > 1 ? a.n_planes : 1;
  const int k = blockIdx.y / P, p = blockIdx.y % P;
  const int W = a.W, H = a.H, C = pl.batch, col0 = blockIdx.x * C;
  const size_t sp = (size_t)a.class_slot[k] * P + p;
  float2* f = a.field + sp * H * W;
  const float* T = a.target[k * P + p];
  load_strip(sm, f, col0, C, W, H);
  __syncthreads();
  fft<false>(pl, C, a.tw_col);
  if (!BWD) {
    float s_it = 0.f, s_ii = 0.f, s_tt = 0.f;
    for (int i = threadIdx.x; i < C * H; i += blockDim.x) {
      const int b = i % C, n = i / C, col = col0 + b;
      if (col >= W) continue;
      const float2 u = sm[pidx(b * H + n)];
      const float i2 = fmaf(u.x, u.x, u.y * u.y);
      const float t2 = __ldg(&T[target_index(a, n, col)]);
      s_it = fmaf(i2, t2, s_it);
      s_ii = fmaf(i2, i2, s_ii);
      s_tt = fmaf(t2, t2, s_tt);
    }
    block_partials(s_it, s_ii, s_tt, a.partials + sp * 3 * gridDim.x);
  } else {
    const double* st = a.stats + sp * 4;
    const float su = (float)__ldcg(&st[0]);
    const float coef = (float)(2.0 / P * __ldcg(&st[0]) / (__ldcg(&st[1]) > 0.0 ? __ldcg(&st[1]) : 1.0));
    for (int i = threadIdx.x; i < C * H; i += blockDim.x) {
      const int b = i % C, n = i / C, col = col0 + b;
      float2 gi = make_float2(0.f, 0.f);
      if (col < W) {
        const float2 u = sm[pidx(b * H + n)];
        const float i2 = fmaf(u.x, u.x, u.y * u.y);
        const float t2 = __ldg(&T[target_index(a, n, col)]);
        gi = c_scale(u, coef * fmaf(su, i2, -t2));
      }
      sm[pidx(b * H + n)] = gi;
    }
    __syncthreads();
    fft<true>(pl, C, a.tw_col);
    store_strip(sm, f, col0, C, W, H);
  }
}

// ---------------------------------------------------------------- host side: plans and tables

bool smooth(int n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

// Radices of n: 16s, then one 8 / 4 / 2 for the rest of the factor 2^a, 9s and a 3, then 5s (the
// order fft() runs its stage loops in).
std::vector<int> radices(int n) {
  int a = 0, b = 0, c = 0;
  while (n % 2 == 0) n /= 2, ++a;
  while (n % 3 == 0) n /= 3, ++b;
  while (n % 5 == 0) n /= 5, ++c;
  std::vector<int> r;
  for (; a >= 4; a -= 4) r.push_back(16);
  if (a) r.push_back(1 << a);
  for (; b >= 2; b -= 2) r.push_back(9);
  if (b) r.push_back(3);
  for (; c > 0; --c) r.push_back(5);
  return r;
}

GenPlan make_plan(int n, int batch) {
  GenPlan pl{};
  pl.n = n;
  pl.batch = batch;
  const std::vector<int> r = radices(n);
  pl.stages = (int)r.size();
  int ns = 1, off = 0;
  for (int s = 0; s < pl.stages; ++s) {
    switch (r[s]) {
      case 16: ++pl.n16; break;
      case 9: ++pl.n9; break;
      case 3: ++pl.n3; break;
      case 5: ++pl.n5; break;
      default: pl.r2 = r[s]; break;
    }
    pl.r[s] = r[s];
    pl.ns[s] = ns;
    pl.off[s] = ns > 1 ? off : -1;
    if (ns > 1) off += (r[s] - 1) * ns;
    ns *= r[s];
  }
  return pl;
}

TwiddleLayout layout(const GenPlan& pl) {
  TwiddleLayout l{};
  l.size = 0;
  for (int s = 0; s < pl.stages; ++s)
    if (pl.ns[s] > 1) {
      l.ns[l.count] = pl.ns[s];
      l.r[l.count] = pl.r[s];
      l.off[l.count] = pl.off[s];
      l.size += (pl.r[s] - 1) * pl.ns[s];
      ++l.count;
    }
  return l;
}

// Threads of a tile: enough that no thread holds more than kVmax values in any stage (a multiple of
// 32); 0 when that takes more than 1024.
int threads(const GenPlan& pl) {
  int nt = 32;
  for (int s = 0; s < pl.stages; ++s) {
    const int bf = pl.batch * (pl.n / pl.r[s]), per = kVmax / pl.r[s];
    nt = std::max(nt, (bf + per - 1) / per);
  }
  nt = (nt + 31) / 32 * 32;
  return nt <= 1024 ? nt : 0;
}

// Raises every generic kernel's dynamic shared-memory limit to what the current device allows beside
// the kernel's static shared memory (the block reductions' 768 bytes).
void set_attrs() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const void* fns[] = {(const void*)&kg_row_init,           (const void*)&kg_row_gs<false>,
                       (const void*)&kg_row_gs<true>,       (const void*)&kg_row_fft<false, false>,
                       (const void*)&kg_row_fft<false, true>, (const void*)&kg_row_fft<true, false>,
                       (const void*)&kg_row_fft<true, true>, (const void*)&kg_row_ospr<false>,
                       (const void*)&kg_row_ospr<true>,     (const void*)&kg_row_plane_fwd,
                       (const void*)&kg_row_plane_back,
                       (const void*)&kg_col_gs<false>,      (const void*)&kg_col_gs<true>,
                       (const void*)&kg_col_fft<false, false>, (const void*)&kg_col_fft<false, true>,
                       (const void*)&kg_col_fft<true, false>, (const void*)&kg_col_fft<true, true>,
                       (const void*)&kg_col_ospr<false, true>, (const void*)&kg_col_ospr<true, true>,
                       (const void*)&kg_col_ospr<true, false>, (const void*)&kg_col_gd<false>,
                       (const void*)&kg_col_gd<true>};
  for (const void* f : fns) {
    cudaFuncAttributes at{};
    if (cudaFuncGetAttributes(&at, f) == cudaSuccess)
      cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)at.sharedSizeBytes);
    cudaGetLastError();
  }
}

struct Tables {
  GenPlan prow, pcol;
  RowKernels rk{};
  ColKernels ck{};
};

// Rows per row tile: as many whole rows as fit 4096 values.  Columns per strip: 16 (rows of at most
// 512), 8 (1920), 4 (3840), else 2, halved until the strip's threads fit one CTA.
std::unique_ptr<Tables> make_tables(int n) {
  auto t = std::make_unique<Tables>();
  const int rows = std::min(1024, std::max(1, 4096 / n));
  t->prow = make_plan(n, rows);
  int cols = n <= 512 ? 16 : (n <= 1920 ? 8 : (n <= 3840 ? 4 : 2));
  t->pcol = make_plan(n, cols);
  while (threads(t->pcol) == 0 && cols > 1) t->pcol = make_plan(n, cols /= 2);
  if (threads(t->prow) == 0 || threads(t->pcol) == 0) return nullptr;

  RowKernels& r = t->rk;
  r.rows = rows;
  r.nt = threads(t->prow);
  // the tile + the OSPR row pass's decisions
  r.smem = padded(rows * n) * (int)sizeof(float2) + (rows * n + 15) / 16 * 16;
  r.init[0] = r.init[1] = (const void*)&kg_row_init;
  r.gs[0][0] = r.gs[0][1] = (const void*)&kg_row_gs<false>;
  r.gs[1][0] = r.gs[1][1] = (const void*)&kg_row_gs<true>;
  r.fft[0][0] = (const void*)&kg_row_fft<false, false>;
  r.fft[0][1] = (const void*)&kg_row_fft<false, true>;
  r.fft[1][0] = (const void*)&kg_row_fft<true, false>;
  r.fft[1][1] = (const void*)&kg_row_fft<true, true>;
  r.ospr[0] = (const void*)&kg_row_ospr<false>;
  r.ospr[1] = (const void*)&kg_row_ospr<true>;
  r.smem_ospr = r.smem;
  // multi-plane GS and gradient descent: one launch per plane (see kg_row_plane_fwd)
  r.plane.start[0] = (const void*)&kg_mp_start<false>;
  r.plane.start[1] = (const void*)&kg_mp_start<true>;
  r.plane.fwd = (const void*)&kg_row_plane_fwd;
  r.plane.back = (const void*)&kg_row_plane_back;
  r.plane.project = (const void*)&kg_mp_project;
  r.plane.grad = (const void*)&kg_gd_grad;
  r.set_attrs = &set_attrs;
  r.tw = layout(t->prow);
  r.gen = &t->prow;

  ColKernels& c = t->ck;
  c.cols = cols;
  c.nt = threads(t->pcol);
  c.smem = padded(cols * n) * (int)sizeof(float2);
  c.smem_gs = c.smem;
  c.smem_ospr = c.smem;
  c.gs[0][0] = c.gs[0][1] = (const void*)&kg_col_gs<false>;
  c.gs[1][0] = c.gs[1][1] = (const void*)&kg_col_gs<true>;
  c.tile = 0;
  c.fft[0][0] = (const void*)&kg_col_fft<false, false>;
  c.fft[0][1] = (const void*)&kg_col_fft<false, true>;
  c.fft[1][0] = (const void*)&kg_col_fft<true, false>;
  c.fft[1][1] = (const void*)&kg_col_fft<true, true>;
  c.ospr[0] = (const void*)&kg_col_ospr<false, true>;
  c.ospr[1] = (const void*)&kg_col_ospr<true, true>;
  c.ospr[2] = (const void*)&kg_col_ospr<true, false>;
  c.gd[0] = (const void*)&kg_col_gd<false>;
  c.gd[1] = (const void*)&kg_col_gd<true>;
  c.set_attrs = &set_attrs;
  c.tw = layout(t->pcol);
  c.gen = &t->pcol;
  return t;
}

std::mutex g_mu;
std::map<int, std::unique_ptr<Tables>> g_tables;

const Tables* tables(int n) {
  if (n < 1 || n > kGenMaxLength || !smooth(n)) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_tables.find(n);
  if (it == g_tables.end()) it = g_tables.emplace(n, make_tables(n)).first;
  return it->second.get();
}

}  // namespace gen

const RowKernels* gen_row_kernels(int n) {
  const gen::Tables* t = gen::tables(n);
  return t ? &t->rk : nullptr;
}

const ColKernels* gen_col_kernels(int n) {
  const gen::Tables* t = gen::tables(n);
  return t ? &t->ck : nullptr;
}

}  // namespace hg
