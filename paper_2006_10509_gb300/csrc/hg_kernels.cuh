// Fused row-pass and column-pass kernels of the phase-retrieval loop.
//
// One GS iteration (Gerchberg & Saxton; section "Algorithm Libraries", HoloGenAlgGSCuda and the
// RunIterations() loop of section "Algorithm Interface") is two passes over the field in HBM:
//
//   column pass: Y -> forward column FFTs -> R = F(h c)  [NMSE partials, R' = A R/|R|]
//                  -> inverse column FFTs -> Z                                    (in place)
//   row pass:    Z -> inverse row FFTs -> g (times conj(c)) -> h = P_SLM(g)
//                  -> (times c) -> forward row FFTs -> Y                           (in place)
//
// so the field crosses HBM twice per iteration (read + write each), plus one read of the target.
// Transforms are unnormalised: every projection in the loop is invariant to a positive scale, and
// the NMSE uses the optimal scale, so the unitary 1/sqrt(HW) factors are only applied by the bare
// propagation entry point.
#pragma once

#include <cooperative_groups.h>
#include <type_traits>

#include "hg_fft.cuh"
#include "hg_launch.h"

namespace hg {

constexpr int kMaxBatch = 32;  // items per launch (a size class with more items is launched in chunks)
constexpr int kMaxPlanes = 16;  // replay planes per plan

__host__ __device__ constexpr int hg_max(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int hg_min(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int round_up(int a, int m) { return (a + m - 1) / m * m; }

// The value itself, hidden from the optimiser.  Column kernels re-derive their store addresses
// (which involve the run-time row stride) through it after the second transform, instead of
// keeping every slot's address live across both transforms.
__device__ __forceinline__ int opaque(int x) {
  int y;
  asm volatile("mov.b32 %0, %1;" : "=r"(y) : "r"(x));
  return y;
}
template <class T>
__device__ __forceinline__ T* opaque(T* x) {
  T* y;
  asm volatile("mov.b64 %0, %1;" : "=l"(y) : "l"(x));
  return y;
}

// Row tile: ROWS rows of length W, about 16 values per thread.  TW > 0: the field is stored in
// column-strip tiles of width TW (see fidx); the tile holds 16 / TW rows (2 for TW = 2) whose lanes
// interleave in groups of TW, so each warp access covers whole 128-byte lines of the tiled layout
// (whole 32-byte sectors for TW = 2, where 8-row tiles of 1024 threads measured slower).
// PV: the radix plan (PlanV<W, PV>; 0 the default, 1 the alternative of the lengths that have one).
template <int W, int TW = 0, int PV = 0>
struct RowCfg {
  static constexpr int ROWS = TW ? (TW >= 4 ? 16 / TW : 2) : hg_max(1, 4096 / W);
  static constexpr int NT =
      pick_threads<typename PlanV<W, PV>::type>(W, ROWS, value_budget(W), TW ? 1024 : 512);
  static constexpr int MINB = hg_min(8, hg_max(1, 1024 / NT));  // CTAs per SM at <= 64 registers
  using G = Geo<W, ROWS, NT, false, (TW && ROWS > 1) ? TW : 0>;
  using Fwd = typename PlanV<W, PV>::type;
  using Inv = typename RRev<Fwd>::type;
  static constexpr int RE = RLast<Fwd>::value;   // radix of the global load/store stages
  static constexpr int RM = RFirst<Fwd>::value;  // radix of the pointwise step between the FFTs
  static constexpr int V = MaxV<G, Fwd>::value;
  static constexpr int SMEM = G::SM_ELEMS * 8;
};

// Column strip widths.  On a field tiled in column strips (GS), measured on GB300 (100
// iterations): 2-column strips (256 / 512 threads, several CTAs per SM, so barriers span few warps
// and the last wave is short) beat 8-column ones by 7-11 % at 2048 and 4096 rows and 12 % at 512;
// at 1024 rows 8-column strips are 8 % faster; at 1080 rows (1080 x 1920) 4-column strips are 14 %
// faster than 8 and 20 % faster than 2; 864 rows are indifferent.  On a row-major field a strip
// reads C columns of every row, so it takes at least 4 (one 32-byte sector): 4 at 1080 and from
// 2048 rows (measured: the gradient-descent adjoint column pass at 2048^2, 3 planes, 131 us with 8
// columns, 105 with 4), else 8, and 16 below 640 rows.
__host__ __device__ constexpr int tiled_cols(int h) {
  return h >= 2048 ? 2 : (h == 1080 ? 4 : (h >= 640 ? 8 : (h >= 384 ? 2 : 16)));
}
__host__ __device__ constexpr int natural_cols(int h) {
  return h >= 2048 ? 4 : (h == 1080 ? 4 : (h >= 640 ? 8 : 16));
}

// Column strip: C columns of length H, about 16 values per thread.  CW = 0: the row-major-field
// width; CW > 0: a strip of the tiled GS field of that width (the plan's default is tiled_cols(H),
// the autotuner may pick another).
template <int H, int CW = 0, int PV = 0>
struct ColCfg {
  static constexpr int C = CW ? CW : natural_cols(H);
  static constexpr int NT = pick_threads<typename PlanV<H, PV>::type>(H, C, value_budget(H), 1024);
  using G = Geo<H, C, NT, true>;
  using Fwd = typename PlanV<H, PV>::type;
  using Inv = typename RRev<Fwd>::type;
  static constexpr int RB = RFirst<Fwd>::value;  // radix of the global load/store stage
  static constexpr int V = MaxV<G, Fwd>::value;
  static constexpr int SMEM = G::SM_ELEMS * 8;
  static constexpr int SMEM_T = SMEM + H * C * 4;  // + the strip's target values (GS passes)
  // the OSPR column pass also stages the strip's accumulated intensity where that keeps at least
  // two CTAs per SM (80 KB); otherwise it reads the sum from global memory where it adds to it
  static constexpr bool OSPR_ACC_SM = SMEM_T + H * C * 4 <= 80 * 1024;
  static constexpr int SMEM_OSPR = OSPR_ACC_SM ? SMEM_T + H * C * 4 : SMEM_T;
  static constexpr int MINB = hg_max(1, 1024 / NT);  // CTAs per SM the register budget is cut for
  // the configuration exists: no thread past the value budget, the GS pass's shared memory fits
  static constexpr bool FEASIBLE =
      RValues<Fwd>::max_values(H, C, NT) <= value_budget(H) && SMEM_T <= 227 * 1024;
};

// Global index of field element (row, n) of an [H][W] item: row-major (TW = 0), or column-strip
// tiles of width TW ([W / TW][H][TW]), the layout in which a column pass reads its strip as one
// contiguous block.
template <int W, int TW>
__device__ __forceinline__ size_t fidx(int row, int n, int H) {
  if constexpr (TW == 0)
    return (size_t)row * W + n;
  else
    return ((size_t)(n / TW) * H + row) * TW + (n % TW);
}

// ---------------------------------------------------------------- asynchronous copies

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Starts copying the strip's target values A[n][col0 .. col0 + C) into ts[n * C + b] (zero past W).
// 16-byte copies when every row segment is whole and aligned, else 4-byte copies.
template <int H, int C, int NT>
__device__ __forceinline__ void prefetch_strip(float* ts, const float* __restrict__ A, int col0, int W) {
  const int t = threadIdx.x;
  bool vec = false;
  if constexpr (C % 4 == 0) {
    vec = (W % 4 == 0) && (col0 + C <= W) && (((uintptr_t)A & 15) == 0) &&
          ((__cvta_generic_to_shared(ts) & 15) == 0);
    if (vec) {
      constexpr int CH = C / 4;  // 16-byte chunks per row
      for (int i = t; i < H * CH; i += NT) {
        const int n = i / CH, c = i % CH;
        cp_async16(ts + n * C + 4 * c, A + (size_t)n * W + col0 + 4 * c);
      }
    }
  }
  if (!vec) {
    for (int i = t; i < H * C; i += NT) {
      const int n = i / C, b = i % C;
      if (col0 + b < W)
        cp_async4(ts + i, A + (size_t)n * W + col0 + b);
      else
        ts[i] = 0.f;
    }
  }
  cp_async_commit();
}

// Starts copying COUNT contiguous floats (COUNT % 4 == 0, both ends 16-byte aligned) into ts.
template <int COUNT, int NT>
__device__ __forceinline__ void prefetch_contig(float* ts, const float* __restrict__ src) {
  for (int i = threadIdx.x; i < COUNT / 4; i += NT) cp_async16(ts + 4 * i, src + 4 * i);
  cp_async_commit();
}

// ---------------------------------------------------------------- programmatic dependent launch

// The GS passes are launched with programmatic stream serialisation: a pass may be scheduled
// while its predecessor drains.  It waits here before reading anything an earlier kernel wrote,
// then lets its own successor be scheduled (which happens once every CTA of this pass has got this
// far, so a waiting successor never holds a slot that one of this pass's CTAs still needs).
// Without that launch attribute the wait returns at once.
__device__ __forceinline__ void pdl_wait_then_release() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// ---------------------------------------------------------------- launch arguments

// Per-launch argument block: up to kMaxBatch items of one size class.  Plan-owned buffers
// (field, chirps, partials) are per class; caller buffers are per item.
struct PassArgs {
  int n_items;
  int H, W;
  int n_levels;            // 0 continuous, 2 binary, N >= 3 N-level; -M: M complex SLM values in lev
                           // (multi-amplitude SLM; extended GS kernels only)
  int iter;                // iteration / subframe index of the pass
  int col_blocks;          // column-pass blocks per (item, plane): partial triples to add
  int finalize;            // row passes: 1 = first add up the preceding column pass's NMSE
  int fin_iter;            // nmse slot of that column pass
  int nmse_stride;         // floats between items in nmse_out (n_iter + 1)
  int n_iter;              // whole-run kernels: GS iterations
  const float2* tw_row;    // per-stage twiddle tables of length W (TwBlob<W>)
  const float2* tw_col;    // per-stage twiddle tables of length H (TwBlob<H>)
  const float2* cx;        // Fresnel chirp along a row (W), nullptr for Fourier
  const float2* cy;        // Fresnel chirp along a column (H)
  const float2* lev;       // level field exp(2 pi i q / N), q < N
  const float* lev_phase;  // level phase 2 pi q / N
  float2* field;           // class field buffer: item k at field + k * H * W
  // MRAF (mix > 0): per-item signal-region masks (nonzero = signal; nullptr = the whole plane) and
  // the mixing parameter m; the target copy marks noise-region pixels with -1
  const uint8_t* mask[kMaxBatch];
  float mix;
  // HIO (with mix = 1): the replay-plane input X on the noise region, [slot][strip][H][C] like the
  // target tiles, in the unnormalised forward transform's scale; nullptr for MRAF / GS
  float2* hio;
  float beta;              // HIO feedback: X' = X - beta Y on the noise region
  int centred;             // targets (and signal masks) in display order: DC at (H/2, W/2)
  const float* illum[kMaxBatch];  // GS: SLM illumination amplitude [H][W] per item (nullptr: uniform)
  float2* partials;        // class partial sums (hi, lo): (slot, plane) at partials + (slot P + p) 3 col_blocks
  float* nmse;             // nmse_out of the run (device) or nullptr
  uint64_t seed;           // starting-phase seed when phase_in is null
  float scale;             // output scale (bare propagation)
  int item_index[kMaxBatch];  // plan item index (nmse row, Philox key)
  int class_slot[kMaxBatch];  // slot in the class buffers
  const float* target[kMaxBatch];
  const float* ttile;           // GS column passes: the targets re-laid out per column strip (slot P + p)
                                // blocks of col_blocks strips, strip t holding [H][C] contiguous; or
                                // nullptr to read the caller's [H][W] targets directly
  const float* phase_in[kMaxBatch];
  float* phase_out[kMaxBatch];
  uint8_t* level_out[kMaxBatch];
  const float2* in[kMaxBatch];  // bare propagation input
  float2* out[kMaxBatch];       // bare propagation output
  // OSPR
  float* acc;                   // class accumulated-intensity buffer: item k at acc + k * H * W
  int acc_read;                 // 1: add to the stored sum, 0: start it
  uint32_t* bits[kMaxBatch];    // [S][H][ceil(W/32)] LSB-first hologram bits, or nullptr
  // planes (multi-plane GS, gradient descent).  With P planes a launch covers n_items * P <= kMaxBatch
  // (item, plane) pairs: target[k * P + p]; class buffers are indexed by slot * P + p.
  int n_planes;                        // P (0 is read as 1)
  const float2* cxp[kMaxPlanes];       // per-plane chirp factors (Fresnel)
  const float2* cyp[kMaxPlanes];
  double* stats;                       // class [slot * P + p][4]: s, sum T^2, loss, 1/sqrt(sum A^2)
  // gradient descent
  float* loss;                         // loss_out [n_items][P + 1] (device) or nullptr
  float* phi[kMaxBatch];               // phase parameters (in / out)
  float* adam_m[kMaxBatch];
  float* adam_v[kMaxBatch];
  float* grad[kMaxBatch];              // dL/dphi out, or nullptr
  const float* grad_scale;             // device scalar multiplying the gradient, or nullptr (= 1)
  int adam;                            // 1: apply the Adam update
  float lr, beta1, beta2, eps, bc1, bc2;  // Adam; bc1 = 1 - beta1^t, bc2 = 1 - beta2^t
  // generic kernels (lengths without a compiled instance): the run-time plans of W and H
  GenPlan gen_row, gen_col;
};

// ---------------------------------------------------------------- pointwise pieces

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Starting-phase draw when no phase is given: counter (p, 0, 1, 0), key (seed_lo, seed_hi ^ item).
__device__ __forceinline__ float2 init_unit(uint32_t p, uint64_t seed, int item) {
  const uint4 x = philox4x32_10(make_uint4(p, 0u, 1u, 0u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32) ^ (uint32_t)item));
  const float u2 = (float)(x.x >> 8) * (1.0f / 8388608.0f);  // 2u, u = (x >> 8) 2^-24
  float s, c;
  sincospif(u2, &s, &c);
  return make_float2(c, s);
}

// SLM projection (nearest point of the constraint set).  q receives the level index (quantised).
// One function per kind of phase-only SLM; slm_project picks one from the level count at run time,
// slm_project_lv<LV> at compile time (LV = 0 continuous, 2, 4 or 8 the sector tests, -1 any other
// count by the arctangent).

__device__ __forceinline__ float2 project_continuous(float2 g, int& q) {
  const float m2 = fmaf(g.x, g.x, g.y * g.y);
  q = 0;
  if (m2 > 0.f) {
    const float r = rsqrtf(m2);
    return make_float2(g.x * r, g.y * r);
  }
  return make_float2(1.f, 0.f);
}

__device__ __forceinline__ float2 project_binary(float2 g, int& q) {
  // arg in [pi/2, 3pi/2) -> pi; on Re g = 0, Im > 0 goes to pi and Im < 0 to 0
  q = (g.x < 0.f || (g.x == 0.f && g.y > 0.f)) ? 1 : 0;
  return make_float2(q ? -1.f : 1.f, 0.f);
}

__device__ __forceinline__ float2 project_4(float2 g, const float2* __restrict__ lev, int& q) {
  // levels 0, pi/2, pi, 3pi/2: the sector of g from |x| against |y| and the signs, no arctangent
  // (measured on GB300: the 4-level GS row pass at 2048^2 29.8 -> 26.3 us).  A midpoint goes to
  // the higher index: arg pi/4 -> 1, 3pi/4 -> 2, 5pi/4 -> 3, 7pi/4 -> 0.
  const float ax = fabsf(g.x), ay = fabsf(g.y);
  int qq;
  if (ax > ay || (ax == ay && ((g.x > 0.f) != (g.y > 0.f))))
    qq = g.x >= 0.f ? 0 : 2;
  else
    qq = g.y > 0.f ? 1 : 3;
  if (ax == 0.f && ay == 0.f) qq = 0;
  q = qq;
  return __ldg(&lev[qq]);
}

__device__ __forceinline__ float2 project_8(float2 g, const float2* __restrict__ lev, int& q) {
  // levels k pi/4: fold g into the first quadrant (quarter turns Q, (u, v) with u > 0, v >= 0),
  // then the sector from v against tan(pi/8) u and u against tan(pi/8) v (a midpoint to the
  // higher index, as above; g = 0 -> 0)
  constexpr float t8 = 0.41421356237309504880f;  // tan(pi/8) = sqrt(2) - 1
  int qd;
  float u, v;
  if (g.x > 0.f && g.y >= 0.f) {
    qd = 0, u = g.x, v = g.y;
  } else if (g.x <= 0.f && g.y > 0.f) {
    qd = 1, u = g.y, v = -g.x;
  } else if (g.x < 0.f && g.y <= 0.f) {
    qd = 2, u = -g.x, v = -g.y;
  } else {
    qd = 3, u = -g.y, v = g.x;
  }
  int qq = 2 * qd + (v < t8 * u ? 0 : (t8 * v >= u ? 2 : 1));
  if (qq >= 8) qq -= 8;
  if (g.x == 0.f && g.y == 0.f) qq = 0;
  q = qq;
  return __ldg(&lev[qq]);
}

__device__ __forceinline__ float2 project_levels(float2 g, int n_levels, const float2* __restrict__ lev, int& q) {
  const float a = atan2f(g.y, g.x);  // (-pi, pi]
  float t = a * ((float)n_levels * 0.15915494309189533577f);
  if (t < 0.f) t += (float)n_levels;
  int qq = (int)floorf(t + 0.5f);
  if (qq >= n_levels) qq -= n_levels;
  q = qq;
  return __ldg(&lev[qq]);
}

template <int LV>
__device__ __forceinline__ float2 slm_project_lv(float2 g, int n_levels, const float2* __restrict__ lev, int& q) {
  if constexpr (LV == 0)
    return project_continuous(g, q);
  else if constexpr (LV == 2)
    return project_binary(g, q);
  else if constexpr (LV == 4)
    return project_4(g, lev, q);
  else if constexpr (LV == 8)
    return project_8(g, lev, q);
  else
    return project_levels(g, n_levels, lev, q);
}

__device__ __forceinline__ float2 slm_project(float2 g, int n_levels, const float2* __restrict__ lev, int& q) {
  if (n_levels == 0) return project_continuous(g, q);
  if (n_levels == 2) return project_binary(g, q);
  if (n_levels == 4) return project_4(g, lev, q);
  if (n_levels == 8) return project_8(g, lev, q);
  return project_levels(g, n_levels, lev, q);
}

// Calls f(std::integral_constant<int, LV>) with LV the compile-time projection kind of a run's
// phase-only level count: the kernels whose pixel loops project take the choice once per launch.
// (The run-time choice inside the unrolled loops of the GS row pass cost about three branches per
// pixel and instruction-fetch stalls: measured on GB300, 2048^2 continuous row pass 26.4 us against
// 24.4 us before the 8-level branch was added to it.)
template <class F>
__device__ __forceinline__ void dispatch_levels(int n_levels, F&& f) {
  if (n_levels == 0)
    f(std::integral_constant<int, 0>{});
  else if (n_levels == 2)
    f(std::integral_constant<int, 2>{});
  else if (n_levels == 4)
    f(std::integral_constant<int, 4>{});
  else if (n_levels == 8)
    f(std::integral_constant<int, 8>{});
  else
    f(std::integral_constant<int, -1>{});
}

// Multi-amplitude / complex-modulation SLM: the nearest of the m complex values lev[0..m) (squared
// distance in float32; the lowest index on a tie).
__device__ __forceinline__ float2 table_project(float2 g, int m, const float2* __restrict__ lev, int& q) {
  int best = 0;
  float2 l = __ldg(&lev[0]);
  float bd = fmaf(g.x - l.x, g.x - l.x, (g.y - l.y) * (g.y - l.y));
  for (int i = 1; i < m; ++i) {
    l = __ldg(&lev[i]);
    const float dd = fmaf(g.x - l.x, g.x - l.x, (g.y - l.y) * (g.y - l.y));
    if (dd < bd) {
      bd = dd;
      best = i;
    }
  }
  q = best;
  return __ldg(&lev[best]);
}

// SLM projection of the GS row kernels: the extended instances also take a table of -n_levels
// complex values (n_levels < 0); the plain ones keep the phase-only sets.
template <bool EXT>
__device__ __forceinline__ float2 slm_project_x(float2 g, int n_levels, const float2* __restrict__ lev, int& q) {
  if (EXT && n_levels < 0) return table_project(g, -n_levels, lev, q);
  return slm_project(g, n_levels, lev, q);
}

__device__ __forceinline__ float phase_0_2pi(float2 h) {
  float a = atan2f(h.y, h.x);
  if (a < 0.f) {
    a += 6.28318530717958647693f;
    if (a >= 6.28318530717958647693f) a = 0.f;
  }
  return a;
}

// ---------------------------------------------------------------- reductions
//
// A pass that needs sums over the whole field (NMSE, loss statistics, target energy) only writes
// per-block partials; the next kernel in stream order (the following row pass, or a small finalise
// kernel) adds them in block order.  Nothing spins, nothing waits on another block, and the result
// does not depend on block scheduling.  Within a block the sums run in double-float arithmetic on
// the FP32 pipes (a pair hi + lo, Knuth's two-sum), which keeps FP64-class accuracy without the
// low-rate FP64 units.

struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bp = s - a.hi;
  float e = (a.hi - (s - bp)) + (b.hi - bp);
  e += a.lo + b.lo;
  const float h = s + e;
  return DF{h, e - (h - s)};
}
__device__ __forceinline__ DF df_shfl_down(DF v, int o) {
  return DF{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}

// Block sums of (x0, x1, x2) -> part[3 * blockIdx.x + i] as (hi, lo) pairs.  All threads must call it.
__device__ __forceinline__ void block_partials(float x0, float x1, float x2, float2* __restrict__ part) {
  __shared__ DF red[3][32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = (blockDim.x + 31) >> 5;
  DF a{x0, 0.f}, b{x1, 0.f}, c{x2, 0.f};
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a = df_add(a, df_shfl_down(a, o));
    b = df_add(b, df_shfl_down(b, o));
    c = df_add(c, df_shfl_down(c, o));
  }
  if (lane == 0) {
    red[0][warp] = a;
    red[1][warp] = b;
    red[2][warp] = c;
  }
  __syncthreads();
  if (warp == 0) {
    const DF z{0.f, 0.f};
    a = lane < nw ? red[0][lane] : z;
    b = lane < nw ? red[1][lane] : z;
    c = lane < nw ? red[2][lane] : z;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      a = df_add(a, df_shfl_down(a, o));
      b = df_add(b, df_shfl_down(b, o));
      c = df_add(c, df_shfl_down(c, o));
    }
    if (lane == 0) {
      part[3 * blockIdx.x + 0] = make_float2(a.hi, a.lo);
      part[3 * blockIdx.x + 1] = make_float2(b.hi, b.lo);
      part[3 * blockIdx.x + 2] = make_float2(c.hi, c.lo);
    }
  }
}

// Sums nblk partial triples in a fixed order (lane k takes blocks k, k + 32, ..., then a shuffle
// tree); call from one full warp; lane 0 receives the totals.
__device__ __forceinline__ void sum_partials(const float2* __restrict__ part, int nblk, double* tot) {
  const int lane = threadIdx.x & 31;
  DF a{0.f, 0.f}, b{0.f, 0.f}, c{0.f, 0.f};
  for (int k = lane; k < nblk; k += 32) {
    const float2 x = part[3 * k + 0], y = part[3 * k + 1], z = part[3 * k + 2];
    a = df_add(a, DF{x.x, x.y});
    b = df_add(b, DF{y.x, y.y});
    c = df_add(c, DF{z.x, z.y});
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a = df_add(a, df_shfl_down(a, o));
    b = df_add(b, df_shfl_down(b, o));
    c = df_add(c, df_shfl_down(c, o));
  }
  tot[0] = (double)a.hi + (double)a.lo;
  tot[1] = (double)b.hi + (double)b.lo;
  tot[2] = (double)c.hi + (double)c.lo;
}

// NMSE = 1 - (sum I T)^2 / (sum I^2 sum T^2) from the sums (sum I T, sum I^2, sum T^2).
__device__ __forceinline__ double nmse_of(const double* tot) {
  return (tot[1] > 0.0 && tot[2] > 0.0) ? 1.0 - (tot[0] * tot[0]) / (tot[1] * tot[2]) : 1.0;
}

// NMSE of launch item k from the partials of the preceding column pass (mean over planes), written
// to nmse[item][fin_iter].  Called by one full warp.
__device__ __forceinline__ void finalize_nmse(const PassArgs& a, int k) {
  const int P = a.n_planes > 1 ? a.n_planes : 1;
  const int slot = a.class_slot[k];
  double m = 0.0;
  for (int p = 0; p < P; ++p) {
    double tot[3];
    sum_partials(a.partials + ((size_t)slot * P + p) * 3 * a.col_blocks, a.col_blocks, tot);
    m += nmse_of(tot);
  }
  if ((threadIdx.x & 31) == 0 && a.nmse) a.nmse[(size_t)a.item_index[k] * a.nmse_stride + a.fin_iter] = (float)(m / P);
}

// Finalise kernel, one warp per launch item (blockIdx.y).  MODE 0: NMSE of the preceding column
// pass.  MODE 1: gradient-descent statistics of the forward column pass: per plane s_u = sum I T /
// sum I^2, sum T^2 and the loss, plus the mean loss.  MODE 2: per-plane target amplitude energy,
// stats[4 sp + 3] = 1 / sqrt(sum A^2).
template <int MODE>
__global__ void __launch_bounds__(32) k_finalize(const __grid_constant__ PassArgs a) {
  const int k = blockIdx.y;
  if (MODE == 0) {
    finalize_nmse(a, k);
    return;
  }
  const int P = a.n_planes > 1 ? a.n_planes : 1;
  const int slot = a.class_slot[k];
  double m = 0.0;
  for (int p = 0; p < P; ++p) {
    const int sp = slot * P + p;
    double tot[3];
    sum_partials(a.partials + (size_t)sp * 3 * a.col_blocks, a.col_blocks, tot);
    if (threadIdx.x == 0) {
      double* st = a.stats + (size_t)sp * 4;
      if (MODE == 1) {
        const double loss = nmse_of(tot);
        st[0] = tot[1] > 0.0 ? tot[0] / tot[1] : 0.0;
        st[1] = tot[2];
        st[2] = loss;
        m += loss;
        if (a.loss) a.loss[(size_t)a.item_index[k] * (P + 1) + p] = (float)loss;
      } else {
        st[3] = tot[0] > 0.0 ? 1.0 / sqrt(tot[0]) : 1.0;
      }
    }
  }
  if (MODE == 1 && threadIdx.x == 0 && a.loss) a.loss[(size_t)a.item_index[k] * (P + 1) + P] = (float)(m / P);
}

// ---------------------------------------------------------------- field I/O of row tiles

// Global load / store of the radix-R first / last stage of a row tile.  In the tiled layout element
// (row, j + r N/R) lies at fidx(row, j) + r (N/R) H (N/R is a multiple of the tile width), one
// address per butterfly plus a stride.
template <class K, int R, int TW>
__device__ __forceinline__ void load_row_slots(float2 (&v)[K::V], const float2* __restrict__ f, int t, int row0,
                                               int H) {
  using G = typename K::G;
  for_each_slot_jr<G, R>(t, [&](int s, int b, int j, int r) {
    const int row = row0 + b;
    float2 x = make_float2(0.f, 0.f);
    if (row < H) {
      if constexpr (TW == 0)
        x = f[(size_t)row * G::N + j + r * (G::N / R)];
      else
        x = f[fidx<G::N, TW>(row, j, H) + (size_t)r * (G::N / R) * H];
    }
    v[s] = x;
  });
}

template <class K, int R, int TW>
__device__ __forceinline__ void store_row_slots(const float2 (&v)[K::V], float2* __restrict__ f, int t, int row0,
                                                int H) {
  using G = typename K::G;
  for_each_slot_jr<G, R>(t, [&](int s, int b, int j, int r) {
    const int row = row0 + b;
    if (row < H) {
      if constexpr (TW == 0)
        f[(size_t)row * G::N + j + r * (G::N / R)] = v[s];
      else
        f[fidx<G::N, TW>(row, j, H) + (size_t)r * (G::N / R) * H] = v[s];
    }
  });
}

// ---------------------------------------------------------------- row passes

// GS prologue: h0 = P_SLM(exp(i phi0)) (phi0 given, or drawn from the seed), times the chirp,
// forward row FFTs -> field.  h0 is written out when phase_out / level_out are set.
template <int W, int TW, bool EXT = false, int PV = 0>
__global__ void __launch_bounds__(RowCfg<W, TW, PV>::NT, RowCfg<W, TW, PV>::MINB) k_row_init(const __grid_constant__ PassArgs a) {
  using K = RowCfg<W, TW, PV>;
  using G = typename K::G;
  extern __shared__ __align__(16) float2 sm[];
  const int t = threadIdx.x, k = blockIdx.y;
  const int row0 = blockIdx.x * K::ROWS;
  const int H = a.H;
  float2* f = a.field + (size_t)a.class_slot[k] * H * W;
  const float* ph = a.phase_in[k];
  float* po = a.phase_out[k];  // set only when the run has no iterations (h_0 is the output)
  uint8_t* lo = a.level_out[k];
  float2 v[K::V];
  for_each_slot<G, RFirst<typename K::Fwd>::value>(t, [&](int s, int b, int n) {
    const int row = row0 + b;
    float2 h = make_float2(0.f, 0.f);
    if (row < H) {
      const size_t p = (size_t)row * W + n;
      float2 e;
      if (ph) {
        float sn, cs;
        sincosf(__ldg(&ph[p]), &sn, &cs);
        e = make_float2(cs, sn);
      } else {
        e = init_unit((uint32_t)p, a.seed, a.item_index[k]);
      }
      int q;
      h = slm_project_x<EXT>(e, a.n_levels, a.lev, q);
      if (po) po[p] = a.n_levels ? __ldg(&a.lev_phase[q]) : phase_0_2pi(h);
      if (lo) lo[p] = (uint8_t)q;
      if (EXT && a.illum[k]) h = c_scale(h, __ldg(&a.illum[k][p]));  // the SLM only sets the phase
      if (a.cx) h = c_mul(h, c_mul(__ldg(&a.cx[n]), __ldg(&a.cy[row])));
    }
    v[s] = h;
  });
  FftRun<G, false, 1, typename K::Fwd, typename K::Fwd>::run(v, sm, t, a.tw_row);
  store_row_slots<K, RLast<typename K::Fwd>::value, TW>(v, f, t, row0, H);
}

// GS row pass: inverse row FFTs, conj chirp, SLM projection (optionally written out), chirp,
// forward row FFTs.  SQ (square items, H = W): the tiled field's strip height is the compile-time W,
// so the strided loads and stores of a row take constant offsets from one address (measured on
// GB300, 2048^2 on 2-column strips: 25.0 -> 23.8 us per launch).
template <int W, bool OUT, int TW, bool EXT = false, int PV = 0, bool SQ = false>
__global__ void __launch_bounds__(RowCfg<W, TW, PV>::NT, RowCfg<W, TW, PV>::MINB) k_row_gs(const __grid_constant__ PassArgs a) {
  using K = RowCfg<W, TW, PV>;
  using G = typename K::G;
  extern __shared__ __align__(16) float2 sm[];
  const int t = threadIdx.x, k = blockIdx.y;
  pdl_wait_then_release();
  if (a.finalize && blockIdx.x == 0 && t < 32) finalize_nmse(a, k);
  const int row0 = blockIdx.x * K::ROWS;
  const int H = a.H;
  float2* f = a.field + (size_t)a.class_slot[k] * H * W;
  float2 v[K::V];
  load_row_slots<K, K::RE, TW>(v, f, t, row0, SQ ? W : H);
  FftRun<G, true, 1, typename K::Inv, typename K::Fwd>::run(v, sm, t, a.tw_row);
  float* po = OUT ? a.phase_out[k] : nullptr;
  uint8_t* lo = OUT ? a.level_out[k] : nullptr;
  // a multi-amplitude SLM's projection depends on the scale of g: bring the unnormalised field to
  // the unitary scale of the loop (replay target at a unit-modulus field's energy): 1 / sqrt(sum A^2)
  // for GS, 1 / (H W) under MRAF / HIO, whose column pass already scales the replacement
  // the table branch and the projection kind are chosen once per launch, outside the pixel loop
  // (measured: a per-pixel table test cost MRAF 8 % and HIO 11 % at 2048^2)
  auto pointwise = [&](auto table, auto lv) {
    constexpr bool TABLE = decltype(table)::value;
    constexpr int LV = decltype(lv)::value;
    const float gscale = TABLE ? (a.mix > 0.f ? 1.f / ((float)H * (float)W)
                                              : (float)__ldcg(&a.stats[(size_t)a.class_slot[k] * 4 + 3]))
                               : 1.f;
    for_each_slot<G, K::RM>(t, [&](int s, int b, int n) {
      const int row = row0 + b;
      float2 g = v[s];
      float2 c = make_float2(1.f, 0.f);
      if (a.cx && row < H) {
        c = c_mul(__ldg(&a.cx[n]), __ldg(&a.cy[row]));
        g = c_mulc(g, c);
      }
      int q;
      float2 h = TABLE ? table_project(c_scale(g, gscale), -a.n_levels, a.lev, q)
                       : slm_project_lv<LV>(g, a.n_levels, a.lev, q);
      if (OUT && row < H) {
        const size_t p = (size_t)row * W + n;
        if (po) po[p] = a.n_levels ? __ldg(&a.lev_phase[q]) : phase_0_2pi(h);
        if (lo) lo[p] = (uint8_t)q;
      }
      if (EXT && a.illum[k] && row < H) h = c_scale(h, __ldg(&a.illum[k][(size_t)row * W + n]));  // phase-only SLM
      if (a.cx) h = c_mul(h, c);
      v[s] = row < H ? h : make_float2(0.f, 0.f);
    });
  };
  if (EXT && a.n_levels < 0)
    pointwise(std::true_type{}, std::integral_constant<int, 0>{});
  else
    dispatch_levels(a.n_levels, [&](auto lv) { pointwise(std::false_type{}, lv); });
  FftRun<G, false, 1, typename K::Fwd, typename K::Fwd>::run(v, sm, t, a.tw_row);
  // tiled: re-derive the (run-time stride) store addresses rather than keep the load's live
  if (SQ)
    store_row_slots<K, K::RE, TW>(v, f, t, row0, W);
  else if (TW)
    store_row_slots<K, K::RE, TW>(v, opaque(f), t, row0, opaque(H));
  else
    store_row_slots<K, K::RE, TW>(v, f, t, row0, H);
}

// Bare row FFTs (propagation): in (times the chirp when PRE) -> FFT -> out.
template <int W, bool INV, bool PRE>
__global__ void __launch_bounds__(RowCfg<W>::NT) k_row_fft(const __grid_constant__ PassArgs a) {
  using K = RowCfg<W>;
  using G = typename K::G;
  extern __shared__ __align__(16) float2 sm[];
  const int t = threadIdx.x, k = blockIdx.y;
  const int row0 = blockIdx.x * K::ROWS;
  const int H = a.H;
  const float2* src = a.in[k];
  float2* dst = a.out[k];
  float2 v[K::V];
  for_each_slot<G, RFirst<typename K::Fwd>::value>(t, [&](int s, int b, int n) {
    const int row = row0 + b;
    float2 x = make_float2(0.f, 0.f);
    if (row < H) {
      x = __ldg(&src[(size_t)row * W + n]);
      if (PRE) x = c_mul(x, c_mul(__ldg(&a.cx[n]), __ldg(&a.cy[row])));
    }
    v[s] = x;
  });
  FftRun<G, INV, 1, typename K::Fwd>::run(v, sm, t, a.tw_row);
  for_each_slot<G, RLast<typename K::Fwd>::value>(t, [&](int s, int b, int n) {
    const int row = row0 + b;
    if (row < H) dst[(size_t)row * W + n] = v[s];
  });
}

// Offset of replay-plane pixel (n, col) (FFT order) in a caller's target: the same offset, or for
// targets in display order (DC at (H/2, W/2)) that of the ifftshifted pixel.
template <bool CENTRED>
__device__ __forceinline__ size_t target_index_t(const PassArgs& a, int n, int col) {
  if (CENTRED) {
    n += a.H / 2;
    n -= n >= a.H ? a.H : 0;
    col += a.W / 2;
    col -= col >= a.W ? a.W : 0;
  }
  return (size_t)n * a.W + col;
}
__device__ __forceinline__ size_t target_index(const PassArgs& a, int n, int col) {
  if (a.centred) {
    n += a.H / 2;
    n -= n >= a.H ? a.H : 0;
    col += a.W / 2;
    col -= col >= a.W ? a.W : 0;
  }
  return (size_t)n * a.W + col;
}

// ---------------------------------------------------------------- column passes

// GS column pass: forward column FFTs -> NMSE partials of I = |R|^2 against T = A^2 and
// amplitude replacement R' = A R / |R| -> inverse column FFTs.  With REPLACE = false only the NMSE
// is taken (last iteration) and the field is not written.  CT > 0: the field is tiled in column
// strips of width CT, each CTA's strip one contiguous block; CT = 0: row-major.  EXT instances
// also take the signal / noise regions of MRAF and HIO (the plain ones stay free of the per-pixel
// test).  HIO keeps its noise-region input X between passes: on the signal region X' = A_s Y / |Y|
// is the replacement itself, so X is stored for the noise region only.
template <int H, bool REPLACE, int CT, bool EXT = false, int PV = 0>
__global__ void __launch_bounds__(ColCfg<H, CT, PV>::NT, ColCfg<H, CT, PV>::MINB)
    k_col_gs(const __grid_constant__ PassArgs a) {
  constexpr bool TILED = CT > 0;
  using K = ColCfg<H, CT, PV>;
  using G = typename K::G;
  extern __shared__ __align__(16) float2 sm[];
  const int P = a.n_planes > 1 ? a.n_planes : 1;
  const int t = threadIdx.x, k = blockIdx.y / P, p = blockIdx.y % P;
  const int col0 = blockIdx.x * K::C;
  const int W = a.W;
  const int slot = a.class_slot[k];
  float2* f = a.field + ((size_t)slot * P + p) * H * W;
  const float* A = a.target[k * P + p];
  float* ts = reinterpret_cast<float*>(sm + G::SM_ELEMS);  // the strip's target, [n][C]
  if (a.ttile)
    prefetch_contig<H * K::C, K::NT>(ts, a.ttile + (((size_t)slot * P + p) * gridDim.x + blockIdx.x) * H * K::C);
  else
    prefetch_strip<H, K::C, K::NT>(ts, A, col0, W);
  pdl_wait_then_release();  // the targets were in place before the previous pass began
  // with several planes each plane's amplitude is brought to the energy of a unit-modulus field
  // (A_s = A sqrt(HW / sum A^2)); the common sqrt(HW) is dropped.  One plane needs no scale, except
  // under MRAF, where the signal region m A_s meets the noise region's (1 - m) R: on this
  // unnormalised forward transform (R_u = sqrt(HW) R) the signal amplitude is m A HW / sqrt(sum_S A^2).
  const bool mraf = EXT && a.mix > 0.f;
  const float esc = (P > 1 || mraf) ? (float)__ldcg(&a.stats[((size_t)slot * P + p) * 4 + 3]) : 1.f;
  const float amp_scale = mraf ? a.mix * (float)H * (float)W * esc : esc;
  // tiled: this strip is one contiguous [H][C] block
  float2* fs = TILED ? f + (size_t)blockIdx.x * H * K::C : f;
  float2* hx = EXT && a.hio ? a.hio + (((size_t)slot * P + p) * gridDim.x + blockIdx.x) * H * K::C : nullptr;
  float2 v[K::V];
  for_each_slot<G, K::RB>(t, [&](int s, int b, int n) {
    const int col = col0 + b;
    if (TILED)
      v[s] = fs[n * K::C + b];
    else
      v[s] = col < W ? f[n * W + col] : make_float2(0.f, 0.f);  // 32-bit offsets: H W < 2^31
  });
  FftRun<G, false, 1, typename K::Fwd, typename K::Fwd>::run(v, sm, t, a.tw_col);
  cp_async_wait_all();
  __syncthreads();
  float s_it = 0.f, s_ii = 0.f, s_tt = 0.f;
  for_each_slot<G, RLast<typename K::Fwd>::value>(t, [&](int s, int b, int n) {
    const float2 r = v[s];
    const float amp = ts[n * K::C + b];
    if (mraf && amp < 0.f) {  // noise region, outside the ROI NMSE
      if (REPLACE) {
        if (a.hio) {  // HIO: X' = X - beta Y, with X_0 = Y_0
          float2* xp = hx + n * K::C + b;
          const float2 x0 = a.iter == 0 ? r : __ldcg(xp);
          const float2 xn = make_float2(fmaf(-a.beta, r.x, x0.x), fmaf(-a.beta, r.y, x0.y));
          __stcg(xp, xn);
          v[s] = xn;
        } else {  // MRAF: R' = (1 - m) R
          v[s] = c_scale(r, 1.f - a.mix);
        }
      }
      return;
    }
    const float i2 = fmaf(r.x, r.x, r.y * r.y);
    const float tt = amp * amp;
    s_it = fmaf(i2, tt, s_it);
    s_ii = fmaf(i2, i2, s_ii);
    s_tt = fmaf(tt, tt, s_tt);
    if (REPLACE) {
      const float as = amp * amp_scale;
      v[s] = i2 > 0.f ? c_scale(r, as * rsqrtf(i2)) : make_float2(as, 0.f);
    }
  });
  if (REPLACE) {
    FftRun<G, true, 1, typename K::Inv, typename K::Fwd>::run(v, sm, t, a.tw_col);
    if (TILED) {
      float2* fo = opaque(fs);
      for_each_slot<G, K::RB>(t, [&](int s, int b, int n) { fo[n * K::C + b] = v[s]; });
    } else {
      const int Wo = opaque(W);
      float2* fo = opaque(f);
      for_each_slot<G, K::RB>(t, [&](int s, int b, int n) {
        const int col = col0 + b;
        if (col < Wo) fo[n * Wo + col] = v[s];
      });
    }
  }
  block_partials(s_it, s_ii, s_tt, a.partials + ((size_t)slot * P + p) * 3 * gridDim.x);
}

// Bare column FFTs (propagation), in place on out: FFT -> (times conj chirp when POST) -> scale.
template <int H, bool INV, bool POST>
__global__ void __launch_bounds__(ColCfg<H>::NT) k_col_fft(const __grid_constant__ PassArgs a) {
  using K = ColCfg<H>;
  using G = typename K::G;
  extern __shared__ __align__(16) float2 sm[];
  const int t = threadIdx.x, k = blockIdx.y;
  const int col0 = blockIdx.x * K::C;
  const int W = a.W;
  float2* f = a.out[k];
  float2 v[K::V];
  for_each_slot<G, RFirst<typename K::Fwd>::value>(t, [&](int s, int b, int n) {
    const int col = col0 + b;
    v[s] = col < W ? f[(size_t)n * W + col] : make_float2(0.f, 0.f);
  });
  FftRun<G, INV, 1, typename K::Fwd>::run(v, sm, t, a.tw_col);
  for_each_slot<G, RLast<typename K::Fwd>::value>(t, [&](int s, int b, int n) {
    const int col = col0 + b;
    if (col < W) {
      float2 x = c_scale(v[s], a.scale);
      if (POST) x = c_mulc(x, c_mul(__ldg(&a.cx[col]), __ldg(&a.cy[n])));
      f[(size_t)n * W + col] = x;
    }
  });
}

// ---------------------------------------------------------------- OSPR passes
//
// One-Step Phase-Retrieval (Cable, Buckley et al.; section "Algorithm Libraries",
// HoloGenAlgOSPRCuda).  Subframe s of target t: E = A exp(2 pi i u), u from Philox4x32-10 (counter
// (p, s, 0, 0), key (seed_lo, seed_hi ^ t)); h = binary(conj(c) F^-1(E)); I_acc += |F(h c)|^2;
// NMSE(I_acc, A^2) after each subframe.  Per subframe the field crosses HBM in two passes:
//   column pass: [finish s-1: forward column FFTs, I_acc += |R|^2, NMSE partials]
//                [start s: random-phase field, inverse column FFTs] -> field
//   row pass:    inverse row FFTs, conj chirp, binarise (bits out), chirp, forward row FFTs -> field

namespace ospr {
__device__ __forceinline__ float2 random_field(uint32_t p, int s, uint64_t seed, int target, float amp) {
  const uint4 x = philox4x32_10(make_uint4(p, (uint32_t)s, 0u, 0u),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32) ^ (uint32_t)target));
  const float u2 = (float)(x.x >> 8) * (1.0f / 8388608.0f);  // 2u
  float sn, cs;
  sincospif(u2, &sn, &cs);
  return make_float2(amp * cs, amp * sn);
}
}  // namespace ospr

// FINISH: the field holds rowFFT(h_{s-1} c); accumulate its replay intensity (ACC_READ: add to the
// stored sum, else start it) and write NMSE[s-1].  START: build subframe s and inverse-transform it.
// The strip's target comes from the tiled copy (a.ttile) and the accumulated intensity is kept per
// strip ([strip][H][C], a.acc), so both stream contiguously; both are prefetched into shared memory
// while the forward transform runs (measured on GB300, 1080 x 1920: the sum read where it is added
// left the pass waiting on global loads, 4.97 cycles per issue).
template <int H, bool FINISH, bool START>
__global__ void __launch_bounds__(ColCfg<H>::NT, ColCfg<H>::MINB) k_col_ospr(const __grid_constant__ PassArgs a) {
  using K = ColCfg<H>;
  using G = typename K::G;
  extern __shared__ __align__(16) float2 sm[];
  const int t = threadIdx.x, k = blockIdx.y;
  const int col0 = blockIdx.x * K::C;
  const int W = a.W;
  const int slot = a.class_slot[k];
  float2* f = a.field + (size_t)slot * H * W;
  const size_t strip = ((size_t)slot * gridDim.x + blockIdx.x) * H * K::C;
  float* acc = a.acc + strip;
  float* ts = reinterpret_cast<float*>(sm + G::SM_ELEMS);  // the strip's target, [n][C]
  float* as = ts + H * K::C;                                 // the strip's accumulated intensity
  static_assert((H * K::C) % 4 == 0, "16-byte strip copies");
  prefetch_contig<H * K::C, K::NT>(ts, a.ttile + strip);
  if (K::OSPR_ACC_SM && FINISH && a.acc_read) prefetch_contig<H * K::C, K::NT>(as, acc);
  float2 v[K::V];
  float s_it = 0.f, s_ii = 0.f, s_tt = 0.f;
  if (FINISH) {
    for_each_slot<G, K::RB>(t, [&](int s, int b, int n) {
      const int col = col0 + b;
      v[s] = col < W ? f[(size_t)n * W + col] : make_float2(0.f, 0.f);
    });
    FftRun<G, false, 1, typename K::Fwd>::run(v, sm, t, a.tw_col);
    cp_async_wait_all();
    __syncthreads();  // the target (and accumulated-intensity) strips have landed
    for_each_slot<G, RLast<typename K::Fwd>::value>(t, [&](int s, int b, int n) {
      const int col = col0 + b;
      if (col < W) {
        const int p = n * K::C + b;
        const float2 r = v[s];
        float i2 = fmaf(r.x, r.x, r.y * r.y);
        if (a.acc_read) i2 += K::OSPR_ACC_SM ? as[p] : acc[p];
        acc[p] = i2;
        const float amp = ts[p];
        const float tt = amp * amp;
        s_it = fmaf(i2, tt, s_it);
        s_ii = fmaf(i2, i2, s_ii);
        s_tt = fmaf(tt, tt, s_tt);
      }
    });
  }
  if (START) {
    // FINISH: its barrier above already saw the target land and the last exchange finish
    if (!FINISH) {
      cp_async_wait_all();
      __syncthreads();
    }
    for_each_slot<G, RFirst<typename K::Inv>::value>(t, [&](int s, int b, int n) {
      const int col = col0 + b;
      float2 e = make_float2(0.f, 0.f);
      if (col < W) {
        const uint32_t p = (uint32_t)((size_t)n * W + col);  // Philox counter: the pixel index
        e = ospr::random_field(p, a.iter, a.seed, a.item_index[k], ts[n * K::C + b]);
      }
      v[s] = e;
    });
    // the inverse runs the reversed plan: its first radix is the forward plan's last
    FftRun<G, true, 1, typename K::Inv>::run(v, sm, t, a.tw_col);
    const int Wo = opaque(W);
    float2* fo = opaque(f);
    for_each_slot<G, K::RB>(t, [&](int s, int b, int n) {
      const int col = col0 + b;
      if (col < Wo) fo[n * Wo + col] = v[s];
    });
  }
  if (FINISH) block_partials(s_it, s_ii, s_tt, a.partials + (size_t)slot * 3 * gridDim.x);
}

// OSPR row pass: inverse row FFTs, conj chirp, binary projection (bits written LSB-first, 32 pixels
// per word, when BITS and a bits pointer is set), chirp, forward row FFTs.
template <int W, bool BITS>
__global__ void __launch_bounds__(RowCfg<W>::NT) k_row_ospr(const __grid_constant__ PassArgs a) {
  using K = RowCfg<W>;
  using G = typename K::G;
  constexpr int WORDS = (W + 31) / 32;
  extern __shared__ __align__(16) float2 sm[];
  unsigned char* qs = reinterpret_cast<unsigned char*>(sm + G::SM_ELEMS);  // [ROWS][W] decisions
  const int t = threadIdx.x, k = blockIdx.y;
  const int row0 = blockIdx.x * K::ROWS;
  const int H = a.H;
  float2* f = a.field + (size_t)a.class_slot[k] * H * W;
  uint32_t* bits = BITS ? a.bits[k] : nullptr;
  if (a.finalize && blockIdx.x == 0 && t < 32) finalize_nmse(a, k);
  float2 v[K::V];
  for_each_slot<G, K::RE>(t, [&](int s, int b, int n) {
    const int row = row0 + b;
    v[s] = row < H ? f[(size_t)row * W + n] : make_float2(0.f, 0.f);
  });
  FftRun<G, true, 1, typename K::Inv>::run(v, sm, t, a.tw_row);
  for_each_slot<G, K::RM>(t, [&](int s, int b, int n) {
    const int row = row0 + b;
    float2 g = v[s];
    float2 c = make_float2(1.f, 0.f);
    if (a.cx && row < H) {
      c = c_mul(__ldg(&a.cx[n]), __ldg(&a.cy[row]));
      g = c_mulc(g, c);
    }
    const int q = (g.x < 0.f || (g.x == 0.f && g.y > 0.f)) ? 1 : 0;
    if (BITS) qs[b * W + n] = (unsigned char)q;
    float2 h = make_float2(q ? -1.f : 1.f, 0.f);
    if (a.cx) h = c_mul(h, c);
    v[s] = row < H ? h : make_float2(0.f, 0.f);
  });
  if (BITS) {
    __syncthreads();
    if (bits) {
      uint32_t* dst = bits + (size_t)a.iter * H * WORDS;
      for (int w = t; w < K::ROWS * WORDS; w += K::NT) {
        const int b = w / WORDS, word = w % WORDS;
        const int row = row0 + b;
        if (row >= H) continue;
        uint32_t x = 0;
        if constexpr (W % 16 == 0) {
          // the word's 32 decisions (bytes 0 / 1) as two 16-byte loads, four bits from each 32-bit
          // lane by shifts (measured on GB300, 1920-pixel rows: one byte load per decision was 8-way
          // bank-conflicted); with W a multiple of 16 a half-word is either whole or past the row
          auto pack4 = [](uint32_t u) { return (u | (u >> 7) | (u >> 14) | (u >> 21)) & 0xFu; };
          const uint4* src = reinterpret_cast<const uint4*>(qs + b * W + word * 32);
          const uint4 lo = src[0];
          x = pack4(lo.x) | pack4(lo.y) << 4 | pack4(lo.z) << 8 | pack4(lo.w) << 12;
          if (word * 32 + 16 < W) {
            const uint4 hi = src[1];
            x |= (pack4(hi.x) | pack4(hi.y) << 4 | pack4(hi.z) << 8 | pack4(hi.w) << 12) << 16;
          }
        } else {
          for (int i = 0; i < 32; ++i) {
            const int n = word * 32 + i;
            if (n < W) x |= (uint32_t)qs[b * W + n] << i;
          }
        }
        dst[(size_t)row * WORDS + word] = x;
      }
    }
  }
  FftRun<G, false, 1, typename K::Fwd>::run(v, sm, t, a.tw_row);
  for_each_slot<G, K::RE>(t, [&](int s, int b, int n) {
    const int row = row0 + b;
    if (row < H) f[(size_t)row * W + n] = v[s];
  });
}

// ---------------------------------------------------------------- planes: multi-plane GS and GD
//
// Multi-plane GS (averaged projections):
//   h <- P_SLM( sum_p conj(c_p) F^-1( A_p R_p / |R_p| ) ),  R_p = F(h c_p)
// is alternating projection in the product space of the P replay fields.  Gradient descent
// (Wirtinger) on phase phi with the optimal-scale intensity loss
//   L = (1/P) sum_p sum (s_p I_p - T_p)^2 / sum T_p^2,  I_p = |F(e^{i phi} c_p)|^2
// has dL/dphi = 2 Im(g conj(h)), g = sum_p conj(c_p) F^-1((2/P) s_p (s_p I_p - T_p)/sum T_p^2 U_p).
// With unnormalised transforms (U_u = sqrt(HW) U, s_u = s / HW) the same g is
// sum_p conj(c_p) F_u^-1((2/P) s_u (s_u I_u - T_p)/sum T_p^2 U_u): the HW factors cancel.

__device__ __forceinline__ float2 chirp_at(const PassArgs& a, int p, int n, int row) {
  return c_mul(__ldg(&a.cxp[p][n]), __ldg(&a.cyp[p][row]));
}

// Start of a multi-plane run: h = P_SLM(exp(i phi)) (PROJECT; else h = exp(i phi) exactly, for
// gradient descent), then for every plane p: forward row FFTs of h c_p -> field p.
// GD reads phi from a.phi[k]; GS from a.phase_in[k] or the seed.  TW > 0 (multi-plane GS): the
// field tiled in column strips of width TW.
// (Capped at 64 registers: measured on GB300, 2048^2 with 3 planes, 98 -> 73 us despite a few
// spills; k_row_mp keeps its 128 registers, which measured faster than any cap.)
template <int W, bool PROJECT, int TW = 0>
__global__ void __launch_bounds__(RowCfg<W, TW>::NT, RowCfg<W, TW>::MINB) k_row_mp_init(const __grid_constant__ PassArgs a) {
  using K = RowCfg<W, TW>;
  using G = typename K::G;
  constexpr int R0 = RFirst<typename K::Fwd>::value;
  extern __shared__ __align__(16) float2 sm[];
  const int P = a.n_planes > 1 ? a.n_planes : 1;
  const int t = threadIdx.x, k = blockIdx.y;
  const int row0 = blockIdx.x * K::ROWS;
  const int H = a.H;
  const int slot = a.class_slot[k];
  const float* ph = PROJECT ? a.phase_in[k] : a.phi[k];
  float* po = PROJECT ? a.phase_out[k] : nullptr;
  uint8_t* lo = PROJECT ? a.level_out[k] : nullptr;
  float2 h0[K::V];
  for_each_slot<G, R0>(t, [&](int s, int b, int n) {
    const int row = row0 + b;
    float2 h = make_float2(0.f, 0.f);
    if (row < H) {
      const size_t px = (size_t)row * W + n;
      float2 e;
      if (ph) {
        float sn, cs;
        sincosf(__ldg(&ph[px]), &sn, &cs);
        e = make_float2(cs, sn);
      } else {
        e = init_unit((uint32_t)px, a.seed, a.item_index[k]);
      }
      h = e;
      if (PROJECT) {
        int q;
        h = slm_project(e, a.n_levels, a.lev, q);
        if (po) po[px] = a.n_levels ? __ldg(&a.lev_phase[q]) : phase_0_2pi(h);
        if (lo) lo[px] = (uint8_t)q;
      }
    }
    h0[s] = h;
  });
  for (int p = 0; p < P; ++p) {
    float2 v[K::V];
    for_each_slot<G, R0>(t, [&](int s, int b, int n) {
      const int row = row0 + b;
      v[s] = (a.cxp[p] && row < H) ? c_mul(h0[s], chirp_at(a, p, n, row)) : h0[s];
    });
    FftRun<G, false, 1, typename K::Fwd>::run(v, sm, t, a.tw_row);
    float2* f = a.field + ((size_t)slot * P + p) * H * W;
    if constexpr (TW == 0) {
      for_each_slot<G, RLast<typename K::Fwd>::value>(t, [&](int s, int b, int n) {
        const int row = row0 + b;
        if (row < H) f[(size_t)row * W + n] = v[s];
      });
    } else {
      store_row_slots<K, RLast<typename K::Fwd>::value, TW>(v, f, t, row0, H);
    }
  }
}

// Multi-plane GS row pass: for every plane inverse row FFTs and conj chirp, summed; SLM projection
// of the sum (optionally written out); for every plane chirp and forward row FFTs.
// TW > 0: the field tiled in column strips of width TW (as the tiled GS row pass reads it).
// (Row-major instances have no minimum of CTAs per SM (0): ptxas then takes 128 registers at 2048,
// measured faster than any cap, and an explicit minimum of 1 made it take 191 and the pass 30 %
// longer.  Tiled instances are held to 2 CTAs of 256 threads per SM, which they would exceed.)
// SQ (square items on the tiled field): the strip height W at compile time, as in k_row_gs (the
// tiled instance's spills, 36-48 bytes per thread at 2048, vanish with it).
template <int W, bool OUT, int TW = 0, bool SQ = false>
__global__ void __launch_bounds__(RowCfg<W, TW>::NT, TW ? hg_max(1, 512 / RowCfg<W, TW>::NT) : 0)
    k_row_mp(const __grid_constant__ PassArgs a) {
  using K = RowCfg<W, TW>;
  using G = typename K::G;
  extern __shared__ __align__(16) float2 sm[];
  const int P = a.n_planes > 1 ? a.n_planes : 1;
  const int t = threadIdx.x, k = blockIdx.y;
  if (a.finalize && blockIdx.x == 0 && t < 32) finalize_nmse(a, k);
  const int row0 = blockIdx.x * K::ROWS;
  const int H = a.H;
  const int slot = a.class_slot[k];
  float2 g[K::V];
#pragma unroll
  for (int i = 0; i < K::V; ++i) g[i] = make_float2(0.f, 0.f);
  for (int p = 0; p < P; ++p) {
    float2 v[K::V];
    const float2* f = a.field + ((size_t)slot * P + p) * H * W;
    if constexpr (TW == 0) {
      for_each_slot<G, K::RE>(t, [&](int s, int b, int n) {
        const int row = row0 + b;
        v[s] = row < H ? f[(size_t)row * W + n] : make_float2(0.f, 0.f);
      });
    } else {
      load_row_slots<K, K::RE, TW>(v, f, t, row0, SQ ? W : H);
    }
    FftRun<G, true, 1, typename K::Inv>::run(v, sm, t, a.tw_row);
    for_each_slot<G, K::RM>(t, [&](int s, int b, int n) {
      const int row = row0 + b;
      const float2 x = (a.cxp[p] && row < H) ? c_mulc(v[s], chirp_at(a, p, n, row)) : v[s];
      g[s] = c_add(g[s], x);
    });
  }
  float* po = OUT ? a.phase_out[k] : nullptr;
  uint8_t* lo = OUT ? a.level_out[k] : nullptr;
  dispatch_levels(a.n_levels, [&](auto lv) {
    for_each_slot<G, K::RM>(t, [&](int s, int b, int n) {
      const int row = row0 + b;
      int q;
      const float2 h = slm_project_lv<decltype(lv)::value>(g[s], a.n_levels, a.lev, q);
      if (OUT && row < H) {
        const size_t px = (size_t)row * W + n;
        if (po) po[px] = a.n_levels ? __ldg(&a.lev_phase[q]) : phase_0_2pi(h);
        if (lo) lo[px] = (uint8_t)q;
      }
      g[s] = row < H ? h : make_float2(0.f, 0.f);
    });
  });
  for (int p = 0; p < P; ++p) {
    float2 v[K::V];
    for_each_slot<G, K::RM>(t, [&](int s, int b, int n) {
      const int row = row0 + b;
      v[s] = (a.cxp[p] && row < H) ? c_mul(g[s], chirp_at(a, p, n, row)) : g[s];
    });
    FftRun<G, false, 1, typename K::Fwd>::run(v, sm, t, a.tw_row);
    float2* f = a.field + ((size_t)slot * P + p) * H * W;
    if constexpr (TW == 0) {
      for_each_slot<G, K::RE>(t, [&](int s, int b, int n) {
        const int row = row0 + b;
        if (row < H) f[(size_t)row * W + n] = v[s];
      });
    } else {
      store_row_slots<K, K::RE, TW>(v, f, t, row0, SQ ? W : H);
    }
  }
}

// Gradient-descent column pass, one (item, plane) per blockIdx.y.  Forward (BWD = false): the loss
// statistics sum I T, sum I^2, sum T^2 of U = F(h c_p) (I = |U|^2, T the target intensity); the last
// block stores s_u, sum T^2 and the plane loss, and the last plane the mean loss.  Backward: the
// adjoint field (2/P) s_u (s_u I - T) / sum T^2 U, inverse column FFTs -> field p (in place).
// SQ (square items): the row length H at compile time, so the strided field and target accesses
// take constant offsets (measured on GB300, 2048^2 with 3 planes: 99 -> 94 and 103 -> 100 us).
template <int H, bool BWD, bool SQ = false>
__global__ void __launch_bounds__(ColCfg<H>::NT, ColCfg<H>::MINB) k_col_gd(const __grid_constant__ PassArgs a) {
  using K = ColCfg<H>;
  using G = typename K::G;
  extern __shared__ __align__(16) float2 sm[];
  const int P = a.n_planes > 1 ? a.n_planes : 1;
  const int t = threadIdx.x, k = blockIdx.y / P, p = blockIdx.y % P;
  const int col0 = blockIdx.x * K::C;
  const int W = SQ ? H : a.W;
  const int slot = a.class_slot[k];
  const int sp = slot * P + p;
  float2* f = a.field + (size_t)sp * H * W;
  const float* T = a.target[k * P + p];
  float2 v[K::V];
  for_each_slot<G, K::RB>(t, [&](int s, int b, int n) {
    const int col = col0 + b;
    v[s] = col < W ? f[(size_t)n * W + col] : make_float2(0.f, 0.f);
  });
  FftRun<G, false, 1, typename K::Fwd>::run(v, sm, t, a.tw_col);
  // display-order targets: the test is taken once per launch, outside the pixel loops (measured: a
  // per-pixel test cost the gradient-descent step 10 % at 2048^2, 3 planes)
  if (!BWD) {
    float s_it = 0.f, s_ii = 0.f, s_tt = 0.f;
    auto sums = [&](auto centred) {
      for_each_slot<G, RLast<typename K::Fwd>::value>(t, [&](int s, int b, int n) {
        const int col = col0 + b;
        if (col < W) {
          const float2 u = v[s];
          const float i2 = fmaf(u.x, u.x, u.y * u.y);
          const float tt = __ldg(&T[decltype(centred)::value ? target_index_t<true>(a, n, col) : (size_t)n * W + col]);
          s_it = fmaf(i2, tt, s_it);
          s_ii = fmaf(i2, i2, s_ii);
          s_tt = fmaf(tt, tt, s_tt);
        }
      });
    };
    if (a.centred)
      sums(std::true_type{});
    else
      sums(std::false_type{});
    block_partials(s_it, s_ii, s_tt, a.partials + (size_t)sp * 3 * gridDim.x);
  } else {
    const double* st = a.stats + (size_t)sp * 4;
    const float su = (float)__ldcg(&st[0]);
    const float coef = (float)(2.0 / P * __ldcg(&st[0]) / (__ldcg(&st[1]) > 0.0 ? __ldcg(&st[1]) : 1.0));
    auto adjoint = [&](auto centred) {
      for_each_slot<G, RLast<typename K::Fwd>::value>(t, [&](int s, int b, int n) {
        const int col = col0 + b;
        float2 gi = make_float2(0.f, 0.f);
        if (col < W) {
          const float2 u = v[s];
          const float i2 = fmaf(u.x, u.x, u.y * u.y);
          const float tt = __ldg(&T[decltype(centred)::value ? target_index_t<true>(a, n, col) : (size_t)n * W + col]);
          gi = c_scale(u, coef * fmaf(su, i2, -tt));
        }
        v[s] = gi;
      });
    };
    if (a.centred)
      adjoint(std::true_type{});
    else
      adjoint(std::false_type{});
    FftRun<G, true, 1, typename K::Inv>::run(v, sm, t, a.tw_col);
    const int Wo = SQ ? W : opaque(W);
    float2* fo = SQ ? f : opaque(f);
    for_each_slot<G, K::RB>(t, [&](int s, int b, int n) {
      const int col = col0 + b;
      if (col < Wo) fo[n * Wo + col] = v[s];
    });
  }
}

// Gradient-descent backward row pass: g = sum_p conj(c_p) (inverse row FFTs of field p);
// dL/dphi = 2 Im(g conj(e^{i phi})) (times *grad_scale); optional gradient out and Adam update of
// phi, m, v in place.
// (Capped at 64 registers: measured on GB300, 2048^2 with 3 planes, 145 -> 96 us despite spills.)
template <int W>
__global__ void __launch_bounds__(RowCfg<W>::NT, RowCfg<W>::MINB) k_row_gd_bwd(const __grid_constant__ PassArgs a) {
  using K = RowCfg<W>;
  using G = typename K::G;
  extern __shared__ __align__(16) float2 sm[];
  const int P = a.n_planes > 1 ? a.n_planes : 1;
  const int t = threadIdx.x, k = blockIdx.y;
  const int row0 = blockIdx.x * K::ROWS;
  const int H = a.H;
  const int slot = a.class_slot[k];
  float2 g[K::V];
#pragma unroll
  for (int i = 0; i < K::V; ++i) g[i] = make_float2(0.f, 0.f);
  for (int p = 0; p < P; ++p) {
    const float2* f = a.field + ((size_t)slot * P + p) * H * W;
    float2 v[K::V];
    for_each_slot<G, K::RE>(t, [&](int s, int b, int n) {
      const int row = row0 + b;
      v[s] = row < H ? f[(size_t)row * W + n] : make_float2(0.f, 0.f);
    });
    FftRun<G, true, 1, typename K::Inv>::run(v, sm, t, a.tw_row);
    for_each_slot<G, K::RM>(t, [&](int s, int b, int n) {
      const int row = row0 + b;
      const float2 x = (a.cxp[p] && row < H) ? c_mulc(v[s], chirp_at(a, p, n, row)) : v[s];
      g[s] = c_add(g[s], x);
    });
  }
  const float gs = a.grad_scale ? __ldg(a.grad_scale) : 1.f;
  float* phi = a.phi[k];
  float* gout = a.grad[k];
  float* m = a.adam_m[k];
  float* vv = a.adam_v[k];
  for_each_slot<G, K::RM>(t, [&](int s, int b, int n) {
    const int row = row0 + b;
    if (row >= H) return;
    const size_t px = (size_t)row * W + n;
    const float ph = phi[px];
    float sn, cs;
    sincosf(ph, &sn, &cs);
    // Im(g conj(h)) with h = (cs, sn)
    const float gr = 2.f * gs * fmaf(g[s].y, cs, -g[s].x * sn);
    if (gout) gout[px] = gr;
    if (a.adam) {
      const float m1 = fmaf(a.beta1, m[px], (1.f - a.beta1) * gr);
      const float v1 = fmaf(a.beta2, vv[px], (1.f - a.beta2) * gr * gr);
      m[px] = m1;
      vv[px] = v1;
      phi[px] = ph - a.lr * (m1 / a.bc1) / (sqrtf(v1 / a.bc2) + a.eps);
    }
  });
}

// ---------------------------------------------------------------- whole run in one cluster

// GS for small holograms (N x N) with the whole run in one launch: one thread-block cluster of CL
// CTAs per item, the field resident in the cluster's shared memory -- CTA r holds rows
// [r N / CL, (r + 1) N / CL) -- so nothing but the target (once) and the outputs crosses HBM.  The
// column phase of CTA r transforms columns [r N / CL, (r + 1) N / CL) of every CTA's rows, read
// and written back through distributed shared memory; the row phase works on the CTA's own rows.
// The arithmetic per element is that of the two-pass kernels (same radix plans, twiddles and
// pointwise steps); only the NMSE partial sums are grouped per CTA.
template <int N, int CL>
struct ClusterCfg {
  static constexpr int RL = N / CL;  // rows per CTA = columns per CTA in the column phase
  using Fwd = typename PlanFor<N>::type;
  using Inv = typename RRev<Fwd>::type;
  static constexpr int NT = pick_threads<Fwd>(N, RL, value_budget(N), 1024);
  using GR = Geo<N, RL, NT, false>;  // row tile: the CTA's RL rows
  using GC = Geo<N, RL, NT, true>;   // column strip: RL columns of length N
  static constexpr int V = hg_max(MaxV<GR, Fwd>::value, MaxV<GC, Fwd>::value);
  static constexpr int XCH = hg_max(GR::SM_ELEMS, GC::SM_ELEMS);  // exchange float2 slots
  static constexpr int FIELD = RL * N;                            // the CTA's rows, float2
  static constexpr int PARTS = round_up(3 * CL, 2);               // rank 0: NMSE partials, float2
  static constexpr int SMEM = (XCH + FIELD + PARTS) * 8 + N * RL * 4;  // + the target strip
  static constexpr bool FEASIBLE = N % CL == 0 && RL >= 1 &&
                                   RValues<Fwd>::max_values(N, RL, NT) <= value_budget(N) &&
                                   SMEM <= 227 * 1024;
};

template <int N, int CL>
__global__ void __launch_bounds__(ClusterCfg<N, CL>::NT, 1) k_gs_cluster(const __grid_constant__ PassArgs a) {
  using K = ClusterCfg<N, CL>;
  using GR = typename K::GR;
  using GC = typename K::GC;
  using Fwd = typename K::Fwd;
  using Inv = typename K::Inv;
  constexpr int RL = K::RL;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) float2 sm[];
  float2* xs = sm;                                          // FFT exchange
  float2* fld = sm + K::XCH;                                // this CTA's rows [RL][N]
  float2* parts = fld + K::FIELD;                           // rank 0: [CL][3] (hi, lo) partials
  float* ts = reinterpret_cast<float*>(parts + K::PARTS);   // target columns [N][RL] of this CTA
  const int t = threadIdx.x, k = blockIdx.y;
  const int rank = (int)cluster.block_rank();  // == blockIdx.x (gridDim.x == CL)
  const int row0 = rank * RL, col0 = rank * RL;
  const int n_iter = a.n_iter;
  const float* A = a.target[k];
  for (int i = t; i < N * RL; i += K::NT) ts[i] = __ldg(&A[target_index(a, i / RL, col0 + i % RL)]);
  float2* part0 = cluster.map_shared_rank(parts, 0);
  float* po = a.phase_out[k];
  uint8_t* lo = a.level_out[k];
  const float* ph = a.phase_in[k];

  // h_0 on this CTA's rows (written out when there is no iteration), forward row FFTs
  float2 v[K::V];
  for_each_slot<GR, RFirst<Fwd>::value>(t, [&](int s, int b, int n) {
    const int row = row0 + b;
    const size_t p = (size_t)row * N + n;
    float2 e;
    if (ph) {
      float sn, cs;
      sincosf(__ldg(&ph[p]), &sn, &cs);
      e = make_float2(cs, sn);
    } else {
      e = init_unit((uint32_t)p, a.seed, a.item_index[k]);
    }
    int q;
    float2 h = slm_project(e, a.n_levels, a.lev, q);
    if (n_iter == 0) {
      if (po) po[p] = a.n_levels ? __ldg(&a.lev_phase[q]) : phase_0_2pi(h);
      if (lo) lo[p] = (uint8_t)q;
    }
    if (a.cx) h = c_mul(h, c_mul(__ldg(&a.cx[n]), __ldg(&a.cy[row])));
    v[s] = h;
  });
  FftRun<GR, false, 1, Fwd>::run(v, xs, t, a.tw_row);
  for_each_slot<GR, RLast<Fwd>::value>(t, [&](int s, int b, int n) { fld[b * N + n] = v[s]; });
  cluster.sync();

  for (int it = 0;; ++it) {
    const bool replace = it < n_iter;
    // column phase: NMSE of h_it, and unless last, replacement and inverse column FFTs
    for_each_slot<GC, RFirst<Fwd>::value>(t, [&](int s, int b, int n) {
      const float2* src = cluster.map_shared_rank(fld, n / RL);
      v[s] = src[(n % RL) * N + col0 + b];
    });
    FftRun<GC, false, 1, Fwd>::run(v, xs, t, a.tw_col);
    float s_it = 0.f, s_ii = 0.f, s_tt = 0.f;
    for_each_slot<GC, RLast<Fwd>::value>(t, [&](int s, int b, int n) {
      const float2 r = v[s];
      const float amp = ts[n * RL + b];
      const float i2 = fmaf(r.x, r.x, r.y * r.y);
      const float tt = amp * amp;
      s_it = fmaf(i2, tt, s_it);
      s_ii = fmaf(i2, i2, s_ii);
      s_tt = fmaf(tt, tt, s_tt);
      v[s] = i2 > 0.f ? c_scale(r, amp * rsqrtf(i2)) : make_float2(amp, 0.f);
    });
    block_partials(s_it, s_ii, s_tt, part0);
    if (replace) {
      FftRun<GC, true, 1, Inv>::run(v, xs, t, a.tw_col);
      for_each_slot<GC, RLast<Inv>::value>(t, [&](int s, int b, int n) {
        float2* dst = cluster.map_shared_rank(fld, n / RL);
        dst[(n % RL) * N + col0 + b] = v[s];
      });
    }
    cluster.sync();  // field and partials of the column phase in place
    if (rank == 0 && t < 32) {
      double tot[3];
      sum_partials(parts, CL, tot);
      if (t == 0 && a.nmse) a.nmse[(size_t)a.item_index[k] * a.nmse_stride + it] = (float)nmse_of(tot);
    }
    if (!replace) break;
    // row phase on this CTA's rows: inverse row FFTs, SLM projection, forward row FFTs
    for_each_slot<GR, RFirst<Inv>::value>(t, [&](int s, int b, int n) { v[s] = fld[b * N + n]; });
    FftRun<GR, true, 1, Inv>::run(v, xs, t, a.tw_row);
    const bool out = it == n_iter - 1;
    dispatch_levels(a.n_levels, [&](auto lv) {
      for_each_slot<GR, RFirst<Fwd>::value>(t, [&](int s, int b, int n) {
        const int row = row0 + b;
        float2 g = v[s];
        float2 c = make_float2(1.f, 0.f);
        if (a.cx) {
          c = c_mul(__ldg(&a.cx[n]), __ldg(&a.cy[row]));
          g = c_mulc(g, c);
        }
        int q;
        float2 h = slm_project_lv<decltype(lv)::value>(g, a.n_levels, a.lev, q);
        if (out) {
          const size_t p = (size_t)row * N + n;
          if (po) po[p] = a.n_levels ? __ldg(&a.lev_phase[q]) : phase_0_2pi(h);
          if (lo) lo[p] = (uint8_t)q;
        }
        if (a.cx) h = c_mul(h, c);
        v[s] = h;
      });
    });
    FftRun<GR, false, 1, Fwd>::run(v, xs, t, a.tw_row);
    for_each_slot<GR, RLast<Fwd>::value>(t, [&](int s, int b, int n) { fld[b * N + n] = v[s]; });
    cluster.sync();  // rows in place before the next column phase reads them
  }
}

}  // namespace hg
