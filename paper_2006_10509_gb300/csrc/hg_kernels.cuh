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

#include "hg_fft.cuh"

namespace hg {

constexpr int kMaxBatch = 32;  // items per launch (a size class with more items is launched in chunks)

__host__ __device__ constexpr int hg_max(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int hg_min(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int round_up(int a, int m) { return (a + m - 1) / m * m; }

// Row tile: ROWS rows of length W, about 16 values per thread.
template <int W>
struct RowCfg {
  static constexpr int ROWS = hg_max(1, 4096 / W);
  static constexpr int NT = hg_min(512, hg_max(32, round_up(ROWS * W / 16, 32)));
  using G = Geo<W, ROWS, NT, false>;
  using Fwd = typename PlanFor<W>::type;
  using Inv = typename RRev<Fwd>::type;
  static constexpr int RE = RLast<Fwd>::value;   // radix of the global load/store stages
  static constexpr int RM = RFirst<Fwd>::value;  // radix of the pointwise step between the FFTs
  static constexpr int V = MaxV<G, Fwd>::value;
  static constexpr int SMEM = ROWS * W * 8;
};

// Column strip: C columns of length H, about 16 values per thread.
template <int H>
struct ColCfg {
  static constexpr int C = H >= 4096 ? 4 : (H >= 640 ? 8 : 16);
  static constexpr int NT = hg_min(1024, hg_max(32, round_up(C * H / 16, 32)));
  using G = Geo<H, C, NT, true>;
  using Fwd = typename PlanFor<H>::type;
  using Inv = typename RRev<Fwd>::type;
  static constexpr int RB = RFirst<Fwd>::value;  // radix of the global load/store stage
  static constexpr int V = MaxV<G, Fwd>::value;
  static constexpr int SMEM = C * H * 8;
};

// ---------------------------------------------------------------- launch arguments

// Per-launch argument block: up to kMaxBatch items of one size class.  Plan-owned buffers
// (field, chirps, partials) are per class; caller buffers are per item.
struct PassArgs {
  int n_items;
  int H, W;
  int n_levels;            // 0 continuous, 2 binary, N >= 3 N-level
  int iter;                // iteration index written by column passes (NMSE slot)
  int nmse_stride;         // floats between items in nmse_out (n_iter + 1)
  const float2* tw_row;    // twiddles exp(-2 pi i t / W), t < W
  const float2* tw_col;    // twiddles exp(-2 pi i t / H), t < H
  const float2* cx;        // Fresnel chirp along a row (W), nullptr for Fourier
  const float2* cy;        // Fresnel chirp along a column (H)
  const float2* lev;       // level field exp(2 pi i q / N), q < N
  const float* lev_phase;  // level phase 2 pi q / N
  float2* field;           // class field buffer: item k at field + k * H * W
  double* partials;        // class partial sums: item k at partials + k * 3 * blocks_x
  unsigned* counters;      // class block counters: one per item
  float* nmse;             // nmse_out of the run (device) or nullptr
  uint64_t seed;           // starting-phase seed when phase_in is null
  float scale;             // output scale (bare propagation)
  int item_index[kMaxBatch];  // plan item index (nmse row, Philox key)
  int class_slot[kMaxBatch];  // slot in the class buffers
  const float* target[kMaxBatch];
  const float* phase_in[kMaxBatch];
  float* phase_out[kMaxBatch];
  uint8_t* level_out[kMaxBatch];
  const float2* in[kMaxBatch];  // bare propagation input
  float2* out[kMaxBatch];       // bare propagation output
  // OSPR
  float* acc;                   // class accumulated-intensity buffer: item k at acc + k * H * W
  int acc_read;                 // 1: add to the stored sum, 0: start it
  uint32_t* bits[kMaxBatch];    // [S][H][ceil(W/32)] LSB-first hologram bits, or nullptr
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
__device__ __forceinline__ float2 slm_project(float2 g, int n_levels, const float2* __restrict__ lev, int& q) {
  if (n_levels == 0) {
    const float m2 = fmaf(g.x, g.x, g.y * g.y);
    q = 0;
    if (m2 > 0.f) {
      const float r = rsqrtf(m2);
      return make_float2(g.x * r, g.y * r);
    }
    return make_float2(1.f, 0.f);
  }
  if (n_levels == 2) {
    // arg in [pi/2, 3pi/2) -> pi; on Re g = 0, Im > 0 goes to pi and Im < 0 to 0
    q = (g.x < 0.f || (g.x == 0.f && g.y > 0.f)) ? 1 : 0;
    return make_float2(q ? -1.f : 1.f, 0.f);
  }
  const float a = atan2f(g.y, g.x);  // (-pi, pi]
  float t = a * ((float)n_levels * 0.15915494309189533577f);
  if (t < 0.f) t += (float)n_levels;
  int qq = (int)floorf(t + 0.5f);
  if (qq >= n_levels) qq -= n_levels;
  q = qq;
  return __ldg(&lev[qq]);
}

__device__ __forceinline__ float phase_0_2pi(float2 h) {
  float a = atan2f(h.y, h.x);
  if (a < 0.f) {
    a += 6.28318530717958647693f;
    if (a >= 6.28318530717958647693f) a = 0.f;
  }
  return a;
}

// Block-wide (ab, bb, tt) sums in double, written as this block's partials; the last block to
// arrive adds all partials in block order (deterministic) and writes
// NMSE = 1 - ab^2 / (bb tt) to *dst.  No block waits on another.
__device__ __forceinline__ void nmse_reduce(float ab, float bb, float tt, double* __restrict__ part,
                                            unsigned* counter, int nblk, float* dst) {
  __shared__ double red[3][32];
  __shared__ bool is_last;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = (blockDim.x + 31) >> 5;
  double a = ab, b = bb, c = tt;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  if (lane == 0) {
    red[0][warp] = a;
    red[1][warp] = b;
    red[2][warp] = c;
  }
  __syncthreads();
  if (warp == 0) {
    a = lane < nw ? red[0][lane] : 0.0;
    b = lane < nw ? red[1][lane] : 0.0;
    c = lane < nw ? red[2][lane] : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
      c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
      part[3 * blockIdx.x + 0] = a;
      part[3 * blockIdx.x + 1] = b;
      part[3 * blockIdx.x + 2] = c;
      __threadfence();
      const unsigned prev = atomicAdd(counter, 1u);
      is_last = (prev == (unsigned)nblk - 1u);
    }
  }
  __syncthreads();
  if (is_last && warp == 0) {
    __threadfence();
    a = b = c = 0.0;
    for (int k = lane; k < nblk; k += 32) {
      a += __ldcg(&part[3 * k + 0]);
      b += __ldcg(&part[3 * k + 1]);
      c += __ldcg(&part[3 * k + 2]);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
      c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
      double e = 1.0;
      if (b > 0.0 && c > 0.0) e = 1.0 - (a * a) / (b * c);
      if (dst) *dst = (float)e;
      *counter = 0u;
    }
  }
}

// ---------------------------------------------------------------- row passes

// GS prologue: h0 = P_SLM(exp(i phi0)) (phi0 given, or drawn from the seed), times the chirp,
// forward row FFTs -> field.  h0 is written out when phase_out / level_out are set.
template <int W>
__global__ void __launch_bounds__(RowCfg<W>::NT) k_row_init(const __grid_constant__ PassArgs a) {
  using K = RowCfg<W>;
  using G = typename K::G;
  extern __shared__ float2 sm[];
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
      h = slm_project(e, a.n_levels, a.lev, q);
      if (po) po[p] = a.n_levels ? __ldg(&a.lev_phase[q]) : phase_0_2pi(h);
      if (lo) lo[p] = (uint8_t)q;
      if (a.cx) h = c_mul(h, c_mul(__ldg(&a.cx[n]), __ldg(&a.cy[row])));
    }
    v[s] = h;
  });
  FftRun<G, false, 1, typename K::Fwd>::run(v, sm, t, a.tw_row);
  for_each_slot<G, RLast<typename K::Fwd>::value>(t, [&](int s, int b, int n) {
    const int row = row0 + b;
    if (row < H) f[(size_t)row * W + n] = v[s];
  });
}

// GS row pass: inverse row FFTs, conj chirp, SLM projection (optionally written out), chirp,
// forward row FFTs.
template <int W, bool OUT>
__global__ void __launch_bounds__(RowCfg<W>::NT) k_row_gs(const __grid_constant__ PassArgs a) {
  using K = RowCfg<W>;
  using G = typename K::G;
  extern __shared__ float2 sm[];
  const int t = threadIdx.x, k = blockIdx.y;
  const int row0 = blockIdx.x * K::ROWS;
  const int H = a.H;
  float2* f = a.field + (size_t)a.class_slot[k] * H * W;
  float2 v[K::V];
  for_each_slot<G, K::RE>(t, [&](int s, int b, int n) {
    const int row = row0 + b;
    v[s] = row < H ? f[(size_t)row * W + n] : make_float2(0.f, 0.f);
  });
  FftRun<G, true, 1, typename K::Inv>::run(v, sm, t, a.tw_row);
  float* po = OUT ? a.phase_out[k] : nullptr;
  uint8_t* lo = OUT ? a.level_out[k] : nullptr;
  for_each_slot<G, K::RM>(t, [&](int s, int b, int n) {
    const int row = row0 + b;
    float2 g = v[s];
    float2 c = make_float2(1.f, 0.f);
    if (a.cx && row < H) {
      c = c_mul(__ldg(&a.cx[n]), __ldg(&a.cy[row]));
      g = c_mulc(g, c);
    }
    int q;
    float2 h = slm_project(g, a.n_levels, a.lev, q);
    if (OUT && row < H) {
      const size_t p = (size_t)row * W + n;
      if (po) po[p] = a.n_levels ? __ldg(&a.lev_phase[q]) : phase_0_2pi(h);
      if (lo) lo[p] = (uint8_t)q;
    }
    if (a.cx) h = c_mul(h, c);
    v[s] = row < H ? h : make_float2(0.f, 0.f);
  });
  FftRun<G, false, 1, typename K::Fwd>::run(v, sm, t, a.tw_row);
  for_each_slot<G, K::RE>(t, [&](int s, int b, int n) {
    const int row = row0 + b;
    if (row < H) f[(size_t)row * W + n] = v[s];
  });
}

// Bare row FFTs (propagation): in (times the chirp when PRE) -> FFT -> out.
template <int W, bool INV, bool PRE>
__global__ void __launch_bounds__(RowCfg<W>::NT) k_row_fft(const __grid_constant__ PassArgs a) {
  using K = RowCfg<W>;
  using G = typename K::G;
  extern __shared__ float2 sm[];
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

// ---------------------------------------------------------------- column passes

// GS column pass: forward column FFTs -> NMSE partials of I = |R|^2 against T = A^2 and
// amplitude replacement R' = A R / |R| -> inverse column FFTs.  With REPLACE = false only the NMSE
// is taken (last iteration) and the field is not written.
template <int H, bool REPLACE>
__global__ void __launch_bounds__(ColCfg<H>::NT) k_col_gs(const __grid_constant__ PassArgs a) {
  using K = ColCfg<H>;
  using G = typename K::G;
  extern __shared__ float2 sm[];
  const int t = threadIdx.x, k = blockIdx.y;
  const int col0 = blockIdx.x * K::C;
  const int W = a.W;
  const int slot = a.class_slot[k];
  float2* f = a.field + (size_t)slot * H * W;
  const float* A = a.target[k];
  float2 v[K::V];
  for_each_slot<G, K::RB>(t, [&](int s, int b, int n) {
    const int col = col0 + b;
    v[s] = col < W ? f[(size_t)n * W + col] : make_float2(0.f, 0.f);
  });
  FftRun<G, false, 1, typename K::Fwd>::run(v, sm, t, a.tw_col);
  float s_it = 0.f, s_ii = 0.f, s_tt = 0.f;
  for_each_slot<G, RLast<typename K::Fwd>::value>(t, [&](int s, int b, int n) {
    const int col = col0 + b;
    const float2 r = v[s];
    const float amp = col < W ? __ldg(&A[(size_t)n * W + col]) : 0.f;
    const float i2 = fmaf(r.x, r.x, r.y * r.y);
    const float tt = amp * amp;
    s_it = fmaf(i2, tt, s_it);
    s_ii = fmaf(i2, i2, s_ii);
    s_tt = fmaf(tt, tt, s_tt);
    if (REPLACE) v[s] = i2 > 0.f ? c_scale(r, amp * rsqrtf(i2)) : make_float2(amp, 0.f);
  });
  if (REPLACE) {
    FftRun<G, true, 1, typename K::Inv>::run(v, sm, t, a.tw_col);
    for_each_slot<G, K::RB>(t, [&](int s, int b, int n) {
      const int col = col0 + b;
      if (col < W) f[(size_t)n * W + col] = v[s];
    });
  }
  float* dst = a.nmse ? a.nmse + (size_t)a.item_index[k] * a.nmse_stride + a.iter : nullptr;
  nmse_reduce(s_it, s_ii, s_tt, a.partials + (size_t)slot * 3 * gridDim.x, a.counters + slot, gridDim.x, dst);
}

// Bare column FFTs (propagation), in place on out: FFT -> (times conj chirp when POST) -> scale.
template <int H, bool INV, bool POST>
__global__ void __launch_bounds__(ColCfg<H>::NT) k_col_fft(const __grid_constant__ PassArgs a) {
  using K = ColCfg<H>;
  using G = typename K::G;
  extern __shared__ float2 sm[];
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
template <int H, bool FINISH, bool START>
__global__ void __launch_bounds__(ColCfg<H>::NT) k_col_ospr(const __grid_constant__ PassArgs a) {
  using K = ColCfg<H>;
  using G = typename K::G;
  extern __shared__ float2 sm[];
  const int t = threadIdx.x, k = blockIdx.y;
  const int col0 = blockIdx.x * K::C;
  const int W = a.W;
  const int slot = a.class_slot[k];
  float2* f = a.field + (size_t)slot * H * W;
  float* acc = a.acc + (size_t)slot * H * W;
  const float* A = a.target[k];
  float2 v[K::V];
  float s_it = 0.f, s_ii = 0.f, s_tt = 0.f;
  if (FINISH) {
    for_each_slot<G, K::RB>(t, [&](int s, int b, int n) {
      const int col = col0 + b;
      v[s] = col < W ? f[(size_t)n * W + col] : make_float2(0.f, 0.f);
    });
    FftRun<G, false, 1, typename K::Fwd>::run(v, sm, t, a.tw_col);
    for_each_slot<G, RLast<typename K::Fwd>::value>(t, [&](int s, int b, int n) {
      const int col = col0 + b;
      if (col < W) {
        const size_t p = (size_t)n * W + col;
        const float2 r = v[s];
        float i2 = fmaf(r.x, r.x, r.y * r.y);
        if (a.acc_read) i2 += acc[p];
        acc[p] = i2;
        const float amp = __ldg(&A[p]);
        const float tt = amp * amp;
        s_it = fmaf(i2, tt, s_it);
        s_ii = fmaf(i2, i2, s_ii);
        s_tt = fmaf(tt, tt, s_tt);
      }
    });
  }
  if (START) {
    if (FINISH) __syncthreads();  // the forward transform's last exchange is done with sm
    for_each_slot<G, RFirst<typename K::Inv>::value>(t, [&](int s, int b, int n) {
      const int col = col0 + b;
      float2 e = make_float2(0.f, 0.f);
      if (col < W) {
        const uint32_t p = (uint32_t)((size_t)n * W + col);
        e = ospr::random_field(p, a.iter, a.seed, a.item_index[k], __ldg(&A[p]));
      }
      v[s] = e;
    });
    // the inverse runs the reversed plan: its first radix is the forward plan's last
    FftRun<G, true, 1, typename K::Inv>::run(v, sm, t, a.tw_col);
    for_each_slot<G, K::RB>(t, [&](int s, int b, int n) {
      const int col = col0 + b;
      if (col < W) f[(size_t)n * W + col] = v[s];
    });
  }
  if (FINISH) {
    float* dst = a.nmse ? a.nmse + (size_t)a.item_index[k] * a.nmse_stride + (a.iter - 1) : nullptr;
    nmse_reduce(s_it, s_ii, s_tt, a.partials + (size_t)slot * 3 * gridDim.x, a.counters + slot, gridDim.x, dst);
  }
}

// OSPR row pass: inverse row FFTs, conj chirp, binary projection (bits written LSB-first, 32 pixels
// per word, when BITS and a bits pointer is set), chirp, forward row FFTs.
template <int W, bool BITS>
__global__ void __launch_bounds__(RowCfg<W>::NT) k_row_ospr(const __grid_constant__ PassArgs a) {
  using K = RowCfg<W>;
  using G = typename K::G;
  constexpr int WORDS = (W + 31) / 32;
  extern __shared__ float2 sm[];
  unsigned char* qs = reinterpret_cast<unsigned char*>(sm + K::ROWS * W);  // [ROWS][W] decisions
  const int t = threadIdx.x, k = blockIdx.y;
  const int row0 = blockIdx.x * K::ROWS;
  const int H = a.H;
  float2* f = a.field + (size_t)a.class_slot[k] * H * W;
  uint32_t* bits = BITS ? a.bits[k] : nullptr;
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
        for (int i = 0; i < 32; ++i) {
          const int n = word * 32 + i;
          if (n < W) x |= (uint32_t)qs[b * W + n] << i;
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

}  // namespace hg
