// Direct binary search on the GPU (section "Algorithm Libraries": the DS class and the single-pixel
// replay updater FFTUpdaterCuda; reading: Seldowitz, Allebach & Sweeney 1987), and simulated
// annealing over the same trial flips (the SA class of the same section; reading: Kirkpatrick,
// Gelatt & Vecchi 1983).
//
// A binary hologram h in {+1, -1} is improved one SLM pixel at a time, in row-major order: the trial
// flip of pixel p = (m, n) changes the unnormalised replay R = F(h c) by
//   dR[k, l] = d exp(-2 pi i (k m / H + l n / W)),   d = -2 h_p c_p,
// and is kept when the NMSE of |R + dR|^2 against T = A^2 is strictly lower.  With the sums
// S_IT = sum I T, S_II = sum I^2 (S_TT fixed) that is S_IT'^2 S_II > S_IT^2 S_II', and the trial
// needs only the changes dI = |R + dR|^2 - |R|^2 = 2 Re(conj(R) dR) + |d|^2:
//   dS_IT = sum dI T,   dS_II = sum dI (2 I + dI).
//
// The trials are sequential; each is a reduction over the whole replay plane.  One thread-block
// cluster per item holds the replay plane in registers (each thread 8 fixed replay pixels with R,
// T and I), so a trial moves no memory: every thread adds its pixels' changes, the CTA sums them in
// double-float arithmetic, thread 0 writes the CTA's sums into every CTA of the cluster (distributed
// shared memory, double-buffered by trial parity), one cluster barrier, and thread 0 of every CTA
// adds the CL partials in rank order -- the same numbers in the same order, so every CTA takes the
// same decision -- and keeps S_IT, S_II in double.  A kept flip updates R, I in registers and the
// sign in each CTA's copy of h.  Exact sums are recomputed at every sweep boundary (the NMSE curve).
#include <cooperative_groups.h>

#include "hg_dbs.h"
#include "hg_kernels.cuh"

namespace hg {

namespace {

namespace cg = cooperative_groups;

// Sum of two per-thread values over the CTA in double-float arithmetic; thread 0 receives the totals.
__device__ __forceinline__ void block_df(DF& a, DF& b, DF& c) {
  __shared__ DF red[3][kDbsThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
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
    constexpr int NW = kDbsThreads / 32;
    const DF z{0.f, 0.f};
    a = lane < NW ? red[0][lane] : z;
    b = lane < NW ? red[1][lane] : z;
    c = lane < NW ? red[2][lane] : z;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      a = df_add(a, df_shfl_down(a, o));
      b = df_add(b, df_shfl_down(b, o));
      c = df_add(c, df_shfl_down(c, o));
    }
  }
}

// Thread 0: this CTA's sums into slot (par, rank) of every CTA of the cluster.
__device__ __forceinline__ void scatter_sums(cg::cluster_group& cluster, float4* slots, int par, int rank, int cl,
                                             DF a, DF b, DF c) {
  const float4 v0 = make_float4(a.hi, a.lo, b.hi, b.lo), v1 = make_float4(c.hi, c.lo, 0.f, 0.f);
  for (int r = 0; r < cl; ++r) {
    float4* dst = cluster.map_shared_rank(slots, r) + (par * kDbsMaxCluster + rank) * 2;
    dst[0] = v0;
    dst[1] = v1;
  }
}

// Thread 0: the cluster totals of slot par, added in rank order.
__device__ __forceinline__ void gather_sums(const float4* slots, int par, int cl, double* tot) {
  DF a{0.f, 0.f}, b{0.f, 0.f}, c{0.f, 0.f};
  for (int r = 0; r < cl; ++r) {
    const float4 v0 = slots[(par * kDbsMaxCluster + r) * 2], v1 = slots[(par * kDbsMaxCluster + r) * 2 + 1];
    a = df_add(a, DF{v0.x, v0.y});
    b = df_add(b, DF{v0.z, v0.w});
    c = df_add(c, DF{v1.x, v1.y});
  }
  tot[0] = (double)a.hi + (double)a.lo;
  tot[1] = (double)b.hi + (double)b.lo;
  tot[2] = (double)c.hi + (double)c.lo;
}

__global__ void __launch_bounds__(kDbsThreads, 1) k_dbs(const __grid_constant__ DbsArgs d) {
  cg::cluster_group cluster = cg::this_cluster();
  const int cl = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int t = threadIdx.x, k = blockIdx.y;
  const int H = d.H, W = d.W, px = H * W;
  extern __shared__ __align__(16) unsigned char smraw[];
  float4* slots = reinterpret_cast<float4*>(smraw);               // [2][kDbsMaxCluster][2]
  float2* wy = reinterpret_cast<float2*>(slots + 4 * kDbsMaxCluster);  // [H]
  float2* wx = wy + H;                                              // [W]
  signed char* hs = reinterpret_cast<signed char*>(wx + W);        // [px] current hologram, +1 / -1
  __shared__ int s_accept;

  for (int i = t; i < H; i += kDbsThreads) wy[i] = __ldg(&d.wy[i]);
  for (int i = t; i < W; i += kDbsThreads) wx[i] = __ldg(&d.wx[i]);
  // h_0 = P_2(exp(i phi_0)), the same projection as the GS start
  const float* ph = d.phase_in[k];
  for (int p = t; p < px; p += kDbsThreads) {
    float2 e;
    if (ph) {
      float sn, cs;
      sincosf(__ldg(&ph[p]), &sn, &cs);
      e = make_float2(cs, sn);
    } else {
      e = init_unit((uint32_t)p, d.seed, d.item_index[k]);
    }
    int q;
    slm_project(e, 2, nullptr, q);
    hs[p] = q ? -1 : 1;
  }
  // this thread's replay pixels: R, T = A^2, I = |R|^2 and the phase indices of the trial pixel
  float2 R[kDbsValues], dr[kDbsValues];
  float T[kDbsValues], I[kDbsValues];
  int ky[kDbsValues], kx[kDbsValues], iy[kDbsValues], ix[kDbsValues];
  const float2* f = d.field[k];
  const float* A = d.target[k];
#pragma unroll
  for (int j = 0; j < kDbsValues; ++j) {
    const int kk = rank * kDbsPixelsPerCta + t + j * kDbsThreads;
    ky[j] = kk < px ? kk / W : 0;
    kx[j] = kk < px ? kk - ky[j] * W : 0;
    R[j] = kk < px ? f[kk] : make_float2(0.f, 0.f);
    int yy = ky[j], xx = kx[j];
    if (d.centred) {
      yy += H / 2;
      yy -= yy >= H ? H : 0;
      xx += W / 2;
      xx -= xx >= W ? W : 0;
    }
    const float a = kk < px ? __ldg(&A[(size_t)yy * W + xx]) : 0.f;
    T[j] = a * a;
    I[j] = fmaf(R[j].x, R[j].x, R[j].y * R[j].y);
    dr[j] = make_float2(0.f, 0.f);
  }
  // valid pixels only: padded slots have R = T = 0 and must not see a trial's |d|^2
  int nvalid = 0;
#pragma unroll
  for (int j = 0; j < kDbsValues; ++j) nvalid += (rank * kDbsPixelsPerCta + t + j * kDbsThreads) < px;

  double s_it = 0.0, s_ii = 0.0, s_tt = 0.0;  // thread 0: the cluster's sums
  double temp = d.t0;                         // thread 0: annealing temperature of the sweep
  const uint2 key = make_uint2((uint32_t)d.seed, (uint32_t)(d.seed >> 32) ^ (uint32_t)d.item_index[k]);
  int par = 0;
  for (int sweep = 0;; ++sweep) {
    // exact sums at the sweep boundary (NMSE of the current hologram)
    {
      float x0 = 0.f, x1 = 0.f, x2 = 0.f;
#pragma unroll
      for (int j = 0; j < kDbsValues; ++j) {
        x0 = fmaf(I[j], T[j], x0);
        x1 = fmaf(I[j], I[j], x1);
        x2 = fmaf(T[j], T[j], x2);
      }
      DF a{x0, 0.f}, b{x1, 0.f}, c{x2, 0.f};
      block_df(a, b, c);
      if (t == 0) scatter_sums(cluster, slots, par, rank, cl, a, b, c);
      cluster.sync();
      if (t == 0) {
        double tot[3];
        gather_sums(slots, par, cl, tot);
        s_it = tot[0];
        s_ii = tot[1];
        s_tt = tot[2];
        if (rank == 0 && d.nmse)
          d.nmse[(size_t)d.item_index[k] * d.nmse_stride + sweep] =
              (float)((s_ii > 0.0 && s_tt > 0.0) ? 1.0 - s_it * s_it / (s_ii * s_tt) : 1.0);
      }
      par ^= 1;
    }
    if (sweep == d.n_sweeps) break;
    if (sweep > 0) temp *= d.alpha;
#pragma unroll
    for (int j = 0; j < kDbsValues; ++j) iy[j] = ix[j] = 0;
    for (int m = 0; m < H; ++m) {
      for (int n = 0; n < W; ++n) {
        const int p = m * W + n;
        float2 dd = make_float2(hs[p] > 0 ? -2.f : 2.f, 0.f);
        if (d.cx) dd = c_scale(c_mul(__ldg(&d.cx[n]), __ldg(&d.cy[m])), dd.x);
        const float dd2 = fmaf(dd.x, dd.x, dd.y * dd.y);
        float x0 = 0.f, x1 = 0.f;
#pragma unroll
        for (int j = 0; j < kDbsValues; ++j) {
          if (j < nvalid) {
            dr[j] = c_mul(dd, c_mul(wy[iy[j]], wx[ix[j]]));
            const float di = fmaf(2.f, fmaf(R[j].x, dr[j].x, R[j].y * dr[j].y), dd2);
            x0 = fmaf(di, T[j], x0);
            x1 = fmaf(di, fmaf(2.f, I[j], di), x1);
          }
          // phase index of the next trial pixel: (k m mod H, l n mod W) in raster order
          ix[j] += kx[j];
          ix[j] -= ix[j] >= W ? W : 0;
        }
        DF a{x0, 0.f}, b{x1, 0.f}, c{0.f, 0.f};
        block_df(a, b, c);
        if (t == 0) scatter_sums(cluster, slots, par, rank, cl, a, b, c);
        cluster.sync();
        if (t == 0) {
          double tot[3];
          gather_sums(slots, par, cl, tot);
          const double nit = s_it + tot[0], nii = s_ii + tot[1];
          bool keep = nii > 0.0 && s_ii > 0.0 && nit * nit * s_ii > s_it * s_it * nii;
          if (!keep && d.anneal && nii > 0.0 && s_ii > 0.0 && s_tt > 0.0) {
            // Metropolis: E' - E = (S_IT^2 / S_II - S_IT'^2 / S_II') / S_TT >= 0
            const double de = (s_it * s_it / s_ii - nit * nit / nii) / s_tt;
            const uint4 x = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)sweep, 2u, 0u), key);
            const double u = (double)(x.x >> 8) * (1.0 / 16777216.0);
            keep = u < exp(-de / temp);
          }
          if (keep) {
            s_it = nit;
            s_ii = nii;
            hs[p] = (signed char)-hs[p];
          }
          s_accept = keep;
        }
        par ^= 1;
        __syncthreads();
        if (s_accept) {
#pragma unroll
          for (int j = 0; j < kDbsValues; ++j) {
            if (j < nvalid) {
              R[j] = make_float2(R[j].x + dr[j].x, R[j].y + dr[j].y);
              I[j] = fmaf(R[j].x, R[j].x, R[j].y * R[j].y);
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kDbsValues; ++j) {
        ix[j] = 0;
        iy[j] += ky[j];
        iy[j] -= iy[j] >= H ? H : 0;
      }
    }
  }
  // outputs from this CTA's copy of h (every CTA holds the same hologram)
  float* po = d.phase_out[k];
  uint8_t* lo = d.level_out[k];
  for (int p = rank * kDbsThreads + t; p < px; p += cl * kDbsThreads) {
    const bool pi = hs[p] < 0;
    if (po) po[p] = pi ? 3.14159265358979323846f : 0.f;
    if (lo) lo[p] = pi ? 1 : 0;
  }
}

}  // namespace

const void* dbs_kernel() { return (const void*)&k_dbs; }

int dbs_smem(int H, int W) { return 4 * kDbsMaxCluster * 16 + (H + W) * 8 + H * W; }

void dbs_set_attrs() {
  // the largest item: 65536 pixels with H + W <= 8192 (lengths up to 4096)
  cudaFuncSetAttribute((const void*)&k_dbs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       4 * kDbsMaxCluster * 16 + 8192 * 8 + 65536);
  cudaFuncSetAttribute((const void*)&k_dbs, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

}  // namespace hg
