// Direct binary search (section "Algorithm Libraries": the DS algorithm class and the single-pixel
// replay updater FFTUpdaterCuda): launch arguments and kernel lookup.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace hg {

constexpr int kDbsMaxBatch = 32;                            // items per launch
constexpr int kDbsThreads = 512;                            // threads per CTA
constexpr int kDbsValues = 8;                               // replay pixels per thread
constexpr int kDbsPixelsPerCta = kDbsThreads * kDbsValues;  // 4096
constexpr int kDbsMaxCluster = 16;                          // CTAs per item: at most 65536 pixels

struct DbsArgs {
  int H, W;
  int n_sweeps;
  int nmse_stride;          // floats between items in nmse (n_sweeps + 1)
  uint64_t seed;            // starting-phase seed when phase_in is null
  const float2* wy;         // exp(-2 pi i j / H), j < H
  const float2* wx;         // exp(-2 pi i j / W), j < W
  const float2* cx;         // Fresnel chirp along a row (W), nullptr for Fourier
  const float2* cy;         // Fresnel chirp along a column (H)
  int centred;              // targets in display order (DC at (H/2, W/2))
  // simulated annealing (anneal = 1): a flip that does not lower the NMSE E is still kept when
  // u < exp(-(E' - E) / T_s), T_s = t0 alpha^s, u from Philox4x32-10 word 0 with counter
  // (pixel, sweep, 2, 0) and key (seed_lo, seed_hi ^ item), u = (x >> 8) 2^-24
  int anneal;
  double t0, alpha;
  float* nmse;              // [item][n_sweeps + 1] or nullptr
  const float2* field[kDbsMaxBatch];  // R_0 = unnormalised F(h_0 c), row-major [H][W] (plan workspace)
  const float* target[kDbsMaxBatch];  // amplitude A [H][W]
  const float* phase_in[kDbsMaxBatch];
  float* phase_out[kDbsMaxBatch];
  uint8_t* level_out[kDbsMaxBatch];
  int item_index[kDbsMaxBatch];
};

// k_dbs (one thread-block cluster of ceil(H W / kDbsPixelsPerCta) CTAs per item, kDbsThreads
// threads, dbs_smem(H, W) bytes of dynamic shared memory)
const void* dbs_kernel();
int dbs_smem(int H, int W);
void dbs_set_attrs();

}  // namespace hg
