// Per-length kernel tables: each supported FFT length is instantiated in its own translation unit
// (hg_len.cu compiled once per length with -DHG_LEN=N) and looked up at run time by the plan.
#pragma once

#include <cuda_runtime.h>

namespace hg {

// Per-stage twiddle tables of one FFT length: table i holds w_{ns R}^{r k} at off + (r-1) ns + k.
struct TwiddleLayout {
  int size;       // float2 entries of the blob
  int count;      // tables
  int ns[16], r[16], off[16];
};

// Run-time radix plan of the generic kernels (lengths without a compile-time instance): stage s has
// radix r[s] after ns[s] = r[0] ... r[s-1] points and reads its twiddles w_{ns R}^{q k} at
// tw + off[s] + (q - 1) ns + k (off[s] < 0 for the first stage, which needs none; the tables of the
// later stages follow one another).  The stages are n16 radix-16 ones, one radix-r2 one (r2 = 8, 4,
// 2, or 0 for none), n9 radix-9, n3 (0 or 1) radix-3 and n5 radix-5 ones, in that order: the device
// code runs from these counts, the arrays serve the host.  batch: rows of a row tile, or columns of
// a column strip, per CTA.
constexpr int kGenMaxStages = 12;
struct GenPlan {
  int n;
  int batch;
  int stages;
  int n16, r2, n9, n3, n5;
  int r[kGenMaxStages], ns[kGenMaxStages], off[kGenMaxStages];
};

struct RowKernels {
  int rows;      // rows per CTA
  int nt;        // threads per CTA
  int smem;      // dynamic shared memory bytes
  // [EXT]: the plain kernel, or the one that also applies an SLM illumination profile or projects
  // onto a multi-amplitude SLM table
  const void* init[2];      // k_row_init (row-major field)
  const void* gs[2][2];     // k_row_gs<OUT = false / true> (row-major field)
  // the same on a field tiled in column strips of width 2 / 4 / 8 / 16 (nullptr where the row
  // length does not allow it); rows / threads / shared memory of those tiles
  const void* init_t[4][2];
  const void* gs_t[4][2][2];
  int rows_t[4], nt_t[4], smem_t[4];
  // the plain tiled GS row kernels with the length's alternative radix plan (has_alt; nullptr
  // otherwise or where that plan does not tile): prologue, pass with OUT = false / true; threads and
  // shared memory of those tiles (the rows are rows_t)
  int has_alt;
  const void* init_tp[4];
  const void* gs_tp[4][2];
  int nt_tp[4], smem_tp[4];
  TwiddleLayout tw_alt;     // twiddle tables of the alternative plan
  // the plain GS row pass on 2-column strips for square items (strip height W at compile time):
  // [radix plan 0 / 1][OUT = false / true]; nullptr where that instance does not exist
  const void* gs_sq[2][2];
  const void* fft[2][2];    // k_row_fft<INV><PRE>
  const void* ospr[2];      // k_row_ospr<BITS = false / true>
  int smem_ospr;            // dynamic shared memory of k_row_ospr (field tile + bit decisions)
  const void* mp_init[2];   // k_row_mp_init<PROJECT = false (gradient descent) / true (GS)>
  const void* mp[2];        // k_row_mp<OUT = false / true>
  const void* gd_bwd;       // k_row_gd_bwd
  // multi-plane GS on a field tiled in column strips of width 2 / 4 / 8 (index as init_t; nullptr
  // where the row length does not tile so, and for width 16): k_row_mp_init<PROJECT = true>, k_row_mp
  const void* mp_init_t[4];
  const void* mp_t[4][2];
  const void* mp_sq[2];     // k_row_mp<OUT> on 2-column strips for square items (nullptr: none)
  // generic lengths only (mp_init / mp / gd_bwd are nullptr there): multi-plane GS and gradient
  // descent run one launch per plane through a plan-owned accumulator [slot][H][W] complex64;
  // kernels (PassArgs, int plane, float* accumulator)
  struct Plane {
    const void* start[2];   // h_0 into the accumulator: [0] exp(i phi) (GD), [1] P_SLM(exp(i phi)) (GS)
    const void* fwd;        // plane p: accumulator c_p -> forward row FFTs -> field p
    const void* back;       // plane p: conj(c_p) inverse row FFTs of field p -> accumulator (+=)
    const void* project;    // accumulator -> P_SLM(accumulator), outputs
    const void* grad;       // gradient and Adam from the accumulator
  } plane;
  // GS with the whole run in one thread-block cluster per N x N item (k_gs_cluster; nullptr where
  // not instantiated): [0] clusters of 8 CTAs, [1] of 16
  const void* gs_cluster[2];
  int nt_cluster[2], smem_cluster[2];
  void (*set_attrs)();      // raises the dynamic shared-memory limit on the current device
  TwiddleLayout tw;         // twiddle tables of length W
  const GenPlan* gen;       // generic kernels: their run-time plan (nullptr for compiled lengths)
};

struct ColKernels {
  int cols;                 // strip width on a row-major field (all kernels but gs_t)
  int nt;
  int smem;
  int smem_gs;              // dynamic shared memory of k_col_gs (exchange + target strip)
  int smem_ospr;            // of k_col_ospr (exchange + target strip + accumulated-intensity strip)
  // [EXT]: the plain kernel, or the one that also takes the signal / noise regions of MRAF and HIO
  const void* gs[2][2];     // k_col_gs<REPLACE = false / true> (row-major field)
  // k_col_gs on the GS field tiled in strips of width 2 / 4 / 8 / 16 (gs nullptr where that
  // configuration does not exist for this length); tile: the default width (tiled_cols)
  struct Tiled {
    int nt, smem_gs;
    const void* gs[2][2];
    // the plain kernel with the alternative radix plan (REPLACE = false / true), its threads and
    // shared memory; nullptr where the length has none or it does not fit
    const void* gs_p[2];
    int nt_p, smem_gs_p;
  } tiled[4];
  int has_alt;
  TwiddleLayout tw_alt;     // twiddle tables of the alternative plan
  int tile;
  const void* fft[2][2];    // k_col_fft<INV><POST>
  const void* ospr[3];      // k_col_ospr: [0] start only, [1] finish + start, [2] finish only
  const void* gd[2];        // k_col_gd<BWD = false / true>
  const void* gd_sq[2];     // the same for square items (row length at compile time)
  void (*set_attrs)();
  TwiddleLayout tw;         // twiddle tables of length H
  const GenPlan* gen;       // generic kernels: their run-time plan (nullptr for compiled lengths)
};

// X-macro of every supported FFT length (rows and columns).
#define HG_FOR_EACH_LENGTH(X) \
  X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) \
  X(12) X(15) X(30) X(60) X(120) X(864) X(1080) X(1536) X(1920) \
  X(720) X(1152) X(1200) X(1280) X(1440) X(1600) X(2160) X(2560) X(3840)

#define HG_DECLARE_LEN(N)                  \
  const RowKernels& row_kernels_##N();     \
  const ColKernels& col_kernels_##N();
HG_FOR_EACH_LENGTH(HG_DECLARE_LEN)
#undef HG_DECLARE_LEN

// nullptr when the length is not supported
const RowKernels* row_kernels(int n);
const ColKernels* col_kernels(int n);

// The generic kernels' tables for a length that has no compiled instance: every n = 2^a 3^b 5^c
// with 1 <= n <= kGenMaxLength (nullptr otherwise).  Built on first use and kept for the process.
constexpr int kGenMaxLength = 4096;
const RowKernels* gen_row_kernels(int n);
const ColKernels* gen_col_kernels(int n);

// Sets the detail string returned by hg_last_error() on this host thread.
void set_last_error(const char* msg);

}  // namespace hg
