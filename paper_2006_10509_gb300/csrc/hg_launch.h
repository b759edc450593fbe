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
  const void* fft[2][2];    // k_row_fft<INV><PRE>
  const void* ospr[2];      // k_row_ospr<BITS = false / true>
  int smem_ospr;            // dynamic shared memory of k_row_ospr (field tile + bit decisions)
  const void* mp_init[2];   // k_row_mp_init<PROJECT = false (gradient descent) / true (GS)>
  const void* mp[2];        // k_row_mp<OUT = false / true>
  const void* gd_bwd;       // k_row_gd_bwd
  // GS with the whole run in one thread-block cluster per N x N item (k_gs_cluster; nullptr where
  // not instantiated): [0] clusters of 8 CTAs, [1] of 16
  const void* gs_cluster[2];
  int nt_cluster[2], smem_cluster[2];
  void (*set_attrs)();      // raises the dynamic shared-memory limit on the current device
  TwiddleLayout tw;         // twiddle tables of length W
};

struct ColKernels {
  int cols;                 // strip width on a row-major field (all kernels but gs_t)
  int nt;
  int smem;
  int smem_gs;              // dynamic shared memory of k_col_gs / k_col_ospr (exchange + target strip)
  // [EXT]: the plain kernel, or the one that also takes the signal / noise regions of MRAF and HIO
  const void* gs[2][2];     // k_col_gs<REPLACE = false / true> (row-major field)
  // k_col_gs on the GS field tiled in strips of width 2 / 4 / 8 / 16 (gs nullptr where that
  // configuration does not exist for this length); tile: the default width (tiled_cols)
  struct Tiled {
    int nt, smem_gs;
    const void* gs[2][2];
  } tiled[4];
  int tile;
  const void* fft[2][2];    // k_col_fft<INV><POST>
  const void* ospr[3];      // k_col_ospr: [0] start only, [1] finish + start, [2] finish only
  const void* gd[2];        // k_col_gd<BWD = false / true>
  void (*set_attrs)();
  TwiddleLayout tw;         // twiddle tables of length H
};

// X-macro of every supported FFT length (rows and columns).
#define HG_FOR_EACH_LENGTH(X) \
  X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096) \
  X(12) X(15) X(30) X(60) X(120) X(864) X(1080) X(1536) X(1920)

#define HG_DECLARE_LEN(N)                  \
  const RowKernels& row_kernels_##N();     \
  const ColKernels& col_kernels_##N();
HG_FOR_EACH_LENGTH(HG_DECLARE_LEN)
#undef HG_DECLARE_LEN

// nullptr when the length is not supported
const RowKernels* row_kernels(int n);
const ColKernels* col_kernels(int n);

// Sets the detail string returned by hg_last_error() on this host thread.
void set_last_error(const char* msg);

}  // namespace hg
