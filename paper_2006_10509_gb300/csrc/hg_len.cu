// Instantiates the row- and column-pass kernels for one FFT length, HG_LEN (set by the build).
#include "hg_kernels.cuh"
#include "hg_launch.h"

#ifndef HG_LEN
#error "HG_LEN must be defined"
#endif

namespace hg {

namespace {

template <class F>
void allow_smem(F* f, int bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <int N, class F = typename PlanFor<N>::type>
TwiddleLayout make_tw() {
  using T = TwBlob<N, F>;
  static_assert(T::count() <= 16, "too many twiddle tables");
  TwiddleLayout l{};
  l.size = T::size;
  l.count = T::count();
  for (int i = 0; i < l.count; ++i) {
    l.ns[i] = T::table(i, 0);
    l.r[i] = T::table(i, 1);
    l.off[i] = T::table(i, 2);
  }
  return l;
}

template <int N, int TW>
void fill_tiled(RowKernels& r, int i) {
  if constexpr (row_tileable<N, TW>()) {
    using K = RowCfg<N, TW>;
    r.init_t[i][0] = (const void*)&k_row_init<N, TW, false>;
    r.init_t[i][1] = (const void*)&k_row_init<N, TW, true>;
    r.gs_t[i][0][0] = (const void*)&k_row_gs<N, false, TW, false>;
    r.gs_t[i][0][1] = (const void*)&k_row_gs<N, false, TW, true>;
    r.gs_t[i][1][0] = (const void*)&k_row_gs<N, true, TW, false>;
    r.gs_t[i][1][1] = (const void*)&k_row_gs<N, true, TW, true>;
    r.rows_t[i] = K::ROWS;
    r.nt_t[i] = K::NT;
    r.smem_t[i] = K::SMEM;
  }
}

// the alternative radix plan's plain tiled GS row kernels
template <int N, int TW>
void fill_tiled_alt(RowKernels& r, int i) {
  if constexpr (has_alt_plan<N>() && row_tileable<N, TW, 1>()) {
    using K = RowCfg<N, TW, 1>;
    r.init_tp[i] = (const void*)&k_row_init<N, TW, false, 1>;
    r.gs_tp[i][0] = (const void*)&k_row_gs<N, false, TW, false, 1>;
    r.gs_tp[i][1] = (const void*)&k_row_gs<N, true, TW, false, 1>;
    r.nt_tp[i] = K::NT;
    r.smem_tp[i] = K::SMEM;
  }
}

// the plain row pass on 2-column strips for square items, both radix plans
template <int N>
void fill_square(RowKernels& r) {
  if constexpr (row_tileable<N, 2>()) {
    r.gs_sq[0][0] = (const void*)&k_row_gs<N, false, 2, false, 0, true>;
    r.gs_sq[0][1] = (const void*)&k_row_gs<N, true, 2, false, 0, true>;
    r.mp_sq[0] = (const void*)&k_row_mp<N, false, 2, true>;
    r.mp_sq[1] = (const void*)&k_row_mp<N, true, 2, true>;
  }
  if constexpr (has_alt_plan<N>() && row_tileable<N, 2, 1>()) {
    r.gs_sq[1][0] = (const void*)&k_row_gs<N, false, 2, false, 1, true>;
    r.gs_sq[1][1] = (const void*)&k_row_gs<N, true, 2, false, 1, true>;
  }
}

template <int N>
void set_square_attrs() {
  if constexpr (row_tileable<N, 2>()) {
    allow_smem(&k_row_gs<N, false, 2, false, 0, true>, RowCfg<N, 2>::SMEM);
    allow_smem(&k_row_gs<N, true, 2, false, 0, true>, RowCfg<N, 2>::SMEM);
    allow_smem(&k_row_mp<N, false, 2, true>, RowCfg<N, 2>::SMEM);
    allow_smem(&k_row_mp<N, true, 2, true>, RowCfg<N, 2>::SMEM);
  }
  if constexpr (has_alt_plan<N>() && row_tileable<N, 2, 1>()) {
    allow_smem(&k_row_gs<N, false, 2, false, 1, true>, RowCfg<N, 2, 1>::SMEM);
    allow_smem(&k_row_gs<N, true, 2, false, 1, true>, RowCfg<N, 2, 1>::SMEM);
  }
}

template <int N, int TW>
void set_tiled_alt_attrs() {
  if constexpr (has_alt_plan<N>() && row_tileable<N, TW, 1>()) {
    allow_smem(&k_row_init<N, TW, false, 1>, RowCfg<N, TW, 1>::SMEM);
    allow_smem(&k_row_gs<N, false, TW, false, 1>, RowCfg<N, TW, 1>::SMEM);
    allow_smem(&k_row_gs<N, true, TW, false, 1>, RowCfg<N, TW, 1>::SMEM);
  }
}

// multi-plane GS row kernels on the tiled field (widths up to 8)
template <int N, int TW>
void fill_tiled_planes(RowKernels& r, int i) {
  if constexpr (TW <= 8 && row_tileable<N, TW>()) {
    r.mp_init_t[i] = (const void*)&k_row_mp_init<N, true, TW>;
    r.mp_t[i][0] = (const void*)&k_row_mp<N, false, TW>;
    r.mp_t[i][1] = (const void*)&k_row_mp<N, true, TW>;
  }
}

template <int N, int TW>
void set_tiled_planes_attrs() {
  if constexpr (TW <= 8 && row_tileable<N, TW>()) {
    constexpr int smem = RowCfg<N, TW>::SMEM;
    allow_smem(&k_row_mp_init<N, true, TW>, smem);
    allow_smem(&k_row_mp<N, false, TW>, smem);
    allow_smem(&k_row_mp<N, true, TW>, smem);
  }
}

template <int N, int TW>
void set_tiled_attrs() {
  if constexpr (row_tileable<N, TW>()) {
    allow_smem(&k_row_init<N, TW, false>, RowCfg<N, TW>::SMEM);
    allow_smem(&k_row_init<N, TW, true>, RowCfg<N, TW>::SMEM);
    allow_smem(&k_row_gs<N, false, TW, false>, RowCfg<N, TW>::SMEM);
    allow_smem(&k_row_gs<N, true, TW, false>, RowCfg<N, TW>::SMEM);
    allow_smem(&k_row_gs<N, false, TW, true>, RowCfg<N, TW>::SMEM);
    allow_smem(&k_row_gs<N, true, TW, true>, RowCfg<N, TW>::SMEM);
  }
}

// whole-run cluster kernels for the small square sizes (the field of one item fits the shared
// memory of one cluster)
constexpr bool cluster_len(int n) { return n == 64 || n == 128 || n == 256; }

template <int N, int CL>
void fill_cluster(RowKernels& r, int i) {
  if constexpr (cluster_len(N) && ClusterCfg<N, CL>::FEASIBLE) {
    r.gs_cluster[i] = (const void*)&k_gs_cluster<N, CL>;
    r.nt_cluster[i] = ClusterCfg<N, CL>::NT;
    r.smem_cluster[i] = ClusterCfg<N, CL>::SMEM;
  }
}

template <int N, int CL>
void set_cluster_attrs() {
  if constexpr (cluster_len(N) && ClusterCfg<N, CL>::FEASIBLE) {
    allow_smem(&k_gs_cluster<N, CL>, ClusterCfg<N, CL>::SMEM);
    if (CL > 8) cudaFuncSetAttribute((const void*)&k_gs_cluster<N, CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
}

template <int N>
RowKernels make_row() {
  using K = RowCfg<N>;
  RowKernels r{};
  r.rows = K::ROWS;
  r.nt = K::NT;
  r.smem = K::SMEM;
  r.init[0] = (const void*)&k_row_init<N, 0, false>;
  r.init[1] = (const void*)&k_row_init<N, 0, true>;
  r.gs[0][0] = (const void*)&k_row_gs<N, false, 0, false>;
  r.gs[0][1] = (const void*)&k_row_gs<N, false, 0, true>;
  r.gs[1][0] = (const void*)&k_row_gs<N, true, 0, false>;
  r.gs[1][1] = (const void*)&k_row_gs<N, true, 0, true>;
  fill_tiled<N, 2>(r, 0);
  fill_tiled<N, 4>(r, 1);
  fill_tiled<N, 8>(r, 2);
  fill_tiled<N, 16>(r, 3);
  r.has_alt = has_alt_plan<N>() ? 1 : 0;
  fill_tiled_alt<N, 2>(r, 0);
  fill_tiled_alt<N, 4>(r, 1);
  fill_tiled_alt<N, 8>(r, 2);
  fill_tiled_alt<N, 16>(r, 3);
  fill_tiled_planes<N, 2>(r, 0);
  fill_tiled_planes<N, 4>(r, 1);
  fill_tiled_planes<N, 8>(r, 2);
  fill_square<N>(r);
  r.fft[0][0] = (const void*)&k_row_fft<N, false, false>;
  r.fft[0][1] = (const void*)&k_row_fft<N, false, true>;
  r.fft[1][0] = (const void*)&k_row_fft<N, true, false>;
  r.fft[1][1] = (const void*)&k_row_fft<N, true, true>;
  r.ospr[0] = (const void*)&k_row_ospr<N, false>;
  r.ospr[1] = (const void*)&k_row_ospr<N, true>;
  r.smem_ospr = K::SMEM + K::ROWS * N;
  r.mp_init[0] = (const void*)&k_row_mp_init<N, false>;
  r.mp_init[1] = (const void*)&k_row_mp_init<N, true>;
  r.mp[0] = (const void*)&k_row_mp<N, false>;
  r.mp[1] = (const void*)&k_row_mp<N, true>;
  r.gd_bwd = (const void*)&k_row_gd_bwd<N>;
  fill_cluster<N, 8>(r, 0);
  fill_cluster<N, 16>(r, 1);
  r.tw = make_tw<N>();
  r.tw_alt = make_tw<N, typename PlanV<N, 1>::type>();
  return r;
}

template <int N, int C>
void fill_col_tiled(ColKernels::Tiled& t) {
  using K = ColCfg<N, C>;
  if constexpr (K::FEASIBLE) {
    t.nt = K::NT;
    t.smem_gs = K::SMEM_T;
    t.gs[0][0] = (const void*)&k_col_gs<N, false, C, false>;
    t.gs[0][1] = (const void*)&k_col_gs<N, false, C, true>;
    t.gs[1][0] = (const void*)&k_col_gs<N, true, C, false>;
    t.gs[1][1] = (const void*)&k_col_gs<N, true, C, true>;
  }
  using KP = ColCfg<N, C, 1>;
  if constexpr (has_alt_plan<N>() && K::FEASIBLE && KP::FEASIBLE) {
    t.nt_p = KP::NT;
    t.smem_gs_p = KP::SMEM_T;
    t.gs_p[0] = (const void*)&k_col_gs<N, false, C, false, 1>;
    t.gs_p[1] = (const void*)&k_col_gs<N, true, C, false, 1>;
  }
}

template <int N, int C>
void set_col_tiled_attrs() {
  using K = ColCfg<N, C>;
  if constexpr (K::FEASIBLE) {
    allow_smem(&k_col_gs<N, false, C, false>, K::SMEM_T);
    allow_smem(&k_col_gs<N, true, C, false>, K::SMEM_T);
    allow_smem(&k_col_gs<N, false, C, true>, K::SMEM_T);
    allow_smem(&k_col_gs<N, true, C, true>, K::SMEM_T);
  }
  using KP = ColCfg<N, C, 1>;
  if constexpr (has_alt_plan<N>() && K::FEASIBLE && KP::FEASIBLE) {
    allow_smem(&k_col_gs<N, false, C, false, 1>, KP::SMEM_T);
    allow_smem(&k_col_gs<N, true, C, false, 1>, KP::SMEM_T);
  }
}

template <int N>
ColKernels make_col() {
  using K = ColCfg<N>;
  ColKernels c{};
  c.cols = K::C;
  c.nt = K::NT;
  c.smem = K::SMEM;
  c.smem_gs = K::SMEM_T;
  c.smem_ospr = K::SMEM_OSPR;
  c.gs[0][0] = (const void*)&k_col_gs<N, false, 0, false>;
  c.gs[0][1] = (const void*)&k_col_gs<N, false, 0, true>;
  c.gs[1][0] = (const void*)&k_col_gs<N, true, 0, false>;
  c.gs[1][1] = (const void*)&k_col_gs<N, true, 0, true>;
  fill_col_tiled<N, 2>(c.tiled[0]);
  fill_col_tiled<N, 4>(c.tiled[1]);
  fill_col_tiled<N, 8>(c.tiled[2]);
  fill_col_tiled<N, 16>(c.tiled[3]);
  c.tile = tiled_cols(N);
  c.has_alt = has_alt_plan<N>() ? 1 : 0;
  c.tw_alt = make_tw<N, typename PlanV<N, 1>::type>();
  c.fft[0][0] = (const void*)&k_col_fft<N, false, false>;
  c.fft[0][1] = (const void*)&k_col_fft<N, false, true>;
  c.fft[1][0] = (const void*)&k_col_fft<N, true, false>;
  c.fft[1][1] = (const void*)&k_col_fft<N, true, true>;
  c.ospr[0] = (const void*)&k_col_ospr<N, false, true>;
  c.ospr[1] = (const void*)&k_col_ospr<N, true, true>;
  c.ospr[2] = (const void*)&k_col_ospr<N, true, false>;
  c.gd[0] = (const void*)&k_col_gd<N, false>;
  c.gd[1] = (const void*)&k_col_gd<N, true>;
  c.gd_sq[0] = (const void*)&k_col_gd<N, false, true>;
  c.gd_sq[1] = (const void*)&k_col_gd<N, true, true>;
  c.tw = make_tw<N>();
  return c;
}

void set_row_attrs(const RowKernels& r) {
  allow_smem(&k_row_init<HG_LEN, 0, false>, r.smem);
  allow_smem(&k_row_init<HG_LEN, 0, true>, r.smem);
  allow_smem(&k_row_gs<HG_LEN, false, 0, false>, r.smem);
  allow_smem(&k_row_gs<HG_LEN, true, 0, false>, r.smem);
  allow_smem(&k_row_gs<HG_LEN, false, 0, true>, r.smem);
  allow_smem(&k_row_gs<HG_LEN, true, 0, true>, r.smem);
  set_tiled_attrs<HG_LEN, 2>();
  set_tiled_attrs<HG_LEN, 4>();
  set_tiled_attrs<HG_LEN, 8>();
  set_tiled_attrs<HG_LEN, 16>();
  set_tiled_alt_attrs<HG_LEN, 2>();
  set_tiled_alt_attrs<HG_LEN, 4>();
  set_tiled_alt_attrs<HG_LEN, 8>();
  set_tiled_alt_attrs<HG_LEN, 16>();
  set_tiled_planes_attrs<HG_LEN, 2>();
  set_tiled_planes_attrs<HG_LEN, 4>();
  set_tiled_planes_attrs<HG_LEN, 8>();
  set_square_attrs<HG_LEN>();
  allow_smem(&k_row_fft<HG_LEN, false, false>, r.smem);
  allow_smem(&k_row_fft<HG_LEN, false, true>, r.smem);
  allow_smem(&k_row_fft<HG_LEN, true, false>, r.smem);
  allow_smem(&k_row_fft<HG_LEN, true, true>, r.smem);
  allow_smem(&k_row_ospr<HG_LEN, false>, r.smem_ospr);
  allow_smem(&k_row_ospr<HG_LEN, true>, r.smem_ospr);
  allow_smem(&k_row_mp_init<HG_LEN, false>, r.smem);
  allow_smem(&k_row_mp_init<HG_LEN, true>, r.smem);
  allow_smem(&k_row_mp<HG_LEN, false>, r.smem);
  allow_smem(&k_row_mp<HG_LEN, true>, r.smem);
  allow_smem(&k_row_gd_bwd<HG_LEN>, r.smem);
  set_cluster_attrs<HG_LEN, 8>();
  set_cluster_attrs<HG_LEN, 16>();
}

void set_col_attrs(const ColKernels& c) {
  allow_smem(&k_col_gs<HG_LEN, false, 0, false>, c.smem_gs);
  allow_smem(&k_col_gs<HG_LEN, true, 0, false>, c.smem_gs);
  allow_smem(&k_col_gs<HG_LEN, false, 0, true>, c.smem_gs);
  allow_smem(&k_col_gs<HG_LEN, true, 0, true>, c.smem_gs);
  set_col_tiled_attrs<HG_LEN, 2>();
  set_col_tiled_attrs<HG_LEN, 4>();
  set_col_tiled_attrs<HG_LEN, 8>();
  set_col_tiled_attrs<HG_LEN, 16>();
  allow_smem(&k_col_fft<HG_LEN, false, false>, c.smem);
  allow_smem(&k_col_fft<HG_LEN, false, true>, c.smem);
  allow_smem(&k_col_fft<HG_LEN, true, false>, c.smem);
  allow_smem(&k_col_fft<HG_LEN, true, true>, c.smem);
  allow_smem(&k_col_ospr<HG_LEN, false, true>, c.smem_ospr);
  allow_smem(&k_col_ospr<HG_LEN, true, true>, c.smem_ospr);
  allow_smem(&k_col_ospr<HG_LEN, true, false>, c.smem_ospr);
  allow_smem(&k_col_gd<HG_LEN, false>, c.smem);
  allow_smem(&k_col_gd<HG_LEN, true>, c.smem);
  allow_smem(&k_col_gd<HG_LEN, false, true>, c.smem);
  allow_smem(&k_col_gd<HG_LEN, true, true>, c.smem);
}

}  // namespace

#define HG_CAT2(a, b) a##b
#define HG_CAT(a, b) HG_CAT2(a, b)

const RowKernels& HG_CAT(row_kernels_, HG_LEN)() {
  static const RowKernels r = [] {
    RowKernels x = make_row<HG_LEN>();
    x.set_attrs = [] { set_row_attrs(make_row<HG_LEN>()); };
    return x;
  }();
  return r;
}

const ColKernels& HG_CAT(col_kernels_, HG_LEN)() {
  static const ColKernels c = [] {
    ColKernels x = make_col<HG_LEN>();
    x.set_attrs = [] { set_col_attrs(make_col<HG_LEN>()); };
    return x;
  }();
  return c;
}

}  // namespace hg
