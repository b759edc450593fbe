// Device-side mixed-radix Stockham FFT engine for the row and column passes.
//
// The paper's FFT handler (section "Algorithm Libraries", FFTHandlerCuda) wraps cuFFT; this is a
// hand-written replacement whose stages can be fused with the pointwise steps of the iteration.
//
// A CTA transforms B independent sequences of length N ("rows" of a row tile, or "columns" of a
// column strip).  Data lives in registers; a stage of radix R with Ns = product of earlier radices
// runs butterfly j (0 <= j < N/R): it takes inputs n = j + r N/R, multiplies input r by
// w_{Ns R}^{r (j mod Ns)}, applies an R-point DFT and produces outputs at
// (j / Ns) Ns R + (j mod Ns) + r Ns (Stockham autosort: natural order out, no bit reversal).
// Between stages the values are exchanged through shared memory.
//
// Two properties are used by the fused kernels:
//  * the inputs of the first stage and the outputs of the last stage both sit at n = j + r N/R, so a
//    kernel loads/stores global memory directly from/to the registers of those stages;
//  * if transform B's first radix equals transform A's last radix, B's first stage takes A's
//    last-stage outputs without any exchange (plans are run forward, then reversed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace hg {

// ---------------------------------------------------------------- complex helpers

// complex add / subtract as one packed FP32x2 instruction (sm_100+), same rounding as two scalar ones
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 c_mulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }

// multiply by the quarter-turn root of unity of the transform direction: -i (forward), +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 c_rot(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos / sin of 2 pi k / 16 for k = 0..15 (exact decimal expansions of cos(pi/8), sin(pi/8), sqrt(2)/2)
#define HG_C1 0.92387953251128675613f
#define HG_S1 0.38268343236508977173f
#define HG_R2 0.70710678118654752440f

// a * w16^K with w16 = exp(-+ 2 pi i / 16)
template <int K, bool INV>
__device__ __forceinline__ float2 c_w16(float2 a) {
  constexpr int k = K & 15;
  constexpr float cs[16] = {1.f, HG_C1, HG_R2, HG_S1, 0.f, -HG_S1, -HG_R2, -HG_C1,
                            -1.f, -HG_C1, -HG_R2, -HG_S1, 0.f, HG_S1, HG_R2, HG_C1};
  constexpr float sn[16] = {0.f, HG_S1, HG_R2, HG_C1, 1.f, HG_C1, HG_R2, HG_S1,
                            0.f, -HG_S1, -HG_R2, -HG_C1, -1.f, -HG_C1, -HG_R2, -HG_S1};
  if constexpr (k == 0) {
    return a;
  } else if constexpr (k == 4) {
    return c_rot<INV>(a);
  } else if constexpr (k == 8) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (k == 12) {
    return c_rot<!INV>(a);
  } else {
    // w = cs - i sn (forward) or cs + i sn (inverse)
    constexpr float c = cs[k];
    constexpr float s = INV ? sn[k] : -sn[k];
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
  }
}

// ---------------------------------------------------------------- small DFTs (in place, natural order)

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = c_add(t, b);
  b = c_sub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 a = c_add(x0, x2), b = c_sub(x0, x2);
  float2 c = c_add(x1, x3), s = c_sub(x1, x3);
  x0 = c_add(a, c);
  x2 = c_sub(a, c);
  // b -+ i s (forward) / b +- i s (inverse) in scalar form: a packed form would need a swapped pair
  x1 = INV ? make_float2(b.x - s.y, b.y + s.x) : make_float2(b.x + s.y, b.y - s.x);
  x3 = INV ? make_float2(b.x + s.y, b.y - s.x) : make_float2(b.x - s.y, b.y + s.x);
}

template <bool INV>
__device__ __forceinline__ void dft3(float2* v) {
  // X1,2 = x0 - (x1+x2)/2 -+ i (sqrt(3)/2)(x1 - x2)   (forward; signs flip for inverse)
  constexpr float h = 0.86602540378443864676f;
  float2 s = c_add(v[1], v[2]);
  float2 d = c_sub(v[1], v[2]);
  float2 m = make_float2(fmaf(-0.5f, s.x, v[0].x), fmaf(-0.5f, s.y, v[0].y));
  float2 r = c_rot<INV>(make_float2(h * d.x, h * d.y));  // -+ i (sqrt3/2) d
  v[0] = c_add(v[0], s);
  v[1] = c_add(m, r);
  v[2] = c_sub(m, r);
}

template <bool INV>
__device__ __forceinline__ void dft5(float2* v) {
  constexpr float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
  constexpr float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
  constexpr float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
  constexpr float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
  float2 a1 = c_add(v[1], v[4]), b1 = c_sub(v[1], v[4]);
  float2 a2 = c_add(v[2], v[3]), b2 = c_sub(v[2], v[3]);
  float2 x0 = v[0];
  float2 p1 = make_float2(x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y);
  float2 p2 = make_float2(x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y);
  // q1 = s1 b1 + s2 b2, q2 = s2 b1 - s1 b2 ; X1 = p1 - i q1, X4 = p1 + i q1 (forward)
  float2 q1 = make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y);
  float2 q2 = make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y);
  float2 r1 = c_rot<INV>(q1);
  float2 r2 = c_rot<INV>(q2);
  v[0] = make_float2(x0.x + a1.x + a2.x, x0.y + a1.y + a2.y);
  v[1] = c_add(p1, r1);
  v[4] = c_sub(p1, r1);
  v[2] = c_add(p2, r2);
  v[3] = c_sub(p2, r2);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  o1 = c_w16<2, INV>(o1);
  o2 = c_w16<4, INV>(o2);
  o3 = c_w16<6, INV>(o3);
  v[0] = c_add(e0, o0);
  v[4] = c_sub(e0, o0);
  v[1] = c_add(e1, o1);
  v[5] = c_sub(e1, o1);
  v[2] = c_add(e2, o2);
  v[6] = c_sub(e2, o2);
  v[3] = c_add(e3, o3);
  v[7] = c_sub(e3, o3);
}

template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
  // r = 4a + b, q = c + 4d:  X[c + 4d] = sum_b w4^{bd} w16^{bc} sum_a x[4a + b] w4^{ac}
#pragma unroll
  for (int b = 0; b < 4; ++b) dft4<INV>(v[b], v[b + 4], v[b + 8], v[b + 12]);
  // now v[b + 4c] = Y_b[c]; twiddle by w16^{bc}
  v[5] = c_w16<1, INV>(v[5]);
  v[9] = c_w16<2, INV>(v[9]);
  v[13] = c_w16<3, INV>(v[13]);
  v[6] = c_w16<2, INV>(v[6]);
  v[10] = c_w16<4, INV>(v[10]);
  v[14] = c_w16<6, INV>(v[14]);
  v[7] = c_w16<3, INV>(v[7]);
  v[11] = c_w16<6, INV>(v[11]);
  v[15] = c_w16<9, INV>(v[15]);
#pragma unroll
  for (int c = 0; c < 4; ++c) dft4<INV>(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
  // v[4c + d] = X[c + 4d]: transpose the 4x4 block
  float2 t[16];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int d = 0; d < 4; ++d) t[c + 4 * d] = v[4 * c + d];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = t[i];
}

// cos and sin of 2 pi m / r, evaluated at compile time in double: the angle is brought to
// [-pi, pi] and summed as a Taylor series (30 terms: truncation far below double rounding there).
__host__ __device__ constexpr double turn_angle(int m, int r) {
  const int k = ((m % r) + r) % r;
  const double pi = 3.14159265358979323846264338327950288;
  return 2.0 * k > r ? 2.0 * pi * (double)(k - r) / r : 2.0 * pi * (double)k / r;
}
__host__ __device__ constexpr double cos_turn(int m, int r) {
  const double x = turn_angle(m, r);
  double term = 1.0, sum = 1.0;
  for (int i = 1; i <= 30; ++i) {
    term *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double sin_turn(int m, int r) {
  const double x = turn_angle(m, r);
  double term = x, sum = x;
  for (int i = 1; i <= 30; ++i) {
    term *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
    sum += term;
  }
  return sum;
}

// a * w_R^M, w_R = exp(-+ 2 pi i / R) (forward / inverse), M a compile-time constant
template <int R, int M, bool INV>
__device__ __forceinline__ float2 c_wt(float2 a) {
  constexpr int m = ((M % R) + R) % R;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (4 * m == R) {
    return c_rot<INV>(a);
  } else if constexpr (2 * m == R) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (4 * m == 3 * R) {
    return c_rot<!INV>(a);
  } else {
    constexpr float c = (float)cos_turn(m, R);
    constexpr float sn = (float)sin_turn(m, R);
    constexpr float s = INV ? sn : -sn;
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
  }
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v);

// Compile-time loop: f(std::integral_constant<int, I>) for I = B .. E-1.
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// R = P Q point DFT (Cooley-Tukey, one level): with n = Q n1 + n2 and k = k1 + P k2,
// X[k] = sum_n2 w_R^(n2 k1) w_Q^(n2 k2) sum_n1 x[Q n1 + n2] w_P^(n1 k1): Q P-point DFTs, twiddles,
// P Q-point DFTs, natural order out.
template <int P, int Q, bool INV>
__device__ __forceinline__ void dft_pq(float2* v) {
  constexpr int R = P * Q;
  static_for<0, Q>([&](auto n2c) {
    constexpr int n2 = decltype(n2c)::value;
    float2 t[P];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) t[n1] = v[Q * n1 + n2];
    dft<P, INV>(t);
    static_for<0, P>([&](auto k1c) {
      constexpr int k1 = decltype(k1c)::value;
      v[Q * k1 + n2] = c_wt<R, n2 * k1, INV>(t[k1]);
    });
  });
  float2 o[R];
#pragma unroll
  for (int k1 = 0; k1 < P; ++k1) {
    float2 u[Q];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) u[n2] = v[Q * k1 + n2];
    dft<Q, INV>(u);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) o[k1 + P * k2] = u[k2];
  }
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = o[i];
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v) {
  if constexpr (R == 2) {
    dft2<INV>(v[0], v[1]);
  } else if constexpr (R == 3) {
    dft3<INV>(v);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 5) {
    dft5<INV>(v);
  } else if constexpr (R == 8) {
    dft8<INV>(v);
  } else if constexpr (R == 16) {
    dft16<INV>(v);
  } else if constexpr (R == 6) {
    dft_pq<2, 3, INV>(v);
  } else if constexpr (R == 9) {
    dft_pq<3, 3, INV>(v);
  } else if constexpr (R == 10) {
    dft_pq<2, 5, INV>(v);
  } else if constexpr (R == 12) {
    dft_pq<4, 3, INV>(v);
  } else if constexpr (R == 15) {
    dft_pq<3, 5, INV>(v);
  } else {
    static_assert(R == 2, "unsupported radix");
  }
}

// ---------------------------------------------------------------- radix plans

template <int... Rs>
struct RList {};

template <class L>
struct RFirst;
template <int R, int... Rs>
struct RFirst<RList<R, Rs...>> {
  static constexpr int value = R;
};

template <class L>
struct RLast;
template <int R>
struct RLast<RList<R>> {
  static constexpr int value = R;
};
template <int R, int R2, int... Rs>
struct RLast<RList<R, R2, Rs...>> {
  static constexpr int value = RLast<RList<R2, Rs...>>::value;
};

template <class L, class Acc = RList<>>
struct RRev;
template <int... As>
struct RRev<RList<>, RList<As...>> {
  using type = RList<As...>;
};
template <int R, int... Rs, int... As>
struct RRev<RList<R, Rs...>, RList<As...>> {
  using type = typename RRev<RList<Rs...>, RList<R, As...>>::type;
};

template <class L>
struct RProd;
template <>
struct RProd<RList<>> {
  static constexpr int value = 1;
};
template <int R, int... Rs>
struct RProd<RList<R, Rs...>> {
  static constexpr int value = R * RProd<RList<Rs...>>::value;
};

template <class L>
struct RArr;
template <int... Rs>
struct RArr<RList<Rs...>> {
  static constexpr int n = sizeof...(Rs);
  __host__ __device__ static constexpr int at(int s) {
    const int a[] = {Rs...};
    return a[s];
  }
};

// Radix plan for each supported length (forward order; the inverse of a fused pair runs reversed).
template <int N>
struct PlanFor;
#define HG_PLAN(N, ...)              \
  template <>                        \
  struct PlanFor<N> {                \
    using type = RList<__VA_ARGS__>; \
  };
HG_PLAN(8, 8)
HG_PLAN(16, 16)
HG_PLAN(32, 8, 4)
HG_PLAN(64, 8, 8)
HG_PLAN(128, 16, 8)
HG_PLAN(256, 16, 16)
HG_PLAN(512, 8, 8, 8)
HG_PLAN(1024, 16, 8, 8)
HG_PLAN(2048, 16, 16, 8)
HG_PLAN(4096, 16, 16, 16)
// lengths with factors 3 and 5 use the composite radices 6, 9, 12, 15 so that no plan needs more
// than three stages (two shared-memory exchanges)
HG_PLAN(12, 12)
HG_PLAN(15, 15)
HG_PLAN(30, 2, 15)
HG_PLAN(60, 4, 15)
HG_PLAN(120, 8, 15)
HG_PLAN(864, 16, 6, 9)
HG_PLAN(1080, 8, 9, 15)
HG_PLAN(1536, 16, 16, 6)
HG_PLAN(1920, 16, 8, 15)
// common SLM sides (1280 x 720, 1280 x 1024, 1920 x 1152, 1920 x 1200, 2560 x 1440, 2560 x 1600,
// 3840 x 2160): measured on GB300 two to four times faster per pixel than the generic kernels;
// stage orders from a bank-conflict model of every tile shape
HG_PLAN(720, 16, 9, 5)
HG_PLAN(1152, 16, 9, 8)
HG_PLAN(1200, 16, 5, 15)
HG_PLAN(1280, 16, 5, 16)
HG_PLAN(1440, 16, 6, 15)
HG_PLAN(1600, 16, 10, 10)
HG_PLAN(2160, 16, 9, 15)
HG_PLAN(2560, 16, 10, 16)
HG_PLAN(3840, 16, 15, 16)
#undef HG_PLAN

// A second radix plan for some lengths (the same three-stage split in another order, or another
// split).  The order changes the stages' twiddle tables, exchange patterns and thread counts, and
// which plan is faster differs between the row and the column pass (measured on GB300, 2048^2
// GS: 16-8-16 rows 24.4 us against 25.1 with 16-16-8, columns 21.8 against 21.6), so the GS passes
// are compiled with both and hg_plan_autotune picks per pass.  PlanV<N, 0> is the default plan.
template <int N, int PV>
struct PlanV {
  using type = typename PlanFor<N>::type;
};
#define HG_ALT_PLAN(N, ...)          \
  template <>                        \
  struct PlanV<N, 1> {               \
    using type = RList<__VA_ARGS__>; \
  };
HG_ALT_PLAN(864, 9, 6, 16)
HG_ALT_PLAN(1024, 4, 16, 16)
HG_ALT_PLAN(1080, 15, 9, 8)
HG_ALT_PLAN(1536, 16, 6, 16)
HG_ALT_PLAN(1920, 15, 8, 16)
HG_ALT_PLAN(2048, 16, 8, 16)
#undef HG_ALT_PLAN
template <int N>
__host__ __device__ constexpr bool has_alt_plan() {
  return !std::is_same<typename PlanV<N, 1>::type, typename PlanFor<N>::type>::value;
}

// Values a thread holds in the widest stage of plan L when NT threads transform B sequences of
// length N (each stage: ceil(B N / R / NT) butterflies of R values).
template <class L>
struct RValues;
template <int... Rs>
struct RValues<RList<Rs...>> {
  __host__ __device__ static constexpr int max_values(int n, int b, int nt) {
    int v = 0;
    ((v = v > (b * n / Rs + nt - 1) / nt * Rs ? v : (b * n / Rs + nt - 1) / nt * Rs), ...);
    return v;
  }
};
// Fewest threads (a multiple of 32, at most cap) with which no thread holds more than vmax values;
// cap when none is that small.
template <class L>
__host__ __device__ constexpr int pick_threads(int n, int b, int vmax, int cap) {
  for (int nt = 32; nt < cap; nt += 32)
    if (RValues<L>::max_values(n, b, nt) <= vmax) return nt;
  return cap;
}
// value budget per thread: 16 for power-of-two lengths (radix-16 stages), 18 with factors 3 and 5
__host__ __device__ constexpr int value_budget(int n) { return (n & (n - 1)) == 0 ? 16 : 18; }

// Whether rows of length N can be processed as interleaved groups of G butterflies (every stage's
// butterfly count N / R a multiple of G) with the n ^ (G b) swizzle (N a multiple of 16).
template <class L>
struct RAll;
template <int... Rs>
struct RAll<RList<Rs...>> {
  __host__ __device__ static constexpr bool divisible(int n, int g) { return ((n / Rs % g == 0) && ...); }
};
template <int N, int G, int PV = 0>
__host__ __device__ constexpr bool row_tileable() {
  return G > 0 && N % 16 == 0 && N % G == 0 && RAll<typename PlanV<N, PV>::type>::divisible(N, G);
}

// Per-stage twiddle tables of length N.  A stage of radix R after Ns earlier points needs
// w_{Ns R}^{r k} for r = 1..R-1, k = 0..Ns-1; its table stores them r-major, entry (r-1) Ns + k, so a
// warp whose lanes hold consecutive k reads consecutive entries.  The stages read only the r = 1
// row and form the higher powers by multiplication (stage_compute).  The blob holds the tables of
// every stage (Ns > 1) of the forward plan F, then those of the reversed plan that are not already
// present.
template <int N, class F = typename PlanFor<N>::type>
struct TwBlob {
  using Bk = typename RRev<F>::type;
  static constexpr int S = RArr<F>::n;
  __host__ __device__ static constexpr int stage_r(int which, int s) {
    return which == 0 ? RArr<F>::at(s) : RArr<Bk>::at(s);
  }
  __host__ __device__ static constexpr int stage_ns(int which, int s) {
    int ns = 1;
    for (int i = 0; i < s; ++i) ns *= stage_r(which, i);
    return ns;
  }
  __host__ __device__ static constexpr bool in_forward(int ns, int r) {
    for (int s = 1; s < S; ++s)
      if (stage_ns(0, s) == ns && stage_r(0, s) == r) return true;
    return false;
  }
  // offset of the (ns, r) table, or the blob size when (ns, r) == (0, 0)
  __host__ __device__ static constexpr int offset(int ns, int r) {
    int off = 0;
    for (int which = 0; which < 2; ++which)
      for (int s = 1; s < S; ++s) {
        const int ns2 = stage_ns(which, s), r2 = stage_r(which, s);
        if (which == 1 && in_forward(ns2, r2)) continue;
        if (ns2 == ns && r2 == r) return off;
        off += (r2 - 1) * ns2;
      }
    return (ns == 0 && r == 0) ? off : -1;
  }
  static constexpr int size = offset(0, 0);
  // number of distinct stage tables and their (ns, r, offset)
  __host__ __device__ static constexpr int count() {
    int c = 0;
    for (int which = 0; which < 2; ++which)
      for (int s = 1; s < S; ++s)
        if (!(which == 1 && in_forward(stage_ns(which, s), stage_r(which, s)))) ++c;
    return c;
  }
  __host__ __device__ static constexpr int table(int idx, int field) {
    int c = 0;
    for (int which = 0; which < 2; ++which)
      for (int s = 1; s < S; ++s) {
        const int ns2 = stage_ns(which, s), r2 = stage_r(which, s);
        if (which == 1 && in_forward(ns2, r2)) continue;
        if (c == idx) return field == 0 ? ns2 : (field == 1 ? r2 : offset(ns2, r2));
        ++c;
      }
    return -1;
  }
};

// ---------------------------------------------------------------- tile geometry

// B sequences of length N, NT threads.  COLS: a column strip (element (b, n) of the strip at global
// row n, column col0 + b; in shared memory at n * B + b).  Otherwise a row tile (element (b, n) at
// global row row0 + b, column n; in shared memory at b * N + n).
// G_ > 1 (row tiles only): lanes interleave the B rows in groups of G_ consecutive butterflies, so that
// a warp's global accesses of a column-strip-tiled field (G_ = tile width, B G_ = 16) cover whole
// 128-byte lines; shared-memory rows are then swizzled (n ^ G_ b) to keep the exchange conflict-free.
template <int N_, int B_, int NT_, bool COLS_, int G_ = 0>
struct Geo {
  static constexpr int N = N_;
  static constexpr int B = B_;
  static constexpr int NT = NT_;
  static constexpr bool COLS = COLS_;
  static constexpr bool ILV = !COLS_ && G_ > 1 && B_ > 1;

  template <int R>
  __host__ __device__ static constexpr int nbf() {
    return B * N / R;
  }
  template <int R>
  __host__ __device__ static constexpr int bpt() {
    return (nbf<R>() + NT - 1) / NT;
  }
  template <int R>
  __host__ __device__ static constexpr bool exact() {
    return nbf<R>() % NT == 0;
  }

  // Shared-memory slot of element (b, n) in an exchange of layout LAY (exchange_layout below).
  // LAY 0 pads by one float2 per 16: the Stockham stores of a power-of-two radix R = 4, 8, 16 after
  // a power-of-two number of points land on distinct banks within each half-warp.  Interleaved row
  // tiles also swizzle row b by (16 / B) b within each 16-element block, so that the B rows a warp
  // touches at once start on different banks.
  // LAY 1: the exchange after a radix-8 first stage (each thread stores 8 consecutive values).  For
  // 2-row tiles the 8 b swizzle leaves that exchange 2-way conflicted and 12 b makes it
  // conflict-free (measured: row pass 31.2 -> 29.9 us at 2048).  Column strips keep their layout
  // (a row-style one removes the conflicts there too, but measured no faster).
  // LAY 2: unpadded (swizzle kept), for exchanges whose radix or point count is odd (3, 5, 9, 15) or
  // whose radix is not a power of two (6, 12): an odd store stride already meets every bank within a
  // half-warp, and the padding then folds strides onto one another (modelled for every plan and tile
  // shape: 1920-point row tiles after a radix-15 first stage 6-8x the ideal wavefronts padded, 1x
  // unpadded).
  static constexpr int SWZ = B >= 16 ? 1 : 16 / B;
  static constexpr bool ROW_ALT = B == 2 && !COLS;
  template <int LAY = 0>
  __device__ __forceinline__ static int sidx(int b, int n) {
    int i;
    if constexpr (LAY == 1 && ROW_ALT)
      i = ILV ? b * N + (n ^ (12 * b)) : b * N + n;
    else
      i = COLS ? n * B + b : (ILV ? b * N + (n ^ (SWZ * b)) : b * N + n);
    if constexpr (LAY == 2)
      return i;
    else
      return i + (i >> 4);
  }
  // float2 slots of the exchange buffer, rounded up to 128 bytes so that data placed after it is
  // 16-byte aligned (cp.async destinations)
  static constexpr int SM_ELEMS = (B * N + ((B * N) >> 4) + 15) / 16 * 16;

  // butterfly i of thread t in a radix-R stage -> (sequence b, butterfly j); false when past the end
  template <int R>
  __device__ __forceinline__ static bool bf(int t, int i, int& b, int& j) {
    const int u = t + i * NT;
    if constexpr (COLS) {
      b = u % B;
      j = u / B;
    } else if constexpr (ILV) {
      b = (u / G_) % B;
      j = (u / (G_ * B)) * G_ + u % G_;
    } else {
      j = u % (N / R);
      b = u / (N / R);
    }
    return exact<R>() || u < nbf<R>();
  }
};

template <class G, class L>
struct MaxV;
template <class G, int R>
struct MaxV<G, RList<R>> {
  static constexpr int value = G::template bpt<R>() * R;
};
template <class G, int R, int R2, int... Rs>
struct MaxV<G, RList<R, R2, Rs...>> {
  static constexpr int a = G::template bpt<R>() * R;
  static constexpr int b = MaxV<G, RList<R2, Rs...>>::value;
  static constexpr int value = a > b ? a : b;
};

// ---------------------------------------------------------------- stage engine

// Visit every value held for a radix-R first/last stage: f(slot, b, n) with n = j + r N / R.
template <class G, int R, class F>
__device__ __forceinline__ void for_each_slot(int t, F&& f) {
#pragma unroll
  for (int i = 0; i < G::template bpt<R>(); ++i) {
    int b, j;
    if (!G::template bf<R>(t, i, b, j)) continue;
#pragma unroll
    for (int r = 0; r < R; ++r) f(i * R + r, b, j + r * (G::N / R));
  }
}

// As for_each_slot, but f(slot, b, j, r) (n = j + r N / R), for linear addressing in the caller.
template <class G, int R, class F>
__device__ __forceinline__ void for_each_slot_jr(int t, F&& f) {
#pragma unroll
  for (int i = 0; i < G::template bpt<R>(); ++i) {
    int b, j;
    if (!G::template bf<R>(t, i, b, j)) continue;
#pragma unroll
    for (int r = 0; r < R; ++r) f(i * R + r, b, j, r);
  }
}

template <class G, int R, int NS, bool INV, class F, int V>
__device__ __forceinline__ void stage_compute(float2 (&v)[V], int t, const float2* __restrict__ tw) {
#pragma unroll
  for (int i = 0; i < G::template bpt<R>(); ++i) {
    int b, j;
    if (!G::template bf<R>(t, i, b, j)) continue;
    float2* x = &v[i * R];
    if constexpr (NS > 1) {
      constexpr int off = TwBlob<G::N, F>::offset(NS, R);
      static_assert(off >= 0, "missing twiddle table");
      // w^r for r >= 2 by repeated multiplication from the table's w = w_{Ns R}^{j mod Ns}: one load
      // per butterfly instead of R - 1 (the loads measured ~8 % of a GS iteration, the extra
      // multiplications ~1/3 of that); at most R - 2 roundings, relative error < 1e-6
      const float2 w1 = __ldg(tw + off + (j % NS));
      float2 wr = w1;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        if (r > 1) wr = c_mul(wr, w1);
        x[r] = INV ? c_mulc(x[r], wr) : c_mul(x[r], wr);
      }
    }
    dft<R, INV>(x);
  }
}

// Slot index steps of a stage: element n + r * STEP for r = 0..R-1.  When the step in the unpadded
// index (STEP, times B in a column strip) is a multiple of 16, the padded (and swizzled) slot of
// n + r * STEP is the slot of n plus r * 17 * step / 16, so one index is computed per butterfly; an
// unpadded layout steps by the raw index (for interleaved row tiles only when the step leaves the
// swizzled low four bits alone).  -1: no constant step.
template <class G, int STEP, int LAY = 0>
__host__ __device__ constexpr int padded_step() {
  constexpr int raw = G::COLS ? STEP * G::B : STEP;
  if constexpr (LAY == 2) return (!G::ILV || STEP % 16 == 0) ? raw : -1;
  return raw % 16 == 0 ? raw / 16 * 17 : -1;
}

// Layout of the exchange after stage (R, NS) (Geo::sidx): 1 after a radix-8 first stage, 2 when R
// is not a power of two or NS is odd and above 1, else 0.
template <int R, int NS>
__host__ __device__ constexpr int exchange_layout() {
  if (R == 8 && NS == 1) return 1;
  return ((R & (R - 1)) != 0 || (NS > 1 && NS % 2 == 1)) ? 2 : 0;
}

template <class G, int R, int NS, int V>
__device__ __forceinline__ void stage_store(const float2 (&v)[V], float2* sm, int t) {
  constexpr int LAY = exchange_layout<R, NS>();
  constexpr int PS = padded_step<G, NS, LAY>();
#pragma unroll
  for (int i = 0; i < G::template bpt<R>(); ++i) {
    int b, j;
    if (!G::template bf<R>(t, i, b, j)) continue;
    const int base = (j / NS) * NS * R + (j % NS);
    if constexpr (PS > 0) {
      float2* q = sm + G::template sidx<LAY>(b, base);
#pragma unroll
      for (int r = 0; r < R; ++r) q[r * PS] = v[i * R + r];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) sm[G::template sidx<LAY>(b, base + r * NS)] = v[i * R + r];
    }
  }
}

template <class G, int R, int LAY, int V>
__device__ __forceinline__ void stage_load(float2 (&v)[V], const float2* sm, int t) {
  constexpr int PS = padded_step<G, G::N / R, LAY>();
#pragma unroll
  for (int i = 0; i < G::template bpt<R>(); ++i) {
    int b, j;
    if (!G::template bf<R>(t, i, b, j)) continue;
    if constexpr (PS > 0) {
      const float2* q = sm + G::template sidx<LAY>(b, j);
#pragma unroll
      for (int r = 0; r < R; ++r) v[i * R + r] = q[r * PS];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) v[i * R + r] = sm[G::template sidx<LAY>(b, j + r * (G::N / R))];
    }
  }
}

// Run all stages of plan L (registers already hold the first stage's inputs); on return the
// registers hold the last stage's outputs.  Uses sm as the exchange buffer (B*N float2).  F is the
// forward plan of the pass (L is F or F reversed): it names the twiddle blob tw holds.
template <class G, bool INV, int NS, class L, class F = typename PlanFor<G::N>::type>
struct FftRun;
template <class G, bool INV, int NS, int R, int... Rs, class F>
struct FftRun<G, INV, NS, RList<R, Rs...>, F> {
  template <int V>
  __device__ __forceinline__ static void run(float2 (&v)[V], float2* sm, int t, const float2* __restrict__ tw) {
    stage_compute<G, R, NS, INV, F>(v, t, tw);
    if constexpr (sizeof...(Rs) > 0) {
      __syncthreads();  // everyone is done reading sm from the previous exchange
      stage_store<G, R, NS>(v, sm, t);
      __syncthreads();
      stage_load<G, RFirst<RList<Rs...>>::value, exchange_layout<R, NS>()>(v, sm, t);
      FftRun<G, INV, NS * R, RList<Rs...>, F>::run(v, sm, t, tw);
    }
  }
};

}  // namespace hg
