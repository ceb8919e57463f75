// Register-resident mixed-radix FFT of one line of N complex points (N = 2^a 3^b).
//
// Each thread holds the N points of its line in registers; every stage is a Stockham
// autosort step (radix 8, 4, 2 or 3) whose indices and twiddle factors are compile-time
// constants, so the whole transform unrolls into straight-line FMA code with no memory
// traffic.  The order of the radices (the schedule) is a per-(precision, N) choice made by the
// tuner from timings (tuned_radix.h); without an entry the stages take 4, then 2, then 3.  DIR = -1 computes X_k = sum_n x_n e^{-2 pi i k n / N}; DIR = +1 the unnormalised
// inverse.  The twiddles e^{DIR 2 pi i m / N} are evaluated at compile time from the Taylor
// series of sin and cos on [0, pi/4] after an exact octant reduction of m/N.
#pragma once

#include <cuda_runtime.h>

namespace dgfs {

template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using C = typename cplx_t<T>::type;

template <typename T> __device__ __forceinline__ C<T> mk(T x, T y) { C<T> r; r.x = x; r.y = y; return r; }
template <typename T> __device__ __forceinline__ C<T> add(C<T> a, C<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C<T> sub(C<T> a, C<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ C<T> cmul(C<T> a, C<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ C<T> scale(C<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// multiply by DIR * i
template <typename T, int DIR> __device__ __forceinline__ C<T> mul_i(C<T> a) {
  return DIR > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}

// ---- compile-time cos / sin of 2 pi a / b -------------------------------------------
constexpr double kTwoPi = 6.283185307179586476925286766559005768;

__host__ __device__ constexpr double taylor_sin(double x) {
  double x2 = x * x, term = x, sum = x;
  for (int k = 1; k < 16; ++k) { term *= -x2 / double((2 * k) * (2 * k + 1)); sum += term; }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int k = 1; k < 16; ++k) { term *= -x2 / double((2 * k - 1) * (2 * k)); sum += term; }
  return sum;
}
// which = 0: cos(2 pi a/b), which = 1: sin(2 pi a/b); exact reduction to [0, pi/4]
__host__ __device__ constexpr double trig2pi(long a, long b, int which) {
  a %= b;
  if (a < 0) a += b;
  bool neg_s = false, neg_c = false, swap = false;
  if (2 * a > b) { a = b - a; neg_s = true; }                 // t -> 1 - t
  if (4 * a > b) { a = b - 2 * a; b = 2 * b; neg_c = true; }  // t -> 1/2 - t
  if (8 * a > b) { a = b - 4 * a; b = 4 * b; swap = true; }   // t -> 1/4 - t
  const double x = kTwoPi * double(a) / double(b);
  double c = taylor_cos(x), s = taylor_sin(x);
  if (swap) { const double t = c; c = s; s = t; }
  if (neg_c) c = -c;
  if (neg_s) s = -s;
  return which == 0 ? c : s;
}

// x * e^{DIR 2 pi i M / N} with trivial factors special-cased
template <typename T, int N, int M, int DIR>
__device__ __forceinline__ C<T> twiddle(C<T> a) {
  constexpr int m = ((M % N) + N) % N;
  if constexpr (m == 0) {
    return a;
  } else if constexpr (2 * m == N) {
    return mk<T>(-a.x, -a.y);
  } else if constexpr (4 * m == N) {
    return mul_i<T, DIR>(a);
  } else if constexpr (4 * m == 3 * N) {
    return mul_i<T, -DIR>(a);
  } else {
    constexpr T c = T(trig2pi(m, N, 0));
    constexpr T s = T(DIR * trig2pi(m, N, 1));
    return mk<T>(a.x * c - a.y * s, a.x * s + a.y * c);
  }
}

// ---- small DFTs ---------------------------------------------------------------------
template <typename T, int DIR> __device__ __forceinline__ void dft2(C<T>* v) {
  const C<T> a = v[0], b = v[1];
  v[0] = add<T>(a, b);
  v[1] = sub<T>(a, b);
}
template <typename T, int DIR> __device__ __forceinline__ void dft4(C<T>* v) {
  const C<T> s02 = add<T>(v[0], v[2]), d02 = sub<T>(v[0], v[2]);
  const C<T> s13 = add<T>(v[1], v[3]), d13 = mul_i<T, DIR>(sub<T>(v[1], v[3]));
  v[0] = add<T>(s02, s13);
  v[2] = sub<T>(s02, s13);
  v[1] = add<T>(d02, d13);
  v[3] = sub<T>(d02, d13);
}
template <typename T, int DIR> __device__ __forceinline__ void dft3(C<T>* v) {
  constexpr T h = T(0.866025403784438646763723170752936183);  // sqrt(3)/2
  const C<T> t = add<T>(v[1], v[2]);
  const C<T> d = mul_i<T, DIR>(sub<T>(v[1], v[2]));
  const C<T> m = mk<T>(v[0].x - T(0.5) * t.x, v[0].y - T(0.5) * t.y);
  v[0] = add<T>(v[0], t);
  v[1] = mk<T>(m.x + h * d.x, m.y + h * d.y);
  v[2] = mk<T>(m.x - h * d.x, m.y - h * d.y);
}
// 8-point DFT: two 4-point DFTs of the even and odd points joined by the eighth roots of unity
// w = e^{DIR 2 pi i / 8}: X_k = E_k + w^k O_k, X_{k+4} = E_k - w^k O_k
template <typename T, int DIR> __device__ __forceinline__ void dft8(C<T>* v) {
  constexpr T r = T(0.707106781186547524400844362104849039);  // 1 / sqrt(2)
  C<T> e[4] = {v[0], v[2], v[4], v[6]};
  C<T> o[4] = {v[1], v[3], v[5], v[7]};
  dft4<T, DIR>(e);
  dft4<T, DIR>(o);
  // w^1 = (1 + DIR i) / sqrt 2, w^2 = DIR i, w^3 = (-1 + DIR i) / sqrt 2
  o[1] = mk<T>(r * (o[1].x - DIR * o[1].y), r * (o[1].y + DIR * o[1].x));
  o[2] = mul_i<T, DIR>(o[2]);
  o[3] = mk<T>(r * (-o[3].x - DIR * o[3].y), r * (-o[3].y + DIR * o[3].x));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = add<T>(e[k], o[k]);
    v[k + 4] = sub<T>(e[k], o[k]);
  }
}
template <typename T, int R, int DIR> __device__ __forceinline__ void dft_small(C<T>* v) {
  if constexpr (R == 2) dft2<T, DIR>(v);
  else if constexpr (R == 3) dft3<T, DIR>(v);
  else if constexpr (R == 8) dft8<T, DIR>(v);
  else dft4<T, DIR>(v);
}

template <int Rem> __host__ __device__ constexpr int pick_radix() { return Rem % 4 == 0 ? 4 : (Rem % 2 == 0 ? 2 : 3); }

// Radix schedule of a line length: the decimal digits of the code, first stage first (442 =
// radix 4, 4, then 2); 0 selects the default order (4, then 2, then 3).
template <typename T, int N> struct RadixCode { static constexpr int value = 0; };
__host__ __device__ constexpr int code_digits(int c) { return c < 10 ? 1 : 1 + code_digits(c / 10); }
__host__ __device__ constexpr int pow10_int(int e) { return e == 0 ? 1 : 10 * pow10_int(e - 1); }
__host__ __device__ constexpr int code_radix(int code, int stage) {
  return (code / pow10_int(code_digits(code) - 1 - stage)) % 10;
}
__host__ __device__ constexpr int code_product(int code) { return code < 10 ? code : (code % 10) * code_product(code / 10); }
#define DGFS_RADIX(TT, NN, CODE)                                                      \
  template <> struct RadixCode<TT, NN> {                                              \
    static constexpr int value = CODE;                                                \
    static_assert(code_product(CODE) == NN, "a radix schedule must multiply to N");   \
  };
#include "tuned_radix.h"
#undef DGFS_RADIX

// twiddles of the radix-R butterfly with k S = KS: v[q] *= e^{DIR 2 pi i q KS / N}, q >= 1
template <typename T, int N, int R, int KS, int DIR, int Q>
__device__ __forceinline__ void twiddle_all(C<T>* v) {
  if constexpr (Q < R) {
    v[Q] = twiddle<T, N, Q * KS, DIR>(v[Q]);
    twiddle_all<T, N, R, KS, DIR, Q + 1>(v);
  }
}

// one Stockham butterfly J of a radix-R stage with span Ns
template <typename T, int N, int R, int Ns, int DIR, int J>
__device__ __forceinline__ void stage_body(const C<T> (&x)[N], C<T> (&y)[N]) {
  if constexpr (J < N / R) {
    constexpr int k = J % Ns;
    constexpr int S = N / (Ns * R);
    C<T> v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = x[J + q * (N / R)];
    twiddle_all<T, N, R, k * S, DIR, 1>(v);
    dft_small<T, R, DIR>(v);
    constexpr int base = (J / Ns) * Ns * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) y[base + q * Ns] = v[q];
    stage_body<T, N, R, Ns, DIR, J + 1>(x, y);
  }
}

template <typename T, int N, int Ns, int DIR, int CODE, int STAGE>
__device__ __forceinline__ void fft_stages(C<T> (&x)[N]) {
  if constexpr (Ns < N) {
    constexpr int R = CODE != 0 ? code_radix(CODE, STAGE) : pick_radix<N / Ns>();
    static_assert(R == 2 || R == 3 || R == 4 || R == 8, "radices 2, 3, 4, 8");
    static_assert((N / Ns) % R == 0, "N must be 2^a 3^b and the schedule must divide it");
    C<T> y[N];
    stage_body<T, N, R, Ns, DIR, 0>(x, y);
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = y[i];
    fft_stages<T, N, Ns * R, DIR, CODE, STAGE + 1>(x);
  }
}

// In-register FFT of one line: DIR = -1 forward, +1 unnormalised inverse.
template <typename T, int N, int DIR>
__device__ __forceinline__ void fft_line(C<T> (&x)[N]) {
  fft_stages<T, N, 1, DIR, RadixCode<T, N>::value, 0>(x);
}

}  // namespace dgfs
