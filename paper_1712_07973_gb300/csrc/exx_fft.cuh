// Register-resident mixed-radix DFTs for the exact-exchange Poisson path.
//
// Every transform length used on the path is 2n = L = L1 * L2 with small
// factors of 2, 3, 5 and 7.  A line of length L is transformed by the
// four-step (two-pass) decomposition: L2 sub-DFTs of length L1, a twiddle,
// then L1 sub-DFTs of length L2.  Each sub-DFT runs entirely in one thread's
// registers (fully unrolled, twiddles known at compile time); the exchange
// between the two passes goes through shared memory.
//
// Zero padding (Sec. 2.1.2 of arXiv 1712.07973: the free-boundary convolution
// is computed exactly with a padded FFT) makes half of every forward input
// and half of every inverse output unneeded; dft_halfin / dft_halfout prune
// the first / last butterfly level accordingly.
//
// Sign convention: SIGN = -1 forward (exp(-2 pi i nk/P)), +1 inverse, both
// unnormalised.
#pragma once

#include <cuda_runtime.h>
#include <type_traits>
#include <utility>

#ifndef EXX_HD
#define EXX_HD __host__ __device__ __forceinline__
#endif

namespace exx {

// ---------------------------------------------------------------- complex
template <typename R> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };
template <typename R> using cplx = typename cvec<R>::type;

template <typename C> struct creal;
template <> struct creal<float2> { using type = float; };
template <> struct creal<double2> { using type = double; };

template <typename C>
EXX_HD C mkc(typename creal<C>::type x, typename creal<C>::type y) {
  C r;
  r.x = x;
  r.y = y;
  return r;
}
// Complex sum and difference.  FP32 on the device: one packed two-lane
// instruction (add.rn.f32x2, sm_100 and later) for the real and imaginary
// parts, each lane rounded like a scalar add, in half the issue slots; the
// butterflies' additions are most of a sub-DFT's arithmetic (pipeline -2.1%
// at 160^3, inv_yx -5.7%).  Sums the compiler used to fuse with a product
// into one FMA are now rounded twice, so FP32 results move in the last bits.
template <typename C> EXX_HD C cadd(C a, C b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  if constexpr (std::is_same<C, float2>::value) return __fadd2_rn(a, b);
#endif
  return mkc<C>(a.x + b.x, a.y + b.y);
}
template <typename C> EXX_HD C csub(C a, C b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  if constexpr (std::is_same<C, float2>::value) return __fadd2_rn(a, make_float2(-b.x, -b.y));
#endif
  return mkc<C>(a.x - b.x, a.y - b.y);
}
template <typename C> EXX_HD C cmul(C a, C b) {
  return mkc<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> EXX_HD C cmulc(C a, C b) {
  return mkc<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> EXX_HD C cscale(C a, typename creal<C>::type s) {
  return mkc<C>(a.x * s, a.y * s);
}
template <typename C> EXX_HD C cconj(C a) { return mkc<C>(a.x, -a.y); }
// multiply by i * SIGN  (SIGN = +1: i, SIGN = -1: -i)
template <int SIGN, typename C> EXX_HD C mul_si(C a) {
  return SIGN > 0 ? mkc<C>(-a.y, a.x) : mkc<C>(a.y, -a.x);
}

// ------------------------------------------------- compile-time trigonometry
// cos / sin of 2 pi num / den: exact reduction of the rational argument to
// the nearest quarter turn, |x| <= pi/4, then the Taylor series (Horner form,
// 13 terms: the first neglected term is below 1e-22).
__host__ __device__ constexpr double tsin_q(double x) {
  const double x2 = x * x;
  double s = 0.0;
  for (int k = 13; k >= 1; --k) s = 1.0 - s * x2 / ((2.0 * k) * (2.0 * k + 1.0));
  return x * s;
}
__host__ __device__ constexpr double tcos_q(double x) {
  const double x2 = x * x;
  double s = 0.0;
  for (int k = 13; k >= 1; --k) s = 1.0 - s * x2 / ((2.0 * k - 1.0) * (2.0 * k));
  return s;
}
constexpr double kTwoPi = 6.283185307179586476925286766559;
__host__ __device__ constexpr long pmod(long a, long m) { return ((a % m) + m) % m; }
// 2 pi a / den = q * pi/2 + x with q = nearest quarter, x = 2 pi (4a - q den) / (4 den)
__host__ __device__ constexpr long quarter(long a, long den) { return (8 * a + den) / (2 * den); }
__host__ __device__ constexpr double cos2pi(long num, long den) {
  const long a = pmod(num, den);
  const long q = quarter(a, den);
  const double x = (kTwoPi / (4.0 * den)) * (double)(4 * a - q * den);
  const double c = tcos_q(x), s = tsin_q(x);
  switch (q & 3) {
    case 0: return c;
    case 1: return -s;
    case 2: return -c;
    default: return s;
  }
}
__host__ __device__ constexpr double sin2pi(long num, long den) {
  const long a = pmod(num, den);
  const long q = quarter(a, den);
  const double x = (kTwoPi / (4.0 * den)) * (double)(4 * a - q * den);
  const double c = tcos_q(x), s = tsin_q(x);
  switch (q & 3) {
    case 0: return s;
    case 1: return c;
    case 2: return -s;
    default: return -c;
  }
}

// compile-time loop: f is called with ic<0>, ic<1>, ... (usable as constants)
template <int I> struct ic {
  static constexpr int value = I;
  __host__ __device__ constexpr operator int() const { return I; }
};
template <int... I, typename F>
EXX_HD void sfor_impl(std::integer_sequence<int, I...>, F&& f) {
  (f(ic<I>{}), ...);
}
template <int N, typename F> EXX_HD void sfor(F&& f) {
  sfor_impl(std::make_integer_sequence<int, N>{}, f);
}

// ------------------------------------------------------ constant products
// x * k and y + x * k for a constant k (rounded to the working precision), and
// a * (c + i s).  In FP32 the rounding of the constants makes each forward
// transform a fixed map whose per-frequency gain differs from 1 by ~1e-7;
// the gain is modelled on the host (exx_gain.cuh) and divided out of the
// kernel table used for the energy.
template <typename R> EXX_HD R kmul(R x, double k) { return x * (R)k; }
template <typename R> EXX_HD R kfma(R x, double k, R y) { return x * (R)k + y; }
template <typename C> EXX_HD C crot(C a, double c, double s) {
  using R = typename creal<C>::type;
  return cmul(a, mkc<C>((R)c, (R)s));
}

// a * omega^E, omega = exp(SIGN 2 pi i / P)
template <int SIGN, int P, int E, typename C> EXX_HD C twmul(C a) {
  constexpr long e = pmod(E, P);
  if constexpr (e == 0) {
    return a;
  } else if constexpr (4 * e == P) {  // omega^{P/4} = SIGN i
    return mul_si<SIGN>(a);
  } else if constexpr (2 * e == P) {
    return mkc<C>(-a.x, -a.y);
  } else if constexpr (4 * e == 3 * P) {
    return mul_si<-SIGN>(a);
  } else if constexpr (8 * e == P || 8 * e == 3 * P || 8 * e == 5 * P || 8 * e == 7 * P) {
    // odd multiples of pi/4: (cs + i ss) / sqrt2 with cs, ss = +-1
    constexpr double r = 0.70710678118654752440084436210485;
    constexpr bool cp = cos2pi(E, P) > 0;
    constexpr bool sp = (SIGN * sin2pi(E, P)) > 0;
    const auto re = cp ? (sp ? a.x - a.y : a.x + a.y) : (sp ? -a.x - a.y : -a.x + a.y);
    const auto im = cp ? (sp ? a.y + a.x : a.y - a.x) : (sp ? -a.y + a.x : -a.y - a.x);
    return mkc<C>(kmul(re, r), kmul(im, r));
  } else {
    return crot(a, cos2pi(E, P), SIGN * sin2pi(E, P));
  }
}

// ------------------------------------------------------------ DFT kernels
// v[S*i], i < P : in-place DFT, natural order in and out.

template <int P> struct first_factor {
  static constexpr int value = (P % 4 == 0 && P > 4) ? 4
                               : (P % 2 == 0) ? 2
                               : (P % 3 == 0) ? 3
                               : (P % 5 == 0) ? 5
                               : (P % 7 == 0) ? 7
                                              : P;
};

template <int P, int S, int SIGN, typename C> EXX_HD void dft(C* v);

template <int S, typename C> EXX_HD void dft2(C* v) {
  C a = v[0], b = v[S];
  v[0] = cadd(a, b);
  v[S] = csub(a, b);
}

template <int S, int SIGN, typename C> EXX_HD void dft3(C* v) {
  using R = typename creal<C>::type;
  constexpr double s3 = SIGN * 0.86602540378443864676372317075294;
  C a = v[0], b = v[S], c = v[2 * S];
  C t1 = cadd(b, c);
  C t2 = mkc<C>(a.x - R(0.5) * t1.x, a.y - R(0.5) * t1.y);
  C d = csub(b, c);
  C t3 = mkc<C>(-kmul(d.y, s3), kmul(d.x, s3));  // i * s3 * (b - c)
  v[0] = cadd(a, t1);
  v[S] = cadd(t2, t3);
  v[2 * S] = csub(t2, t3);
}

template <int S, int SIGN, typename C> EXX_HD void dft4(C* v) {
  C a = v[0], b = v[S], c = v[2 * S], d = v[3 * S];
  C s0 = cadd(a, c), s1 = csub(a, c), s2 = cadd(b, d), s3 = mul_si<SIGN>(csub(b, d));
  v[0] = cadd(s0, s2);
  v[2 * S] = csub(s0, s2);
  v[S] = cadd(s1, s3);
  v[3 * S] = csub(s1, s3);
}

// odd prime P: X_k = x0 + sum_{j=1}^{(P-1)/2} [(x_j + x_{P-j}) cos(2 pi jk/P)
//                                               + SIGN i (x_j - x_{P-j}) sin(2 pi jk/P)]
template <int P, int S, int SIGN, typename C> EXX_HD void dft_prime(C* v) {
  using R = typename creal<C>::type;
  constexpr int H = (P - 1) / 2;
  C sp[H], sm[H];
  sfor<H>([&](auto J) {
    constexpr int j = J + 1;
    sp[J] = cadd(v[j * S], v[(P - j) * S]);
    sm[J] = csub(v[j * S], v[(P - j) * S]);
  });
  C x0 = v[0];
  C tot = x0;
  sfor<H>([&](auto J) { tot = cadd(tot, sp[J]); });
  sfor<H>([&](auto K) {
    constexpr int k = K + 1;
    R re = x0.x, im = x0.y, qre = 0, qim = 0;
    sfor<H>([&](auto J) {
      constexpr int j = J + 1;
      constexpr double c = cos2pi((long)j * k, P);
      constexpr double s = SIGN * sin2pi((long)j * k, P);
      re = kfma(sp[J].x, c, re);
      im = kfma(sp[J].y, c, im);
      qre = kfma(sm[J].y, -s, qre);  // real part of i * s * sm
      qim = kfma(sm[J].x, s, qim);
    });
    v[k * S] = mkc<C>(re + qre, im + qim);
    v[(P - k) * S] = mkc<C>(re - qre, im - qim);
  });
  v[0] = tot;
}

// composite P = A * B (A = first factor): input n = B*n1 + n2, output k1 + A*k2
template <int P, int S, int SIGN, typename C> EXX_HD void dft_composite(C* v) {
  constexpr int A = first_factor<P>::value;
  constexpr int B = P / A;
  // step 1: B DFTs of length A over n1 (stride B*S), in place
  sfor<B>([&](auto N2) { dft<A, B * S, SIGN>(v + N2 * S); });
  // twiddle: element at (B*k1 + n2) *= omega_P^{n2 k1}
  sfor<A>([&](auto K1) {
    sfor<B>([&](auto N2) {
      constexpr int idx = (B * K1 + N2) * S;
      v[idx] = twmul<SIGN, P, (int)(N2 * K1)>(v[idx]);
    });
  });
  // step 2: A DFTs of length B over n2 (contiguous blocks of B)
  sfor<A>([&](auto K1) { dft<B, S, SIGN>(v + B * K1 * S); });
  // position (B*k1 + k2) holds X[k1 + A*k2]: transpose to natural order
  C t[P];
  sfor<A>([&](auto K1) { sfor<B>([&](auto K2) { t[K1 + A * K2] = v[(B * K1 + K2) * S]; }); });
  sfor<P>([&](auto I) { v[I * S] = t[I]; });
}

// Coprime split P = A * B (A the largest power of P's smallest prime factor;
// B = 1 for a prime power) and modular inverses, for the prime-factor
// (Good-Thomas) form below.
__host__ __device__ constexpr int pfa_a(int p) {
  int q = 2;
  while (p % q != 0) ++q;
  int a = 1;
  while (p % q == 0) {
    p /= q;
    a *= q;
  }
  return a;
}
__host__ __device__ constexpr int inv_mod(int a, int m) {
  for (int x = 1; x < m; ++x)
    if ((a * x) % m == 1) return x;
  return 1;
}

// P = A * B with gcd(A, B) = 1, no twiddle factors (Good-Thomas): input
// index n = (B n1 + A n2) mod P, output index k = (B b k1 + A a k2) mod P with
// b = B^-1 mod A and a = A^-1 mod B; then omega_P^(n k) = omega_A^(n1 k1)
// omega_B^(n2 k2), so X = DFT_B over n2 of DFT_A over n1.  Both index maps are
// register renames; the twiddles of the Cooley-Tukey form (4(A-1)(B-1) real
// operations) disappear.
template <int P, int S, int SIGN, typename C> EXX_HD void dft_pfa(C* v) {
  constexpr int A = pfa_a(P), B = P / A;
  constexpr int bi = inv_mod(B % A, A), ai = inv_mod(A % B, B);
  C t[P];
  sfor<A>([&](auto N1) { sfor<B>([&](auto N2) { t[N1 * B + N2] = v[((B * N1 + A * N2) % P) * S]; }); });
  sfor<B>([&](auto N2) { dft<A, B, SIGN>(t + N2); });       // over n1 (stride B)
  sfor<A>([&](auto K1) { dft<B, 1, SIGN>(t + K1 * B); });   // over n2
  sfor<A>([&](auto K1) {
    sfor<B>([&](auto K2) { v[(((long)B * bi * K1 + (long)A * ai * K2) % P) * S] = t[K1 * B + K2]; });
  });
}

template <int P, int S, int SIGN, typename C> EXX_HD void dft(C* v) {
  if constexpr (P == 1) {
  } else if constexpr (P == 2) {
    dft2<S>(v);
  } else if constexpr (P == 3) {
    dft3<S, SIGN>(v);
  } else if constexpr (P == 4) {
    dft4<S, SIGN>(v);
  } else if constexpr (P == 5 || P == 7) {
    dft_prime<P, S, SIGN>(v);
  } else {
    static_assert(first_factor<P>::value != P, "DFT length with a prime factor > 7");
    if constexpr (pfa_a(P) != P) dft_pfa<P, S, SIGN>(v);  // coprime factors
    else dft_composite<P, S, SIGN>(v);                     // a prime power
  }
}

// Pruned input: only v[0..P/2) are nonzero (the rest is ignored).  Output all
// P values in natural order.  X[2k] = DFT_{P/2}(x), X[2k+1] = DFT_{P/2}(x w^j).
template <int P, int SIGN, typename C> EXX_HD void dft_halfin(C* v) {
  static_assert(P % 2 == 0, "pruned DFT needs an even length");
  constexpr int H = P / 2;
  C e[H], o[H];
  sfor<H>([&](auto J) {
    e[J] = v[J];
    o[J] = twmul<SIGN, P, (int)J>(v[J]);
  });
  dft<H, 1, SIGN>(e);
  dft<H, 1, SIGN>(o);
  sfor<H>([&](auto K) {
    v[2 * K] = e[K];
    v[2 * K + 1] = o[K];
  });
}

// Pruned output: all P inputs, only outputs y[0..P/2) are produced (into
// v[0..P/2)).  y[j] = DFT_{P/2}(x_even)[j] + w^j DFT_{P/2}(x_odd)[j].
template <int P, int SIGN, typename C> EXX_HD void dft_halfout(C* v) {
  static_assert(P % 2 == 0, "pruned DFT needs an even length");
  constexpr int H = P / 2;
  C e[H], o[H];
  sfor<H>([&](auto J) {
    e[J] = v[2 * J];
    o[J] = v[2 * J + 1];
  });
  dft<H, 1, SIGN>(e);
  dft<H, 1, SIGN>(o);
  sfor<H>([&](auto J) { v[J] = cadd(e[J], twmul<SIGN, P, (int)J>(o[J])); });
}

// Four-step split of a line length L = L1 * L2: L1 even (pruning), L1 <= 16,
// L2 <= 20, both with factors in {2, 3, 5, 7}.
__host__ __device__ constexpr bool smooth7(int p) {
  while (p % 2 == 0) p /= 2;
  while (p % 3 == 0) p /= 3;
  while (p % 5 == 0) p /= 5;
  while (p % 7 == 0) p /= 7;
  return p == 1;
}
__host__ __device__ constexpr int split_l1(int L) {
  for (int a = 16; a >= 2; a -= 2)
    if (L % a == 0 && L / a <= 20 && smooth7(a) && smooth7(L / a)) return a;
  return 0;
}
// Split of the z lines (zconv).  Its middle pass, the heaviest (forward DFT
// of length L2, kernel multiply, inverse), has L1 units over the CTA's warps:
// where L = 20 L2 with 12 <= L2 <= 16 (L = 320), L1 = 20 and L2 = 16 give ten
// warps two full rounds there, against 16 units of DFT20 for the 16 x 20
// split (six of ten warps busy in the second round).
__host__ __device__ constexpr int split_z(int L) {
  return (L % 20 == 0 && L / 20 >= 12 && L / 20 <= 16 && smooth7(L / 20)) ? 20 : split_l1(L);
}

}  // namespace exx
