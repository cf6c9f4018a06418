// Systematic gain of the FP32 forward transforms, and its removal from the
// Parseval energy.
//
// FP32 constants (sub-DFT rotations and twiddle tables) are rounded to
// nearest; the rounding changes the modulus of each constant slightly, and a
// transform chains several of them per output, so the FP32 forward transform
// is a fixed linear map Ft = F + dF whose outputs come out scaled by a
// frequency-dependent factor d(k) = <F_k, Ft_k> / <F_k, F_k> (rows over the
// unpadded inputs).  The energy sum over |rho_hat|^2 inherits |d|^2 - 1
// (~ -5e-8 per transform) as a bias, while the remaining part of dF only adds
// unbiased noise.  The factors are computed here on the host, from a model
// that runs the kernels' own sub-DFT code with FP64 arithmetic and FP32-
// rounded constants, and are divided out of the kernel spectrum used for the
// energy: Ghat'(kx, ky, kz) = Ghat / (|dx(kx)|^2 |dy(ky)|^2 |dz(kz)|^2).  The y
// and z passes are the same operator (dy = dz).
#pragma once

#include <cmath>
#include <complex>
#include <vector>

#include "exx_kernels.cuh"

namespace exx {

// Scalar of the model: FP64 value and arithmetic; a conversion from double
// (how the sub-DFT code forms its constants) rounds to FP32 first.
struct F32c {
  struct Raw {};
  double v;
  F32c() = default;
  __host__ __device__ constexpr F32c(double x) : v((double)(float)x) {}
  __host__ __device__ constexpr F32c(double x, Raw) : v(x) {}
};
__host__ __device__ inline F32c operator+(F32c a, F32c b) { return F32c(a.v + b.v, F32c::Raw{}); }
__host__ __device__ inline F32c operator-(F32c a, F32c b) { return F32c(a.v - b.v, F32c::Raw{}); }
__host__ __device__ inline F32c operator*(F32c a, F32c b) { return F32c(a.v * b.v, F32c::Raw{}); }
__host__ __device__ inline F32c operator-(F32c a) { return F32c(-a.v, F32c::Raw{}); }
struct F32c2 {
  F32c x, y;
};
template <> struct cvec<F32c> { using type = F32c2; };
template <> struct creal<F32c2> { using type = F32c; };

// PER: periodic boundary conditions (full lines of 2N points, nothing pruned);
// otherwise free (lines of N points padded to 2N).  S: the model's scalar
// (F32c; a type with the same interface that does not round gives |d|^2 = 1).
// L1O: the line split of the modelled pass (0: split_l1, the y pass; the z
// pass of zconv uses split_z).
template <int N, bool PER = false, typename S = F32c, int L1O = 0> struct GainModel {
  using R = S;
  using C = typename cvec<S>::type;
  static constexpr int L = 2 * N, L1 = L1O ? L1O : split_l1(L), L2 = L / L1, H1 = L1 / 2;
  static constexpr int X1 = split_x(N), X2 = N / X1;
  static constexpr int G = PER ? L : N;  // input samples per line
  static constexpr int NIN = PER ? L1 : H1;
  static constexpr bool PX = !PER && (N % 2) == 0;
  static constexpr int XIN = PX ? X1 / 2 : X1;

  // table entry w^e = exp(-2 pi i e / L), rounded as build_twiddles rounds it
  static C tw(long e) {
    const double a = -M_PI * (double)(e % L) / (double)N;
    return mkc<C>(R(std::cos(a)), R(std::sin(a)));
  }
  static C raw(double a, double b) { return mkc<C>(R(a, typename R::Raw{}), R(b, typename R::Raw{})); }

  // forward line transform of the y and z passes: in[n], n < G -> out[k]
  static void line(const C* in, C* out) {
    C B[L];  // [n2][k1]
    for (int n2 = 0; n2 < L2; ++n2) {
      C v[L1];
      for (int n1 = 0; n1 < NIN; ++n1) v[n1] = in[L2 * n1 + n2];
      dft_fwd_in<L1, PER>(v);
      B[n2 * L1] = v[0];
      for (int k1 = 1; k1 < L1; ++k1) B[n2 * L1 + k1] = cmul(v[k1], tw((long)n2 * k1));
    }
    for (int k1 = 0; k1 < L1; ++k1) {
      C v[L2];
      for (int n2 = 0; n2 < L2; ++n2) v[n2] = B[n2 * L1 + k1];
      dft<L2, 1, -1>(v);
      for (int k2 = 0; k2 < L2; ++k2) out[k1 + L1 * k2] = v[k2];
    }
  }

  // forward x pass: real in[m], m < G -> half spectrum out[k], k = 0..N
  static void xline(const double* in, C* out) {
    C Z1[N], Z[N];
    for (int n2 = 0; n2 < X2; ++n2) {
      C v[X1];
      for (int n1 = 0; n1 < X1; ++n1) v[n1] = raw(0.0, 0.0);
      for (int n1 = 0; n1 < XIN; ++n1) {
        const int m = X2 * n1 + n2;
        v[n1] = raw(2 * m < G ? in[2 * m] : 0.0, 2 * m + 1 < G ? in[2 * m + 1] : 0.0);
      }
      if constexpr (PX) dft_halfin<X1, -1>(v);
      else dft<X1, 1, -1>(v);
      Z1[n2 * X1] = v[0];
      for (int k1 = 1; k1 < X1; ++k1) Z1[n2 * X1 + k1] = cmul(v[k1], tw((long)2 * n2 * k1));
    }
    for (int k1 = 0; k1 < X1; ++k1) {
      C v[X2];
      for (int n2 = 0; n2 < X2; ++n2) v[n2] = Z1[n2 * X1 + k1];
      dft<X2, 1, -1>(v);
      for (int k2 = 0; k2 < X2; ++k2) Z[k1 + X1 * k2] = v[k2];
    }
    out[0] = raw(Z[0].x.v + Z[0].y.v, 0.0);
    out[N] = raw(Z[0].x.v - Z[0].y.v, 0.0);
    for (int k = 1; k <= N / 2; ++k) {
      if (2 * k == N) out[k] = mkc<C>(Z[k].x, -Z[k].y);
      else split_step(Z[k], Z[N - k], tw(k), out[k], out[N - k]);
    }
  }

  // |d|^2 per output: gx[k], k = 0..N (x pass); gz[k], k < L (y and z passes)
  static void gains(double* gx, double* gz) {
    std::vector<std::complex<double>> az(L), ax(N + 1);
    std::vector<C> in(G), out(L), xo(N + 1);
    std::vector<double> rin(G);
    for (int n = 0; n < G; ++n) {
      for (int j = 0; j < G; ++j) {
        in[j] = raw(j == n ? 1.0 : 0.0, 0.0);
        rin[j] = j == n ? 1.0 : 0.0;
      }
      line(in.data(), out.data());
      xline(rin.data(), xo.data());
      for (int k = 0; k < L; ++k) {
        const double a = M_PI * (double)(((long)k * n) % L) / (double)N;  // conj of F_kn
        az[k] += std::complex<double>(std::cos(a), std::sin(a)) *
                 std::complex<double>(out[k].x.v, out[k].y.v);
        if (k <= N)
          ax[k] += std::complex<double>(std::cos(a), std::sin(a)) *
                   std::complex<double>(xo[k].x.v, xo[k].y.v);
      }
    }
    for (int k = 0; k < L; ++k) gz[k] = std::norm(az[k] / (double)G);
    for (int k = 0; k <= N; ++k) gx[k] = std::norm(ax[k] / (double)G);
  }
};

}  // namespace exx
