// Host-only check of the register DFT templates (exx_fft.cuh): every length
// the transforms use, in FP64 on the CPU (no kernel is launched), against the
// DFT written out as a sum.  For each length P and sign it prints one JSON
// line with the largest deviation of
//   full:    dft<P>           (all P outputs, natural order)
//   halfin:  dft_halfin<P>    (inputs P/2..P-1 taken as zero), even P
//   halfout: dft_halfout<P>   (outputs 0..P/2-1 only), even P
// from the direct sum, relative to the largest output, and whether the length
// takes the prime-factor form (pfa: coprime factors, no twiddles).
#include <cmath>
#include <complex>
#include <cstdio>

#include "exx_fft.cuh"

using namespace exx;
using cd = std::complex<double>;

// seeded inputs in [-1, 1) (64-bit linear congruential generator)
static double next_uniform(unsigned long long& s) {
  s = s * 6364136223846793005ull + 1442695040888963407ull;
  return (double)(s >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

static void direct(const cd* x, cd* X, int P, int sign, int nin) {
  for (int k = 0; k < P; ++k) {
    cd s = 0;
    for (int n = 0; n < nin; ++n) {
      const double a = sign * 2.0 * M_PI * (double)(((long)n * k) % P) / P;
      s += x[n] * cd(std::cos(a), std::sin(a));
    }
    X[k] = s;
  }
}

template <int P, int SIGN> void check() {
  unsigned long long seed = 1000003ull * P + (SIGN > 0);
  cd x[P], X[P];
  double2 v[P];
  for (int n = 0; n < P; ++n) x[n] = cd(next_uniform(seed), next_uniform(seed));
  double full = 0, hin = -1, hout = -1, scale = 0;
  direct(x, X, P, SIGN, P);
  for (int k = 0; k < P; ++k) scale = std::fmax(scale, std::abs(X[k]));
  for (int n = 0; n < P; ++n) v[n] = make_double2(x[n].real(), x[n].imag());
  dft<P, 1, SIGN>(v);
  for (int k = 0; k < P; ++k) full = std::fmax(full, std::abs(cd(v[k].x, v[k].y) - X[k]) / scale);
  if constexpr (P % 2 == 0) {
    direct(x, X, P, SIGN, P / 2);
    double sc = 0;
    for (int k = 0; k < P; ++k) sc = std::fmax(sc, std::abs(X[k]));
    for (int n = 0; n < P; ++n) v[n] = make_double2(n < P / 2 ? x[n].real() : 7.0, n < P / 2 ? x[n].imag() : 7.0);
    dft_halfin<P, SIGN>(v);
    hin = 0;
    for (int k = 0; k < P; ++k) hin = std::fmax(hin, std::abs(cd(v[k].x, v[k].y) - X[k]) / sc);
    direct(x, X, P, SIGN, P);
    for (int n = 0; n < P; ++n) v[n] = make_double2(x[n].real(), x[n].imag());
    dft_halfout<P, SIGN>(v);
    hout = 0;
    for (int k = 0; k < P / 2; ++k) hout = std::fmax(hout, std::abs(cd(v[k].x, v[k].y) - X[k]) / scale);
  }
  std::printf("{\"P\": %d, \"sign\": %d, \"pfa\": %d, \"full\": %.3e, \"halfin\": %.3e, \"halfout\": %.3e}\n",
              P, SIGN, (int)(P != 2 && P != 3 && P != 4 && P != 5 && P != 7 && pfa_a(P) != P), full, hin, hout);
}

template <int... Ps> void check_all() {
  (check<Ps, -1>(), ...);
  (check<Ps, 1>(), ...);
}

int main() {
  // every length with prime factors <= 7 up to 20, and a few longer ones
  check_all<2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 18, 20, 21, 24, 28, 30, 32>();
  return 0;
}
