// Host-only checks of the FP32 transform-gain model (exx_gain.cuh), compiled
// by nvcc and run on the CPU (no kernel is launched).  For each line size it
// prints, as one JSON line:
//   err32 / err64: max |model transform - exact DFT| over unit impulses, with
//                  FP32-rounded constants (the model) and with unrounded ones
//   gdev32 / gdev64: max | |d|^2 - 1 | over the x and y/z gains
#include <cmath>
#include <complex>
#include <cstdio>
#include <vector>

#include "exx_gain.cuh"

namespace exx {
// the model's scalar without the FP32 rounding of constants
struct F64x {
  struct Raw {};
  double v;
  F64x() = default;
  __host__ __device__ constexpr F64x(double x) : v(x) {}
  __host__ __device__ constexpr F64x(double x, Raw) : v(x) {}
};
__host__ __device__ inline F64x operator+(F64x a, F64x b) { return F64x(a.v + b.v); }
__host__ __device__ inline F64x operator-(F64x a, F64x b) { return F64x(a.v - b.v); }
__host__ __device__ inline F64x operator*(F64x a, F64x b) { return F64x(a.v * b.v); }
__host__ __device__ inline F64x operator-(F64x a) { return F64x(-a.v); }
struct F64x2 {
  F64x x, y;
};
template <> struct cvec<F64x> { using type = F64x2; };
template <> struct creal<F64x2> { using type = F64x; };
}  // namespace exx

using namespace exx;

// max deviation of the y/z line transform and of the x (real) transform from
// the exact DFT of length 2N over every unit impulse within the inputs
template <int N, bool PER, typename S, int L1O = 0> double transform_error() {
  using M = GainModel<N, PER, S, L1O>;
  using C = typename M::C;
  constexpr int L = M::L, G = M::G;
  double err = 0.0;
  std::vector<C> in(G), out(L), xo(N + 1);
  std::vector<double> rin(G);
  for (int n = 0; n < G; ++n) {
    for (int j = 0; j < G; ++j) {
      in[j] = M::raw(j == n ? 1.0 : 0.0, 0.0);
      rin[j] = j == n ? 1.0 : 0.0;
    }
    M::line(in.data(), out.data());
    M::xline(rin.data(), xo.data());
    for (int k = 0; k < L; ++k) {
      const double a = -2.0 * M_PI * (double)(((long)k * n) % L) / L;
      const std::complex<double> e(std::cos(a), std::sin(a));
      err = std::fmax(err, std::abs(std::complex<double>(out[k].x.v, out[k].y.v) - e));
      if (k <= N) err = std::fmax(err, std::abs(std::complex<double>(xo[k].x.v, xo[k].y.v) - e));
    }
  }
  return err;
}

template <int N, bool PER, typename S, int L1O = 0> double gain_deviation() {
  std::vector<double> gx(N + 1), gz(2 * N);
  GainModel<N, PER, S, L1O>::gains(gx.data(), gz.data());
  double d = 0.0;
  for (double g : gx) d = std::fmax(d, std::fabs(g - 1.0));
  for (double g : gz) d = std::fmax(d, std::fabs(g - 1.0));
  return d;
}

// L1O: the line split of the modelled pass (0: the y pass; split_z(2N): zconv)
template <int N, bool PER, int L1O = 0> void report() {
  std::printf("{\"N\": %d, \"periodic\": %d, \"L1\": %d, \"err32\": %.3e, \"err64\": %.3e, "
              "\"gdev32\": %.3e, \"gdev64\": %.3e}\n",
              N, (int)PER, GainModel<N, PER, F32c, L1O>::L1, transform_error<N, PER, F32c, L1O>(),
              transform_error<N, PER, F64x, L1O>(), gain_deviation<N, PER, F32c, L1O>(),
              gain_deviation<N, PER, F64x, L1O>());
}

int main() {
  report<8, false>();
  report<12, false>();
  report<48, false>();
  report<96, false>();
  report<160, false>();
  report<160, false, split_z(320)>();  // zconv's 20 x 16 split of 320-point lines
  report<4, true>();
  report<24, true>();
  report<48, true>();
  return 0;
}
