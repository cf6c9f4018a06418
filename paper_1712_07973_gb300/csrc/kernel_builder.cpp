// Host-side FP64 builder of the free-boundary Poisson kernel spectrum.
//
// The paper solves lap V_ij = -4 pi rho_ij by convolving rho_ij with a Green's
// function discretised on the uniform mesh, exactly, through an FFT on a grid
// zero-padded to 2n points per axis (arXiv 1712.07973, Sec. 2.1.2).  It does
// not print the discretisation; this library uses the band-limited kernel
//
//   G[m] = h^3 G_BL(m h),  G_BL(r) = (2 pi)^-3 int_{|k_d| <= pi/h} 4 pi/k^2 e^{ik.r} d^3k,
//
// (the exact potential of densities band-limited to the mesh's Brillouin zone)
// or, on request, the point-sampled Hockney kernel h^3/|m h|, or the
// band-limited short-range kernel erfc(omega r)/r of screened hybrids, whose
// t-integral below runs from omega (erfc(w r)/r = (2/sqrt pi) int_w^inf e^{-t^2 r^2} dt).
//
// Route used here (distinct from the FP64 oracle's real-space route): with
// 1/r = (2/sqrt pi) int_0^inf exp(-t^2 r^2) dt every term of the t-integral is
// separable, so the padded spectrum itself separates per t:
//
//   Ghat[kx,ky,kz] = h^2 (2/sqrt pi) int_0^inf  gh(t,kx) gh(t,ky) gh(t,kz) dt,
//   gh(t,k) = sum_{d=-(n-1)}^{n} g(t,d) cos(pi k d / n)          (windowed DFT)
//   g(t,x)  = 1/(sqrt(pi) t) int_0^pi exp(-q^2/(4t^2)) cos(q x) dq (h = 1 units)
//
// The t-integral uses the exp-sinh rule t = t0 + exp(pi/2 sinh s) (double
// exponential decay at both ends); g uses composite 16-point Gauss-Legendre in
// q, or exp(-t^2 x^2) when t <= 0.2 (the neglected tail is below erfc(2.5 pi)).
// The slot d = n of the periodic embedding is never reached by outputs in
// [0, n) and carries G[n], which keeps the spectrum real and even.

#include <cmath>
#include <cstddef>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace exx_host {

namespace {

const double kPi = 3.14159265358979323846264338327950288;

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_m.
void gauss_legendre(int m, std::vector<double>& x, std::vector<double>& w) {
  x.assign(m, 0.0);
  w.assign(m, 0.0);
  for (int i = 0; i < m; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (m + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= m; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_m(z), p0 = P_{m-1}(z)
      dp = m * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Separable (t-node) spectrum: A[t][k] = gh(t,k) at the nodes of the t rule
// on [t0, inf) (t0 = 0: full Coulomb kernel; t0 = omega h: erfc(omega r)/r).
// Optionally also AD[t][k], the windowed DFT of g(t,d) - g(t,0) (equal to A
// for k != 0, without its cancellation where t is small), g(t,0) per node in
// g0 and the nodes themselves in ts.
void sinc_factors(int n, double t0, std::vector<double>& A, std::vector<double>& wt,
                  std::vector<double>* AD = nullptr, std::vector<double>* g0 = nullptr,
                  std::vector<double>* tsout = nullptr) {
  // composite Gauss-Legendre on q in [0, pi]: one panel per cosine period of
  // the largest distance, plus margin
  const int gl = 16;
  std::vector<double> gx, gw;
  gauss_legendre(gl, gx, gw);
  const int panels = n / 2 + 8;
  const int nq = gl * panels;
  std::vector<double> q(nq), qw(nq);
  for (int p = 0; p < panels; ++p) {
    double a = kPi * p / panels, b = kPi * (p + 1) / panels;
    for (int i = 0; i < gl; ++i) {
      q[p * gl + i] = 0.5 * (a + b) + 0.5 * (b - a) * gx[i];
      qw[p * gl + i] = 0.5 * (b - a) * gw[i];
    }
  }
  std::vector<double> cq((size_t)nq * (n + 1));
  for (int j = 0; j < nq; ++j)
    for (int d = 0; d <= n; ++d) cq[(size_t)j * (n + 1) + d] = std::cos(q[j] * d);
  // windowed DFT matrix cos(pi k d / n) with end weights 1, 2, ..., 2, 1
  std::vector<double> ck((size_t)(n + 1) * (n + 1));
  for (int k = 0; k <= n; ++k)
    for (int d = 0; d <= n; ++d) {
      double c = (d == 0 || d == n) ? 1.0 : 2.0;
      // exact argument reduction of k*d mod 2n keeps the cosine accurate
      long r = ((long)k * d) % (2L * n);
      ck[(size_t)k * (n + 1) + d] = c * std::cos(kPi * (double)r / n);
    }
  // exp-sinh nodes
  const double step = 1.0 / 64.0;
  const double smin = -4.5, smax = 3.6;
  std::vector<double> ts, ws;
  for (double s = smin; s <= smax + 1e-12; s += step) {
    const double e = std::exp(0.5 * kPi * std::sinh(s));
    const double dtds = 0.5 * kPi * std::cosh(s) * e;
    ts.push_back(t0 + e);
    ws.push_back(step * dtds);
  }
  const int nt = (int)ts.size();
  A.assign((size_t)nt * (n + 1), 0.0);
  wt = ws;
  if (tsout) *tsout = ts;
  if (AD) AD->assign((size_t)nt * (n + 1), 0.0);
  if (g0) g0->assign(nt, 0.0);
  std::vector<double> g(n + 1), D(n + 1);
  for (int it = 0; it < nt; ++it) {
    const double t = ts[it];
    if (t <= 0.2) {
      for (int d = 0; d <= n; ++d) {
        g[d] = std::exp(-t * t * (double)d * d);
        D[d] = std::expm1(-t * t * (double)d * d);
      }
    } else {
      std::vector<double> e(nq);
      for (int j = 0; j < nq; ++j) e[j] = qw[j] * std::exp(-q[j] * q[j] / (4.0 * t * t));
      const double pre = 1.0 / (std::sqrt(kPi) * t);
      for (int d = 0; d <= n; ++d) {
        double acc = 0.0;
        for (int j = 0; j < nq; ++j) acc += e[j] * cq[(size_t)j * (n + 1) + d];
        g[d] = pre * acc;
      }
      for (int d = 0; d <= n; ++d) D[d] = g[d] - g[0];
    }
    for (int k = 0; k <= n; ++k) {
      double acc = 0.0, accd = 0.0;
      for (int d = 0; d <= n; ++d) {
        acc += ck[(size_t)k * (n + 1) + d] * g[d];
        accd += ck[(size_t)k * (n + 1) + d] * D[d];
      }
      A[(size_t)it * (n + 1) + k] = acc;
      if (AD) (*AD)[(size_t)it * (n + 1) + k] = accd;
    }
    if (g0) (*g0)[it] = g[0];
  }
}

void sinc_spectrum(int n, double h, double a, double* out) {
  std::vector<double> A, wt;
  sinc_factors(n, a, A, wt);
  const int nt = (int)wt.size();
  const int m = n + 1;
  const double pre = h * h * 2.0 / std::sqrt(kPi);
  // Ghat is symmetric under permutations of (kx, ky, kz) on a cubic grid:
  // evaluate kz >= ky >= kx and mirror.
#pragma omp parallel for schedule(dynamic, 1)
  for (int kz = 0; kz < m; ++kz) {
    std::vector<double> b(nt);
    for (int ky = 0; ky <= kz; ++ky) {
      for (int it = 0; it < nt; ++it)
        b[it] = wt[it] * A[(size_t)it * m + kz] * A[(size_t)it * m + ky];
      for (int kx = 0; kx <= ky; ++kx) {
        double acc = 0.0;
        for (int it = 0; it < nt; ++it) acc += b[it] * A[(size_t)it * m + kx];
        const double v = pre * acc;
        const int p[3] = {kz, ky, kx};
        // all 6 permutations
        const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
        for (int q = 0; q < 6; ++q) {
          const int a = p[perm[q][0]], bb = p[perm[q][1]], c = p[perm[q][2]];
          out[((size_t)a * m + bb) * m + c] = v;
        }
      }
    }
  }
}

void hockney_spectrum(int n, double h, double* out) {
  const int m = n + 1;
  const double origin = 3.0 * std::log(2.0 + std::sqrt(3.0)) - 0.5 * kPi;
  std::vector<double> G((size_t)m * m * m), T((size_t)m * m * m);
  for (int z = 0; z < m; ++z)
    for (int y = 0; y < m; ++y)
      for (int x = 0; x < m; ++x) {
        const double r = std::sqrt((double)x * x + (double)y * y + (double)z * z);
        G[((size_t)z * m + y) * m + x] = h * h * (r > 0.0 ? 1.0 / r : origin);
      }
  std::vector<double> ck((size_t)m * m);
  for (int k = 0; k < m; ++k)
    for (int d = 0; d < m; ++d) {
      double c = (d == 0 || d == n) ? 1.0 : 2.0;
      long r = ((long)k * d) % (2L * n);
      ck[(size_t)k * m + d] = c * std::cos(kPi * (double)r / n);
    }
  // three separable passes of the windowed cosine transform
  for (int axis = 0; axis < 3; ++axis) {
#pragma omp parallel for
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b)
        for (int k = 0; k < m; ++k) {
          double acc = 0.0;
          for (int d = 0; d < m; ++d) {
            size_t src;
            if (axis == 0) src = ((size_t)a * m + b) * m + d;       // along x
            else if (axis == 1) src = ((size_t)a * m + d) * m + b;  // along y
            else src = ((size_t)d * m + a) * m + b;                 // along z
            acc += ck[(size_t)k * m + d] * G[src];
          }
          size_t dst;
          if (axis == 0) dst = ((size_t)a * m + b) * m + k;
          else if (axis == 1) dst = ((size_t)a * m + k) * m + b;
          else dst = ((size_t)k * m + a) * m + b;
          T[dst] = acc;
        }
    G.swap(T);
  }
  for (size_t i = 0; i < G.size(); ++i) out[i] = G[i];
}

// Periodic cell of n points per axis (n even): 4 pi / |k|^2 with
// k = 2 pi m / (n h), m in [0, n/2]^3 (the signed frequencies fold onto this
// octant), the k = 0 term removed.  out: (n/2+1)^3 doubles.
void periodic_spectrum(int n, double h, double* out) {
  const int m = n / 2 + 1;
  const double c = 2.0 * kPi / (n * h);
  for (int kz = 0; kz < m; ++kz)
    for (int ky = 0; ky < m; ++ky)
      for (int kx = 0; kx < m; ++kx) {
        const double k2 = c * c * ((double)kx * kx + (double)ky * ky + (double)kz * kz);
        out[((size_t)kz * m + ky) * m + kx] = k2 > 0.0 ? 4.0 * kPi / k2 : 0.0;
      }
}

// Slab and wire boundary conditions (n even).  With
// 4 pi / k^2 = int_0^inf (2 pi / t^3) e^{-k^2/(4t^2)} dt every axis contributes
// one factor: on a free axis (zero-padded to 2n) the windowed DFT of the
// band-limited 1D Gaussian, (t/sqrt(pi)) gh(t h, k) in the units above; on a
// periodic axis e^{-k^2/(4t^2)} at k = 2 pi m / (n h).  In h = 1 units
// (tau = t h, kappa = k h), per spectrum entry:
//   slab:  Ghat = 2 sqrt(pi) h^2 int e^{-kappa^2/(4tau^2)} gh(tau, kz) / tau^2 dtau
//   wire:  Ghat = 2 h^2 int e^{-kappa^2/(4tau^2)} gh(tau, kx) gh(tau, ky) / tau dtau
// Each diverges at its (0, 0, 0) entry only (the 1D and 2D Coulomb potentials
// have no finite mean); that entry is the windowed sum of the regularised
// real-space kernel whose constant makes band-limited densities see exactly
// -2 pi |z| (slab) or -2 ln(r / bohr) (wire):
//   slab:  h^2 [2 sqrt(pi) int AD(tau, 0) / tau^2 dtau - 2n 4/pi]
//   wire:  h^2 [2 int AD(tau, 0) (gh(tau, 0) + 2n g(tau, 0)) / tau dtau
//               + (2n)^2 (2 ln(pi/h) + 2 gamma - 4 Catalan / pi)]
// with AD the windowed DFT of g(tau, d) - g(tau, 0) (so that the t-integrals
// converge at tau -> 0 without cancellation); for kz != 0 (slab) and kx or
// ky != 0 (wire) the factor is taken from AD too.
// Slab: out[(kz (n/2+1) + ky) (n/2+1) + kx], kz <= n, kx, ky <= n/2.
// Wire: out[(kz (n+1) + ky) (n+1) + kx], kz <= n/2, kx, ky <= n.
void slab_spectrum(int n, double h, double* out) {
  std::vector<double> A, AD, wt, g0, ts;
  sinc_factors(n, 0.0, A, wt, &AD, &g0, &ts);
  const int nt = (int)wt.size(), m = n + 1, m2 = n / 2 + 1;
  const double pre = 2.0 * std::sqrt(kPi) * h * h;
  const double c = 2.0 * kPi / n;
#pragma omp parallel for schedule(dynamic, 1)
  for (int ky = 0; ky < m2; ++ky) {
    std::vector<double> e(nt);
    for (int kx = 0; kx <= ky; ++kx) {
      const double kap2 = c * c * ((double)kx * kx + (double)ky * ky);
      for (int it = 0; it < nt; ++it)
        e[it] = wt[it] * std::exp(-kap2 / (4.0 * ts[it] * ts[it])) / (ts[it] * ts[it]);
      for (int kz = 0; kz < m; ++kz) {
        const std::vector<double>& F = (kz != 0 || kap2 == 0.0) ? AD : A;
        double acc = 0.0;
        for (int it = 0; it < nt; ++it) acc += e[it] * F[(size_t)it * m + kz];
        double v = pre * acc;
        if (kz == 0 && kap2 == 0.0) v -= h * h * 2.0 * n * 4.0 / kPi;
        out[((size_t)kz * m2 + ky) * m2 + kx] = v;
        out[((size_t)kz * m2 + kx) * m2 + ky] = v;
      }
    }
  }
}

void wire_spectrum(int n, double h, double* out) {
  std::vector<double> A, AD, wt, g0, ts;
  sinc_factors(n, 0.0, A, wt, &AD, &g0, &ts);
  const int nt = (int)wt.size(), m = n + 1, m2 = n / 2 + 1;
  const double pre = 2.0 * h * h;
  const double c = 2.0 * kPi / n;
  const double kEulerGamma = 0.57721566490153286061, kCatalan = 0.91596559417721901505;
  const double creg = 2.0 * std::log(kPi / h) + 2.0 * kEulerGamma - 4.0 * kCatalan / kPi;
#pragma omp parallel for schedule(dynamic, 1)
  for (int kz = 0; kz < m2; ++kz) {
    const double kap2 = c * c * (double)kz * kz;
    std::vector<double> e(nt);
    for (int it = 0; it < nt; ++it)
      e[it] = wt[it] * std::exp(-kap2 / (4.0 * ts[it] * ts[it])) / ts[it];
    for (int ky = 0; ky < m; ++ky) {
      const std::vector<double>& Fy = ky != 0 ? AD : A;
      for (int kx = 0; kx <= ky; ++kx) {
        const std::vector<double>& Fx = kx != 0 ? AD : A;
        double v;
        if (kap2 == 0.0 && kx == 0 && ky == 0) {
          double acc = 0.0;
          for (int it = 0; it < nt; ++it)
            acc += e[it] * AD[(size_t)it * m] * (A[(size_t)it * m] + 2.0 * n * g0[it]);
          v = pre * acc + h * h * (2.0 * n) * (2.0 * n) * creg;
        } else {
          double acc = 0.0;
          for (int it = 0; it < nt; ++it)
            acc += e[it] * Fx[(size_t)it * m + kx] * Fy[(size_t)it * m + ky];
          v = pre * acc;
        }
        out[((size_t)kz * m + ky) * m + kx] = v;
        out[((size_t)kz * m + kx) * m + ky] = v;
      }
    }
  }
}

}  // namespace

// kind: 0 = band-limited (sinc), 1 = Hockney, 2 = band-limited erfc(omega r)/r
// (omega > 0): out (n+1)^3 doubles; 3 = periodic (n even): out (n/2+1)^3;
// 4 = slab (n even): out (n+1) (n/2+1)^2; 5 = wire (n even): out (n/2+1) (n+1)^2.
bool kernel_spectrum_octant(int n, double h, int kind, double omega, double* out) {
  if (n < 1 || !(h > 0.0) || out == nullptr) return false;
  if (kind == 3 || kind == 4 || kind == 5) {
    if (n % 2 != 0) return false;
    if (kind == 3) periodic_spectrum(n, h, out);
    else if (kind == 4) slab_spectrum(n, h, out);
    else wire_spectrum(n, h, out);
    return true;
  }
  if (kind == 0) sinc_spectrum(n, h, 0.0, out);
  else if (kind == 1) hockney_spectrum(n, h, out);
  else if (kind == 2 && omega > 0.0 && std::isfinite(omega)) sinc_spectrum(n, h, omega * h, out);
  else return false;
  return true;
}

}  // namespace exx_host
