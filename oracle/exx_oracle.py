"""Plain FP64 CPU oracle of the free-boundary exact-exchange (EXX) operator.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (``paper_1712_07973_gb300``), and it does not import
that package.

What it computes (arXiv 1712.07973, Ratcliff et al.):

* Sec. 2, Eq. 1 defines the one-body density matrix with occupations f_i; for
  real orbitals the co-density of a pair is rho_ij = psi_i * psi_j (Sec. 2.1,
  "Kernel 1"), and rho_ij = rho_ji.
* Sec. 2, the equation after Eq. daction: V_ij solves the Poisson equation
  lap V_ij = -4 pi rho_ij, i.e. V_ij = rho_ij convolved with 1/|r - r'|.
  Sec. 2.1.2 states that this convolution is done exactly, with appropriate
  zero padding, by Fourier techniques, with a Green's function discretised on
  the uniform mesh for free boundary conditions.
* Sec. 2, Eq. HF and the E_X equation that follows the pair-count paragraph:
  E_x = -(alpha/2) * sum_{i,j} f_i f_j  int rho_ij V_ij.  The factor alpha is
  the exact-exchange fraction of the hybrid (PBE0: 1/4, Sec. 3).
* Sec. 2, Eq. daction: (Vx psi)_i = -alpha * sum_j f_j V_ij psi_j.
* Sec. 2, pair-count paragraph: all N(N+1)/2 co-densities are formed; the
  symmetry V_ij = V_ji lets pair (i, j) serve both (Vx psi)_i and (Vx psi)_j
  (Sec. 2.1, round-robin paragraph).

Readings where the paper is silent:

* The paper names the interpolating-scaling-function Green's function but
  prints no formula for it.  This oracle uses the band-limited ("sinc basis")
  free-space kernel: G[m] = h^3 * G_BL(m h) with
  G_BL(r) = (2 pi)^-3 * int over the cube |k_d| <= pi/h of (4 pi / k^2) e^{i k.r} d^3k,
  which is the exact Coulomb potential of any density band-limited to the
  grid's Brillouin zone.  The point-sampled Hockney kernel (G[m] = h^3/|m h|,
  G[0] = h^2 times the cell average of 1/r) is offered as a second option.
* Grid nodes sit at x_m = m h, m = 0..n-1, per axis; arrays are indexed
  [z, y, x] with x fastest.
* Occupations are used exactly as passed (no sum over spin channels).
* E_ij = h^3 * sum_m rho_ij[m] V_ij[m] (rectangle-rule quadrature on the mesh).
* Periodic boundary conditions (the paper's own H2O and UO2 runs, Sec. 3, are
  periodic; Sec. 2.1.2 only states that other boundary conditions use other
  Green's functions): the n^3 cell of side n h repeats, no padding, and
  V_hat(k) = 4 pi rho_hat(k) / |k|^2 for the band-limited density with the
  k = 0 term removed (a neutralising background), |k|^2 from the signed
  frequencies 2 pi m / (n h), |m| <= n/2.
* Slab ("surface") boundary conditions: periodic in x and y with the cell
  n h, free in z (zero-padded to 2n along z only).  Per in-plane frequency
  k = |(k_x, k_y)| the kernel along z is the band-limited 1D Green's function
  of d^2/dz^2 - k^2,  g(k, z) = 4 int_0^{pi/h} cos(q z) / (k^2 + q^2) dq
  (-> (2 pi / k) e^{-k|z|} without the band limit); for k = 0 it is
  regularised to g0(z) = 4 int_0^{pi/h} (cos(q z) - 1) / q^2 dq - 4 h / pi,
  the constant chosen so that densities band-limited in z see exactly the
  continuum potential -2 pi int |z - z'| rho(z') dz'.
* Wire boundary conditions: free in x and y (zero-padded to 2n), periodic in
  z with the cell n h.  Per axial frequency k the kernel in the (x, y) plane is
  the band-limited 2D Green's function of lap_2 - k^2,
  (2 pi)^-2 int over |q_d| <= pi/h of 4 pi e^{i q.r} / (k^2 + q^2) d^2q
  (-> 2 K0(k r)); for k = 0 it is regularised to
  (1/pi) int (e^{i q.r} - 1) / q^2 d^2q + 2 ln(pi/h) + 2 gamma - 4 Catalan / pi,
  the constant chosen so that band-limited densities see exactly the
  continuum potential -2 int ln|r - r'| rho(r') d^2r' (r in bohr).

Precision: FP64 throughout.
"""

import math

import numpy as np
from scipy import fft as sfft
from scipy import special as sspecial
from scipy import integrate as sint

__all__ = [
    "KERNEL_SINC",
    "KERNEL_HOCKNEY",
    "KERNEL_ERFC",
    "sinc_kernel_g1d",
    "kernel_real_space",
    "kernel_spectrum",
    "kernel_spectrum_periodic",
    "kernel_spectrum_slab",
    "kernel_spectrum_wire",
    "poisson",
    "direct_sum_potential",
    "pair_list",
    "exx",
    "exx_pair",
    "exx_energy_gradient",
]

KERNEL_SINC = "sinc"
KERNEL_HOCKNEY = "hockney"
KERNEL_ERFC = "erfc"  # band-limited short-range kernel erfc(omega r)/r (screened hybrids)

# --------------------------------------------------------------------------
# Free-boundary Green's function on the mesh (Sec. 2.1.2; reading above)
# --------------------------------------------------------------------------
#
# With 1/r = (2/sqrt(pi)) int_0^inf exp(-t^2 r^2) dt and the Fourier pair of a
# Gaussian, the band-limited kernel separates per axis:
#     G_BL(r) = (2/sqrt(pi)) int_0^inf  prod_{d=x,y,z} g(t, r_d)  dt,
#     g(t, x) = (1/2pi) int_{-pi/h}^{pi/h} (sqrt(pi)/t) exp(-k^2/(4t^2)) cos(kx) dk.
# For h = 1 and integer x = m this 1D factor has the closed form
#     g(t, m) = exp(-t^2 m^2) - (-1)^m exp(-pi^2/(4t^2)) Re w(-t m + i pi/(2t)),
# with w the Faddeeva function (w(z) = exp(-z^2) erfc(-iz)), and g(t, 0) =
# erf(pi/(2t)).  Scaling: G[m] = h^3 G_BL(m h; h) = h^2 G_BL(m; 1).

# t-integral: trapezoid rule in s = ln t.  The integrand t * prod g is analytic
# in the strip |Im s| < pi/4 and decays like e^{s} (s -> -inf) and e^{-2s}
# (s -> +inf), so the rule converges geometrically with the step.
_S_MIN, _S_MAX, _S_STEP = -40.0, 20.0, 0.1


def sinc_kernel_g1d(t, m):
    """1D factor g(t, m) of the band-limited kernel for h = 1 (closed form)."""
    t = np.asarray(t, dtype=np.float64)[:, None]
    m = np.asarray(m, dtype=np.float64)[None, :]
    a = np.pi / (2.0 * t)
    z = -t * m + 1j * a
    sign = np.where(np.mod(m, 2.0) == 0.0, 1.0, -1.0)
    out = np.exp(-(t * m) ** 2) - sign * np.exp(-a * a) * np.real(sspecial.wofz(z))
    # m = 0: g = erf(pi/(2t)) evaluated directly (the form above cancels there).
    zero = (m == 0.0)[0]
    if np.any(zero):
        out[:, zero] = sspecial.erf(a[:, 0])[:, None]
    return out


def _sinc_kernel_octant(n):
    """G_BL(m; h=1) for m in [0, n]^3 (octant; G is even per axis)."""
    # nodes at exact multiples of the step (a float-step arange drifts by a few
    # ulp per node, which biases the rule at the 1e-13 level)
    K = int(round((_S_MAX - _S_MIN) / _S_STEP))
    s = _S_MIN + _S_STEP * np.arange(K + 1, dtype=np.float64)
    t = np.exp(s)
    w = _S_STEP * t * (2.0 / math.sqrt(math.pi))
    w[0] *= 0.5
    w[-1] *= 0.5
    m = np.arange(n + 1)
    g = sinc_kernel_g1d(t, m)  # (nt, n+1)
    nt = t.size
    # G[a, b, c] = sum_t w_t g[t,a] g[t,b] g[t,c]   (a plain contraction)
    gw = g * w[:, None]
    ab = (gw[:, :, None] * g[:, None, :]).reshape(nt, -1)  # (nt, (n+1)^2)
    G = (ab.T @ g).reshape(n + 1, n + 1, n + 1)
    # tail t > e^{S_MAX}: only m = 0 is not negligible; prod g ~ pi^{3/2} t^-3
    # there, so (2/sqrt(pi)) int_T^inf pi^{3/2} t^-3 dt = pi / T^2.
    G[0, 0, 0] += math.pi * math.exp(-2.0 * _S_MAX)
    return G


def _longrange_octant(n, a):
    """(2/sqrt(pi)) int_0^a prod_d g(t, m_d) dt for m in [0, n]^3, h = 1.

    The band-limited long-range part erf-like kernel; composite Gauss-Legendre
    in t on [0, a] (the integrand is analytic there), 64 panels of 16 nodes.
    """
    x, w = np.polynomial.legendre.leggauss(16)
    panels = 64
    edges = np.linspace(0.0, a, panels + 1)
    t = (0.5 * (edges[:-1] + edges[1:])[:, None] + 0.5 * np.diff(edges)[:, None] * x[None, :]).ravel()
    wt = (0.5 * np.diff(edges)[:, None] * w[None, :]).ravel() * (2.0 / math.sqrt(math.pi))
    m = np.arange(n + 1)
    g = sinc_kernel_g1d(t, m)
    gw = g * wt[:, None]
    ab = (gw[:, :, None] * g[:, None, :]).reshape(t.size, -1)
    return (ab.T @ g).reshape(n + 1, n + 1, n + 1)


def _hockney_cell_average():
    """Average of 1/r over the unit cube centred at the origin.

    Splitting the cube into the 24 pyramids where one |coordinate| is largest
    and scaling the two others by it gives 3 * int_0^1 asinh(1/sqrt(1+a^2)) da.
    """
    val, _ = sint.quad(lambda a: np.arcsinh(1.0 / np.sqrt(1.0 + a * a)), 0.0, 1.0,
                       epsabs=1e-14, epsrel=1e-14, limit=200)
    return 3.0 * val


def kernel_real_space(n, h, kind=KERNEL_SINC, omega=0.0):
    """Real-space mesh kernel G[m] for m in [0, n]^3, including the h^3 weight.

    V[m] = sum_{m'} G[|m - m'|] rho[m'] (absolute difference per axis) is the
    discrete free-boundary potential of the co-density rho.  KERNEL_ERFC is the
    band-limited erfc(omega r)/r: the t-integral of the sinc kernel restricted
    to t > omega (erfc(w r)/r = (2/sqrt pi) int_w^inf exp(-t^2 r^2) dt), i.e.
    the full kernel minus its t < omega part; in h = 1 units omega becomes
    omega h.
    """
    if kind == KERNEL_SINC:
        return (h * h) * _sinc_kernel_octant(n)
    if kind == KERNEL_ERFC:
        if not omega > 0.0:
            raise ValueError("the erfc kernel needs omega > 0")
        return (h * h) * (_sinc_kernel_octant(n) - _longrange_octant(n, omega * h))
    if kind == KERNEL_HOCKNEY:
        m = np.arange(n + 1, dtype=np.float64)
        r = np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2)
        with np.errstate(divide="ignore"):
            G = 1.0 / r
        G[0, 0, 0] = _hockney_cell_average()
        return (h * h) * G
    raise ValueError(f"unknown kernel kind {kind!r}")


def kernel_spectrum(G):
    """Spectrum of the zero-padded (2n)^3 periodic embedding of G.

    G~[d mod 2n] = G[|d|] for d in [-(n-1), n]; the slot d = n is never used by
    outputs in [0, n) and carries G[n] so that G~ stays even and its DFT real.
    Returns the real half spectrum of shape (2n, 2n, n+1) in scipy's rfftn
    layout (last axis = x, k_x in [0, n]).
    """
    n = G.shape[0] - 1
    idx = np.concatenate([np.arange(n + 1), np.arange(n - 1, 0, -1)])
    Gt = G[np.ix_(idx, idx, idx)]
    Ghat = sfft.rfftn(Gt, workers=-1)
    return np.ascontiguousarray(Ghat.real)


def kernel_spectrum_periodic(n, h):
    """Periodic Coulomb spectrum 4 pi / |k|^2 (k = 0 removed) on the n^3 cell,
    in scipy's rfftn layout (n, n, n//2 + 1) (see the module header)."""
    m = np.fft.fftfreq(n, d=1.0 / n)  # signed integer frequencies
    mx = np.arange(n // 2 + 1, dtype=np.float64)
    k2 = (2.0 * math.pi / (n * h)) ** 2 * (m[:, None, None] ** 2 + m[None, :, None] ** 2
                                             + mx[None, None, :] ** 2)
    with np.errstate(divide="ignore"):
        G = np.where(k2 > 0, 4.0 * math.pi / np.where(k2 > 0, k2, 1.0), 0.0)
    return G


# --------------------------------------------------------------------------
# Slab and wire boundary conditions (readings in the module header)
# --------------------------------------------------------------------------
# Both kernels come from 4 pi / k^2 = int_0^inf (2 pi / t^3) e^{-k^2/(4t^2)} dt,
# whose factor per axis is, on a free axis, the band-limited 1D function
# (1/2pi) int_{-pi/h}^{pi/h} e^{-q^2/(4t^2)} cos(q x) dq = (t/sqrt(pi)) g(t h, x/h) / h
# (g = sinc_kernel_g1d), and on a periodic axis its Fourier coefficient
# e^{-k^2/(4t^2)} itself.  In h = 1 units (tau = t h, kappa = k h):
#   slab, kappa > 0:  h g(k, d h) = h^2 2 sqrt(pi) int e^{-kappa^2/(4tau^2)} g(tau, d) / tau^2 dtau
#   wire, kappa > 0:  h^2 g2(k, d h) = h^2 2 int e^{-kappa^2/(4tau^2)} g(tau, dx) g(tau, dy) / tau dtau
# The t-integrals use the trapezoid rule in s = ln tau of the free kernel.
_EULER_GAMMA = 0.57721566490153286061
_CATALAN = 0.91596559417721901505


def _s_nodes():
    K = int(round((_S_MAX - _S_MIN) / _S_STEP))
    s = _S_MIN + _S_STEP * np.arange(K + 1, dtype=np.float64)
    w = np.full(s.size, _S_STEP)
    w[0] *= 0.5
    w[-1] *= 0.5
    return np.exp(s), w


def _g1d_minus_g0(t, m):
    """g(t, m) - g(t, 0) without cancellation where t is small:
    expm1(-t^2 m^2) - (-1)^m e^{-a^2} Re w(-t m + i a) + erfc(a), a = pi/(2t)."""
    t = np.asarray(t, dtype=np.float64)[:, None]
    m = np.asarray(m, dtype=np.float64)[None, :]
    a = np.pi / (2.0 * t)
    sign = np.where(np.mod(m, 2.0) == 0.0, 1.0, -1.0)
    out = (np.expm1(-(t * m) ** 2) - sign * np.exp(-a * a) * np.real(sspecial.wofz(-t * m + 1j * a))
           + sspecial.erfc(a))
    out[:, (m == 0.0)[0]] = 0.0
    return out


def slab_kernel_z(n, h, kappa):
    """K[c][d] = h g(kappa_c / h, d h) for d in [0, n]: the slab kernel along z
    with its quadrature weight h, per in-plane frequency kappa_c = k h."""
    kappa = np.atleast_1d(np.asarray(kappa, dtype=np.float64))
    d = np.arange(n + 1, dtype=np.float64)
    out = np.empty((kappa.size, n + 1))
    pos = kappa > 0
    if np.any(pos):
        t, w = _s_nodes()
        g = sinc_kernel_g1d(t, d)                      # (nt, n+1)
        with np.errstate(over="ignore"):
            e = np.exp(-kappa[pos, None] ** 2 / (4.0 * t[None, :] ** 2))
        out[pos] = (e * (w / t)[None, :]) @ g * (2.0 * math.sqrt(math.pi))
    if np.any(~pos):
        # k = 0: 4 [ (1 - cos(K z)) / K - z Si(K z) ] - 4 / K at z = d h, K = pi / h
        si, _ = sspecial.sici(np.pi * d)
        out[~pos] = -(4.0 / np.pi) * np.where(d % 2 == 0, 1.0, -1.0) - 4.0 * d * si
    return (h * h) * out


def wire_kernel_xy(n, h, kappa):
    """K2[c][dy][dx] = h^2 g2(kappa_c / h, (dx, dy) h) for dx, dy in [0, n]:
    the wire kernel in the (x, y) plane with its weight h^2, per axial
    frequency kappa_c = k h."""
    kappa = np.atleast_1d(np.asarray(kappa, dtype=np.float64))
    d = np.arange(n + 1, dtype=np.float64)
    t, w = _s_nodes()
    g = sinc_kernel_g1d(t, d)                          # (nt, n+1)
    out = np.empty((kappa.size, n + 1, n + 1))
    pos = kappa > 0
    if np.any(pos):
        with np.errstate(over="ignore"):
            e = np.exp(-kappa[pos, None] ** 2 / (4.0 * t[None, :] ** 2)) * w[None, :]
        gg = (g[:, :, None] * g[:, None, :]).reshape(t.size, -1)
        out[pos] = (2.0 * (e @ gg)).reshape(-1, n + 1, n + 1)
    if np.any(~pos):
        # k = 0: g(t,dx) g(t,dy) - g(t,0)^2 = D(dx) g(dy) + g(0) D(dy), D = g - g(t,0)
        D = _g1d_minus_g0(t, d)
        g0 = g[:, :1]
        reg = (D[:, None, :] * g[:, :, None] + (g0 * D)[:, :, None]) * w[:, None, None]
        c = 2.0 * math.log(math.pi / h) + 2.0 * _EULER_GAMMA - 4.0 * _CATALAN / math.pi
        out[~pos] = 2.0 * reg.sum(axis=0) + c
    return (h * h) * out


def _window(n):
    """Indices of the zero-padded periodic embedding: slot d mod 2n <- |d|,
    d in [-(n-1), n] (slot n carries the value at n, as in kernel_spectrum)."""
    return np.concatenate([np.arange(n + 1), np.arange(n - 1, 0, -1)])


def kernel_spectrum_slab(n, h):
    """Slab spectrum in scipy's rfftn layout of the (2n, n, n) grid [z, y, x]:
    shape (2n, n, n//2 + 1); z zero-padded, x and y periodic (n even)."""
    if n % 2:
        raise ValueError("the slab kernel needs an even n")
    my = np.fft.fftfreq(n, d=1.0 / n)
    mx = np.arange(n // 2 + 1, dtype=np.float64)
    m2 = my[:, None] ** 2 + mx[None, :] ** 2
    uq, inv = np.unique(m2, return_inverse=True)
    K = slab_kernel_z(n, h, 2.0 * np.pi * np.sqrt(uq) / n)     # (nu, n+1)
    spec = sfft.rfft(K[:, _window(n)], axis=1, workers=-1).real  # (nu, n+1): kz in [0, n]
    kz = np.concatenate([np.arange(n + 1), np.arange(n - 1, 0, -1)])
    return np.ascontiguousarray(spec[inv.reshape(m2.shape)][..., kz].transpose(2, 0, 1))


def kernel_spectrum_wire(n, h):
    """Wire spectrum in scipy's rfftn layout of the (n, 2n, 2n) grid [z, y, x]:
    shape (n, 2n, n + 1); x and y zero-padded, z periodic (n even)."""
    if n % 2:
        raise ValueError("the wire kernel needs an even n")
    mz = np.abs(np.fft.fftfreq(n, d=1.0 / n))
    uq, inv = np.unique(mz, return_inverse=True)
    K2 = wire_kernel_xy(n, h, 2.0 * np.pi * uq / n)            # (nu, n+1, n+1)
    idx = _window(n)
    spec = sfft.rfft2(K2[:, idx][:, :, idx], workers=-1).real   # (nu, 2n, n+1)
    return np.ascontiguousarray(spec[inv])


def poisson(rho, Ghat):
    """V = G * rho on the n^3 grid.  The spectrum's shape says which axes are
    zero-padded to 2n (free: the aperiodic convolution of Sec. 2.1.2) and which
    are periodic: (2n, 2n, n+1) free (kernel_spectrum), (n, n, n/2+1) periodic,
    (2n, n, n/2+1) slab, (n, 2n, n+1) wire."""
    n = rho.shape[0]
    shape = (2 * n if Ghat.shape[0] == 2 * n else n,
             2 * n if Ghat.shape[1] == 2 * n else n,
             2 * n if Ghat.shape[2] == n + 1 else n)
    if shape == rho.shape:
        return np.ascontiguousarray(sfft.irfftn(sfft.rfftn(rho, workers=-1) * Ghat, s=rho.shape,
                                                workers=-1))
    pad = np.zeros(shape, dtype=np.float64)
    pad[:n, :n, :n] = rho
    V = sfft.irfftn(sfft.rfftn(pad, workers=-1) * Ghat, s=shape, workers=-1)
    return np.ascontiguousarray(V[:n, :n, :n])


def direct_sum_potential(rho, G):
    """Brute force V[m] = sum_{m'} G[|m-m'|] rho[m'] (O(n^6); tiny grids only)."""
    n = rho.shape[0]
    idx = np.arange(n)
    dif = np.abs(idx[:, None] - idx[None, :])  # (m, m')
    V = np.empty_like(rho)
    for z in range(n):
        for y in range(n):
            for x in range(n):
                V[z, y, x] = np.sum(G[dif[z][:, None, None], dif[y][None, :, None],
                                      dif[x][None, None, :]] * rho)
    return V


def pair_list(N):
    """All N(N+1)/2 pairs (i, j), i <= j (Sec. 2, pair-count paragraph)."""
    return [(i, j) for i in range(N) for j in range(i, N)]


def exx_pair(psi_i, psi_j, Ghat, h):
    """One pair: co-density, potential and E_ij = h^3 sum rho_ij V_ij."""
    rho = psi_i * psi_j
    V = poisson(rho, Ghat)
    return V, (h ** 3) * float(np.sum(rho * V))


def exx(psi, occ, alpha, h, Ghat, want_vx=True):
    """Exact exchange of real orbitals psi[N, n, n, n] (FP64).

    Returns (E_x, Vxpsi or None, Eij) with
      E_x      = -(alpha/2) sum_{i,j} f_i f_j E_ij,
      Vxpsi[i] = -alpha sum_j f_j V_ij psi_j,
      Eij      = symmetric matrix of h^3 sum rho_ij V_ij.
    Pair (i, j), i < j, feeds both i and j; i = j feeds i once.
    """
    psi = np.asarray(psi, dtype=np.float64)
    occ = np.asarray(occ, dtype=np.float64)
    N = psi.shape[0]
    Eij = np.zeros((N, N))
    vx = np.zeros_like(psi) if want_vx else None
    for i, j in pair_list(N):
        V, e = exx_pair(psi[i], psi[j], Ghat, h)
        Eij[i, j] = Eij[j, i] = e
        if want_vx:
            vx[i] += (-alpha * occ[j]) * V * psi[j]
            if i != j:
                vx[j] += (-alpha * occ[i]) * V * psi[i]
    Ex = -0.5 * alpha * float(occ @ Eij @ occ)
    return Ex, vx, Eij


def exx_energy_gradient(psi, occ, alpha, h, Ghat):
    """E_x and dE_x/dpsi_k = 2 f_k h^3 (Vx psi)_k (Eq. daction from delta E/delta F)."""
    Ex, vx, _ = exx(psi, occ, alpha, h, Ghat, want_vx=True)
    grad = 2.0 * (h ** 3) * np.asarray(occ)[:, None, None, None] * vx
    return Ex, grad
