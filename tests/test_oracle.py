"""Pins of the FP64 oracle against facts the paper and mathematics fix.

None of these retypes the oracle's own formula: each compares it with an
independent route (direct sums, closed forms, other quadratures, invariants).
"""

import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

from oracle import exx_oracle as o

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- kernel G

def test_sinc_kernel_origin_closed_form():
    # G_BL(0) over the Brillouin-zone cube reduces (24 symmetric pyramids,
    # scaling k_y, k_z by k_x) to 12 C / pi with C = int int da db/(1+a^2+b^2).
    C, _ = integrate.dblquad(lambda a, b: 1.0 / (1.0 + a * a + b * b), 0, 1, 0, 1,
                             epsabs=1e-14, epsrel=1e-14)
    for h in (1.0, 0.4, 0.37):
        G = o.kernel_real_space(4, h)
        assert G[0, 0, 0] == pytest.approx(h * h * 12.0 * C / math.pi, rel=2e-14)


def test_hockney_kernel_origin_closed_form():
    # Average of 1/r over the unit cube: 3 ln(2 + sqrt 3) - pi/2.
    G = o.kernel_real_space(4, 0.5, kind=o.KERNEL_HOCKNEY)
    c0 = 3.0 * math.log(2.0 + math.sqrt(3.0)) - 0.5 * math.pi
    assert G[0, 0, 0] == pytest.approx(0.25 * c0, rel=1e-14)
    assert G[3, 0, 4] == pytest.approx(0.25 / 5.0, rel=1e-15)


def test_sinc_kernel_far_field():
    # Away from the axes the band-limited kernel approaches the point Coulomb
    # value h^3/|m h| quickly; along an axis the cube band edge leaves an
    # alternating ~0.11/|m| relative ripple, which must also shrink like 1/|m|.
    n, h = 64, 0.4
    G = o.kernel_real_space(n, h)
    for m in [(20, 10, 7), (30, 20, 11), (40, 40, 40), (60, 33, 21), (64, 64, 30)]:
        r = h * math.sqrt(sum(c * c for c in m))
        rel = G[m] * r / h ** 3 - 1.0
        assert abs(rel) < 1e-6 * (20.0 / (r / h)) ** 2, (m, rel)
    ax = np.array([G[m, 0, 0] * m * h / h ** 3 - 1.0 for m in range(16, 64)])
    assert np.all(np.abs(ax) * np.arange(16, 64) < 0.12)
    assert np.all(np.sign(ax[:-1]) != np.sign(ax[1:]))  # alternating ripple


def test_kernel_symmetry_and_real_spectrum():
    G = o.kernel_real_space(12, 0.3)
    assert np.allclose(G, G.transpose(1, 0, 2), rtol=0, atol=1e-15)
    assert np.allclose(G, G.transpose(2, 1, 0), rtol=0, atol=1e-15)
    n = 12
    idx = np.concatenate([np.arange(n + 1), np.arange(n - 1, 0, -1)])
    Gt = G[np.ix_(idx, idx, idx)]
    full = np.fft.fftn(Gt)
    assert np.max(np.abs(full.imag)) < 1e-12 * np.max(np.abs(full.real))
    Gh = o.kernel_spectrum(G)
    assert np.allclose(Gh, full.real[:, :, : n + 1], rtol=1e-13, atol=1e-13)


# ------------------------------------------------- padded FFT = direct sum

@pytest.mark.parametrize("n", [4, 5, 6, 7, 8, 10])
@pytest.mark.parametrize("kind", [o.KERNEL_SINC, o.KERNEL_HOCKNEY])
def test_padded_fft_equals_direct_sum(n, kind):
    # The paper's zero-padded convolution is exact: compare with the O(n^6)
    # direct sum over every source point.
    rho = _rng(n).standard_normal((n, n, n))
    G = o.kernel_real_space(n, 0.45, kind)
    V = o.poisson(rho, o.kernel_spectrum(G))
    Vd = o.direct_sum_potential(rho, G)
    assert np.max(np.abs(V - Vd)) <= 1e-13 * np.max(np.abs(Vd))


# ------------------------------------------------------ Gaussian physics

def _centered_grid(n, h):
    x = np.arange(n) * h - 0.5 * (n - 1) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return np.sqrt(X * X + Y * Y + Z * Z)


def test_gaussian_potential_and_self_energy():
    # A normalised Gaussian charge of width sigma has V(r) = erf(r/(sqrt2 sigma))/r
    # and self energy 1/(2 sigma sqrt(pi)).  sigma = 3h keeps its spectrum inside
    # the Brillouin zone (tail e^{-(pi sigma/h)^2/2} ~ 1e-19) and the box holds
    # more than 7 sigma on each side.
    n, h, sig = 48, 0.2, 0.6
    r = _centered_grid(n, h)
    rho = np.exp(-r * r / (2 * sig * sig)) / (2 * math.pi * sig * sig) ** 1.5
    V = o.poisson(rho, o.kernel_spectrum(o.kernel_real_space(n, h)))
    with np.errstate(invalid="ignore", divide="ignore"):
        Vex = np.where(r > 0, special.erf(r / (math.sqrt(2) * sig)) / np.where(r > 0, r, 1),
                       math.sqrt(2 / math.pi) / sig)
    assert np.max(np.abs(V / Vex - 1)) < 1e-12
    E = 0.5 * h ** 3 * np.sum(rho * V)
    assert E == pytest.approx(1.0 / (2 * sig * math.sqrt(math.pi)), rel=1e-12)


def test_hockney_gaussian_is_second_order():
    # The point-sampled kernel is only O(h^2) accurate: halving h must cut the
    # self-energy error by roughly 4.
    sig = 0.6
    errs = []
    for n, h in ((24, 0.4), (48, 0.2)):
        r = _centered_grid(n, h)
        rho = np.exp(-r * r / (2 * sig * sig)) / (2 * math.pi * sig * sig) ** 1.5
        V = o.poisson(rho, o.kernel_spectrum(o.kernel_real_space(n, h, o.KERNEL_HOCKNEY)))
        E = 0.5 * h ** 3 * np.sum(rho * V)
        errs.append(abs(E * 2 * sig * math.sqrt(math.pi) - 1))
    assert 2.5 < errs[0] / errs[1] < 6.0


def test_single_orbital_exchange_closed_form():
    # psi = (pi s^2)^{-3/4} exp(-r^2/(2 s^2)) has rho = psi^2 of width s/sqrt2,
    # so E_x = -(alpha/2) f^2 / (sigma_rho sqrt(pi)), and (Vx psi)/psi is
    # -alpha f erf(r/(sqrt2 sigma_rho))/r.
    n, h, s = 48, 0.2, 0.6 * math.sqrt(2.0)
    r = _centered_grid(n, h)
    psi = (math.pi * s * s) ** -0.75 * np.exp(-r * r / (2 * s * s))
    alpha, f = 0.25, 2.0
    Gh = o.kernel_spectrum(o.kernel_real_space(n, h))
    Ex, vx, Eij = o.exx(psi[None], np.array([f]), alpha, h, Gh)
    sr = s / math.sqrt(2.0)
    assert Ex == pytest.approx(-0.5 * alpha * f * f / (sr * math.sqrt(math.pi)), rel=1e-11)
    with np.errstate(invalid="ignore", divide="ignore"):
        Vex = np.where(r > 0, special.erf(r / (math.sqrt(2) * sr)) / np.where(r > 0, r, 1),
                       math.sqrt(2 / math.pi) / sr)
    mask = psi > 1e-12 * psi.max()
    assert np.max(np.abs(vx[0][mask] / psi[mask] / (-alpha * f * Vex[mask]) - 1)) < 1e-10


def test_two_distant_gaussians_add():
    # Two orbitals too far apart to overlap: the cross term vanishes and E_x is
    # the sum of the single-orbital values.
    n, h, s = 64, 0.25, 0.5 * math.sqrt(2.0)
    x = np.arange(n) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    c1, c2 = np.array([4.0, 8.0, 8.0]), np.array([12.0, 8.0, 8.0])
    def orb(c):
        r2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
        return (math.pi * s * s) ** -0.75 * np.exp(-r2 / (2 * s * s))
    psi = np.stack([orb(c1), orb(c2)])
    Gh = o.kernel_spectrum(o.kernel_real_space(n, h))
    Ex, _, Eij = o.exx(psi, np.array([2.0, 1.0]), 0.25, h, Gh)
    sr = s / math.sqrt(2)
    e1 = 1.0 / (sr * math.sqrt(math.pi))
    assert abs(Eij[0, 1]) < 1e-20
    assert Ex == pytest.approx(-0.125 * (4.0 * e1 + 1.0 * e1), rel=1e-10)


# ----------------------------------------------- full operator, brute force

def test_exx_matches_ordered_pair_direct_sum():
    # Every ordered pair (i, j), direct-sum potentials, no triangle bookkeeping:
    # catches a dropped factor 2 on off-diagonal pairs or a wrong occupation.
    rng = _rng(7)
    n, N, h, alpha = 6, 3, 0.5, 0.3
    psi = rng.standard_normal((N, n, n, n))
    occ = rng.uniform(0.5, 2.0, N)
    G = o.kernel_real_space(n, h)
    Ex_bf = 0.0
    vx_bf = np.zeros_like(psi)
    for i in range(N):
        for j in range(N):
            rho = psi[i] * psi[j]
            V = o.direct_sum_potential(rho, G)
            Ex_bf += -0.5 * alpha * occ[i] * occ[j] * h ** 3 * np.sum(rho * V)
            vx_bf[i] += -alpha * occ[j] * V * psi[j]
    Ex, vx, _ = o.exx(psi, occ, alpha, h, o.kernel_spectrum(G))
    assert Ex == pytest.approx(Ex_bf, rel=1e-13)
    assert np.max(np.abs(vx - vx_bf)) <= 1e-13 * np.max(np.abs(vx_bf))


def _small_case(seed=3, n=10, N=4):
    from paper_1712_07973_gb300 import synth
    r = synth.OrbitalRecipe(n=n, h=0.5, norb=N, nsites=3, seed=seed, gauss_per_orb=3,
                            sigma=(0.6, 1.0), p_type=True)
    return r, synth.make_orbitals(r)


def test_invariants():
    r, psi = _small_case()
    h, N = r.h, r.norb
    occ = np.full(N, 2.0)
    Gh = o.kernel_spectrum(o.kernel_real_space(r.n, h))
    Ex, vx, Eij = o.exx(psi, occ, 0.25, h, Gh)
    # exchange is negative, every pair energy positive (positive-definite kernel)
    assert Ex < 0
    assert np.all(np.linalg.eigvalsh(Eij) > -1e-14) and np.all(np.diag(Eij) > 0)
    # E_x = 1/2 sum_i f_i h^3 <psi_i, (Vx psi)_i>
    cons = 0.5 * sum(occ[i] * h ** 3 * np.sum(psi[i] * vx[i]) for i in range(N))
    assert cons == pytest.approx(Ex, rel=1e-13)
    # homogeneity and linearity in alpha
    Ex2, vx2, _ = o.exx(1.7 * psi, occ, 0.25, h, Gh)
    assert Ex2 == pytest.approx(1.7 ** 4 * Ex, rel=1e-13)
    assert np.allclose(vx2, 1.7 ** 3 * vx, rtol=1e-12, atol=1e-14)
    Ex3, _, _ = o.exx(psi, occ, 0.5, h, Gh)
    assert Ex3 == pytest.approx(2 * Ex, rel=1e-14)
    # orthogonal rotation among equally occupied orbitals
    U, _ = np.linalg.qr(_rng(11).standard_normal((N, N)))
    psiU = np.einsum("ij,jzyx->izyx", U, psi)
    ExU, vxU, _ = o.exx(psiU, occ, 0.25, h, Gh)
    assert ExU == pytest.approx(Ex, rel=1e-12)
    assert np.allclose(vxU, np.einsum("ij,jzyx->izyx", U, vx), rtol=0,
                       atol=1e-12 * np.abs(vx).max())
    # V_ij = V_ji: the pair potential does not depend on the order
    V1, e1 = o.exx_pair(psi[0], psi[2], Gh, h)
    V2, e2 = o.exx_pair(psi[2], psi[0], Gh, h)
    assert np.array_equal(V1, V2) and e1 == e2


def test_gradient_finite_differences_and_euler():
    # dE_x/dpsi_k = 2 f_k h^3 (Vx psi)_k: central differences with step 1e-4
    # along 20 seeded directions normalised so that h^3 sum d^2 = 1.
    r, psi = _small_case(seed=5, n=8, N=3)
    h = r.h
    occ = np.array([2.0, 1.5, 0.5])
    Gh = o.kernel_spectrum(o.kernel_real_space(r.n, h))
    Ex, grad = o.exx_energy_gradient(psi, occ, 0.25, h, Gh)
    rng = _rng(21)
    eps = 1e-4
    for _ in range(20):
        d = rng.standard_normal(psi.shape)
        d /= math.sqrt(h ** 3 * np.sum(d * d))
        Ep, _, _ = o.exx(psi + eps * d, occ, 0.25, h, Gh, want_vx=False)
        Em, _, _ = o.exx(psi - eps * d, occ, 0.25, h, Gh, want_vx=False)
        fd = (Ep - Em) / (2 * eps)
        an = float(np.sum(grad * d))
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3 * abs(Ex)), (fd, an)
    # E_x is homogeneous of degree 4 in psi
    assert float(np.sum(psi * grad)) == pytest.approx(4 * Ex, rel=1e-12)


def test_pair_count_matches_paper_table():
    with open(os.path.join(GOLDEN, "pscount.json")) as fh:
        table = json.load(fh)
    for N, count in table["h2o"]:
        assert N * (N + 1) // 2 == count
    for N in (1, 2, 4, 7, 64):
        pl = o.pair_list(N)
        assert len(pl) == N * (N + 1) // 2 and len(set(pl)) == len(pl)
        assert all(i <= j for i, j in pl)


# ------------------------------------------------------ screened kernel

def test_erfc_kernel_gaussian_potential_and_energy():
    # Gaussian charge (variance s^2) in the short-range kernel erfc(w r)/r:
    # V = [erf(r/(sqrt2 s)) - erf(r/sqrt(2 s^2 + 1/w^2))]/r, because erf(w r)/r is
    # the potential of a Gaussian of variance 1/(2 w^2) and variances add under
    # convolution; E = int rho V = sqrt(2/pi) [1/sqrt(2 s^2) - 1/sqrt(2 s^2 + 1/(2 w^2))]
    n, h, sig = 48, 0.2, 0.6
    for w in (0.11, 0.6, 2.0):
        r = _centered_grid(n, h)
        rho = np.exp(-r * r / (2 * sig * sig)) / (2 * math.pi * sig * sig) ** 1.5
        G = o.kernel_real_space(n, h, o.KERNEL_ERFC, omega=w)
        V = o.poisson(rho, o.kernel_spectrum(G))
        s2 = 2 * sig * sig + 1.0 / (w * w)
        with np.errstate(invalid="ignore", divide="ignore"):
            Vex = np.where(r > 0, (special.erf(r / (math.sqrt(2) * sig)) - special.erf(r / math.sqrt(s2)))
                           / np.where(r > 0, r, 1),
                           math.sqrt(2 / math.pi) / sig - 2.0 / math.sqrt(math.pi * s2))
        assert np.max(np.abs(V - Vex)) <= 1e-11 * np.max(np.abs(Vex)), w
        E = h ** 3 * np.sum(rho * V)
        Eex = math.sqrt(2 / math.pi) * (1 / math.sqrt(2 * sig * sig) - 1 / math.sqrt(2 * sig * sig + 0.5 / (w * w)))
        assert E == pytest.approx(Eex, rel=1e-11), w


def test_erfc_kernel_small_omega_longrange_part_is_point_erf():
    # for omega h << 1 the t < omega part of the band-limited kernel is the
    # plain point value h^3 erf(omega |m| h)/(|m| h) (the band edge is far)
    n, h, w = 12, 0.4, 0.11
    Gf = o.kernel_real_space(n, h)
    Gs = o.kernel_real_space(n, h, o.KERNEL_ERFC, omega=w)
    m = np.arange(n + 1, dtype=float)
    R = h * np.sqrt(m[:, None, None] ** 2 + m[None, :, None] ** 2 + m[None, None, :] ** 2)
    with np.errstate(invalid="ignore", divide="ignore"):
        lr = np.where(R > 0, special.erf(w * R) / np.where(R > 0, R, 1), 2 * w / math.sqrt(math.pi))
    assert np.max(np.abs((Gf - Gs) - h ** 3 * lr)) <= 1e-13 * np.max(np.abs(Gf))


def test_closed_shell_as_two_spin_channels():
    # Eq. HF with per-spin occupations: identical up and down channels with
    # f = 1 give half the value of the spinless formula with f = 2 (the
    # occupations enter quadratically), i.e. twice one channel with f = 1
    r, psi = _small_case(seed=8, n=8, N=3)
    Gh = o.kernel_spectrum(o.kernel_real_space(r.n, r.h))
    E1, vx1, _ = o.exx(psi, np.ones(3), 0.25, r.h, Gh)
    E2, vx2, _ = o.exx(psi, np.full(3, 2.0), 0.25, r.h, Gh)
    assert 2 * E1 == pytest.approx(0.5 * E2, rel=1e-14)
    assert np.allclose(2 * vx1, vx2, rtol=1e-14, atol=0)


# ------------------------------------------------------ periodic boundary conditions

def test_periodic_plane_wave_exact():
    # rho = cos(k0 . r) on the periodic cell solves lap V = -4 pi rho with
    # V = (4 pi / |k0|^2) rho exactly
    n, h = 12, 0.5
    x = np.arange(n) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    Lb = n * h
    for m in [(1, 0, 0), (2, 1, 0), (1, 3, 2), (0, 0, 6)]:
        k0 = 2 * math.pi / Lb * np.array(m, dtype=float)
        rho = np.cos(k0[0] * X + k0[1] * Y + k0[2] * Z)
        V = o.poisson(rho, o.kernel_spectrum_periodic(n, h))
        assert np.max(np.abs(V - 4 * math.pi / (k0 @ k0) * rho)) <= 1e-12 * 4 * math.pi / (k0 @ k0)


def test_periodic_constant_density_has_zero_potential():
    n, h = 8, 0.4
    V = o.poisson(np.full((n, n, n), 0.7), o.kernel_spectrum_periodic(n, h))
    assert np.max(np.abs(V)) <= 1e-14


def test_periodic_gaussian_madelung_constant():
    # A unit Gaussian charge (sigma) with a neutralising background in a cubic
    # cell of side Lb: E = 1/(2 sigma sqrt(pi)) - xi/(2 Lb) + c/Lb^3 + ...,
    # xi = 2.837297479 the Madelung constant of the simple cubic lattice with a
    # uniform compensating background.  Fitting xi and c over three cells pins
    # the periodic kernel's normalisation, its k = 0 treatment and |k|.
    sig, h = 1.0, 0.25
    Ls, Es = [], []
    for n in (40, 56, 72):
        Lb = n * h
        x = np.arange(n) * h - 0.5 * Lb
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        rho = np.exp(-(X * X + Y * Y + Z * Z) / (2 * sig * sig)) / (2 * math.pi * sig * sig) ** 1.5
        V = o.poisson(rho, o.kernel_spectrum_periodic(n, h))
        Ls.append(Lb)
        Es.append(0.5 * h ** 3 * float(np.sum(rho * V)))
    Ls, Es = np.array(Ls), np.array(Es)
    A = np.stack([-0.5 / Ls, 1.0 / Ls ** 3], axis=1)
    (xi, c), *_ = np.linalg.lstsq(A, Es - 1.0 / (2 * sig * math.sqrt(math.pi)), rcond=None)
    assert xi == pytest.approx(2.837297479, abs=1e-5), (xi, c)


def test_periodic_exchange_invariants():
    r, psi = _small_case(seed=9, n=8, N=3)
    Gp = o.kernel_spectrum_periodic(r.n, r.h)
    Ex, vx, Eij = o.exx(psi, np.full(3, 2.0), 0.25, r.h, Gp)
    assert Ex < 0 and np.all(np.diag(Eij) > 0)
    assert np.all(np.linalg.eigvalsh(Eij) > -1e-14)
    assert Ex == pytest.approx(0.5 * 2.0 * r.h ** 3 * float(np.sum(psi * vx)), rel=1e-13)
    # V_ij = V_ji and the pair sum by brute force over ordered pairs
    tot = 0.0
    for i in range(3):
        for j in range(3):
            V = o.poisson(psi[i] * psi[j], Gp)
            tot += 4.0 * r.h ** 3 * float(np.sum(psi[i] * psi[j] * V))
    assert Ex == pytest.approx(-0.5 * 0.25 * tot, rel=1e-13)


# ------------------------------------------------ slab and wire boundary conditions
# Slab: x, y periodic (cell n h), z free.  Wire: x, y free, z periodic.  The
# densities below are band-limited on the free axes (sigma >= 2.5 h) and fit
# the box (sigma <= half-box / 7), so the band-limited kernels must reproduce
# the continuum potentials to rounding.

def _gauss1(u, s):
    return np.exp(-u * u / (2 * s * s)) / (s * math.sqrt(2 * math.pi))


def test_slab_charged_sheet_potential():
    # uniform in the plane, Gaussian profile in z (unit charge per area):
    # V(z) = -2 pi int |z - z'| rho(z') dz' = -2 pi [z erf(z / (s sqrt 2)) + s sqrt(2/pi) e^{-z^2/2s^2}]
    n, h, s = 48, 0.2, 0.6
    zz = np.arange(n) * h - (n - 1) * h / 2
    rho = np.broadcast_to(_gauss1(zz, s)[:, None, None], (n, n, n)).copy()
    V = o.poisson(rho, o.kernel_spectrum_slab(n, h))
    ref = -2 * math.pi * (zz * special.erf(zz / (s * math.sqrt(2)))
                          + s * math.sqrt(2 / math.pi) * np.exp(-zz ** 2 / (2 * s * s)))
    assert np.max(np.abs(V - ref[:, None, None])) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("mx,my", [(1, 0), (3, 2), (7, 0), (0, 5)])
def test_slab_plane_wave_times_gaussian(mx, my):
    # rho = cos(k . r_par) g(z): V = cos(k . r_par) (2 pi / k) int e^{-k|z-z'|} g(z') dz'
    #     = cos(k . r_par) (pi / k) e^{-z^2/2s^2} [erfcx((k s^2 - z)/(s sqrt 2)) + erfcx((k s^2 + z)/(s sqrt 2))]
    n, h, s = 48, 0.2, 0.6
    x = np.arange(n) * h
    zz = x - (n - 1) * h / 2
    kx, ky = 2 * math.pi * mx / (n * h), 2 * math.pi * my / (n * h)
    k = math.hypot(kx, ky)
    plane = np.cos(ky * x[:, None] + kx * x[None, :])        # [y, x]
    rho = _gauss1(zz, s)[:, None, None] * plane[None]
    V = o.poisson(rho, o.kernel_spectrum_slab(n, h))
    a = (k * s * s - zz) / (s * math.sqrt(2))
    b = (k * s * s + zz) / (s * math.sqrt(2))
    Vz = (math.pi / k) * np.exp(-zz ** 2 / (2 * s * s)) * (special.erfcx(a) + special.erfcx(b))
    ref = Vz[:, None, None] * plane[None]
    assert np.max(np.abs(V - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("kappa,d", [(0.3, 0), (0.3, 5), (1.7, 2), (2.9, 11)])
def test_slab_kernel_entries_against_quadpack(kappa, d):
    # h g(k, d h) = h 4 int_0^{pi/h} cos(q d h) / (k^2 + q^2) dq (QUADPACK's
    # cosine-weighted rule, not the oracle's t-integral)
    # (d = 0: the closed form (4 / k) atan(pi / (h k)))
    n, h = 16, 0.4
    k = kappa / h
    if d == 0:
        val = 4.0 / k * math.atan(math.pi / (h * k))
    else:
        val, _ = integrate.quad(lambda q: 4.0 / (k * k + q * q), 0.0, math.pi / h, weight="cos",
                                wvar=d * h, epsabs=1e-13, epsrel=1e-13)
    got = o.slab_kernel_z(n, h, [kappa])[0, d]
    assert got == pytest.approx(h * val, rel=1e-12, abs=1e-14)


def test_wire_line_charge_potential():
    # uniform along z, 2D Gaussian across (unit charge per length):
    # V(r) = -2 ln r - E1(r^2 / (2 s^2))  (-> -2 ln r far away; gamma - ln(2 s^2) at r = 0)
    n, h, s = 48, 0.2, 0.6
    u = np.arange(n) * h - (n // 2) * h
    r2 = u[:, None] ** 2 + u[None, :] ** 2                     # [y, x]
    rho2 = np.exp(-r2 / (2 * s * s)) / (2 * math.pi * s * s)
    V = o.poisson(np.broadcast_to(rho2[None], (n, n, n)).copy(), o.kernel_spectrum_wire(n, h))
    ref = np.empty_like(r2)
    nz = r2 > 0
    ref[nz] = -np.log(r2[nz]) - special.exp1(r2[nz] / (2 * s * s))
    ref[~nz] = np.euler_gamma - math.log(2 * s * s)
    assert np.max(np.abs(V - ref[None])) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("mz", [1, 2, 5])
def test_wire_axial_wave_times_gaussian(mz):
    # rho = cos(k z) g2(r): V = cos(k z) 2 int_0^inf q J0(q r) e^{-q^2 s^2/2} / (k^2 + q^2) dq,
    # = cos(k z) e^{k^2 s^2/2} E1(k^2 s^2/2) on the axis
    n, h, s = 48, 0.2, 0.6
    x = np.arange(n) * h
    u = x - (n // 2) * h
    r2 = u[:, None] ** 2 + u[None, :] ** 2
    k = 2 * math.pi * mz / (n * h)
    rho = np.cos(k * x)[:, None, None] * (np.exp(-r2 / (2 * s * s)) / (2 * math.pi * s * s))[None]
    V = o.poisson(rho, o.kernel_spectrum_wire(n, h))
    axis = math.exp(k * k * s * s / 2) * special.exp1(k * k * s * s / 2)
    assert V[0, n // 2, n // 2] == pytest.approx(axis, rel=1e-12)
    for (iy, ix) in [(n // 2, n // 2 + 3), (n // 2 + 7, n // 2 - 4), (3, 40)]:
        rr = math.sqrt(r2[iy, ix])
        val, _ = integrate.quad(lambda q: 2 * q * special.j0(q * rr) * math.exp(-q * q * s * s / 2)
                                / (k * k + q * q), 0, 15.0 / s, epsabs=1e-14, epsrel=1e-13, limit=400)
        assert V[0, iy, ix] == pytest.approx(val, rel=1e-11, abs=1e-13)


def _mixed_direct_sum(rho, K, per_axes):
    """V[m] = sum_m' Kr[m - m'] rho[m'] with per-axis differences taken mod n on
    the periodic axes and as |m - m'| on the free ones (O(n^6), tiny n)."""
    n = rho.shape[0]
    idx = np.arange(n)
    dif = [((idx[:, None] - idx[None, :]) % n) if p else np.abs(idx[:, None] - idx[None, :])
           for p in per_axes]
    V = np.empty_like(rho)
    for z in range(n):
        for y in range(n):
            for x in range(n):
                V[z, y, x] = np.sum(K[dif[0][z][:, None, None], dif[1][y][None, :, None],
                                      dif[2][x][None, None, :]] * rho)
    return V


def test_slab_and_wire_padded_fft_equal_direct_sums():
    # the real-space kernels, periodised by an explicit inverse DFT over the
    # periodic axes, summed directly: pins the zero padding, the window and the
    # spectrum assembly of kernel_spectrum_slab / _wire
    n, h = 6, 0.45
    rng = _rng(21)
    rho = rng.standard_normal((n, n, n))
    m = np.fft.fftfreq(n, d=1.0 / n)
    # slab: Kr[dz][dy][dx] = (1/n^2) sum_{my, mx} e^{2 pi i (my dy + mx dx)/n} K[kappa(my, mx)][dz]
    kap = 2 * math.pi * np.sqrt(m[:, None] ** 2 + m[None, :] ** 2) / n
    Kz = o.slab_kernel_z(n, h, kap.ravel()).reshape(n, n, n + 1)      # [my][mx][dz]
    Kr = np.real(np.fft.ifft2(Kz, axes=(0, 1))).transpose(2, 0, 1)    # [dz][dy][dx]
    V = o.poisson(rho, o.kernel_spectrum_slab(n, h))
    assert np.max(np.abs(V - _mixed_direct_sum(rho, Kr, (False, True, True)))) <= 1e-12 * np.max(np.abs(V))
    # wire: Kr[dz][dy][dx] = (1/n) sum_mz e^{2 pi i mz dz/n} K2[kappa(mz)][dy][dx]
    K2 = o.wire_kernel_xy(n, h, 2 * math.pi * np.abs(m) / n)          # [mz][dy][dx]
    Kr = np.real(np.fft.ifft(K2, axis=0))
    V = o.poisson(rho, o.kernel_spectrum_wire(n, h))
    assert np.max(np.abs(V - _mixed_direct_sum(rho, Kr, (True, False, False)))) <= 1e-12 * np.max(np.abs(V))


def test_slab_and_wire_exchange_invariants():
    r, psi = _small_case(seed=10, n=8, N=3)
    for Gm in (o.kernel_spectrum_slab(r.n, r.h), o.kernel_spectrum_wire(r.n, r.h)):
        Ex, vx, Eij = o.exx(psi, np.full(3, 2.0), 0.25, r.h, Gm)
        assert np.allclose(Eij, Eij.T, rtol=0, atol=0)
        assert Ex == pytest.approx(0.5 * 2.0 * r.h ** 3 * float(np.sum(psi * vx)), rel=1e-12)
        # homogeneity: E_x(c psi) = c^4 E_x
        E2, _, _ = o.exx(1.3 * psi, np.full(3, 2.0), 0.25, r.h, Gm, want_vx=False)
        assert E2 == pytest.approx(1.3 ** 4 * Ex, rel=1e-12)
