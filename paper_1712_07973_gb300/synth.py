"""Seeded synthetic Kohn-Sham-like orbitals on a uniform cubic mesh.

This module only manufactures inputs.  It holds none of the exact-exchange
arithmetic, so both the FP64 oracle's tests and the CUDA path can consume the
same arrays.  Everything is FP64 NumPy, driven by ``numpy.random.default_rng``
so that the same seed gives the same orbitals on every machine (up to the last
bits of the LAPACK eigensolver used by the Lowdin step).

Recipe (stands in for the pseudopotential orbitals of the paper's H2O / UO2
runs, Sec. 3, whose structures and grids are not published):

* grid nodes at x_m = m h, m = 0..n-1 per axis, arrays indexed [z, y, x];
* "atom" sites uniform in the central 60% of the box, or on a jittered cubic
  lattice (the large cluster workload);
* each orbital is a sum of Gaussians exp(-|r-R|^2 / (2 sigma^2)) centred on
  random sites, of type s, or x/y/z times the Gaussian (p type), with
  N(0,1) coefficients and sigma uniform in a given range;
* the set is Lowdin-orthonormalised with the discrete inner product
  S_ij = h^3 sum_m phi_i phi_j, psi = S^{-1/2} phi.
"""

from dataclasses import dataclass, field

import numpy as np

__all__ = ["OrbitalRecipe", "make_orbitals", "orbital_subset", "workload", "WORKLOADS",
           "batched_workload", "small_batched_workload"]


@dataclass
class OrbitalRecipe:
    n: int                       # grid points per axis
    h: float                     # grid spacing (bohr)
    norb: int                    # number of orbitals
    nsites: int                  # number of atom sites
    seed: int
    gauss_per_orb: int = 3
    sigma: tuple = (0.8, 1.5)
    p_type: bool = False         # include x/y/z * Gaussian terms
    lattice: float = 0.0         # >0: sites on a jittered cubic lattice (bohr)
    occupation: float = 2.0
    alpha: float = 0.25
    extra: dict = field(default_factory=dict)


def _sites(rng, r: OrbitalRecipe):
    L = (r.n - 1) * r.h
    if r.lattice > 0.0:
        a = r.lattice
        c = 0.5 * L
        k = int(np.ceil(np.cbrt(r.nsites))) + 3
        g = np.arange(-k, k + 1, dtype=np.float64)
        P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
        d2 = np.sum(P * P, axis=1)
        # nearest to the centre; ties broken by lexicographic index (stable sort)
        order = np.argsort(d2, kind="stable")[: r.nsites]
        P = c + a * P[order]
        P = P + rng.uniform(-0.1 * a, 0.1 * a, size=P.shape)
        return P
    return rng.uniform(0.2 * L, 0.8 * L, size=(r.nsites, 3))


def make_orbitals(r: OrbitalRecipe, dtype=np.float64, device=None):
    """Return psi[norb, n, n, n] (Lowdin-orthonormal, FP64 unless dtype given).

    With ``device`` (a torch device) the per-orbital contractions and the
    Lowdin step run there in FP64 and a torch tensor on that device is
    returned; the random draws are the same NumPy ones.
    """
    if device is not None:
        return _make_orbitals_torch(r, dtype, device)
    rng = np.random.default_rng(r.seed)
    sites = _sites(rng, r)
    x = np.arange(r.n, dtype=np.float64) * r.h
    n, G = r.n, r.gauss_per_orb
    phi = np.empty((r.norb, n, n, n), dtype=np.float64)
    for o in range(r.norb):
        at = rng.integers(0, r.nsites, size=G)
        sig = rng.uniform(r.sigma[0], r.sigma[1], size=G)
        coef = rng.standard_normal(G)
        typ = rng.integers(0, 4, size=G) if r.p_type else np.zeros(G, int)
        R = sites[at]                                   # (G, 3) as (x, y, z)
        s2 = 2.0 * sig ** 2
        dz = x[:, None] - R[None, :, 2]                 # (n, G)
        dy = x[:, None] - R[None, :, 1]
        dx = x[:, None] - R[None, :, 0]
        gz = np.exp(-dz * dz / s2) * np.where(typ == 3, dz, 1.0) * coef
        gy = np.exp(-dy * dy / s2) * np.where(typ == 2, dy, 1.0)
        gx = np.exp(-dx * dx / s2) * np.where(typ == 1, dx, 1.0)
        # sum over the G separable terms as one contraction: (n, G) @ (G, n^2)
        yx = (gy[:, None, :] * gx[None, :, :]).reshape(n * n, G)
        phi[o] = (gz @ yx.T).reshape(n, n, n)
    flat = phi.reshape(r.norb, -1)
    S = (r.h ** 3) * (flat @ flat.T)
    w, U = np.linalg.eigh(S)
    Sm12 = (U / np.sqrt(w)) @ U.T
    psi = (Sm12 @ flat).reshape(phi.shape)
    return np.ascontiguousarray(psi.astype(dtype, copy=False))


def _make_orbitals_torch(r: OrbitalRecipe, dtype, device):
    import torch
    rng = np.random.default_rng(r.seed)
    sites = _sites(rng, r)
    x = np.arange(r.n, dtype=np.float64) * r.h
    n, G = r.n, r.gauss_per_orb
    phi = torch.empty((r.norb, n * n * n), dtype=torch.float64, device=device)
    for o in range(r.norb):
        at = rng.integers(0, r.nsites, size=G)
        sig = rng.uniform(r.sigma[0], r.sigma[1], size=G)
        coef = rng.standard_normal(G)
        typ = rng.integers(0, 4, size=G) if r.p_type else np.zeros(G, int)
        R = sites[at]
        s2 = 2.0 * sig ** 2
        dz = x[:, None] - R[None, :, 2]
        dy = x[:, None] - R[None, :, 1]
        dx = x[:, None] - R[None, :, 0]
        gz = np.exp(-dz * dz / s2) * np.where(typ == 3, dz, 1.0) * coef
        gy = np.exp(-dy * dy / s2) * np.where(typ == 2, dy, 1.0)
        gx = np.exp(-dx * dx / s2) * np.where(typ == 1, dx, 1.0)
        gz_t = torch.from_numpy(gz).to(device)
        yx_t = torch.from_numpy((gy[:, None, :] * gx[None, :, :]).reshape(n * n, G)).to(device)
        phi[o] = (gz_t @ yx_t.T).reshape(-1)
    S = (r.h ** 3) * (phi @ phi.T)
    # the norb x norb eigenproblem on the host (NumPy, as in make_orbitals)
    w, U = np.linalg.eigh(S.cpu().numpy())
    Sm12 = torch.from_numpy((U / np.sqrt(w)) @ U.T).to(device)
    psi = (Sm12 @ phi).reshape(r.norb, n, n, n)
    tdt = {np.float64: torch.float64, np.float32: torch.float32}[np.dtype(dtype).type]
    return psi.to(tdt).contiguous()


def _terms(r: OrbitalRecipe):
    """The separable terms of every orbital, with the same random draws as
    make_orbitals: per-axis profiles Z, Y, X (coefficient folded into Z) of
    shape (norb * G, n) and the orbital of each term."""
    rng = np.random.default_rng(r.seed)
    sites = _sites(rng, r)
    x = np.arange(r.n, dtype=np.float64) * r.h
    G = r.gauss_per_orb
    Z, Y, X = [], [], []
    for o in range(r.norb):
        at = rng.integers(0, r.nsites, size=G)
        sig = rng.uniform(r.sigma[0], r.sigma[1], size=G)
        coef = rng.standard_normal(G)
        typ = rng.integers(0, 4, size=G) if r.p_type else np.zeros(G, int)
        R = sites[at]
        s2 = 2.0 * sig ** 2
        dz = x[None, :] - R[:, 2, None]                 # (G, n)
        dy = x[None, :] - R[:, 1, None]
        dx = x[None, :] - R[:, 0, None]
        Z.append(np.exp(-dz * dz / s2[:, None]) * np.where(typ[:, None] == 3, dz, 1.0) * coef[:, None])
        Y.append(np.exp(-dy * dy / s2[:, None]) * np.where(typ[:, None] == 2, dy, 1.0))
        X.append(np.exp(-dx * dx / s2[:, None]) * np.where(typ[:, None] == 1, dx, 1.0))
    owner = np.repeat(np.arange(r.norb), G)
    return np.concatenate(Z), np.concatenate(Y), np.concatenate(X), owner


def orbital_subset(r: OrbitalRecipe, idx, chunk=1024):
    """Orbitals idx of the workload (the rows psi[idx] of make_orbitals, to
    rounding) without forming the others: every orbital is a sum of separable
    terms, so the overlap matrix S_ij = h^3 sum_m phi_i phi_j is a sum of
    products of one-dimensional overlaps, and psi_k = sum_j (S^-1/2)_kj phi_j
    is a weighted sum of the separable terms.  Memory O(norb^2 G^2 / blocks +
    len(idx) n^3); used for large workloads on the host."""
    Z, Y, X, owner = _terms(r)
    N, G, n = r.norb, r.gauss_per_orb, r.n
    S = np.zeros((N, N))
    for b0 in range(0, N, max(1, chunk // G)):
        b1 = min(N, b0 + max(1, chunk // G))
        rows = slice(b0 * G, b1 * G)
        W = (Z[rows] @ Z.T) * (Y[rows] @ Y.T) * (X[rows] @ X.T)   # term overlaps
        S[b0:b1] = W.reshape(b1 - b0, G, N, G).sum(axis=(1, 3))
    S *= r.h ** 3
    S = 0.5 * (S + S.T)
    w, U = np.linalg.eigh(S)
    Sm12 = (U / np.sqrt(w)) @ U.T
    idx = np.asarray(idx, dtype=np.int64)
    A = Sm12[idx][:, owner]                                       # (K, terms)
    out = np.zeros((len(idx), n, n * n))
    for t0 in range(0, Z.shape[0], chunk):
        t1 = min(Z.shape[0], t0 + chunk)
        YX = (Y[t0:t1, :, None] * X[t0:t1, None, :]).reshape(t1 - t0, n * n)
        for k in range(len(idx)):
            out[k] += (Z[t0:t1] * A[k, t0:t1, None]).T @ YX
    return out.reshape(len(idx), n, n, n)


# Workloads: the five configurations the benchmarks and parity tests use.
WORKLOADS = {
    # plain FP64: 4 orbitals, 32^3 grid (64^3 padded), 3 s-Gaussians each
    "c1_fp64_n32_N4": OrbitalRecipe(n=32, h=0.4, norb=4, nsites=4, seed=0,
                                    gauss_per_orb=3, sigma=(0.8, 1.5)),
    # FP32 forward: 64 orbitals, 96^3 (192^3 padded), 16 s/p Gaussians each
    "c2_fp32_n96_N64": OrbitalRecipe(n=96, h=0.4, norb=64, nsites=32, seed=1,
                                     gauss_per_orb=16, sigma=(0.7, 1.8), p_type=True),
    # autograd: 128 orbitals, 128^3 (256^3 padded)
    "c3_grad_n128_N128": OrbitalRecipe(n=128, h=0.37, norb=128, nsites=64, seed=2,
                                       gauss_per_orb=16, sigma=(0.7, 1.8), p_type=True),
    # large cluster: 512 orbitals, 160^3 (320^3 padded), jittered 0.35 nm lattice
    "c5_large_n160_N512": OrbitalRecipe(n=160, h=0.42, norb=512, nsites=256, seed=4,
                                        gauss_per_orb=16, sigma=(0.7, 1.8), p_type=True,
                                        lattice=6.614),
}


def workload(name, dtype=np.float64, device=None):
    r = WORKLOADS[name]
    return r, make_orbitals(r, dtype=dtype, device=device)


def batched_workload(seed=3, nmol=16, grids=(48, 64, 80, 96, 112, 128), nrange=(8, 96)):
    """Recipes of the batched, uneven workload: nmol molecules, N_m ~ U{8..96},
    n_m drawn from ``grids``, h = 0.4, sites proportional to N_m / 2."""
    rng = np.random.default_rng(seed)
    out = []
    for mol in range(nmol):
        N = int(rng.integers(nrange[0], nrange[1] + 1))
        n = int(grids[int(rng.integers(0, len(grids)))])
        out.append(OrbitalRecipe(n=n, h=0.4, norb=N, nsites=max(2, N // 2),
                                 seed=int(rng.integers(0, 2 ** 31 - 1)),
                                 gauss_per_orb=16, sigma=(0.7, 1.8), p_type=True))
    return out


def small_batched_workload(seed=5, nmol=64, grids=(32, 40, 48), nrange=(8, 24)):
    """Recipes of many small molecules (N_m ~ U{8..24}, n_m from ``grids``,
    h = 0.4): per-launch work is small, so launch count and tail effects
    dominate a per-molecule schedule."""
    return batched_workload(seed=seed, nmol=nmol, grids=grids, nrange=nrange)
