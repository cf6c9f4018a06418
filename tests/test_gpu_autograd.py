"""GPU checks of the autograd wrapper: its backward is the exchange action.

* FP64: central finite differences (step 1e-4) along 20 seeded directions
  normalised so that h^3 sum d^2 = 1 agree with <grad, d> to 1e-7 relative, and
  the gradient equals the oracle's 2 f_k h^3 (Vx psi)_k.
* FP32: the gradient matches the FP64 gradient in relative L2 (1e-5), also on
  the 128-orbital 128^3 workload itself, where the FP64 gradient is the
  analytic one of the FP64 path.  There the FP32 energy is accurate to ~1e-8
  relative, so central differences at step 1e-4 carry ~1e-4 relative noise;
  that check uses random localised directions (Gaussian bumps) and a 2e-3
  bound.
* The library's gradient (exx_gradient, the factor 2 f_k h^3 folded into the
  accumulation) equals 2 f_k h^3 times exx_apply's action.
"""

import json
import math
import os

import numpy as np
import pytest

from oracle import exx_oracle as o
from paper_1712_07973_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1712_07973_gb300 import autograd, build, exx
    build.build()
    return torch, torch.device("cuda:0"), exx, autograd


def _orbitals(n, N, seed, h):
    r = synth.OrbitalRecipe(n=n, h=h, norb=N, nsites=3, seed=seed, gauss_per_orb=3,
                            sigma=(0.12 * n * h, 0.2 * n * h), p_type=True)
    return synth.make_orbitals(r)


def _grad(env, psi_np, occ, h, precision, recompute=False):
    torch, dev, exx, ag = env
    n = psi_np.shape[1]
    plan = exx.ExxPlan(n, h, 0.25, occ, precision=precision)
    psi = torch.from_numpy(psi_np).to(dev, plan.dtype).requires_grad_(True)
    E = ag.exx_energy(psi, plan, recompute=recompute)
    E.backward()
    g = psi.grad.detach().double().cpu().numpy()
    return float(E.item()), g, plan


def test_fp64_gradient_fd_oracle_and_euler(env):
    torch, dev, exx, ag = env
    n, N, h = 16, 4, 0.45
    psi = _orbitals(n, N, seed=71, h=h)
    occ = np.array([2.0, 1.5, 1.0, 0.5])
    E, g, plan = _grad(env, psi, occ, h, "fp64")
    # oracle gradient
    Gh = o.kernel_spectrum(o.kernel_real_space(n, h))
    Eo, go = o.exx_energy_gradient(psi, occ, 0.25, h, Gh)
    assert abs(E - Eo) <= 1e-10 * abs(Eo)
    assert np.max(np.abs(g - go)) <= 1e-10 * np.max(np.abs(go))
    # Euler: E_x is homogeneous of degree 4
    assert float(np.sum(psi * g)) == pytest.approx(4 * E, rel=1e-10)
    # central differences on the GPU energy
    rng = np.random.default_rng(5)
    eps = 1e-4
    for _ in range(20):
        d = rng.standard_normal(psi.shape)
        d /= math.sqrt(h ** 3 * np.sum(d * d))
        Ep = plan.energy(torch.from_numpy(psi + eps * d).to(dev))
        Em = plan.energy(torch.from_numpy(psi - eps * d).to(dev))
        fd = (Ep - Em) / (2 * eps)
        an = float(np.sum(g * d))
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3 * abs(E)), (fd, an)
    plan.close()


def test_recompute_mode_and_grad_scaling(env):
    torch, dev, exx, ag = env
    psi = _orbitals(12, 3, seed=72, h=0.45)
    occ = np.array([2.0, 2.0, 1.0])
    E1, g1, p1 = _grad(env, psi, occ, 0.45, "fp64")
    E2, g2, p2 = _grad(env, psi, occ, 0.45, "fp64", recompute=True)
    assert E1 == E2 and np.array_equal(g1, g2)
    # d(c E)/dpsi = c dE/dpsi through grad_out
    pt = torch.from_numpy(psi).to(dev).requires_grad_(True)
    (3.0 * ag.exx_energy(pt, p1)).backward()
    assert np.allclose(pt.grad.cpu().numpy(), 3.0 * g1, rtol=1e-14, atol=0)
    # no gradient requested: energy path only
    with torch.no_grad():
        E3 = ag.exx_energy(torch.from_numpy(psi).to(dev), p1)
    assert float(E3) == pytest.approx(E1, rel=1e-13)
    p1.close()
    p2.close()


def test_fp32_gradient_matches_fp64(env):
    psi = _orbitals(24, 5, seed=73, h=0.4)
    occ = np.full(5, 2.0)
    E64, g64, p64 = _grad(env, psi, occ, 0.4, "fp64")
    E32, g32, p32 = _grad(env, psi, occ, 0.4, "fp32")
    assert abs(E32 - E64) <= 1e-6
    assert np.linalg.norm(g32 - g64) <= 1e-5 * np.linalg.norm(g64)
    p64.close()
    p32.close()


def test_library_gradient_is_scaled_action(env):
    torch, dev, exx, ag = env
    n, N, h = 16, 5, 0.45
    psi_np = _orbitals(n, N, seed=74, h=h)
    occ = np.array([2.0, 1.5, 1.0, 0.5, 0.25])
    for prec in ("fp64", "fp32"):
        plan = exx.ExxPlan(n, h, 0.25, occ, precision=prec, vx_fp64=True)
        psi = torch.from_numpy(psi_np).to(dev, plan.dtype)
        E1, vx = plan.apply(psi)
        E2, g = plan.gradient(psi)
        plan.close()
        assert E1 == E2
        sc = torch.as_tensor(2.0 * h ** 3 * occ, device=dev).view(-1, 1, 1, 1)
        assert torch.allclose(g, sc * vx, rtol=1e-14, atol=0)


def test_fp32_gradient_matches_fp64_on_the_128_orbital_workload(env):
    # 128 orbitals on 128^3: FP32 autograd gradient against the FP64 path's
    # analytic gradient 2 f_k h^3 (Vx psi)_k, relative L2 <= 1e-5
    torch, dev, exx, ag = env
    r, psi64 = synth.workload("c3_grad_n128_N128", dtype=np.float64, device=dev)
    occ = np.full(r.norb, r.occupation)
    p64 = exx.ExxPlan(r.n, r.h, r.alpha, occ, precision="fp64")
    E64, g64 = p64.gradient(psi64)
    Eij64 = p64.pair_energies()
    p64.close()
    p32 = exx.ExxPlan(r.n, r.h, r.alpha, occ, precision="fp32")
    psi = psi64.float().requires_grad_(True)
    E32 = ag.exx_energy(psi, p32)
    E32.backward()
    Eij32 = p32.pair_energies()
    p32.close()
    assert abs(float(E32.item()) - E64) <= 1e-6
    num = float(torch.linalg.vector_norm(psi.grad.double() - g64).item())
    den = float(torch.linalg.vector_norm(g64).item())
    assert num <= 1e-5 * den, num / den
    # both against the stored oracle values of this workload (E_x, all 8,256
    # E_ij, the action at 256 seeded points), written by tests/golden/make_golden.py
    path = os.path.join(os.path.dirname(__file__), "golden", "c3_grad_n128_N128.json")
    with open(path) as fh:
        gold = json.load(fh)
    assert abs(E64 - gold["E_x"]) <= 1e-10 * abs(gold["E_x"])
    assert abs(float(E32.item()) - gold["E_x"]) <= 1e-6
    Eo = np.asarray(gold["E_ij"])
    assert np.max(np.abs(Eij64 - Eo)) <= 1e-10 * np.max(np.abs(Eo))
    assert np.max(np.abs(Eij32 - Eo)) <= 1e-6
    pts = np.asarray(gold["sample_points"])
    vxo = np.asarray(gold["vx_samples"])
    vx64 = (g64 / (2.0 * r.occupation * r.h ** 3)).cpu().numpy()
    got = vx64[pts[:, 0], pts[:, 1], pts[:, 2], pts[:, 3]]
    assert np.max(np.abs(got - vxo)) <= 1e-10 * np.max(np.abs(vxo))


def test_autograd_workload_128_orbitals_n128_fd(env):
    # 128 orbitals on 128^3 (256^3 padded), h = 0.37: forward + hand-written
    # backward, central differences (step 1e-4) along 20 seeded directions
    torch, dev, exx, ag = env
    r, psi_np = synth.workload("c3_grad_n128_N128", dtype=np.float32)
    occ = np.full(r.norb, r.occupation)
    plan = exx.ExxPlan(r.n, r.h, r.alpha, occ, precision="fp32")
    psi = torch.from_numpy(psi_np).to(dev).requires_grad_(True)
    E = ag.exx_energy(psi, plan)
    E.backward()
    g = psi.grad.detach()
    Ev = float(E.item())
    # Euler identity in FP64 on the device
    euler = float((psi.detach().double() * g.double()).sum().item())
    assert euler == pytest.approx(4 * Ev, rel=1e-5)
    # directions: a Gaussian bump of random width (0.8-1.5 bohr) on a random
    # orbital, normalised to h^3 sum d^2 = 1.  A delocalised direction spreads the 1e-4 step over
    # 2.7e8 values, below the FP32 resolution of psi; a bump keeps it resolved.
    rng = np.random.default_rng(9)
    eps = 1e-4
    base = psi.detach()
    x = torch.arange(r.n, device=dev, dtype=torch.float64) * r.h
    for _ in range(20):
        k = int(rng.integers(0, r.norb))
        # centre: within 1 bohr of the orbital's largest value, so that the
        # derivative stands well above the FP32 energy-difference floor
        # (~2e-9 Ha, i.e. ~1e-5 on the difference quotient)
        am = int(base[k].abs().argmax().item())
        iz, iy, ix = am // (r.n * r.n), (am // r.n) % r.n, am % r.n
        c = np.array([ix, iy, iz]) * r.h + rng.uniform(-1.0, 1.0, 3)
        w = rng.uniform(0.8, 1.5)
        gz = torch.exp(-(x - c[2]) ** 2 / (2 * w * w))
        gy = torch.exp(-(x - c[1]) ** 2 / (2 * w * w))
        gx = torch.exp(-(x - c[0]) ** 2 / (2 * w * w))
        bump = gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
        bump /= math.sqrt(r.h ** 3 * float((bump * bump).sum().item()))
        pp = base.double().clone()
        pm = base.double().clone()
        pp[k] += eps * bump
        pm[k] -= eps * bump
        Ep = plan.energy(pp.float())
        Em = plan.energy(pm.float())
        fd = (Ep - Em) / (2 * eps)
        an = float((g[k].double() * bump).sum().item())
        assert abs(fd - an) <= 2e-3 * abs(an) + 2e-5, (fd, an)
    plan.close()
