"""GPU checks of the batched, uneven path (exx_batch_*).

Each molecule's pair energies and Vx psi must equal those of its own plan
(same kernels, same tile edge, same accumulation order; E_x to rounding, as
its final sum runs in another order) and the FP64 oracle within the FP32
tolerance (1e-6 Ha on E_x).
"""

import numpy as np
import pytest

from oracle import exx_oracle as o
from paper_1712_07973_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1712_07973_gb300 import build, exx
    build.build()
    return torch, torch.device("cuda:0"), exx


def _mol(n, N, seed, h):
    r = synth.OrbitalRecipe(n=n, h=h, norb=N, nsites=3, seed=seed, gauss_per_orb=3,
                            sigma=(0.12 * n * h, 0.2 * n * h), p_type=True)
    return synth.make_orbitals(r)


SMALL = [  # (n, N, h, alpha): uneven sizes, two molecules share (n, h)
    (8, 3, 0.45, 0.25), (12, 7, 0.4, 0.25), (12, 11, 0.4, 0.3), (16, 2, 0.35, 0.25), (10, 9, 0.5, 0.2),
]


def _small(env):
    torch, dev, exx = env
    psis, occs, mols = [], [], []
    for k, (n, N, h, a) in enumerate(SMALL):
        psi = _mol(n, N, 300 + k, h)
        occ = np.linspace(0.5, 2.0, N)
        psis.append(psi)
        occs.append(occ)
        mols.append({"n": n, "h": h, "alpha": a, "occupations": occ})
    return psis, occs, mols


def test_batch_equals_single_plans_and_oracle(env):
    torch, dev, exx = env
    psis, occs, mols = _small(env)
    b = exx.ExxBatch(mols)
    assert b.info()["groups"] == 4
    pt = [torch.from_numpy(p).to(dev, torch.float32) for p in psis]
    vx = [torch.empty_like(p) for p in pt]
    b.set_buffers(pt, vx)
    E = b.apply().cpu().numpy()
    Ee = b.energy().cpu().numpy()
    for k, (m, p, occ) in enumerate(zip(mols, psis, occs)):
        plan = exx.ExxPlan(m["n"], m["h"], m["alpha"], occ, precision="fp32")
        Es, vs = plan.apply(pt[k])
        # the final FP64 sum runs in another order: equal to rounding
        assert abs(E[k] - Es) <= 1e-14 * abs(Es) and abs(Ee[k] - Es) <= 1e-14 * abs(Es)
        assert torch.equal(vx[k], vs)
        assert np.array_equal(b.pair_energies(k), plan.pair_energies())
        plan.close()
        Gh = o.kernel_spectrum(o.kernel_real_space(m["n"], m["h"]))
        Eo, vxo, _ = o.exx(p, occ, m["alpha"], m["h"], Gh)
        assert abs(E[k] - Eo) <= 1e-6
        assert np.max(np.abs(vx[k].double().cpu().numpy() - vxo)) <= 2e-6 * np.max(np.abs(vxo))
    b.close()


def test_batch_graph_capture_replay_and_rebinding(env):
    torch, dev, exx = env
    psis, occs, mols = _small(env)
    b = exx.ExxBatch(mols)
    pt = [torch.from_numpy(p).to(dev, torch.float32) for p in psis]
    vx = [torch.empty_like(p) for p in pt]
    b.set_buffers(pt, vx)
    E_ref = b.apply().clone()
    vx_ref = [v.clone() for v in vx]
    s = torch.cuda.Stream()
    E = torch.zeros(len(mols), dtype=torch.float64, device=dev)
    b.graph(True)
    with torch.cuda.stream(s):
        for _ in range(3):  # capture once, then replay
            b.apply(E, stream=s)
    s.synchronize()
    assert torch.equal(E, E_ref)
    assert all(torch.equal(a, c) for a, c in zip(vx, vx_ref))
    # rebinding new orbitals (scaled by 2: E x16, Vx psi x8) reuses the graph
    pt2 = [2.0 * p for p in pt]
    vx2 = [torch.empty_like(p) for p in pt]
    b.set_buffers(pt2, vx2)
    with torch.cuda.stream(s):
        b.apply(E, stream=s)
    s.synchronize()
    assert torch.allclose(E, 16.0 * E_ref, rtol=1e-6, atol=0)
    for a, c in zip(vx2, vx_ref):
        assert torch.allclose(a, 8.0 * c, rtol=1e-5, atol=1e-6 * float(c.abs().max()))
    b.close()


def test_batched_autograd_equals_single_plan_autograd(env):
    # ExxBatchEnergy (one batched gradient call) against ExxEnergy on each
    # molecule's own plan: identical gradients (same tiles, same accumulation
    # order, same per-orbital factor) and E_x to rounding; grad_out weights
    # per molecule go through the chain rule
    torch, dev, exx = env
    from paper_1712_07973_gb300 import autograd as ag
    psis, occs, mols = _small(env)
    b = exx.ExxBatch(mols)
    pt = [torch.from_numpy(p).to(dev, torch.float32).requires_grad_(True) for p in psis]
    E = ag.exx_batch_energy(b, pt)
    w = torch.linspace(0.5, 1.5, len(mols), dtype=torch.float64, device=dev)
    (w * E).sum().backward()
    for k, (m, occ) in enumerate(zip(mols, occs)):
        plan = exx.ExxPlan(m["n"], m["h"], m["alpha"], occ, precision="fp32")
        q = pt[k].detach().clone().requires_grad_(True)
        Es = ag.exx_energy(q, plan)
        Es.backward()
        plan.close()
        assert abs(float(E[k]) - float(Es)) <= 1e-14 * abs(float(Es))
        assert torch.equal(pt[k].grad, q.grad * w[k].float())
    # energy only (no gradient requested)
    with torch.no_grad():
        E2 = ag.exx_batch_energy(b, [p.detach() for p in pt])
    assert torch.allclose(E2, E.detach(), rtol=1e-14, atol=0)
    b.close()


def test_batch_rejects_bad_descriptors(env):
    torch, dev, exx = env
    with pytest.raises(exx.ExxError):
        exx.ExxBatch([{"n": 11, "h": 0.4, "alpha": 0.25, "occupations": [2.0]}])
    with pytest.raises(exx.ExxError):
        exx.ExxBatch([{"n": 8, "h": -0.4, "alpha": 0.25, "occupations": [2.0]}])
    b = exx.ExxBatch([{"n": 8, "h": 0.4, "alpha": 0.25, "occupations": [2.0, 2.0]}])
    with pytest.raises(exx.ExxError):  # no buffers bound yet
        b.apply()
    with pytest.raises(exx.ExxError):
        b.set_buffers([torch.zeros((3, 8, 8, 8), device=dev)])
    b.close()


def test_batched_workload_16_uneven_molecules(env):
    # 16 molecules, N_m uniform in [8, 96], grids from {48..128}^3, h = 0.4,
    # one graph launch; every molecule equals its own plan, and a seeded sample
    # of pair energies per molecule equals the oracle's
    torch, dev, exx = env
    recipes = synth.batched_workload()
    mols, pt, occs = [], [], []
    for r in recipes:
        occ = np.full(r.norb, r.occupation)
        mols.append({"n": r.n, "h": r.h, "alpha": r.alpha, "occupations": occ})
        pt.append(torch.from_numpy(synth.make_orbitals(r, dtype=np.float32)).to(dev))
        occs.append(occ)
    b = exx.ExxBatch(mols)
    vx = [torch.empty_like(p) for p in pt]
    b.set_buffers(pt, vx)
    b.graph(True)
    s = torch.cuda.Stream()
    E = torch.zeros(len(mols), dtype=torch.float64, device=dev)
    with torch.cuda.stream(s):
        b.apply(E, stream=s)
    s.synchronize()
    rng = np.random.default_rng(4)
    for k, (r, m) in enumerate(zip(recipes, mols)):
        plan = exx.ExxPlan(r.n, r.h, r.alpha, occs[k], precision="fp32")
        Es, vs = plan.apply(pt[k])
        assert abs(float(E[k]) - Es) <= 1e-14 * abs(Es)
        assert torch.equal(vx[k], vs)
        Eij = plan.pair_energies()
        plan.close()
        Gh = o.kernel_spectrum(o.kernel_real_space(r.n, r.h))
        pairs = o.pair_list(r.norb)
        psi = pt[k].double().cpu().numpy()
        for g in rng.choice(len(pairs), size=2, replace=False):
            i, j = pairs[g]
            _, eo = o.exx_pair(psi[i], psi[j], Gh, r.h)
            assert abs(Eij[g] - eo) <= 1e-6 * max(1.0, abs(eo)), (k, i, j, Eij[g], eo)
    b.close()


def test_tuned_tile_gives_same_results(env, tmp_path, monkeypatch):
    # the tuner times real applies; any tile edge gives the same result up to
    # the FP64 accumulation order
    torch, dev, exx = env
    from paper_1712_07973_gb300 import tune
    monkeypatch.setenv("EXX_TUNE_CACHE", str(tmp_path / "tiles.json"))
    n, N = 16, 10
    best, timings = tune.tune(n, N, "fp32", reps=2)
    assert best in timings and len(timings) == 4
    assert tune.best_tile(n, N, "fp32") == best
    psi = torch.from_numpy(_mol(n, N, 77, 0.4)).to(dev, torch.float32)
    occ = np.full(N, 2.0)
    p0 = exx.ExxPlan(n, 0.4, 0.25, occ, precision="fp32", vx_fp64=True)
    pa = exx.ExxPlan(n, 0.4, 0.25, occ, precision="fp32", vx_fp64=True, tile="auto")
    assert pa.info()["tile"] == best
    E0, v0 = p0.apply(psi)
    Ea, va = pa.apply(psi)
    assert abs(Ea - E0) <= 1e-13 * abs(E0)
    assert torch.allclose(va, v0, rtol=0, atol=1e-12 * float(v0.abs().max()))
    p0.close()
    pa.close()


def test_batch_two_lanes_equal_one_lane(env, monkeypatch):
    # consecutive waves on two streams (the default) against one stream:
    # identical results (the accumulation runs in wave order either way),
    # eagerly and through the captured graph
    torch, dev, exx = env
    psis, occs, mols = _small(env)
    pt = [torch.from_numpy(p).to(dev, torch.float32) for p in psis]
    out = []
    for lanes in ("1", "2"):
        monkeypatch.setenv("EXX_LANES", lanes)
        b = exx.ExxBatch(mols)
        vx = [torch.empty_like(p) for p in pt]
        b.set_buffers(pt, vx)
        E = b.apply().cpu()
        b.graph(True)  # capture needs a created stream
        s = torch.cuda.Stream()
        Eg = torch.zeros(len(mols), dtype=torch.float64, device=dev)
        with torch.cuda.stream(s):
            b.apply(Eg, stream=s)
        s.synchronize()
        assert torch.equal(E, Eg.cpu())
        out.append((E, [v.cpu() for v in vx]))
        b.close()
    (E1, v1), (E2, v2) = out
    assert torch.equal(E1, E2)
    for a, c in zip(v1, v2):
        assert torch.equal(a, c)


MANY = [  # (n, N, h, alpha): several waves per group (slot reuse, tile order)
    (12, 20, 0.45, 0.25), (12, 13, 0.45, 0.25), (16, 17, 0.4, 0.25), (8, 5, 0.5, 0.3),
    (10, 9, 0.5, 0.2),
]


@pytest.mark.parametrize("lanes", ["1", "2"])
def test_persistent_queue_equals_launch_per_pass(env, monkeypatch, lanes):
    # one persistent launch per (n, h) group over a device work queue against
    # five launches per wave: the same per-CTA code and tile order, compiled
    # into another kernel (the compiler may contract other multiply-adds, so
    # equal to FP32 rounding: Vx psi to 1e-6 of its largest entry, E_ij to
    # 1e-7 relative); each schedule bit-identical eagerly and through the
    # captured graph, and both against the oracle
    torch, dev, exx = env
    monkeypatch.setenv("EXX_LANES", lanes)
    psis, occs, mols = [], [], []
    for k, (n, N, h, a) in enumerate(MANY):
        psis.append(_mol(n, N, 400 + k, h))
        occs.append(np.linspace(0.5, 2.0, N))
        mols.append({"n": n, "h": h, "alpha": a, "occupations": occs[-1]})
    pt = [torch.from_numpy(p).to(dev, torch.float32) for p in psis]
    res = []
    for persistent in (False, True):
        b = exx.ExxBatch(mols)
        b.persistent(persistent)
        vx = [torch.empty_like(p) for p in pt]
        b.set_buffers(pt, vx)
        Ea = b.apply().cpu()
        va = [v.clone() for v in vx]
        Eij = [b.pair_energies(k) for k in range(len(mols))]
        Eg = b.gradient().cpu()
        vg = [v.clone() for v in vx]
        Ee = b.energy().cpu()
        b.graph(True)
        s = torch.cuda.Stream()
        E2 = torch.zeros(len(mols), dtype=torch.float64, device=dev)
        with torch.cuda.stream(s):
            for _ in range(2):
                b.apply(E2, stream=s)
        s.synchronize()
        assert torch.equal(E2.cpu(), Ea)
        assert all(torch.equal(a, c) for a, c in zip(vx, va))
        info = b.info()
        b.close()
        res.append((Ea, va, Eij, Eg, vg, Ee, info))
    (Ea0, va0, Eij0, Eg0, vg0, Ee0, i0), (Ea1, va1, Eij1, Eg1, vg1, Ee1, i1) = res
    assert i1["launches_apply"] == len({(m["n"], m["h"]) for m in mols}) + 2
    assert torch.allclose(Ea1, Ea0, rtol=1e-7, atol=0)
    assert torch.allclose(Eg1, Eg0, rtol=1e-7, atol=0)
    assert torch.allclose(Ee1, Ee0, rtol=1e-7, atol=0)
    for k in range(len(mols)):
        for x1, x0 in ((va1[k], va0[k]), (vg1[k], vg0[k])):
            assert torch.allclose(x1, x0, rtol=0, atol=1e-6 * float(x0.abs().max()))
        assert np.allclose(Eij1[k], Eij0[k], rtol=1e-7, atol=0)
    # and the oracle
    for k, (m, p, occ) in enumerate(zip(mols, psis, occs)):
        Gh = o.kernel_spectrum(o.kernel_real_space(m["n"], m["h"]))
        Eo, vxo, _ = o.exx(p, occ, m["alpha"], m["h"], Gh)
        assert abs(float(Ea1[k]) - Eo) <= 1e-6
        assert np.max(np.abs(va1[k].double().cpu().numpy() - vxo)) <= 2e-6 * np.max(np.abs(vxo))


def test_persistent_queue_wait_times_out_and_context_survives(env, monkeypatch):
    # a queue segment made to wait for one that never completes (host-side
    # test hook): the bounded device-side wait runs out, the launch skips the
    # rest and ends, the next synchronising call reports EXX_ERR_TIMEOUT, and
    # the context still computes correct energies
    torch, dev, exx = env
    psis, occs, mols = _small(env)
    pt = [torch.from_numpy(p).to(dev, torch.float32) for p in psis]
    monkeypatch.setenv("EXX_TEST_STALL_QUEUE", "1")
    b = exx.ExxBatch(mols)
    b.persistent(True)
    vx = [torch.empty_like(p) for p in pt]
    b.set_buffers(pt, vx)
    b.apply()
    with pytest.raises(exx.ExxError) as ei:
        b.pair_energies(0)
    assert ei.value.status == 4
    b.close()
    monkeypatch.delenv("EXX_TEST_STALL_QUEUE")
    b = exx.ExxBatch(mols)
    b.persistent(True)
    b.set_buffers(pt, vx)
    E = b.apply().cpu()
    for k, (m, p, occ) in enumerate(zip(mols, psis, occs)):
        Gh = o.kernel_spectrum(o.kernel_real_space(m["n"], m["h"]))
        Eo, vxo, _ = o.exx(p, occ, m["alpha"], m["h"], Gh)
        assert abs(float(E[k]) - Eo) <= 1e-6
        assert np.max(np.abs(vx[k].double().cpu().numpy() - vxo)) <= 2e-6 * np.max(np.abs(vxo))
    b.close()


def test_persistent_mixed_groups_and_single_pair(env):
    # persistent schedule with a group that keeps the launch-per-pass schedule
    # (160^3: clustered slab kernels) next to persistent groups, and a molecule
    # of one orbital (one pair, one wave): equal to the launch-per-pass
    # schedule to FP32 rounding, and to the oracle
    torch, dev, exx = env
    spec = [(160, 2, 0.42, 0.25), (12, 1, 0.45, 0.25), (12, 6, 0.45, 0.25), (16, 9, 0.4, 0.3)]
    psis, occs, mols = [], [], []
    for k, (n, N, h, a) in enumerate(spec):
        r = synth.OrbitalRecipe(n=n, h=h, norb=N, nsites=3, seed=700 + k, gauss_per_orb=6,
                                sigma=(0.7, 1.8), p_type=True)
        psis.append(synth.make_orbitals(r))
        occs.append(np.linspace(1.0, 2.0, N))
        mols.append({"n": n, "h": h, "alpha": a, "occupations": occs[-1]})
    pt = [torch.from_numpy(p).to(dev, torch.float32) for p in psis]
    res = []
    for persistent in (False, True):
        b = exx.ExxBatch(mols)
        b.persistent(persistent)
        vx = [torch.empty_like(p) for p in pt]
        b.set_buffers(pt, vx)
        E = b.gradient().cpu()
        res.append((E, [v.clone() for v in vx], b.info()))
        b.close()
    (E0, v0, i0), (E1, v1, i1) = res
    # groups (160, 0.42): one wave of five launches; (12, 0.45) and (16, 0.4): one
    # persistent launch each; E_x totals and output conversion: two
    assert i1["launches_apply"] == 5 + 2 + 2
    assert torch.allclose(E1, E0, rtol=1e-7, atol=0)
    for k, (m, p, occ) in enumerate(zip(mols, psis, occs)):
        assert torch.allclose(v1[k], v0[k], rtol=0, atol=1e-6 * float(v0[k].abs().max()))
        Gh = o.kernel_spectrum(o.kernel_real_space(m["n"], m["h"]))
        Eo, go = o.exx_energy_gradient(p, occ, m["alpha"], m["h"], Gh)
        assert abs(float(E1[k]) - Eo) <= 1e-6
        assert np.max(np.abs(v1[k].double().cpu().numpy() - go)) <= 2e-6 * np.max(np.abs(go))
