"""Sharding over ranks on the CPU: the tile assignment (host logic of the C
ABI) and a world-size-2 gloo run in which each rank computes its own tiles'
pairs with the FP64 oracle and the partial E_x and Vx psi are all-reduced."""

import os
import socket

import numpy as np
import pytest

from oracle import exx_oracle as o


@pytest.fixture(scope="module")
def exx():
    from paper_1712_07973_gb300 import build, exx as ex
    build.build()
    ex.load_library()
    return ex


def _tile_pairs(d):
    i0, ti, j0, tj, diag = (int(x) for x in d)
    return [(i0 + a, j0 + b) for a in range(ti) for b in range(a if diag else 0, tj)]


@pytest.mark.parametrize("N,T,R", [(1, 8, 2), (5, 2, 3), (17, 4, 2), (64, 8, 8), (30, 8, 7)])
def test_shard_assignment_covers_every_pair_once_and_balances(exx, N, T, R):
    desc, own = exx.shard_tiles(N, T, R)
    assert len(desc) == len(own)
    seen = [p for d in desc for p in _tile_pairs(d)]
    assert sorted(seen) == o.pair_list(N)
    loads = np.zeros(R)
    for d, r in zip(desc, own):
        assert 0 <= r < R
        loads[r] += len(_tile_pairs(d))
    biggest = max(len(_tile_pairs(d)) for d in desc)
    assert loads.max() - loads.min() <= biggest
    # deterministic
    d2, o2 = exx.shard_tiles(N, T, R)
    assert np.array_equal(d2, desc) and np.array_equal(o2, own)


def _rank_main(rank, world, port, path):
    import torch
    import torch.distributed as dist

    from paper_1712_07973_gb300 import exx, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r = synth.OrbitalRecipe(n=8, h=0.5, norb=7, nsites=3, seed=41, gauss_per_orb=3,
                            sigma=(0.6, 1.0), p_type=True)
    psi = synth.make_orbitals(r)
    occ = np.linspace(0.5, 2.0, r.norb)
    alpha = 0.25
    Gh = o.kernel_spectrum(o.kernel_real_space(r.n, r.h))
    desc, own = exx.shard_tiles(r.norb, 3, world)
    E = 0.0
    vx = np.zeros_like(psi)
    for d, owner in zip(desc, own):
        if owner != rank:
            continue
        for i, j in _tile_pairs(d):
            V, e = o.exx_pair(psi[i], psi[j], Gh, r.h)
            E += -0.5 * alpha * occ[i] * occ[j] * e * (1.0 if i == j else 2.0)
            vx[i] += -alpha * occ[j] * V * psi[j]
            if i != j:
                vx[j] += -alpha * occ[i] * V * psi[i]
    tE = torch.tensor([E], dtype=torch.float64)
    tV = torch.from_numpy(vx)
    dist.all_reduce(tE)
    dist.all_reduce(tV)
    if rank == 0:
        Ef, vxf, _ = o.exx(psi, occ, alpha, r.h, Gh)
        err_e = abs(float(tE.item()) - Ef) / abs(Ef)
        err_v = float(np.max(np.abs(tV.numpy() - vxf)) / np.max(np.abs(vxf)))
        with open(path, "w") as fh:
            fh.write(f"{err_e} {err_v}")
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_sum_to_full_oracle(exx, tmp_path):
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    path = str(tmp_path / "res.txt")
    mp.start_processes(_rank_main, args=(2, port, path), nprocs=2, join=True, start_method="spawn")
    err_e, err_v = map(float, open(path).read().split())
    assert err_e < 1e-13 and err_v < 1e-13


class _OracleShardPlan:
    """CPU stand-in for ExxPlan with the interface dist.sharded_apply uses:
    set_shard restricts it to the rank's pair tiles (the library's own
    assignment, exx_shard_tiles), apply_async / gradient_async write the
    partial E_x and Vx psi (or gradient) of those tiles, computed by the
    oracle."""

    def __init__(self, exx, occ, alpha, h, T, Gh):
        import torch
        self.exx, self.occ, self.alpha, self.h, self.T, self.Gh = exx, occ, alpha, h, T, Gh
        self.vx_dtype = torch.float64
        self.rank, self.world = 0, 1

    def set_shard(self, rank, world):
        self.rank, self.world = rank, world

    def _partial(self, psi, out, E, grad):
        import torch
        p = psi.numpy()
        desc, own = self.exx.shard_tiles(p.shape[0], self.T, self.world)
        e, vx = 0.0, np.zeros_like(p)
        for d, owner in zip(desc, own):
            if owner != self.rank:
                continue
            for i, j in _tile_pairs(d):
                V, eij = o.exx_pair(p[i], p[j], self.Gh, self.h)
                e += -0.5 * self.alpha * self.occ[i] * self.occ[j] * eij * (1.0 if i == j else 2.0)
                vx[i] += -self.alpha * self.occ[j] * V * p[j]
                if i != j:
                    vx[j] += -self.alpha * self.occ[i] * V * p[i]
        if grad:
            vx *= (2.0 * self.h ** 3 * self.occ)[:, None, None, None]
        out.copy_(torch.from_numpy(vx))
        E.fill_(e)

    def apply_async(self, psi, out, E):
        self._partial(psi, out, E, False)

    def gradient_async(self, psi, out, E):
        self._partial(psi, out, E, True)


def _rank_main_sharded_apply(rank, world, port, path):
    import torch
    import torch.distributed as dist

    from paper_1712_07973_gb300 import dist as xdist, exx, synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r = synth.OrbitalRecipe(n=8, h=0.5, norb=6, nsites=3, seed=43, gauss_per_orb=3,
                            sigma=(0.6, 1.0), p_type=True)
    psi = synth.make_orbitals(r)
    occ = np.linspace(0.5, 2.0, r.norb)
    alpha = 0.25
    Gh = o.kernel_spectrum(o.kernel_real_space(r.n, r.h))
    plan = _OracleShardPlan(exx, occ, alpha, r.h, 2, Gh)
    tpsi = torch.from_numpy(psi)
    E_a, vx_a = xdist.sharded_apply(plan, tpsi)
    E_g, g = xdist.sharded_apply(plan, tpsi, gradient=True, sync=False)
    if rank == 0:
        Ef, vxf, _ = o.exx(psi, occ, alpha, r.h, Gh)
        gf = vxf * (2.0 * r.h ** 3 * occ)[:, None, None, None]
        errs = [abs(E_a - Ef) / abs(Ef),
                float(np.max(np.abs(vx_a.numpy() - vxf)) / np.max(np.abs(vxf))),
                abs(float(E_g.item()) - Ef) / abs(Ef),
                float(np.max(np.abs(g.numpy() - gf)) / np.max(np.abs(gf)))]
        with open(path, "w") as fh:
            fh.write(" ".join(str(x) for x in errs))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_sharded_apply_equals_full_oracle(exx, tmp_path):
    # dist.sharded_apply itself at world size 2 (gloo, CPU tensors): each rank
    # sets its shard, computes its tiles' partial results and the function's
    # two all-reduces give the full E_x and action (and gradient) on every rank
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    path = str(tmp_path / "res.txt")
    mp.start_processes(_rank_main_sharded_apply, args=(2, port, path), nprocs=2, join=True,
                       start_method="spawn")
    errs = [float(x) for x in open(path).read().split()]
    assert len(errs) == 4 and max(errs) < 1e-13, errs
