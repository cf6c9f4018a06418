"""The allocation-free pair energy against the plan-based path.

exx_pair_energy_noalloc serves callers that cannot call cudaMalloc (codes that
give the whole device memory to their own pool allocator, or that keep
allocation latency and its implicit synchronisation out of their iteration
loop): its scratch lives in device arrays inside the library.  Here it is
called through the C ABI twice in a row for several pairs and compared with
the per-pair energies of exx_energy on a plan, within the FP32 tolerance used
by the other tests (1e-6 Ha).  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

from paper_1712_07973_gb300 import synth

pytestmark = pytest.mark.gpu


def _orbitals(n, N, seed, h):
    r = synth.OrbitalRecipe(n=n, h=h, norb=N, nsites=3, seed=seed, gauss_per_orb=3,
                            sigma=(0.12 * n * h, 0.2 * n * h), p_type=True)
    return synth.make_orbitals(r)


@pytest.mark.parametrize("n,h", [(12, 0.45), (40, 0.35), (96, 0.4)])
def test_noalloc_pair_energy_matches_plan(n, h):
    import torch
    from paper_1712_07973_gb300 import build, exx
    build.build()
    lib = exx.load_library()
    dev = torch.device("cuda:0")
    N = 3
    psi = torch.from_numpy(_orbitals(n, N, seed=50 + n, h=h)).to(dev, torch.float32)
    plan = exx.ExxPlan(n, h, 0.25, np.full(N, 2.0), precision="fp32")
    plan.energy(psi)
    ref = plan.pair_energies()  # (0,0),(0,1),(0,2),(1,1),(1,2),(2,2)
    plan.close()
    gid = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):  # two calls in a row: the shared scratch is reused
        for (i, j) in [(0, 1), (2, 2), (1, 2), (0, 0)]:
            st = lib.exx_pair_energy_noalloc(n, h, exx.KERNEL_SINC, ctypes.c_void_p(psi.data_ptr()),
                                             N, i, j, ctypes.c_void_p(E.data_ptr()), stream)
            assert st == 0, exx.STATUS[st]
            torch.cuda.synchronize()
            assert abs(E.item() - ref[gid[(i, j)]]) <= 1e-6, (n, i, j, E.item(), ref[gid[(i, j)]])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1712_07973_gb300 import build, exx
    build.build()
    lib = exx.load_library()
    dev = torch.device("cuda:0")
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    psi = torch.zeros(2 * 8 ** 3, dtype=torch.float32, device=dev)
    p, e = ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(E.data_ptr())
    maxn = 96
    assert lib.exx_pair_energy_noalloc(maxn + 16, 0.4, 0, p, 2, 0, 1, e, None) == 5
    assert lib.exx_pair_energy_noalloc(11, 0.4, 0, p, 2, 0, 1, e, None) == 5
    assert lib.exx_pair_energy_noalloc(8, 0.4, 0, p, 2, 0, 2, e, None) == 1
    assert lib.exx_pair_energy_noalloc(8, -0.4, 0, p, 2, 0, 1, e, None) == 1
    assert lib.exx_pair_energy_noalloc(8, 0.4, 0, None, 2, 0, 1, e, None) == 1
