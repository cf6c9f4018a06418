"""Write the oracle's expected values for the seeded workloads to tests/golden/.

Calls only the FP64 oracle (``oracle/``) and the seeded input generator; no
value here ever comes from the CUDA path.  Usage:

    python tests/golden/make_golden.py c1_fp64_n32_N4 c2_fp32_n96_N64

Each output ``<workload>.json`` holds E_x, all pair energies E_ij (i <= j,
row-major), the norms h^3 <(Vx psi)_i, (Vx psi)_i> and (Vx psi) at 256 seeded
sample points, plus input fingerprints that let a test detect drift of the
generator on another machine.
"""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import exx_oracle as o  # noqa: E402
from paper_1712_07973_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def sample_points(N, n, count=256, seed=1234):
    rng = np.random.default_rng(seed)
    return np.stack([rng.integers(0, N, count), rng.integers(0, n, count),
                     rng.integers(0, n, count), rng.integers(0, n, count)], axis=1)


def fingerprint(psi):
    flat = psi.reshape(psi.shape[0], -1)
    return {"abs_sum": [float(np.abs(r).sum()) for r in flat],
            "first": [float(r[len(r) // 3]) for r in flat]}


def make(name):
    r, psi = synth.workload(name)
    occ = np.full(r.norb, r.occupation)
    t0 = time.time()
    Gh = o.kernel_spectrum(o.kernel_real_space(r.n, r.h))
    Ex, vx, Eij = o.exx(psi, occ, r.alpha, r.h, Gh)
    dt = time.time() - t0
    iu = np.triu_indices(r.norb)
    pts = sample_points(r.norb, r.n)
    out = {
        "workload": name,
        "source": "FP64 oracle (oracle/exx_oracle.py), band-limited kernel, written by "
                  "tests/golden/make_golden.py",
        "n": r.n, "h": r.h, "norb": r.norb, "alpha": r.alpha, "occupation": r.occupation,
        "E_x": Ex,
        "E_ij": Eij[iu].tolist(),
        "vx_norm2": [float(r.h ** 3 * np.sum(v * v)) for v in vx],
        "sample_points": pts.tolist(),
        "vx_samples": [float(vx[a, b, c, d]) for a, b, c, d in pts],
        "psi_fingerprint": fingerprint(psi),
        "oracle_seconds": dt,
        "host_cores": os.cpu_count(),
    }
    with open(os.path.join(HERE, f"{name}.json"), "w") as fh:
        json.dump(out, fh)
    print(f"{name}: E_x = {Ex:.12f}  ({dt:.1f} s)")


if __name__ == "__main__":
    for nm in sys.argv[1:]:
        make(nm)
