"""Pair-tile autotuner.

The tile edge T (orbitals per tile side, 1..8) trades the amortisation of the
orbital reads and FP64 accumulator updates (which fall as 1/T per pair) against
the size of each launch and of the workspace (T^2 pairs per tile).  ``tune``
times exx_apply for a few candidates on seeded orbitals of the requested size
and keeps the fastest in a JSON cache keyed by (n, N, precision, SM count);
``best_tile`` reads it.  The cache path is $EXX_TUNE_CACHE, else
~/.cache/exx_gb300/tiles.json.
"""

import json
import os
import statistics

__all__ = ["CANDIDATES", "cache_path", "cache_key", "load_cache", "store", "best_tile", "tune"]

CANDIDATES = (2, 4, 6, 8)


def cache_path():
    p = os.environ.get("EXX_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "exx_gb300", "tiles.json")


def cache_key(n, N, precision, sm_count):
    return f"n{int(n)}:N{int(N)}:{precision}:sm{int(sm_count)}"


def load_cache(path=None):
    path = path or cache_path()
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store(key, tile, timings, path=None):
    path = path or cache_path()
    d = load_cache(path)
    d[key] = {"tile": int(tile), "ms": {str(k): float(v) for k, v in timings.items()}}
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _sm_count():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def best_tile(n, N, precision="fp32", tune_if_missing=False, path=None):
    """Cached tile edge for (n, N, precision) on this GPU, or 0 (library default)."""
    key = cache_key(n, N, precision, _sm_count())
    e = load_cache(path).get(key)
    if e:
        return int(e["tile"])
    if tune_if_missing:
        return tune(n, N, precision, path=path)[0]
    return 0


def select(timings):
    """Fastest candidate; ties go to the larger tile (less accumulator traffic)."""
    return min(timings, key=lambda t: (timings[t], -t))


def tune(n, N, precision="fp32", h=0.4, reps=3, candidates=CANDIDATES, path=None, measure=None,
         sm_count=None):
    """Time exx_apply for each candidate tile edge; store and return (best, timings).

    ``measure(tile) -> ms`` replaces the GPU timing and ``sm_count`` the device
    query (both used to test the host logic without a GPU).
    """
    cands = sorted({min(int(t), N) for t in candidates if t >= 1})
    if measure is None:
        measure = _gpu_measure(n, N, precision, h, reps)
    timings = {t: float(measure(t)) for t in cands}
    best = select(timings)
    sm = _sm_count() if sm_count is None else sm_count
    store(cache_key(n, N, precision, sm), best, timings, path)
    return best, timings


def _gpu_measure(n, N, precision, h, reps):
    import numpy as np
    import torch

    from . import exx, synth
    r = synth.OrbitalRecipe(n=n, h=h, norb=N, nsites=max(2, N // 2), seed=1234, gauss_per_orb=4,
                            sigma=(0.7, 1.8), p_type=True)
    dt = torch.float64 if precision == "fp64" else torch.float32
    psi = torch.from_numpy(synth.make_orbitals(r)).to("cuda", dt)
    occ = np.full(N, 2.0)

    def measure(tile):
        plan = exx.ExxPlan(n, h, 0.25, occ, precision=precision, tile=tile)
        out = torch.empty(psi.shape, dtype=plan.vx_dtype, device=psi.device)
        plan.apply_async(psi, out)
        torch.cuda.synchronize()
        times = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            plan.apply_async(psi, out)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        plan.close()
        return statistics.median(times)

    return measure
