"""Host-side logic of bench.py (no GPU): the pair-tile table, the algorithmic
byte counts behind the roofline, and the committed ncu traffic lookup."""

import json
import os

import pytest

import bench


@pytest.mark.parametrize("N,T", [(1, 8), (5, 8), (8, 8), (10, 8), (64, 8), (19, 4), (128, 8)])
def test_tile_list_covers_every_pair_once(N, T):
    tiles = bench.tile_list(N, T)
    assert sum(t[0] for t in tiles) == N * (N + 1) // 2
    nb = (N + T - 1) // T
    assert len(tiles) == nb * (nb + 1) // 2
    assert sum(1 for t in tiles if t[3]) == nb


def test_algorithmic_bytes_per_kernel():
    # one diagonal tile of 8 orbitals, n = 96: 36 pairs
    n, N, T, rs = 96, 8, 8, 4
    S = (n + 1) * n * 2 * n * 8                      # spectrum per pair (complex FP32)
    a = bench.algorithmic_bytes(n, N, T, rs)
    n3 = n ** 3
    assert a["fwd_xy"] == 8 * n3 * 4 + 36 * S
    assert a["zconv"] == 2 * 36 * S + (n + 1) * (2 * n) ** 2 * 4
    assert a["inv_yx"] == 36 * S + 36 * n3 * 4
    assert a["accum"] == 36 * n3 * 4 + 8 * n3 * 4 + 2 * 8 * n3 * 8


def test_half_lines_and_mixed_boundary_bytes():
    n = 96
    assert bench.half_lines(n, "free") == (96, 96)
    assert bench.half_lines(n, "periodic") == (48, 48)
    assert bench.half_lines(n, "slab") == (48, 96)
    assert bench.half_lines(n, "wire") == (96, 48)
    # the spectrum follows the x, y lines; the kernel table also the z line
    per = bench.algorithmic_bytes(n, 8, 8, bc="periodic")
    slab = bench.algorithmic_bytes(n, 8, 8, bc="slab")
    assert per["fwd_xy"] == slab["fwd_xy"]
    assert slab["zconv"] - per["zconv"] == 49 * (192 - 96) * 96 * 4
    free = bench.algorithmic_bytes(n, 8, 8)
    wire = bench.algorithmic_bytes(n, 8, 8, bc="wire")
    assert free["inv_yx"] == wire["inv_yx"]
    assert free["zconv"] - wire["zconv"] == 97 * (192 - 96) * 192 * 4


def test_committed_traffic_only_for_the_captured_sources():
    # profiles/traffic.json carries the hash of the kernel sources' code it was
    # captured from; the bench reports the counters only while that hash
    # matches, and null otherwise
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    with open(path) as fh:
        d = json.load(fh)
    for wl in d:
        for kern, entry in d[wl].items():
            assert 0.85 <= entry["traffic_over_algorithmic"] <= 1.05, (wl, kern)
            if entry["source_hash"] == bench.kernel_source_hash():
                assert bench.committed_traffic(kern, wl) == entry["dram_bytes_per_launch"]
            else:
                assert bench.committed_traffic(kern, wl) is None


def test_pair_sample_decode_and_cpu_model():
    # sampled pair ids decode to (i, j), i <= j, in the row-major order of the
    # pair energies
    N = 37
    order = [(i, j) for i in range(N) for j in range(i, N)]
    for i, j, g in bench.sample_pairs(N, 50, seed=3):
        assert order[g] == (i, j)
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()


def _run_bench(args, env_extra=None):
    import subprocess
    import sys
    env = dict(os.environ, **(env_extra or {}))
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py")] + args,
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


def test_reference_arm_prints_the_contract_line():
    # the reference arm (the FP64 oracle on the host cores) on the 64-orbital
    # 96^3 workload: one JSON line with the base contract's keys, the oracle
    # described as the CPU baseline, and an e2e record without copies
    out = _run_bench(["--impl", "reference", "--workload", "c2_fp32_n96_N64",
                      "--steps", "1", "--warmup", "0"])
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["config"]["workload"] == "c2_fp32_n96_N64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # one step is a measured sample of pair solves; the full-workload time is
    # a separate, labelled extrapolation
    assert "measured" in d["ms_per_step_is"]
    assert d["ms_per_full_workload_extrapolated"] > d["ms_per_step"]


def test_reference_arm_other_ranks_exit_quietly():
    # under torchrun only rank 0 runs the oracle and prints
    out = _run_bench(["--impl", "reference", "--workload", "c2_fp32_n96_N64", "--steps", "1",
                      "--warmup", "0"], {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out.strip() == ""
