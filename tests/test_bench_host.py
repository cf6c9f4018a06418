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
