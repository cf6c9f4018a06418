"""The host model of the FP32 transform gains (csrc/exx_gain.cuh) on the CPU.

The model runs the kernels' own sub-DFT templates with FP64 arithmetic and
FP32-rounded constants.  Pinned here against the exact DFT: with unrounded
constants it is the exact transform (to rounding) and its gains are 1; with
rounded constants it stays within FP32 accuracy of the exact transform and
its gains differ from 1 by the rounding of the constants only.
"""

import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rows(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("gain") / "gain_model")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "paper_1712_07973_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "c", "gain_model.cu"), "-o", exe],
                   check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return [json.loads(ln) for ln in out.splitlines()]


def test_both_splits_of_320_point_lines_are_modelled(rows):
    # y pass 16 x 20, zconv 20 x 16 (split_z)
    assert sorted(r["L1"] for r in rows if r["N"] == 160) == [16, 20]


def test_model_with_exact_constants_is_the_dft(rows):
    for r in rows:
        assert r["err64"] <= 1e-12, r
        assert r["gdev64"] <= 1e-12, r


def test_model_with_fp32_constants(rows):
    for r in rows:
        assert r["err32"] <= 2e-6, r           # FP32 accuracy of the transform itself
        assert 1e-9 <= r["gdev32"] <= 1e-6, r  # gains: rounding of the constants, visible and small
