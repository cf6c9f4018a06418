"""The register DFT templates of the transforms (csrc/exx_fft.cuh) on the CPU.

Every sub-DFT length the line splits use (2..20 with prime factors up to 7,
and 21, 24, 28, 30, 32) is run in FP64 by a host program (tests/c/dft_check.cu,
compiled by nvcc; no kernel is launched) against the DFT written out as a
sum, in both directions, in full and in the pruned forms (half the inputs
zero; half the outputs kept).  Lengths with coprime factors take the
prime-factor (Good-Thomas) form, whose index maps a wrong modular inverse or
a transposed factor would break; prime powers take the Cooley-Tukey form.
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
    exe = str(tmp_path_factory.mktemp("dft") / "dft_check")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "paper_1712_07973_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "c", "dft_check.cu"), "-o", exe],
                   check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return [json.loads(ln) for ln in out.splitlines()]


def test_every_length_is_the_dft(rows):
    assert len(rows) == 40
    for r in rows:
        assert r["full"] <= 1e-14, r
        if r["P"] % 2 == 0:
            assert 0 <= r["halfin"] <= 1e-14, r
            assert 0 <= r["halfout"] <= 1e-14, r


def test_prime_factor_form_where_the_factors_are_coprime(rows):
    pfa = sorted({r["P"] for r in rows if r["pfa"]})
    assert pfa == [6, 10, 12, 14, 15, 18, 20, 21, 24, 28, 30]
