"""The C ABI used from a plain C program (tests/c/exx_c_example.c), compiled
with gcc against include/exx.h and the in-tree library."""

import os
import subprocess

import numpy as np
import pytest

from oracle import exx_oracle as o
from paper_1712_07973_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    from paper_1712_07973_gb300 import build
    build.build()
    lib = build.lib_path()
    out = str(tmp_path_factory.mktemp("c") / "exx_c_example")
    subprocess.run(["gcc", "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "exx_c_example.c"), lib,
                    "-Wl,-rpath," + os.path.dirname(lib), "-o", out], check=True)
    return out


def test_c_program_kernel_spectrum(exe):
    # host-only entry point, no GPU: against the oracle's independent route
    n, h = 12, 0.4
    res = subprocess.run([exe, "spectrum", str(n), str(h)], capture_output=True, text=True, check=True)
    g0, gn = (float(v) for v in res.stdout.split())
    ref = o.kernel_spectrum(o.kernel_real_space(n, h))
    assert g0 == pytest.approx(ref[0, 0, 0], rel=1e-13)
    assert gn == pytest.approx(ref[n, n, n], rel=1e-12, abs=1e-13 * abs(ref[0, 0, 0]))


@pytest.mark.gpu
def test_c_program_apply_host_matches_oracle(exe, tmp_path):
    n, N, h = 16, 3, 0.45
    r = synth.OrbitalRecipe(n=n, h=h, norb=N, nsites=3, seed=61, gauss_per_orb=3,
                            sigma=(0.12 * n * h, 0.2 * n * h), p_type=True)
    psi = synth.make_orbitals(r)
    pin, pout = tmp_path / "psi.bin", tmp_path / "vx.bin"
    psi.astype(np.float64).tofile(pin)
    res = subprocess.run([exe, "apply", str(n), str(h), str(N), str(pin), str(pout)],
                         capture_output=True, text=True, check=True)
    E = float(res.stdout.strip())
    vx = np.fromfile(pout, dtype=np.float64).reshape(psi.shape)
    Eo, vxo, _ = o.exx(psi, np.full(N, 2.0), 0.25, h, o.kernel_spectrum(o.kernel_real_space(n, h)))
    assert abs(E - Eo) <= 1e-10 * abs(Eo)
    assert np.max(np.abs(vx - vxo)) <= 1e-10 * np.max(np.abs(vxo))
