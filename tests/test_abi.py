"""CPU-side checks of the C ABI: the library builds, loads and exports every
declared symbol; argument validation and the host kernel builder need no GPU."""

import ctypes
import os
import re

import numpy as np
import pytest

from oracle import exx_oracle as o

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    from paper_1712_07973_gb300 import build, exx
    build.build()
    return exx.load_library()


def _declared_symbols():
    with open(os.path.join(ROOT, "include", "exx.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"\b(exx_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    from paper_1712_07973_gb300 import exx
    names = _declared_symbols()
    assert names, "no declarations found"
    for nm in names:
        assert hasattr(lib, nm), nm
        assert nm in exx.EXPORTS, f"binding lacks {nm}"
    assert set(exx.EXPORTS) == set(names)
    assert lib.exx_version().startswith(b"exx-gb300")


def test_status_strings(lib):
    assert lib.exx_status_string(0) == b"EXX_OK"
    assert lib.exx_status_string(5) == b"EXX_ERR_NOT_SUPPORTED"
    assert lib.exx_status_string(99) == b"EXX_UNKNOWN_STATUS"


def _create(lib, grid=(8, 8, 8), h=(0.4, 0.4, 0.4), occ=(2.0, 2.0), prec=1, kernel=0, flags=0,
            out=True):
    handle = ctypes.c_void_p(123)
    g = (ctypes.c_int * 3)(*grid)
    hh = (ctypes.c_double * 3)(*h)
    oc = (ctypes.c_double * max(1, len(occ)))(*occ)
    st = lib.exx_plan_create(ctypes.byref(handle) if out else None, g, hh, 0.25, oc, len(occ),
                             prec, kernel, flags, None)
    return st, handle


def test_argument_validation_before_any_device_work(lib):
    # every one of these is rejected on the host, before CUDA is touched
    assert _create(lib, out=False)[0] == 1
    st, hdl = _create(lib, occ=())
    assert st == 1 and not hdl.value  # out handle cleared on failure
    assert _create(lib, grid=(1, 1, 1))[0] == 1
    assert _create(lib, h=(0.0, 0.0, 0.0))[0] == 1
    assert _create(lib, h=(-0.4, -0.4, -0.4))[0] == 1
    assert _create(lib, prec=7)[0] == 1
    assert _create(lib, kernel=9)[0] == 1
    assert _create(lib, flags=0x80)[0] == 1
    assert _create(lib, occ=(2.0, float("nan")))[0] == 1
    assert _create(lib, grid=(8, 8, 10))[0] == 5     # not cubic
    assert _create(lib, h=(0.4, 0.4, 0.5))[0] == 5   # not isotropic
    assert _create(lib, grid=(11, 11, 11))[0] == 5   # 2n = 22 has the prime 11
    assert _create(lib, grid=(1000, 1000, 1000))[0] == 5  # beyond the compiled sizes
    assert lib.exx_plan_destroy(None) == 0
    assert lib.exx_apply(None, None, None, None, None) == 1
    assert lib.exx_energy(None, None, None, None) == 1


@pytest.mark.parametrize("n,h", [(4, 0.5), (8, 0.4), (13, 0.33), (32, 0.4), (48, 0.2)])
def test_host_kernel_spectrum_matches_oracle(lib, n, h):
    # the library's kernel builder (t-separable spectral route, exp-sinh nodes)
    # against the oracle's (real-space Faddeeva route + FFT): independent code
    from paper_1712_07973_gb300 import exx
    got = exx.kernel_spectrum(n, h, exx.KERNEL_SINC)
    ref = o.kernel_spectrum(o.kernel_real_space(n, h))[: n + 1, : n + 1, : n + 1]
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))


@pytest.mark.parametrize("n,h", [(6, 0.5), (20, 0.3)])
def test_host_hockney_spectrum_matches_oracle(lib, n, h):
    from paper_1712_07973_gb300 import exx
    got = exx.kernel_spectrum(n, h, exx.KERNEL_HOCKNEY)
    ref = o.kernel_spectrum(o.kernel_real_space(n, h, o.KERNEL_HOCKNEY))[: n + 1, : n + 1, : n + 1]
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_kernel_spectrum_rejects_bad_arguments(lib):
    out = np.zeros(8)
    p = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.exx_kernel_spectrum(0, 0.4, 0, 0.0, p) == 1
    assert lib.exx_kernel_spectrum(1, -1.0, 0, 0.0, p) == 1
    assert lib.exx_kernel_spectrum(1, 0.4, 6, 0.0, p) == 1
    assert lib.exx_kernel_spectrum(1, 0.4, 0, 0.0, None) == 1
    assert lib.exx_kernel_spectrum(1, 0.4, 2, 0.0, p) == 1   # erfc needs omega > 0
    assert lib.exx_kernel_spectrum(1, 0.4, 2, -0.1, p) == 1


@pytest.mark.parametrize("n,h,w", [(8, 0.4, 0.11), (16, 0.3, 0.6), (32, 0.4, 2.0)])
def test_host_erfc_spectrum_matches_oracle(lib, n, h, w):
    from paper_1712_07973_gb300 import exx
    got = exx.kernel_spectrum(n, h, exx.KERNEL_ERFC, omega=w)
    ref = o.kernel_spectrum(o.kernel_real_space(n, h, o.KERNEL_ERFC, omega=w))[: n + 1, : n + 1, : n + 1]
    # the oracle forms the short-range kernel as full minus long-range part, so
    # its rounding is relative to the full kernel's scale
    full = o.kernel_spectrum(o.kernel_real_space(n, h))
    assert np.max(np.abs(got - ref)) <= 5e-14 * np.max(np.abs(full))


def test_erfc_plan_needs_omega(lib):
    # the plain constructor refuses the screened kernel (no omega to pass)
    assert _create(lib, kernel=2)[0] == 1


@pytest.mark.parametrize("n,h", [(8, 0.5), (12, 0.4), (32, 0.3)])
def test_host_periodic_spectrum_matches_oracle(lib, n, h):
    from paper_1712_07973_gb300 import exx
    got = exx.kernel_spectrum(n, h, exx.KERNEL_PERIODIC)  # [kz][ky][kx], k <= n/2
    ref = o.kernel_spectrum_periodic(n, h)                # rfftn layout (n, n, n/2+1)
    m = n // 2 + 1
    assert np.allclose(got, ref[:m, :m, :m], rtol=1e-14, atol=0)


def test_periodic_needs_even_supported_grid(lib):
    assert _create(lib, grid=(9, 9, 9), kernel=3)[0] == 5     # odd
    assert _create(lib, grid=(10, 10, 10), kernel=3)[0] == 5   # 10 not compiled
    out = np.zeros(8)
    assert lib.exx_kernel_spectrum(3, 0.4, 3, 0.0, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == 1


@pytest.mark.parametrize("n,h", [(8, 0.4), (16, 0.3), (48, 0.2)])
def test_host_slab_and_wire_spectra_match_oracle(lib, n, h):
    # library: t-separable spectral factors with exp-sinh nodes and the
    # regularised (0,0,0) entries; oracle: Faddeeva factors, trapezoid in ln t,
    # and the sine-integral closed form of the slab's k = 0 kernel
    from paper_1712_07973_gb300 import exx
    m, m2 = n + 1, n // 2 + 1
    got = exx.kernel_spectrum(n, h, exx.KERNEL_SLAB)         # [kz][ky][kx], kz <= n
    ref = o.kernel_spectrum_slab(n, h)[:m, :m2, :m2]
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    got = exx.kernel_spectrum(n, h, exx.KERNEL_WIRE)         # [kz][ky][kx], kz <= n/2
    ref = o.kernel_spectrum_wire(n, h)[:m2, :m, :m]
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_slab_and_wire_need_even_supported_grid(lib):
    for kernel in (4, 5):
        assert _create(lib, grid=(9, 9, 9), kernel=kernel)[0] == 5
        assert _create(lib, grid=(12, 12, 12), kernel=kernel)[0] == 5   # not compiled
        out = np.zeros(8)
        assert lib.exx_kernel_spectrum(3, 0.4, kernel, 0.0,
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == 1
    assert _create(lib, kernel=6)[0] == 1


def test_no_cpu_fallback_without_a_gpu(lib):
    # the product path fails loudly where CUDA is missing: there is no host
    # implementation behind the binding (this container has no GPU)
    import torch
    from paper_1712_07973_gb300 import exx
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(exx.ExxError, match="no CUDA device"):
        exx.ExxPlan(8, 0.4, 0.25, [2.0, 2.0], precision="fp32")
    with pytest.raises(exx.ExxError, match="no CUDA device"):
        exx.ExxBatch([{"n": 8, "h": 0.4, "alpha": 0.25, "occupations": [2.0]}])
