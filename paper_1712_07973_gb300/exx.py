"""Thin Python binding over the C ABI in ``include/exx.h`` (argument marshalling only).

Every step of the exact-exchange pipeline runs in the CUDA library
``_lib/libexx_gb300.so``; this module passes device pointers from PyTorch
tensors and the current CUDA stream.  There is no CPU path: if the library or
a CUDA device is missing, the calls raise.
"""

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = ["ExxError", "ExxPlan", "ExxBatch", "load_library", "kernel_spectrum", "shard_tiles", "EXPORTS",
           "FP64", "FP32", "KERNEL_SINC", "KERNEL_HOCKNEY", "KERNEL_ERFC", "KERNEL_PERIODIC",
           "KERNEL_SLAB", "KERNEL_WIRE", "FLAG_VX_FP64"]

FP64, FP32 = 0, 1
KERNEL_SINC, KERNEL_HOCKNEY, KERNEL_ERFC, KERNEL_PERIODIC, KERNEL_SLAB, KERNEL_WIRE = range(6)
FLAG_VX_FP64 = 1
STATUS = ["EXX_OK", "EXX_ERR_INVALID_ARG", "EXX_ERR_CUDA", "EXX_ERR_OOM", "EXX_ERR_TIMEOUT",
          "EXX_ERR_NOT_SUPPORTED"]

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_size_p = ctypes.POINTER(ctypes.c_size_t)

# name -> (restype, argtypes), one entry per declaration in include/exx.h
EXPORTS = {
    "exx_plan_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), _c_int_p, _c_double_p,
                                       ctypes.c_double, _c_double_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_uint, ctypes.c_void_p]),
    "exx_energy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _c_double_p, ctypes.c_void_p]),
    "exx_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _c_double_p,
                                 ctypes.c_void_p]),
    "exx_apply_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "exx_energy_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "exx_gradient": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _c_double_p,
                                    ctypes.c_void_p]),
    "exx_gradient_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "exx_pair_energies": (ctypes.c_int, [ctypes.c_void_p, _c_double_p, ctypes.c_void_p]),
    "exx_plan_info": (ctypes.c_int, [ctypes.c_void_p, _c_int_p, _c_int_p, _c_size_p, _c_int_p,
                                     _c_int_p]),
    "exx_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "exx_apply_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _c_double_p,
                                      ctypes.c_void_p]),
    "exx_gradient_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         _c_double_p, ctypes.c_void_p]),
    "exx_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "exx_plan_set_lanes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "exx_plan_get_lanes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "exx_profile_read": (ctypes.c_int, [ctypes.c_void_p, _c_double_p,
                                        ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]),
    "exx_kernel_spectrum": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                           _c_double_p]),
    "exx_plan_create_desc": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "exx_pair_energy_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                               ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "exx_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_void_p]),
    "exx_batch_set_buffers": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]),
    "exx_batch_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "exx_batch_energy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "exx_batch_gradient": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "exx_batch_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "exx_batch_set_persistent": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "exx_batch_pair_energies": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _c_double_p,
                                               ctypes.c_void_p]),
    "exx_batch_info": (ctypes.c_int, [ctypes.c_void_p, _c_int_p, _c_int_p, _c_size_p, _c_int_p,
                                      ctypes.POINTER(ctypes.c_longlong)]),
    "exx_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "exx_shard_tiles": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_int_p, _c_int_p,
                                       _c_int_p]),
    "exx_plan_set_shard": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "exx_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "exx_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "exx_version": (ctypes.c_char_p, []),
}

_LIB = None


class ExxError(RuntimeError):
    """A non-zero exx_status_t from the library (``status``), with the call
    that returned it and, where the plan kept one, the CUDA error text."""

    def __init__(self, status, where, detail=""):
        name = STATUS[status] if 0 <= status < len(STATUS) else f"status {status}"
        super().__init__(f"{where}: {name}" + (f" ({detail})" if detail else ""))
        self.status = status


def load_library(path=None):
    """Load the CUDA library (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or _build.lib_path()
    if not os.path.exists(path):
        raise ExxError(1, "load_library",
                       f"{path} is missing; build it with paper_1712_07973_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status, where, plan=None):
    if status != 0:
        detail = ""
        if plan is not None:
            detail = (load_library().exx_last_error(plan) or b"").decode()
        raise ExxError(status, where, detail)


def kernel_spectrum(n, h, kind=KERNEL_SINC, omega=0.0):
    """Host-only FP64 octant of the kernel spectrum, indexed [kz][ky][kx]:
    (n+1,)*3 for the padded free-boundary kernels, (n/2+1,)*3 for
    KERNEL_PERIODIC, (n+1, n/2+1, n/2+1) for KERNEL_SLAB and
    (n/2+1, n+1, n+1) for KERNEL_WIRE (a periodic axis runs to n/2)."""
    half, full = n // 2 + 1, n + 1
    shape = {KERNEL_PERIODIC: (half,) * 3, KERNEL_SLAB: (full, half, half),
             KERNEL_WIRE: (half, full, full)}.get(int(kind), (full,) * 3)
    out = np.zeros(int(np.prod(shape)), dtype=np.float64)
    _check(load_library().exx_kernel_spectrum(n, float(h), int(kind), float(omega),
                                              out.ctypes.data_as(_c_double_p)), "exx_kernel_spectrum")
    return out.reshape(shape)


def shard_tiles(norb, tile=0, nranks=1):
    """Host-only: tile table (ntiles, 5: i0, ti, j0, tj, diag) and owner ranks."""
    lib = load_library()
    nt = ctypes.c_int()
    _check(lib.exx_shard_tiles(int(norb), int(tile), int(nranks), None, None, ctypes.byref(nt)),
           "exx_shard_tiles")
    desc = np.zeros(5 * nt.value, dtype=np.int32)
    own = np.zeros(nt.value, dtype=np.int32)
    _check(lib.exx_shard_tiles(int(norb), int(tile), int(nranks), desc.ctypes.data_as(_c_int_p),
                               own.ctypes.data_as(_c_int_p), ctypes.byref(nt)), "exx_shard_tiles")
    return desc.reshape(-1, 5), own


def _host_ptr(a):
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if a.is_cuda:
        raise ExxError(1, "host buffer", "a host tensor is required")
    return a.data_ptr()


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class PlanDesc(ctypes.Structure):
    """exx_plan_desc of include/exx.h."""
    _fields_ = [("grid", ctypes.c_int * 3), ("h", ctypes.c_double * 3), ("alpha", ctypes.c_double),
                ("occupations", _c_double_p), ("norb", ctypes.c_int), ("precision", ctypes.c_int),
                ("kernel", ctypes.c_int), ("flags", ctypes.c_uint), ("omega", ctypes.c_double)]


class ExxPlan:
    """Plan of the exact-exchange operator for fixed grid, h, alpha and occupations.

    precision: "fp64" (psi/vxpsi double) or "fp32" (psi float; vxpsi float, or
    double with vx_fp64=True).  kernel: "sinc" (band-limited), "hockney",
    "erfc" (band-limited erfc(omega r)/r, screened hybrids; needs omega > 0),
    "periodic" (the n^3 cell repeats), "slab" (x, y periodic, z free) or
    "wire" (x, y free, z periodic).
    tile: pair-tile edge 1..8 (0: the library default; "auto": the tuned value).
    """

    def __init__(self, n, h, alpha, occupations, precision="fp32", kernel="sinc",
                 vx_fp64=False, tile=0, omega=0.0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise ExxError(2, "ExxPlan", "no CUDA device: the EXX operator runs only on the GPU")
        self.lib = load_library()
        self.n = int(n)
        self.h = float(h)
        self.alpha = float(alpha)
        occ = np.ascontiguousarray(np.asarray(occupations, dtype=np.float64))
        self.occ = occ
        self.norb = int(occ.size)
        self.precision = {"fp64": FP64, "fp32": FP32}[precision]
        self.kernel = {"sinc": KERNEL_SINC, "hockney": KERNEL_HOCKNEY, "erfc": KERNEL_ERFC,
                       "periodic": KERNEL_PERIODIC, "slab": KERNEL_SLAB, "wire": KERNEL_WIRE}[kernel]
        self.omega = float(omega)
        self.vx_fp64 = bool(vx_fp64)
        self.dtype = torch.float64 if self.precision == FP64 else torch.float32
        self.vx_dtype = torch.float64 if (self.precision == FP64 or self.vx_fp64) else torch.float32
        grid = (ctypes.c_int * 3)(self.n, self.n, self.n)
        hh = (ctypes.c_double * 3)(self.h, self.h, self.h)
        handle = ctypes.c_void_p()
        if tile == "auto":
            from . import tune
            tile = tune.best_tile(self.n, self.norb, precision, tune_if_missing=True)
        flags = (FLAG_VX_FP64 if self.vx_fp64 else 0) | ((int(tile) & 15) << 8)
        d = PlanDesc()
        d.grid = grid
        d.h = hh
        d.alpha = self.alpha
        d.occupations = occ.ctypes.data_as(_c_double_p)
        d.norb = self.norb
        d.precision = self.precision
        d.kernel = self.kernel
        d.flags = flags
        d.omega = self.omega
        _check(self.lib.exx_plan_create_desc(ctypes.byref(handle), ctypes.byref(d), _stream_ptr(stream)),
               "exx_plan_create_desc")
        self.handle = handle

    # ---------------------------------------------------------------- checks
    def _psi(self, psi):
        import torch
        if not isinstance(psi, torch.Tensor) or not psi.is_cuda:
            raise ExxError(1, "psi", "a CUDA tensor is required")
        if psi.dtype != self.dtype:
            raise ExxError(1, "psi", f"dtype {psi.dtype}, plan expects {self.dtype}")
        if tuple(psi.shape) != (self.norb, self.n, self.n, self.n) or not psi.is_contiguous():
            raise ExxError(1, "psi", f"contiguous shape {(self.norb,) + (self.n,) * 3} required")
        return ctypes.c_void_p(psi.data_ptr())

    def energy(self, psi, stream=None):
        """E_x of psi ([norb, n, n, n] CUDA tensor of the plan's dtype), in
        hartree (exx_energy; synchronises the stream)."""
        E = ctypes.c_double()
        _check(self.lib.exx_energy(self.handle, self._psi(psi), ctypes.byref(E), _stream_ptr(stream)),
               "exx_energy", self.handle)
        return E.value

    def apply(self, psi, out=None, stream=None):
        """(E_x, Vx psi): the energy and the exchange action for every orbital
        (exx_apply).  out, if given, receives Vx psi (contiguous, psi's shape,
        the plan's output dtype)."""
        import torch
        p = self._psi(psi)
        if out is None:
            out = torch.empty(psi.shape, dtype=self.vx_dtype, device=psi.device)
        elif out.dtype != self.vx_dtype or out.shape != psi.shape or not out.is_contiguous():
            raise ExxError(1, "vxpsi", f"contiguous {self.vx_dtype} tensor of psi's shape required")
        E = ctypes.c_double()
        _check(self.lib.exx_apply(self.handle, p, ctypes.c_void_p(out.data_ptr()), ctypes.byref(E),
                                  _stream_ptr(stream)), "exx_apply", self.handle)
        return E.value, out

    def _out(self, psi, out):
        import torch
        if out is None:
            return torch.empty(psi.shape, dtype=self.vx_dtype, device=psi.device)
        if out.dtype != self.vx_dtype or out.shape != psi.shape or not out.is_contiguous():
            raise ExxError(1, "output", f"contiguous {self.vx_dtype} tensor of psi's shape required")
        return out

    def gradient(self, psi, out=None, stream=None):
        """(E_x, dE_x/dpsi): the energy and its gradient 2 f_k h^3 (Vx psi)_k,
        the per-orbital factor applied inside the library (exx_gradient)."""
        p = self._psi(psi)
        out = self._out(psi, out)
        E = ctypes.c_double()
        _check(self.lib.exx_gradient(self.handle, p, ctypes.c_void_p(out.data_ptr()), ctypes.byref(E),
                                     _stream_ptr(stream)), "exx_gradient", self.handle)
        return E.value, out

    def gradient_async(self, psi, out, E_dev=None, stream=None):
        """exx_gradient without synchronising (E_x into the device tensor E_dev)."""
        p = self._psi(psi)
        out = self._out(psi, out)
        e = ctypes.c_void_p(E_dev.data_ptr()) if E_dev is not None else ctypes.c_void_p()
        _check(self.lib.exx_gradient_async(self.handle, p, ctypes.c_void_p(out.data_ptr()), e,
                                           _stream_ptr(stream)), "exx_gradient_async", self.handle)
        return out

    def apply_async(self, psi, out, E_dev=None, stream=None):
        """exx_apply without synchronising: Vx psi into out and, if given, E_x
        into the one-element FP64 device tensor E_dev (graph-capturable)."""
        p = self._psi(psi)
        e = ctypes.c_void_p(E_dev.data_ptr()) if E_dev is not None else ctypes.c_void_p()
        _check(self.lib.exx_apply_async(self.handle, p, ctypes.c_void_p(out.data_ptr()), e,
                                        _stream_ptr(stream)), "exx_apply_async", self.handle)

    def energy_async(self, psi, E_dev=None, stream=None):
        """exx_energy without synchronising, E_x into E_dev (device)."""
        p = self._psi(psi)
        e = ctypes.c_void_p(E_dev.data_ptr()) if E_dev is not None else ctypes.c_void_p()
        _check(self.lib.exx_energy_async(self.handle, p, e, _stream_ptr(stream)),
               "exx_energy_async", self.handle)

    def pair_energies(self, stream=None):
        """E_ij = h^3 sum rho_ij V_ij of the last call, pairs (0,0), (0,1), ..,
        (N-1, N-1) in row-major order over i <= j (NumPy, FP64)."""
        P = self.norb * (self.norb + 1) // 2
        out = np.zeros(P, dtype=np.float64)
        _check(self.lib.exx_pair_energies(self.handle, out.ctypes.data_as(_c_double_p),
                                          _stream_ptr(stream)), "exx_pair_energies", self.handle)
        return out

    def apply_host(self, psi_host, vx_host, stream=None):
        """exx_apply_host on (page-locked) host tensors/arrays; returns E_x."""
        E = ctypes.c_double()
        _check(self.lib.exx_apply_host(self.handle, ctypes.c_void_p(_host_ptr(psi_host)),
                                       ctypes.c_void_p(_host_ptr(vx_host)), ctypes.byref(E),
                                       _stream_ptr(stream)), "exx_apply_host", self.handle)
        return E.value

    def gradient_host(self, psi_host, grad_host, stream=None):
        """exx_gradient_host on (page-locked) host tensors/arrays; returns E_x."""
        E = ctypes.c_double()
        _check(self.lib.exx_gradient_host(self.handle, ctypes.c_void_p(_host_ptr(psi_host)),
                                          ctypes.c_void_p(_host_ptr(grad_host)), ctypes.byref(E),
                                          _stream_ptr(stream)), "exx_gradient_host", self.handle)
        return E.value

    KINDS = ("fwd_xy", "zconv", "pair_energy", "inv_yx", "accum", "exx_total", "to_float")

    def set_lanes(self, lanes):
        """1: every kernel on the caller's stream; 2: consecutive tiles on two
        internal streams (the default where the plan has several tiles)."""
        _check(self.lib.exx_plan_set_lanes(self.handle, int(lanes)), "exx_plan_set_lanes", self.handle)

    def profile(self, enable=True):
        """Record CUDA events around every launch of later calls (per kernel
        kind; read with profile_read)."""
        _check(self.lib.exx_profile_enable(self.handle, int(bool(enable))), "exx_profile_enable")

    def profile_read(self, reset=True):
        """Summed ms and launch counts per kernel kind since the last reset."""
        ms = (ctypes.c_double * len(self.KINDS))()
        cnt = (ctypes.c_longlong * len(self.KINDS))()
        _check(self.lib.exx_profile_read(self.handle, ms, cnt, int(bool(reset))),
               "exx_profile_read", self.handle)
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.KINDS)}

    def set_shard(self, rank, nranks):
        """Process only this rank's pair tiles (partial E_x and Vx psi)."""
        _check(self.lib.exx_plan_set_shard(self.handle, int(rank), int(nranks)), "exx_plan_set_shard")

    def info(self):
        """Tile edge, tile count, device workspace bytes, kernel launches per
        apply / energy call and pipeline lanes of the plan."""
        t, nt, la, le = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ws = ctypes.c_size_t()
        _check(self.lib.exx_plan_info(self.handle, ctypes.byref(t), ctypes.byref(nt),
                                      ctypes.byref(ws), ctypes.byref(la), ctypes.byref(le)),
               "exx_plan_info")
        lanes = ctypes.c_int()
        _check(self.lib.exx_plan_get_lanes(self.handle, ctypes.byref(lanes)), "exx_plan_get_lanes")
        return {"tile": t.value, "ntiles": nt.value, "workspace_bytes": ws.value,
                "launches_apply": la.value, "launches_energy": le.value, "lanes": lanes.value}

    def close(self):
        """Free the plan's device memory (exx_plan_destroy); idempotent."""
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.exx_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MolDesc(ctypes.Structure):
    """exx_mol_desc of include/exx.h."""
    _fields_ = [("n", ctypes.c_int), ("h", ctypes.c_double), ("alpha", ctypes.c_double),
                ("occupations", _c_double_p), ("norb", ctypes.c_int), ("tile", ctypes.c_int)]


class ExxBatch:
    """Batched FP32 exact exchange over molecules of uneven size.

    mols: list of dicts with keys n, h, alpha, occupations and optional tile
    (1..8, 0 for the default, or "auto" for the tuned edge, see tune.py).
    """

    def __init__(self, mols, kernel="sinc", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise ExxError(2, "ExxBatch", "no CUDA device: the EXX operator runs only on the GPU")
        self.lib = load_library()
        self.nmol = len(mols)
        self._occ = [np.ascontiguousarray(np.asarray(m["occupations"], dtype=np.float64)) for m in mols]
        self.mols = [dict(m) for m in mols]
        descs = (MolDesc * self.nmol)()
        for k, m in enumerate(mols):
            descs[k].n = int(m["n"])
            descs[k].h = float(m["h"])
            descs[k].alpha = float(m["alpha"])
            descs[k].occupations = self._occ[k].ctypes.data_as(_c_double_p)
            descs[k].norb = int(self._occ[k].size)
            tile = m.get("tile", 0)
            if tile == "auto":
                from . import tune
                tile = tune.best_tile(descs[k].n, descs[k].norb, "fp32", tune_if_missing=True)
            descs[k].tile = int(tile)
        handle = ctypes.c_void_p()
        kind = {"sinc": KERNEL_SINC, "hockney": KERNEL_HOCKNEY}[kernel]
        _check(self.lib.exx_batch_create(ctypes.byref(handle), self.nmol, ctypes.cast(descs, ctypes.c_void_p),
                                         kind, _stream_ptr(stream)), "exx_batch_create")
        self.handle = handle
        self._bound = None

    def set_buffers(self, psis, vxs=None, stream=None):
        """Bind each molecule's orbitals (and Vx psi outputs) as contiguous
        CUDA float32 tensors; rebinding keeps a captured graph valid."""
        import torch
        for k, (p, m) in enumerate(zip(psis, self.mols)):
            n = int(m["n"])
            if (not isinstance(p, torch.Tensor) or not p.is_cuda or p.dtype != torch.float32
                    or not p.is_contiguous() or tuple(p.shape) != (self._occ[k].size, n, n, n)):
                raise ExxError(1, "psi", f"molecule {k}: contiguous CUDA float32 tensor required")
        pp = (ctypes.c_void_p * self.nmol)(*[p.data_ptr() for p in psis])
        vv = None
        if vxs is not None:
            for v, p in zip(vxs, psis):
                if v.dtype != torch.float32 or v.shape != p.shape or not v.is_contiguous() or not v.is_cuda:
                    raise ExxError(1, "vxpsi", "contiguous CUDA float32 tensors of psi's shapes required")
            vv = (ctypes.c_void_p * self.nmol)(*[v.data_ptr() for v in vxs])
        _check(self.lib.exx_batch_set_buffers(self.handle, ctypes.cast(pp, ctypes.c_void_p),
                                              ctypes.cast(vv, ctypes.c_void_p) if vv else None,
                                              _stream_ptr(stream)), "exx_batch_set_buffers")
        self._bound = (list(psis), list(vxs) if vxs is not None else None)

    def apply(self, E_dev=None, stream=None):
        """E_x per molecule (FP64 device tensor) and Vx psi into the bound
        outputs, asynchronously on the stream."""
        import torch
        if E_dev is None:
            E_dev = torch.zeros(self.nmol, dtype=torch.float64, device="cuda")
        _check(self.lib.exx_batch_apply(self.handle, ctypes.c_void_p(E_dev.data_ptr()),
                                        _stream_ptr(stream)), "exx_batch_apply")
        return E_dev

    def gradient(self, E_dev=None, stream=None):
        """E_x per molecule (FP64 device tensor) and the gradients
        2 f_k h^3 (Vx psi)_k into the bound outputs, asynchronously."""
        import torch
        if E_dev is None:
            E_dev = torch.zeros(self.nmol, dtype=torch.float64, device="cuda")
        _check(self.lib.exx_batch_gradient(self.handle, ctypes.c_void_p(E_dev.data_ptr()),
                                           _stream_ptr(stream)), "exx_batch_gradient")
        return E_dev

    def energy(self, E_dev=None, stream=None):
        """E_x per molecule only (FP64 device tensor), asynchronously."""
        import torch
        if E_dev is None:
            E_dev = torch.zeros(self.nmol, dtype=torch.float64, device="cuda")
        _check(self.lib.exx_batch_energy(self.handle, ctypes.c_void_p(E_dev.data_ptr()),
                                         _stream_ptr(stream)), "exx_batch_energy")
        return E_dev

    def graph(self, enable=True):
        """Capture each call kind once into a CUDA graph and replay it (needs a
        created, non-default stream)."""
        _check(self.lib.exx_batch_graph(self.handle, int(bool(enable))), "exx_batch_graph")

    def persistent(self, enable=True, stream=None):
        """Run each (n, h) group as one launch of the persistent kernel over a
        device work queue (exx_batch_set_persistent)."""
        _check(self.lib.exx_batch_set_persistent(self.handle, int(bool(enable)), _stream_ptr(stream)),
               "exx_batch_set_persistent")

    def pair_energies(self, mol, stream=None):
        """E_ij of molecule ``mol`` from the last call (as ExxPlan.pair_energies)."""
        N = self._occ[mol].size
        out = np.zeros(N * (N + 1) // 2)
        _check(self.lib.exx_batch_pair_energies(self.handle, int(mol), out.ctypes.data_as(_c_double_p),
                                                _stream_ptr(stream)), "exx_batch_pair_energies")
        return out

    def info(self):
        """Groups of equal (n, h), waves, workspace bytes, launches per apply
        and total pairs of the batch."""
        g, w, la = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ws, pr = ctypes.c_size_t(), ctypes.c_longlong()
        _check(self.lib.exx_batch_info(self.handle, ctypes.byref(g), ctypes.byref(w), ctypes.byref(ws),
                                       ctypes.byref(la), ctypes.byref(pr)), "exx_batch_info")
        return {"groups": g.value, "waves": w.value, "workspace_bytes": ws.value,
                "launches_apply": la.value, "pairs": pr.value}

    def close(self):
        """Free the batch's device memory (exx_batch_destroy); idempotent."""
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.exx_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
