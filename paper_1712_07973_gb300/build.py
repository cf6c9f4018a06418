"""Build the in-tree CUDA library ``_lib/libexx_gb300.so`` for sm_103a.

Every ``csrc/*.cu`` file is compiled by nvcc with
``-gencode arch=compute_103a,code=sm_103a`` (in parallel), the host-side
kernel builder by g++ with OpenMP, and everything is linked into one shared
library with the CUDA runtime linked statically.  The build is skipped when a
fingerprint of the sources, headers and flags is unchanged.
"""

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUTDIR = os.path.join(HERE, "_lib")
LIBNAME = "libexx_gb300.so"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fopenmp",
              f"-I{INCLUDE}"]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-fopenmp"]


def _nvcc():
    cand = [os.environ.get("NVCC", ""), shutil.which("nvcc") or "", "/usr/local/cuda/bin/nvcc"]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the EXX library")


def lib_path():
    return os.path.join(OUTDIR, LIBNAME)


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    hdr = sorted(f for f in os.listdir(CSRC) if f.endswith((".cuh", ".h")))
    return cu, cpp, hdr


def _fingerprint(files):
    h = hashlib.sha256()
    h.update(" ".join(ARCH + NVCC_FLAGS + CXX_FLAGS).encode())
    for f in files:
        with open(f, "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build step failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build(force=False, verbose=False, jobs=None):
    """Compile and link the library; returns its path."""
    cu, cpp, hdr = _sources()
    files = [os.path.join(CSRC, f) for f in cu + cpp + hdr] + [os.path.join(INCLUDE, "exx.h")]
    fp = _fingerprint(files)
    stamp = os.path.join(OUTDIR, "fingerprint")
    out = lib_path()
    if not force and os.path.exists(out) and os.path.exists(stamp):
        with open(stamp) as fh:
            if fh.read().strip() == fp:
                return out
    os.makedirs(OUTDIR, exist_ok=True)
    objdir = os.path.join(OUTDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()
    cmds = []
    objs = []
    for f in cu:
        o = os.path.join(objdir, f[:-3] + ".o")
        cmds.append([nvcc] + ARCH + NVCC_FLAGS + ["-c", os.path.join(CSRC, f), "-o", o])
        objs.append(o)
    cxx = os.environ.get("CXX", "g++")
    for f in cpp:
        o = os.path.join(objdir, f[:-4] + ".o")
        cmds.append([cxx] + CXX_FLAGS + ["-c", os.path.join(CSRC, f), "-o", o])
        objs.append(o)
    jobs = jobs or min(len(cmds), max(1, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(jobs) as ex:
        for log in ex.map(_run, cmds):
            if verbose and log.strip():
                print(log)
    tmp = out + ".tmp"
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lgomp"])
    os.replace(tmp, out)
    with open(stamp, "w") as fh:
        fh.write(fp)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
