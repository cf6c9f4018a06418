"""Launch shapes of every compiled configuration, checked on the host.

A small host program (generated here from the size registries of
csrc/exx_api.cu and compiled by nvcc; it evaluates only the compile-time
constants of OpsImpl, no kernel is compiled or launched) prints the shapes
the library launches.  The checks: every registered configuration is
supported; no CTA asks for more shared memory or threads than an SM gives;
the register budget (threads x CTAs per SM) stays within 2048 threads; CTAs
that stage the kernel table by TMA have 16-byte aligned boxes; the bench
workload's shapes are the measured ones.
"""

import json
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1712_07973_gb300", "csrc")
SMEM_PER_SM = 228 * 1024
SMEM_PER_CTA = 227 * 1024 - 256


def _registry():
    with open(os.path.join(CSRC, "exx_api.cu")) as fh:
        src = fh.read()

    def sizes(name):
        # the macro's body: its line and any continuation lines (ending in "\")
        m = re.search(r"#define " + name + r"\(X\)((?:[^\n]*\\\n)*[^\n]*)", src)
        return [int(v) for v in re.findall(r"X\((\d+)\)", m.group(1))]

    cfg = []
    for n in sizes("EXX_SIZES"):
        cfg.append(("free", n, f"{n}, false, {n}, false"))
    for N in sizes("EXX_PSIZES"):
        cfg.append(("periodic", 2 * N, f"{N}, true, {N}, true"))
    for N in sizes("EXX_SSIZES"):
        cfg.append(("slab", 2 * N, f"{N}, true, {2 * N}, false"))
    for n in sizes("EXX_WSIZES"):
        cfg.append(("wire", n, f"{n}, false, {n // 2}, true"))
    return cfg


@pytest.fixture(scope="module")
def shapes(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    lines = ['#include <cstdio>', '#include "exx_ops.cuh"', "using namespace exx;",
             "template <typename T> void show(const char* bc, int n, const char* prec) {",
             '  std::printf("{\\"bc\\": \\"%s\\", \\"n\\": %d, \\"prec\\": \\"%s\\", \\"ok\\": %d, '
             '\\"nt_a\\": %d, \\"minb_a\\": %d, \\"cl_a\\": %d, \\"smem_a\\": %zu, '
             '\\"nt_c\\": %d, \\"minb_c\\": %d, \\"cl_c\\": %d, \\"smem_c\\": %zu, '
             '\\"nw\\": %d, \\"minb_b\\": %d, \\"smem_b\\": %zu, \\"stage\\": %d, \\"w\\": %d, '
             '\\"lz\\": %d, \\"fold\\": %d}\\n", bc, n, prec, (int)T::ok, T::NT_A, T::MINB_A, '
             'T::CL_A, T::smem_a, T::NT_C, T::MINB_C, T::CL_C, T::smem_c, T::NW, T::MINB_B, '
             'T::smem_b, (int)T::stage_g, T::W, T::LZ, (int)T::fold_y);',
             "}", "int main() {"]
    for bc, n, args in _registry():
        for prec, R in (("fp32", "float"), ("fp64", "double")):
            lines.append(f'  show<OpsImpl<{R}, {args}>>("{bc}", {n}, "{prec}");')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("shapes")
    src, exe = d / "shapes.cu", d / "shapes"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([nvcc, "-std=c++17", "-O0", f"-I{CSRC}", f"-I{os.path.join(ROOT, 'include')}",
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return [json.loads(ln) for ln in out.splitlines()]


def test_every_registered_configuration_is_supported(shapes):
    bad = [(s["bc"], s["n"], s["prec"]) for s in shapes if not s["ok"]]
    assert bad == [], bad
    assert len([s for s in shapes if s["prec"] == "fp32" and s["ok"]]) == len(shapes) // 2


def test_ctas_fit_an_sm(shapes):
    for s in (s for s in shapes if s["ok"]):
        for k in ("a", "c"):
            nt, minb, smem = s["nt_" + k], s["minb_" + k], s["smem_" + k]
            assert nt <= 1024 and smem <= SMEM_PER_CTA, s
            assert nt * minb <= 2048 and minb * (smem + 1024) <= SMEM_PER_SM, s
        nt_b = 32 * s["nw"]
        assert s["smem_b"] <= SMEM_PER_CTA and nt_b * s["minb_b"] <= 2048, s
        assert s["minb_b"] * (s["smem_b"] + 1024) <= SMEM_PER_SM or s["minb_b"] == 2, s


def test_tma_staged_tables_have_aligned_boxes(shapes):
    for s in (s for s in shapes if s["ok"] and s["stage"]):
        assert s["prec"] == "fp32" and (s["w"] * 4) % 16 == 0 and s["lz"] <= 256, s
        assert not s["fold"], s


def test_bench_workload_shapes(shapes):
    s = next(s for s in shapes if s["bc"] == "free" and s["n"] == 96 and s["prec"] == "fp32")
    assert (s["nt_a"], s["minb_a"], s["cl_a"]) == (320, 2, 1)
    assert (s["nt_c"], s["minb_c"], s["cl_c"]) == (320, 2, 1)
    assert (s["nw"], s["minb_b"], s["stage"]) == (8, 4, 0)


def test_largest_grid_shapes(shapes):
    # n = 160: the slab kernels run as four-CTA clusters, two CTAs of 320
    # threads per SM in FP32 and one in FP64 (whose slab quarter and scratch
    # take most of an SM)
    f32 = next(s for s in shapes if s["bc"] == "free" and s["n"] == 160 and s["prec"] == "fp32")
    f64 = next(s for s in shapes if s["bc"] == "free" and s["n"] == 160 and s["prec"] == "fp64")
    assert (f32["nt_a"], f32["minb_a"], f32["cl_a"]) == (320, 2, 4)
    assert (f32["nt_c"], f32["minb_c"], f32["cl_c"]) == (320, 2, 4)
    assert (f64["nt_a"], f64["minb_a"], f64["cl_a"]) == (320, 1, 4)
    assert (f64["nt_c"], f64["minb_c"], f64["cl_c"]) == (320, 1, 4)
    assert f64["minb_b"] == 1
    # FP32 zconv on 320-point lines: 32 columns, ten warps, two CTAs per SM
    assert (f32["w"], f32["nw"], f32["minb_b"]) == (32, 10, 2)
