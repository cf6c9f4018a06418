#!/usr/bin/env python
"""Benchmark of the exact-exchange operator on one GB300 (or N GPUs, sharded).

Workload (one "step" = one E_x + gradient: exx_gradient, i.e. E_x and
dE_x/dpsi_k = 2 f_k h^3 (Vx psi)_k from all pair solves): 512
Lowdin-orthonormal Gaussian-combination orbitals of a 256-site cluster on a
160^3 grid (320^3 zero-padded Poisson grid), h = 0.42 bohr, f = 2,
alpha = 0.25, FP32 FFTs and products with FP64 kernel, E_x and gradient
accumulation: 131,328 pair solves per step (the pair count of the 512-orbital
H2O row of the paper's Table pscount).  Inputs are seeded synthetic orbitals
(no dataset exists for this path), resident in HBM before timing.

Output: one JSON line (rank 0).  ``value`` is pair-solves/s over all ranks;
``roofline`` describes the dominant kernel (CUDA events recorded by the library
on the launching stream around every launch of the timed region); ``e2e`` is
the same metric through exx_gradient_host with pinned host buffers;
``cpu_baseline`` is the FP64 NumPy oracle on the host cores over a bounded
sample of the same pair solves, whose energies also give the FP32 path's
per-pair error.  Sub-records: ``fp32_vs_fp64`` (the metric's FP32-vs-FP64
comparison per E_x + gradient on the 128-orbital 128^3 workload, the largest
whose FP64 step fits the run), ``c2`` (64 orbitals on 96^3) and ``batched``
(the 16-molecule uneven batch and a 64-molecule small-molecule batch, FP32
batched autograd against FP64 plain).

Under torchrun (N > 1 ranks, one GPU each) the step is the sharded path: each
rank solves its share of the pair tiles and the partial E_x and gradients are
summed with NCCL all-reduces (strong scaling: the work per step is fixed).

``--impl reference`` times the FP64 oracle alone (there is no other
implementation of this path to run) on a bounded sample of the same workload's
pair solves per step and prints the same JSON line.
"""

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c5_large_n160_N512"
METRIC = "EXX pair-solves/s and ms per E_x+gradient: FP32 batched vs FP64 plain at ≤1e-6 Ha"
UNIT = "pair-solves/s"
KERNEL_SOURCES = ["exx_fft.cuh", "exx_kernels.cuh", "exx_ops.cuh"]
WORKLOADS = ["c5_large_n160_N512", "c3_grad_n128_N128", "c2_fp32_n96_N64"]


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD, choices=WORKLOADS,
                    help="orbital workload of the timed step (default: 512 orbitals on 160^3)")
    ap.add_argument("--cpu-sample", type=int, default=64,
                    help="pair solves of the oracle sample (CPU baseline and per-pair errors)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP32-vs-FP64 sub-record")
    ap.add_argument("--no-c2", action="store_true", help="skip the 64-orbital 96^3 sub-record")
    ap.add_argument("--batched", action=argparse.BooleanOptionalAction, default=True,
                    help="batched sub-records (16 uneven molecules; 64 small molecules)")
    ap.add_argument("--bc", choices=["free", "periodic", "slab", "wire"], default="free",
                    help="boundary conditions: free (zero-padded 2n FFTs), periodic cell, slab "
                         "(x, y periodic, z free) or wire (x, y free, z periodic)")
    ap.add_argument("--norb", type=int, default=0,
                    help="use only the first NORB orbitals (small profiling cases)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def kernel_source_hash():
    """Hash of the kernel sources' code (line comments and blank lines left
    out, so that a comment edit does not invalidate the committed counters)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1712_07973_gb300", "csrc", f)) as fh:
            code = [ln.split("//", 1)[0].strip() for ln in fh.read().splitlines()]
        h.update("\n".join(ln for ln in code if ln).encode())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_model():
    """Host CPU model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


# ------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"exx_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# -------------------------------------------------------- roofline bytes
def tile_list(N, T):
    nb = (N + T - 1) // T
    out = []
    for bi in range(nb):
        for bj in range(bi, nb):
            ti = min(T, N - bi * T)
            tj = min(T, N - bj * T)
            diag = bi == bj
            npair = ti * (ti + 1) // 2 if diag else ti * tj
            out.append((npair, ti, tj, diag))
    return out


def half_lines(n, bc):
    """Half line lengths (x and y, z) of the transforms: n on a free
    (zero-padded) axis, n/2 on a periodic one."""
    return {"free": (n, n), "periodic": (n // 2, n // 2), "slab": (n // 2, n),
            "wire": (n, n // 2)}[bc]


def algorithmic_bytes(n, N, T, rs=4, bc="free"):
    """Minimal HBM bytes of each kernel kind over one step.

    x and y transforms of length 2h, z transforms of length 2hz (half_lines).
    Per pair: fwd_xy writes the y-transformed spectrum X2 ((h+1) n 2h complex);
    zconv reads it and writes X3 in place; inv_yx reads X3 and writes V (n^3);
    accum reads V.  Per tile: fwd_xy and accum read the tile's orbitals once,
    accum reads and writes their FP64 accumulators once; zconv reads the
    kernel table ((h+1) 2hz 2h) once per launch.
    """
    cs = 2 * rs
    hl, hz = half_lines(n, bc)
    spec = (hl + 1) * n * 2 * hl * cs
    n3 = n ** 3
    tot = {"fwd_xy": 0, "zconv": 0, "inv_yx": 0, "accum": 0}
    for npair, ti, tj, diag in tile_list(N, T):
        orbs = ti if diag else ti + tj
        tot["fwd_xy"] += orbs * n3 * rs + npair * spec
        tot["zconv"] += 2 * npair * spec + (hl + 1) * (2 * hz) * (2 * hl) * rs
        tot["inv_yx"] += npair * spec + npair * n3 * rs
        tot["accum"] += npair * n3 * rs + orbs * n3 * rs + 2 * orbs * n3 * 8
    return tot


def committed_traffic(kernel, workload=WORKLOAD):
    """ncu DRAM bytes per launch from profiles/traffic.json, if the kernel
    sources are unchanged since the capture; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


# ------------------------------------------------------------ CPU oracle
def oracle_spectrum(n, h, bc="free"):
    from oracle import exx_oracle as o
    return {"periodic": lambda: o.kernel_spectrum_periodic(n, h),
            "slab": lambda: o.kernel_spectrum_slab(n, h),
            "wire": lambda: o.kernel_spectrum_wire(n, h),
            "free": lambda: o.kernel_spectrum(o.kernel_real_space(n, h))}[bc]()


def oracle_pairs(orb, pairs, r, Gh):
    """Time the FP64 oracle on the given pair solves (co-density, FFT Poisson
    solve, E_ij, both V psi products).  orb(i) returns orbital i as FP64
    NumPy.  Returns (seconds, {(i, j): E_ij})."""
    import numpy as np
    from oracle import exx_oracle as o
    cache = {}

    def get(i):
        if i not in cache:
            cache[i] = orb(i)
        return cache[i]

    for i, j in pairs:  # inputs ready before the clock starts
        get(i), get(j)
    acc = np.zeros((2,) + cache[pairs[0][0]].shape)
    E = {}
    t0 = time.perf_counter()
    for i, j in pairs:
        V, e = o.exx_pair(get(i), get(j), Gh, r.h)
        acc[0] += (-r.alpha * r.occupation) * V * get(j)
        acc[1] += (-r.alpha * r.occupation) * V * get(i)
        E[(i, j)] = e
    return time.perf_counter() - t0, E


def sample_pairs(N, count, seed):
    import numpy as np
    P = N * (N + 1) // 2
    rng = np.random.default_rng(seed)
    g = np.sort(rng.choice(P, size=min(count, P), replace=False))
    out = []
    for gid in g:  # row-major decode over i <= j
        i, rem = 0, int(gid)
        while rem >= N - i:
            rem -= N - i
            i += 1
        out.append((i, i + rem, int(gid)))
    return out


# ------------------------------------------------------------ timing helpers
def cuda_time(torch, stream, fn, steps):
    """Milliseconds per call of fn over steps calls (CUDA events on stream)."""
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def roofline_of(prof, alg, steps_timed, peak, peak_kind, workload, timed_region):
    """Roofline object of the kernel kind with the largest measured time."""
    dom = max(alg, key=lambda k: prof[k][0])
    kms, kcnt = prof[dom]
    per_launch_bytes = alg[dom] / (kcnt / steps_timed)
    achieved = per_launch_bytes / (kms / kcnt * 1e-3) / 1e9
    tot = sum(x[0] for x in prof.values())
    shares = {k: round(v[0] / max(1e-9, tot), 4) for k, v in prof.items()}
    per_kernel = {}
    for k in alg:
        ms_k, c_k = prof[k]
        if c_k:
            b = alg[k] / (c_k / steps_timed)
            per_kernel[k] = {"avg_launch_ms": ms_k / c_k, "algorithmic_bytes_per_launch": int(b),
                             "achieved_gbs": round(b / (ms_k / c_k * 1e-3) / 1e9, 1),
                             "frac": round(b / (ms_k / c_k * 1e-3) / 1e9 / peak, 4)}
    return {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
            "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": committed_traffic(dom, workload),
            "algorithmic_bytes_per_launch": int(per_launch_bytes),
            "avg_launch_ms": kms / kcnt, "kernel_shares": shares, "per_kernel": per_kernel,
            "timed_region": timed_region}


# ------------------------------------------------------------ sub-records
def c2_record(torch, dev, exx, synth, stream, steps):
    """64 orbitals on 96^3 (two pipeline lanes): throughput, roofline of the
    serialised kernels, E_x error against the stored oracle value."""
    import numpy as np
    r, psi_np = synth.workload("c2_fp32_n96_N64")
    psi = torch.from_numpy(psi_np).to(dev, torch.float32)
    P = r.norb * (r.norb + 1) // 2
    plan = exx.ExxPlan(r.n, r.h, r.alpha, np.full(r.norb, r.occupation), precision="fp32")
    info = plan.info()
    out = torch.empty_like(psi)
    E_dev = torch.zeros(1, dtype=torch.float64, device=dev)
    for _ in range(3):
        plan.gradient_async(psi, out, E_dev)
    ms = cuda_time(torch, stream, lambda: plan.gradient_async(psi, out, E_dev), steps)
    E = float(E_dev.item())
    plan.set_lanes(1)
    plan.gradient_async(psi, out, E_dev)
    plan.profile(True)
    plan.profile_read(reset=True)
    ms1 = cuda_time(torch, stream, lambda: plan.gradient_async(psi, out, E_dev), steps)
    prof = plan.profile_read(reset=True)
    plan.profile(False)
    plan.close()
    peak, kind = measured_peaks()
    rl = roofline_of(prof, algorithmic_bytes(r.n, r.norb, info["tile"]), steps, peak, kind,
                     "c2_fp32_n96_N64", f"{steps} steps, one pipeline lane, events around every launch")
    rl["serialised_ms_per_step"] = ms1
    rec = {"workload": "c2_fp32_n96_N64: 64 orbitals on 96^3 (192^3 padded), h = 0.4",
           "pairs": P, "ms_per_step": ms, "value": P / (ms * 1e-3), "unit": UNIT,
           "lanes": info["lanes"], "E_x": E, "roofline": rl}
    golden = os.path.join(ROOT, "tests", "golden", "c2_fp32_n96_N64.json")
    if os.path.exists(golden):
        with open(golden) as fh:
            rec["E_x_abs_err_vs_oracle_Ha"] = abs(E - json.load(fh)["E_x"])
    return rec


def fp32_vs_fp64_record(torch, dev, exx, synth, stream, ag):
    """The metric's comparison per E_x + gradient (torch.autograd forward +
    backward) on the 128-orbital 128^3 workload: FP32 against the plain FP64
    GPU path, both against the stored FP64 oracle value of E_x."""
    import numpy as np
    name = "c3_grad_n128_N128"
    r, psi64 = synth.workload(name, dtype=np.float64, device=dev)
    occ = np.full(r.norb, r.occupation)
    P = r.norb * (r.norb + 1) // 2

    def step(plan, x):
        def f():
            x.grad = None
            E = ag.exx_energy(x, plan)
            E.backward()
            return E
        return f

    p32 = exx.ExxPlan(r.n, r.h, r.alpha, occ, precision="fp32")
    x32 = psi64.float().requires_grad_(True)
    f32 = step(p32, x32)
    f32()
    ms32 = cuda_time(torch, stream, f32, 3)
    E32 = float(f32().item())
    g32 = x32.grad.detach().double()
    p32.close()
    del x32
    p64 = exx.ExxPlan(r.n, r.h, r.alpha, occ, precision="fp64")
    x64 = psi64.clone().requires_grad_(True)
    f64 = step(p64, x64)
    f64()
    ms64 = cuda_time(torch, stream, f64, 1)
    E64 = float(f64().item())
    g64 = x64.grad.detach()
    p64.close()
    rel = float(torch.linalg.vector_norm(g32 - g64).item() / torch.linalg.vector_norm(g64).item())
    rec = {"workload": f"{name}: 128 orbitals on 128^3 (256^3 padded), h = 0.37 -- the largest "
                       "workload whose FP64 step fits the bench run (an FP64 step of the 512-orbital "
                       "160^3 workload takes minutes)",
           "pairs": P, "what": "ms per E_x + gradient: ExxEnergy forward + backward (torch.autograd)",
           "fp32_ms_per_step": ms32, "fp64_plain_ms_per_step": ms64,
           "fp32_speedup_vs_fp64_plain": ms64 / ms32,
           "fp32_value": P / (ms32 * 1e-3), "fp64_value": P / (ms64 * 1e-3), "unit": UNIT,
           "E_x_fp32": E32, "E_x_fp64": E64, "E_x_abs_diff_fp32_vs_fp64_Ha": abs(E32 - E64),
           "gradient_rel_l2_fp32_vs_fp64": rel}
    golden = os.path.join(ROOT, "tests", "golden", f"{name}.json")
    if os.path.exists(golden):
        with open(golden) as fh:
            Eo = json.load(fh)["E_x"]
        rec["E_x_fp32_abs_err_vs_oracle_Ha"] = abs(E32 - Eo)
        rec["E_x_fp64_abs_err_vs_oracle_Ha"] = abs(E64 - Eo)
    del psi64, x64
    torch.cuda.empty_cache()
    return rec


def batched_record(torch, dev, exx, synth, ag, recipes, label, fp64=True):
    """A batch of uneven molecules: FP32 batched (one CUDA-graph launch) apply
    and autograd per step, against one FP32 plan per molecule and the plain
    FP64 path (one FP64 plan per molecule, autograd)."""
    import numpy as np
    mols, pt = [], []
    for r in recipes:
        mols.append({"n": r.n, "h": r.h, "alpha": r.alpha, "occupations": np.full(r.norb, r.occupation)})
        pt.append(synth.make_orbitals(r, dtype=np.float64, device=dev))
    p32 = [p.float() for p in pt]
    pairs = sum(r.norb * (r.norb + 1) // 2 for r in recipes)
    b = exx.ExxBatch(mols)
    vx = [torch.empty_like(p) for p in p32]
    b.set_buffers(p32, vx)
    b.graph(True)
    s = torch.cuda.Stream()
    E = torch.zeros(len(mols), dtype=torch.float64, device=dev)
    modes = {}
    for mode in ("waves", "persistent"):  # graph of per-wave launches / one persistent launch per group
        b.persistent(mode == "persistent")
        with torch.cuda.stream(s):
            for _ in range(2):
                b.gradient(E, stream=s)
            modes[mode] = (cuda_time(torch, s, lambda: b.gradient(E, stream=s), 3), b.info())
    best = min(modes, key=lambda k: modes[k][0])
    b.persistent(best == "persistent")
    ms, info = modes[best]
    # batched autograd: ExxBatchEnergy forward + backward
    xs = [p.clone().requires_grad_(True) for p in p32]

    def ag_step():
        for x in xs:
            x.grad = None
        ag.exx_batch_energy(b, xs).sum().backward()
    with torch.cuda.stream(s):  # graph replay needs a created stream
        ag_step()
        ms_ag = cuda_time(torch, s, ag_step, 3)
    b.close()
    cur = torch.cuda.current_stream()
    # one FP32 plan per molecule
    plans = [exx.ExxPlan(m["n"], m["h"], m["alpha"], m["occupations"], precision="fp32") for m in mols]
    outs = [torch.empty_like(p) for p in p32]

    def seq():
        for pl, p, o in zip(plans, p32, outs):
            pl.gradient_async(p, o)
    seq()
    ms_seq = cuda_time(torch, cur, seq, 3)
    for pl in plans:
        pl.close()
    rec = {"workload": label, "pairs": pairs, "ms_per_step": ms, "value": pairs / (ms * 1e-3),
           "unit": UNIT, "graph": True, "schedule": best, "groups": info["groups"],
           "waves": info["waves"], "launches_per_step": info["launches_apply"],
           "schedules": {k: {"ms_per_step": v[0], "launches_per_step": v[1]["launches_apply"]}
                         for k, v in modes.items()},
           "autograd_ms_per_step": ms_ag,
           "sequential_plans_ms": ms_seq, "speedup_vs_sequential_plans": ms_seq / ms}
    if fp64:
        plans = [exx.ExxPlan(m["n"], m["h"], m["alpha"], m["occupations"], precision="fp64") for m in mols]
        xs64 = [p.clone().requires_grad_(True) for p in pt]

        def ag64():
            for pl, x in zip(plans, xs64):
                x.grad = None
                ag.exx_energy(x, pl).backward()
        ag64()
        ms64 = cuda_time(torch, cur, ag64, 1)
        for pl in plans:
            pl.close()
        rec["fp64_plain_autograd_ms_per_step"] = ms64
        rec["fp32_batched_autograd_speedup_vs_fp64_plain"] = ms64 / ms_ag
        del xs64
    del pt, p32, xs
    torch.cuda.empty_cache()
    return rec


# ------------------------------------------------------------ reference arm
def run_reference(a):
    """The FP64 oracle on the host cores, each step a bounded sample of the
    workload's pair solves (a few seeded pairs among 16 seeded orbitals)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    from paper_1712_07973_gb300 import synth
    r = synth.WORKLOADS[a.workload]
    if a.norb:
        r.norb = a.norb
    N, P = r.norb, r.norb * (r.norb + 1) // 2
    rng = np.random.default_rng(2024)
    pool = np.sort(rng.choice(N, size=min(16, N), replace=False))
    orbs = dict(zip(pool.tolist(), synth.orbital_subset(r, pool)))
    Gh = oracle_spectrum(r.n, r.h, a.bc)
    per_step = 8 if r.n >= 128 else 32  # about 0.8 s of FP64 oracle work per step on 16 cores
    pool_pairs = [(int(i), int(j)) for k, i in enumerate(pool) for j in pool[k:]]

    def one_step(seed):
        sel = np.random.default_rng(seed).choice(len(pool_pairs), size=per_step, replace=False)
        dt, _ = oracle_pairs(lambda i: orbs[i], [pool_pairs[s] for s in sel], r, Gh)
        return dt

    for k in range(a.warmup):
        one_step(1 + k)
    times = [one_step(100 + k) for k in range(a.steps)]
    tot = sum(times)
    value = per_step * a.steps / tot
    cores = os.cpu_count()
    sample = (f"{per_step} seeded pair solves per step (among the pairs of 16 seeded orbitals) of "
              f"the {P} of the workload; FP64 NumPy/SciPy, scipy.fft workers = all cores")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps,
        "ms_per_step_is": f"measured: one step = {per_step} sampled pair solves",
        "ms_per_full_workload_extrapolated": 1e3 * P / value,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": a.workload, "norb": N, "n": r.n, "pairs": P,
                                        "pairs_per_step": per_step, "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu_model": cpu_model(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- GPU arm
def run_ours(a):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    tdist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1712_07973_gb300 import autograd as ag, build, dist as xdist, exx, synth
    build.build()
    small = a.workload == "c2_fp32_n96_N64"
    if small:
        r, psi_np = synth.workload(a.workload)
        if a.norb:
            psi_np = psi_np[: a.norb].copy()
            r.norb = a.norb
        psi = torch.from_numpy(psi_np).to(dev, torch.float32)
    else:  # large inputs: generated with the device's help, never copied to the host
        r, psi = synth.workload(a.workload, dtype=np.float32, device=dev)
        if a.norb:
            psi = psi[: a.norb].contiguous()
            r.norb = a.norb
    N, n = r.norb, r.n
    P = N * (N + 1) // 2
    occ = np.full(N, r.occupation)
    per = a.bc != "free"
    kern = "sinc" if a.bc == "free" else a.bc
    plan = exx.ExxPlan(n, r.h, r.alpha, occ, precision="fp32", kernel=kern)
    info = plan.info()
    out = torch.empty(psi.shape, dtype=torch.float32, device=dev)
    E_dev = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    if tdist:
        def step():
            xdist.sharded_apply(plan, psi, out=out, gradient=True, sync=False)
        parallelism = f"pair-tile sharding over {world} GPUs + NCCL all-reduce of E_x and the gradient"
    else:
        def step():
            plan.gradient_async(psi, out, E_dev)
        parallelism = "one GPU"

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    # one lane (plans whose slab kernels run as two-CTA clusters): every kernel
    # alone on the stream, so the per-launch events of the roofline are taken
    # in the headline region itself
    inline_prof = info["lanes"] == 1 and not tdist
    if inline_prof:
        plan.profile(True)
        plan.profile_read(reset=True)
    sampler = ClockSampler(local) if rank == 0 else None
    if tdist:
        tdist.barrier()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(a.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    if tdist:
        tdist.barrier()
    clocks = sampler.stop() if sampler else None
    ms = t0.elapsed_time(t1)
    if tdist:
        tt = torch.tensor([ms], device=dev, dtype=torch.float64)
        tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
        ms = float(tt.item())
    if tdist:
        E = float(xdist.sharded_apply(plan, psi, out=out, gradient=True)[0])
    else:
        E = float(E_dev.item())
    value = P * a.steps / (ms * 1e-3)
    ms_step = ms / a.steps

    peak, peak_kind = measured_peaks()
    alg = algorithmic_bytes(n, N, info["tile"], bc=a.bc)
    if inline_prof:
        prof = plan.profile_read(reset=True)
        plan.profile(False)
        region = f"the {a.steps} timed steps (one pipeline lane), events around every launch"
        ms_serial = ms_step
    elif not tdist:
        # two lanes overlap consecutive tiles: a second region of the same
        # steps with one lane times every kernel alone
        plan.set_lanes(1)
        step()
        plan.profile(True)
        plan.profile_read(reset=True)
        ms_serial = cuda_time(torch, stream, step, a.steps)
        prof = plan.profile_read(reset=True)
        plan.profile(False)
        plan.set_lanes(info["lanes"])
        region = f"{a.steps} further steps, one pipeline lane, events around every launch"
    else:
        prof = None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": a.workload, "bc": a.bc, "norb": N, "n": n,
                       "fft_grid": [2 * hh for hh in half_lines(n, a.bc)], "h": r.h,
                       "pairs": P, "tile": info["tile"], "lanes": info["lanes"],
                       "step": "E_x + gradient (exx_gradient: all pair solves, products, FP64 "
                               "accumulation and energy)",
                       "precision": "fp32 ffts and products, fp64 kernel, energies and accumulation",
                       "l2": f"inputs larger than L2 (psi {N * n ** 3 * 4 / 1e9:.2f} GB; pair-tile "
                             "spectra up to 4.2 GB): no flush needed",
                       "parallelism": parallelism},
            "E_x": E, "clocks": clocks,
            "gpu_launches": info["launches_apply"] * a.steps}
    if prof is not None:
        rl = roofline_of(prof, alg, a.steps, peak, peak_kind, a.workload, region)
        rl["serialised_ms_per_step"] = ms_serial
        step_bytes = sum(alg.values())
        rl["pipeline"] = {"algorithmic_bytes_per_step": int(step_bytes),
                          "bytes_per_pair": int(step_bytes / P),
                          "achieved": round(step_bytes / (ms_step * 1e-3) / 1e9, 1), "unit": "GB/s",
                          "frac": round(step_bytes / (ms_step * 1e-3) / 1e9 / peak, 4)}
        if per or a.norb:
            rl["traffic"] = None  # the committed captures are of the free-BC workloads
        line["roofline"] = rl

    # oracle sample: per-pair errors of the FP32 path and the CPU baseline
    if rank == 0 and world == 1 and not a.no_cpu_baseline and not a.norb and not per:
        Eij = plan.pair_energies()
        sp = sample_pairs(N, a.cpu_sample, seed=77)
        Gh = oracle_spectrum(n, r.h, a.bc)

        def orb(i):
            return psi[i].double().cpu().numpy()
        dt, Eo = oracle_pairs(orb, [(i, j) for i, j, _ in sp], r, Gh)
        errs = [abs(Eij[g] - Eo[(i, j)]) for i, j, g in sp]
        w = [(1.0 if i == j else 2.0) * occ[i] * occ[j] * 0.5 * r.alpha for i, j, _ in sp]
        est = (P / len(sp)) * sum(wk * (Eij[g] - Eo[(i, j)]) for wk, (i, j, g) in zip(w, sp))
        line["pair_sample_vs_oracle"] = {
            "pairs": len(sp), "max_abs_err_E_ij_Ha": max(errs),
            "mean_abs_err_E_ij_Ha": sum(errs) / len(errs),
            "E_x_error_estimate_Ha": abs(est),
            "E_x_error_estimate_is": "sampled pairs' weighted errors scaled to all pairs (estimate)",
            "inputs": "the FP32 orbitals of the GPU run, in FP64"}
        line["cpu_baseline"] = {"value": len(sp) / dt, "unit": UNIT, "cores": os.cpu_count(),
                                "cpu_model": cpu_model(), "kind": "oracle", "seconds": dt,
                                "sample": f"{len(sp)} seeded pair solves (of {P}) of the same "
                                          "workload, FP64 NumPy/SciPy, scipy.fft workers = all cores"}
        # out holds the gradient 2 f_k h^3 (Vx psi)_k, so E_x = 1/2 sum_k f_k h^3
        # <psi_k, (Vx psi)_k> = 1/4 sum_k <psi_k, grad_k> (energy by Parseval in
        # the z kernel, gradient in real space after every inverse transform)
        cons = 0.25 * float((psi.double() * out.double()).sum().item())
        line["E_x_vs_gradient_identity_rel"] = abs(cons - E) / abs(E)

    # e2e through the host-buffer entry point (pinned memory): every step copies
    # psi in and the gradient + E_x out
    if not a.no_e2e and world == 1:
        psi_h = psi.cpu().pin_memory()
        g_h = torch.empty(psi_h.shape, dtype=torch.float32).pin_memory()
        e2e_steps = 1 if not small else max(3, min(a.steps, 10))
        plan.gradient_host(psi_h, g_h)
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(e2e_steps):
            plan.gradient_host(psi_h, g_h)
        e2e_s = time.perf_counter() - w0
        nbytes = N * n ** 3 * 4
        line["e2e"] = {"value": P * e2e_steps / e2e_s, "unit": UNIT,
                       "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 8,
                       "api": "exx_gradient_host", "steps": e2e_steps}
        del psi_h, g_h
    plan.close()
    del out
    torch.cuda.empty_cache()

    if rank == 0 and world == 1 and not a.norb and not per:
        if not a.no_fp64:
            line["fp32_vs_fp64"] = fp32_vs_fp64_record(torch, dev, exx, synth, stream, ag)
        if not a.no_c2 and not small:
            line["c2"] = c2_record(torch, dev, exx, synth, stream, 10)
        if a.batched:
            line["batched"] = batched_record(
                torch, dev, exx, synth, ag, synth.batched_workload(),
                "16 molecules, N_m in [8,96], n_m in {48,64,80,96,112,128}, h=0.4, seed 3",
                fp64=not a.no_fp64)
            line["batched_small"] = batched_record(
                torch, dev, exx, synth, ag, synth.small_batched_workload(),
                "64 small molecules, N_m in [8,24], n_m in {32,40,48}, h=0.4, seed 5",
                fp64=not a.no_fp64)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if tdist:
        tdist.barrier()
        tdist.destroy_process_group()
    return 0


def main():
    a = args_parse()
    if a.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
