#!/usr/bin/env python
"""Benchmark of the exact-exchange operator on one GB300 (or N replicas).

Workload (one "step" = one exx_apply: E_x plus the exchange action Vx psi,
i.e. E_x and its gradient): 64 Lowdin-orthonormal Gaussian-combination
orbitals on a 96^3 grid (192^3 zero-padded Poisson grid), h = 0.4 bohr,
f = 2, alpha = 0.25, FP32 FFTs and products with FP64 kernel, E_x and Vx psi
accumulation: 2080 pair solves per step.  Inputs are seeded synthetic
orbitals (no dataset exists for this path), resident in HBM before timing.

Output: one JSON line (rank 0).  ``value`` is pair-solves/s over all ranks;
``roofline`` describes the dominant kernel (per-kernel CUDA events on the
launching stream over the timed region); ``e2e`` is the same metric through
exx_apply_host with pinned host buffers; ``cpu_baseline`` is the FP64 NumPy
oracle on the host cores over a bounded sample of the same pair solves.

``--impl reference`` times that oracle alone (there is no other
implementation of this path to run) and prints the same JSON line.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c2_fp32_n96_N64"
METRIC = "EXX pair-solves/s (exx_apply: E_x + Vx psi gradient, FP32 FFTs, FP64 reductions)"
UNIT = "pair-solves/s"
KERNEL_SOURCES = ["exx_fft.cuh", "exx_kernels.cuh", "exx_ops.cuh"]


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-sample", type=int, default=128, help="pair solves timed on the CPU")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=["c2_fp32_n96_N64", "c3_grad_n128_N128", "c5_large_n160_N512"],
                    help="orbital workload of the timed step (default: 64 orbitals on 96^3)")
    ap.add_argument("--batched", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the 16-molecule batched workload (one graph launch)")
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
    """Minimal HBM bytes of each kernel kind over one exx_apply.

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


def committed_traffic(kernel):
    """ncu DRAM bytes per launch from profiles/traffic.json, if the kernel
    sources are unchanged since the capture; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(WORKLOAD, {}).get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


# ------------------------------------------------------------ CPU oracle
def cpu_oracle_rate(psi, r, npairs, seed=0, bc="free"):
    """Time the FP64 oracle on a seeded sample of the workload's pair solves
    (co-density, FFT Poisson solve, E_ij, both V psi products)."""
    import numpy as np
    from oracle import exx_oracle as o
    Gh = {"periodic": lambda: o.kernel_spectrum_periodic(r.n, r.h),
          "slab": lambda: o.kernel_spectrum_slab(r.n, r.h),
          "wire": lambda: o.kernel_spectrum_wire(r.n, r.h),
          "free": lambda: o.kernel_spectrum(o.kernel_real_space(r.n, r.h))}[bc]()
    rng = np.random.default_rng(seed)
    pairs = o.pair_list(r.norb)
    pick = [pairs[k] for k in rng.choice(len(pairs), size=npairs, replace=False)]
    acc = np.zeros((2,) + psi.shape[1:])
    t0 = time.perf_counter()
    for i, j in pick:
        V, e = o.exx_pair(psi[i], psi[j], Gh, r.h)
        acc[0] += (-r.alpha * r.occupation) * V * psi[j]
        acc[1] += (-r.alpha * r.occupation) * V * psi[i]
    dt = time.perf_counter() - t0
    return npairs / dt, dt


def batched_line(torch, dev, exx, synth, stream):
    """16 molecules of uneven size (N_m in [8, 96], n_m in {48..128}^3), FP32,
    one CUDA-graph launch per step; compared with one plan per molecule."""
    import numpy as np
    recipes = synth.batched_workload()
    mols, pt = [], []
    for r in recipes:
        mols.append({"n": r.n, "h": r.h, "alpha": r.alpha, "occupations": np.full(r.norb, r.occupation)})
        pt.append(torch.from_numpy(synth.make_orbitals(r, dtype=np.float32)).to(dev))
    pairs = sum(r.norb * (r.norb + 1) // 2 for r in recipes)
    b = exx.ExxBatch(mols)
    vx = [torch.empty_like(p) for p in pt]
    b.set_buffers(pt, vx)
    b.graph(True)
    s = torch.cuda.Stream()
    E = torch.zeros(len(mols), dtype=torch.float64, device=dev)
    with torch.cuda.stream(s):
        for _ in range(2):
            b.apply(E, stream=s)
        s.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(s)
        for _ in range(3):
            b.apply(E, stream=s)
        t1.record(s)
    s.synchronize()
    ms = t0.elapsed_time(t1) / 3
    info = b.info()
    b.close()
    plans = [exx.ExxPlan(m["n"], m["h"], m["alpha"], m["occupations"], precision="fp32") for m in mols]
    outs = [torch.empty_like(p) for p in pt]
    for pl, p, o in zip(plans, pt, outs):
        pl.apply_async(p, o)
    torch.cuda.synchronize()
    q0 = torch.cuda.Event(enable_timing=True)
    q1 = torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    for _ in range(3):
        for pl, p, o in zip(plans, pt, outs):
            pl.apply_async(p, o)
    q1.record(stream)
    torch.cuda.synchronize()
    ms_seq = q0.elapsed_time(q1) / 3
    for pl in plans:
        pl.close()
    return {"workload": "16 molecules, N_m in [8,96], n_m in {48,64,80,96,112,128}, h=0.4, seed 3",
            "pairs": pairs, "ms_per_step": ms, "value": pairs / (ms * 1e-3), "unit": UNIT,
            "graph": True, "groups": info["groups"], "waves": info["waves"],
            "launches_per_step": info["launches_apply"],
            "sequential_plans_ms": ms_seq, "speedup_vs_sequential_plans": ms_seq / ms}


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1712_07973_gb300 import synth
    r, psi = synth.workload(WORKLOAD)
    per_step = 32
    for _ in range(a.warmup):
        cpu_oracle_rate(psi, r, per_step, seed=1)
    rates, tot_t = [], 0.0
    for k in range(a.steps):
        rate, dt = cpu_oracle_rate(psi, r, per_step, seed=100 + k)
        rates.append(rate)
        tot_t += dt
    value = per_step * a.steps / tot_t
    P = r.norb * (r.norb + 1) // 2
    cores = os.cpu_count()
    sample = f"{per_step} seeded pair solves per step of the {P} of the 64-orbital 96^3 workload"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * P / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "norb": r.norb, "n": r.n,
                                        "pairs": P, "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- GPU arm
def run_ours(a):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1712_07973_gb300 import build, exx, synth
    build.build()
    big = a.workload != WORKLOAD
    if big:  # large inputs: generated with the device's help, never copied to the host
        r, psi = synth.workload(a.workload, dtype=np.float32, device=dev)
        psi_np = None
    else:
        r, psi_np = synth.workload(a.workload)
        if a.norb:
            psi_np = psi_np[: a.norb].copy()
            r.norb = a.norb
        psi = torch.from_numpy(psi_np).to(dev, torch.float32)
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

    for _ in range(a.warmup):
        plan.apply_async(psi, out, E_dev)
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if rank == 0 else None
    if dist:
        dist.barrier()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(a.steps):
        plan.apply_async(psi, out, E_dev)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    ms = t0.elapsed_time(t1)
    if dist:
        tt = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    E = float(E_dev.item())
    value = world * P * a.steps / (ms * 1e-3)
    ms_step = ms / a.steps

    # roofline of the dominant kernel: a second timed region of the same steps
    # with one pipeline lane (every kernel alone on the stream, as the two-lane
    # headline region overlaps consecutive tiles) and CUDA events recorded by
    # the library around every launch
    plan.set_lanes(1)
    plan.apply_async(psi, out, E_dev)
    torch.cuda.synchronize()
    plan.profile(True)
    plan.profile_read(reset=True)
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for _ in range(a.steps):
        plan.apply_async(psi, out, E_dev)
    s1.record(stream)
    torch.cuda.synchronize()
    ms_serial = s0.elapsed_time(s1) / a.steps
    prof = plan.profile_read(reset=True)
    plan.profile(False)
    plan.set_lanes(info["lanes"])
    alg = algorithmic_bytes(n, N, info["tile"], bc=a.bc)
    dom = max(alg, key=lambda k: prof[k][0])
    kms, kcnt = prof[dom]
    per_launch_bytes = alg[dom] / (kcnt / a.steps)
    achieved = per_launch_bytes / (kms / kcnt * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    shares = {k: round(v[0] / max(1e-9, sum(x[0] for x in prof.values())), 4) for k, v in prof.items()}
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                "peak_source": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": committed_traffic(dom), "algorithmic_bytes_per_launch": int(per_launch_bytes),
                "avg_launch_ms": kms / kcnt, "kernel_shares": shares,
                "timed_region": f"{a.steps} further steps, one pipeline lane, events around every launch",
                "serialised_ms_per_step": ms_serial}

    # whole pipeline: algorithmic bytes of all kernels of a step over the step time
    step_bytes = sum(alg.values())
    pipeline = {"algorithmic_bytes_per_step": int(step_bytes),
                "bytes_per_pair": int(step_bytes / P),
                "achieved": round(step_bytes / (ms_step * 1e-3) / 1e9, 1), "unit": "GB/s",
                "frac": round(step_bytes / (ms_step * 1e-3) / 1e9 / peak, 4)}
    roofline["pipeline"] = pipeline

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": a.workload, "bc": a.bc, "norb": N, "n": n,
                       "fft_grid": [2 * hh for hh in half_lines(n, a.bc)], "h": r.h,
                       "pairs": P, "tile": info["tile"], "lanes": info["lanes"],
                       "precision": "fp32 ffts, fp64 reductions",
                       "l2": "inputs larger than L2 (psi 226 MB; pair-tile spectra 0.2-0.9 GB)",
                       "parallelism": f"replicas x{world}"},
            "E_x": E, "clocks": clocks, "roofline": roofline,
            "gpu_launches": info["launches_apply"] * a.steps}
    if per:
        line["roofline"]["traffic"] = None  # the committed capture is of the free-BC kernels

    golden = os.path.join(ROOT, "tests", "golden", f"{a.workload}.json")
    if a.norb or per:
        golden = ""
    if os.path.exists(golden):
        with open(golden) as fh:
            line["E_x_abs_err_vs_oracle_Ha"] = abs(E - json.load(fh)["E_x"])

    # e2e through the host-buffer entry point (pinned memory), every step copies
    # psi in and Vx psi + E_x out
    psi_h = (psi.cpu() if big else torch.from_numpy(psi_np.astype(np.float32))).pin_memory()
    vx_h = torch.empty(psi_h.shape, dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(a.steps, 10))
    plan.apply_host(psi_h, vx_h)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        plan.apply_host(psi_h, vx_h)
    w1 = time.perf_counter()
    e2e_s = w1 - w0
    if dist:
        tt = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    nbytes = N * n ** 3 * 4
    line["e2e"] = {"value": world * P * e2e_steps / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 8,
                   "api": "exx_apply_host"}

    # autograd path: forward + hand-written backward through ExxEnergy (the
    # backward is the exchange action computed in the same pair solves)
    from paper_1712_07973_gb300 import autograd as ag
    pg = psi.clone().requires_grad_(True)
    for _ in range(2):
        pg.grad = None
        ag.exx_energy(pg, plan).backward()
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    ag_steps = max(3, min(a.steps, 10))
    a0.record(stream)
    for _ in range(ag_steps):
        pg.grad = None
        ag.exx_energy(pg, plan).backward()
    a1.record(stream)
    torch.cuda.synchronize()
    line["autograd"] = {"ms_per_step": a0.elapsed_time(a1) / ag_steps,
                        "what": "E_x forward + gradient backward via torch.autograd"}
    del pg

    # FP64 plain GPU path on the same workload (the comparison the metric names)
    if not a.no_fp64 and (not big or n <= 128):
        p64 = exx.ExxPlan(n, r.h, r.alpha, occ, precision="fp64", kernel=kern)
        if big:  # same seeded orbitals, generated in FP64 on the device
            psi64 = synth.workload(a.workload, dtype=np.float64, device=dev)[1].to(torch.float64)
        else:
            psi64 = torch.from_numpy(psi_np).to(dev)
        out64 = torch.empty(psi64.shape, dtype=torch.float64, device=dev)
        p64.apply_async(psi64, out64, E_dev)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(2):
            p64.apply_async(psi64, out64, E_dev)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / 2
        E64 = float(E_dev.item())
        line["fp64_plain"] = {"ms_per_step": ms64, "value": P / (ms64 * 1e-3), "unit": UNIT,
                              "E_x": E64, "fp32_speedup": ms64 / ms_step,
                              "autograd_fp32_speedup": ms64 / line["autograd"]["ms_per_step"],
                              "E_x_abs_diff_fp32_vs_fp64_Ha": abs(E - E64)}
        if os.path.exists(golden):
            with open(golden) as fh:
                line["fp64_plain"]["E_x_abs_err_vs_oracle_Ha"] = abs(E64 - json.load(fh)["E_x"])
        p64.close()
        del psi64, out64

    if a.batched and not big:
        line["batched"] = batched_line(torch, dev, exx, synth, stream)

    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        sample = a.cpu_sample if not big else max(4, a.cpu_sample // 16)
        if big:
            psi_np = psi.double().cpu().numpy()
        a.cpu_sample = sample
        rate, dt = cpu_oracle_rate(psi_np, r, a.cpu_sample, bc=a.bc)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": os.cpu_count(),
                                "kind": "oracle", "seconds": dt,
                                "sample": f"{a.cpu_sample} seeded pair solves (of {P}) of the same "
                                          "workload, FP64 NumPy/SciPy, scipy.fft workers = all cores"}
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
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
