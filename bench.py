"""Benchmark: Poisson + 3 x screened-Helmholtz solves to 1e-10 relative
residual at 512^3 on one GB300 (per rank), through libmg's C ABI.

One step = one solve set: the variable-permittivity Poisson problem (dielectric
slab eps_r = 4 below z = 0.2, streamer-shell charge, phi = 0 / 1 on the bottom
/ top faces, Neumann sides) plus the three radiative-transfer Helmholtz
problems (kappa L = 10, 100, 1000, Gaussian-smoothed ionisation source), each
from a zero initial guess, mixed precision (FP32 V-cycles inside FP64
iterative refinement).  Inputs are seeded synthetic fields generated on the
host and resident in HBM before timing; every array is 1 GiB, far larger than
the 129 MB L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank solves its own replica (weak scaling, no collective on
the data path); the time is the max over ranks.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Hardware work queues of the device (read when the CUDA context is created,
# so before any CUDA call).  The end-to-end leg drives the solver's four
# problem streams and its own upload, download and solve streams; with the
# default 8 queues some of them share one, and a problem's step then waits
# behind the 4 GiB download of the previous set's answers (141 against 131 ms
# per set measured).
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "Poisson+3×Helmholtz solves/s to 1e-10 rel. residual at 512³; % HBM roofline"
UNIT = "solve sets/s (1 set = 1 Poisson + 3 Helmholtz)"
TOL = 1e-10
KAPPAS = (10.0, 100.0, 1000.0)
COPY_STREAMS = 4  # streams per copy direction in the end-to-end leg


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--inner-cycles", type=int, default=3)
    ap.add_argument("--concurrency", type=int, default=4)
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep --inner-cycles and V(2,2) instead of the autotuned choice")
    ap.add_argument("--e2e-steps", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ir-zchunk", type=int, default=0,
                    help="refinement-pass tile (z planes per CTA column) when not autotuning; "
                         "0 = automatic")
    ap.add_argument("--no-amr", action="store_true",
                    help="skip the composite AMR solve among the extras")
    ap.add_argument("--no-config3", action="store_true",
                    help="skip the 256^3 parent + 16 sub-box pass among the extras")
    ap.add_argument("--no-needle", action="store_true",
                    help="skip the 896^3 needle-plane set among the extras")
    ap.add_argument("--coarse-visits", type=int, default=0,
                    help="V-cycles on the first coarse level per finest-level cycle "
                         "(0 = the library default, one)")
    ap.add_argument("--stack", action="store_true",
                    help="stack the Helmholtz problems' V-cycles (mg_options.stack)")
    ap.add_argument("--no-fp64-leg", action="store_true",
                    help="skip the FP64-mode GPU solve set among the extras")
    return ap.parse_args()


def max_over_ranks(x, world, device):
    """The largest of the ranks' x (every rank passes its own and gets the
    maximum); world == 1 returns x."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, seconds_per_step):
    """Sets per second of the whole job: every rank solves its own replica
    (weak scaling), the step time is the slowest rank's."""
    return world / seconds_per_step


def emit(line, rank):
    """The JSON line, printed by rank 0 only."""
    if rank == 0:
        print(json.dumps(line), flush=True)


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def workload(n):
    from paper_1809_08857_gb300 import workloads as W

    return {"rho": W.streamer_shell(n, 0), "eps": W.dielectric_slab(n),
            "S": W.ionization_source(n, 0)}


def config(args):
    return {"workload": f"poisson_slab_shell_{args.n}^3 + 3x helmholtz_{args.n}^3 (kappa L = 10, 100, 1000)",
            "grid": [args.n] * 3, "tol": TOL, "precision": args.precision,
            "inner_cycles": args.inner_cycles, "concurrency": args.concurrency,
            "graphs": not args.no_graphs, "smoother": "red-black Gauss-Seidel V(nu1, nu2)",
            "l2": "inputs larger than L2 (1 GiB per array), no flush"}


# ---------------------------------------------------------------- CPU oracle


def oracle_problems(n, inputs=None):
    import oracle

    if inputs is None:
        inputs = workload(n)
    h = 1.0 / n
    probs = [(oracle.poisson((n, n, n), h, eps_r=inputs["eps"]), inputs["rho"] / oracle.EPS0)]
    probs += [(oracle.helmholtz((n, n, n), h, k), inputs["S"]) for k in KAPPAS]
    return probs


def oracle_set(inputs, n):
    """One whole solve set by the FP64 CPU oracle on the host cores, as it
    stands: the Poisson problem and the three Helmholtz problems, each from a
    zero guess to the same 1e-10 relative residual as the GPU (the oracle's
    own V(2,2)-cycles, set-up included).  Returns (seconds, [(cycles, rel)])."""
    probs = oracle_problems(n, inputs)
    t0 = time.perf_counter()
    info = []
    for p, f in probs:
        _, cyc, rel, _ = p.solve(f, tol=TOL, max_cycles=200)
        info.append((int(cyc), float(rel)))
    return time.perf_counter() - t0, info


def oracle_sets(inputs, n, max_sets, budget_s):
    """Whole oracle solve sets, one after another, until max_sets have run or
    the next one would end after budget_s seconds (at least one runs).
    Returns (seconds per set, sets run, per-problem (cycles, rel) of the last
    set, threads)."""
    cores = os.cpu_count() or 1
    times, info = [], None
    t_start = time.perf_counter()
    while len(times) < max(1, max_sets):
        if times and (time.perf_counter() - t_start) + statistics.mean(times) > budget_s:
            break
        t, info = oracle_set(inputs, n)
        times.append(t)
    return statistics.mean(times), len(times), info, cores


def oracle_baseline(inputs, n, max_sets=1, budget_s=120.0):
    """cpu_baseline object: whole oracle solve sets at n^3 timed on all host
    cores (no extrapolation from a partial solve)."""
    sec, nsets, info, cores = oracle_sets(inputs, n, max_sets, budget_s)
    return {"value": 1.0 / sec, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"FP64 C oracle (OpenMP, {cores} threads), {nsets} whole solve set(s) at "
                       f"{n}^3: Poisson + 3 Helmholtz, each from zero to 1e-10 relative residual "
                       f"with the oracle's own V(2,2)-cycles (cycles {[c for c, _ in info]}), "
                       f"{sec:.1f} s per set"),
            "seconds_per_set": sec, "sets": nsets,
            "cycles": [c for c, _ in info], "rel_resid": [r for _, r in info]}


# ---------------------------------------------------------------- clocks


class Clocks:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- roofline


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {
    "smooth": ["paper_1809_08857_gb300/csrc/mg_split32.cu", "paper_1809_08857_gb300/csrc/tma.cuh"],
    "restrict": ["paper_1809_08857_gb300/csrc/mg_split32.cu"],
    "prolong": ["paper_1809_08857_gb300/csrc/mg_split32.cu"],
    "resid64": ["paper_1809_08857_gb300/csrc/mg_ir.cu", "paper_1809_08857_gb300/csrc/df.cuh",
                "paper_1809_08857_gb300/csrc/tma.cuh"],
}


def traffic_for(cls, algorithmic_bytes):
    """DRAM bytes per launch of the class: the ratio of DRAM to algorithmic
    bytes that a committed ncu capture of the class's 512^3 launches
    measured (profiles/traffic.json), times this launch's algorithmic bytes;
    None when there is no capture or the kernel source changed since."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    ent = t.get(cls)
    if not ent or ent.get("source_hash") != source_hash(KERNEL_SOURCES.get(cls, [])):
        return None
    return round(ent["dram_over_algorithmic"] * algorithmic_bytes)


def classes(prof):
    total = sum(v["ms"] for v in prof.values())
    return ({k: round(v["ms"] / total, 4) for k, v in prof.items()} if total > 0 else {},
            {k: round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1)
             for k, v in prof.items() if k != "coarse" and v["ms"] > 0})


def roofline(prof_serial, prof_overlap, n):
    """Dominant fine-level kernel class of a profiled step run one problem at
    a time (launches do not overlap, so an event pair brackets one kernel):
    algorithmic bytes per launch / average launch time, against the measured
    copy bandwidth."""
    pk, src = peaks()
    fine = {k: v for k, v in prof_serial.items() if k != "coarse" and v["ms"] > 0}
    if not fine:
        return None
    dom = max(fine, key=lambda k: fine[k]["ms"])
    d = fine[dom]
    avg_ms = d["ms"] / d["launches"]
    avg_bytes = d["bytes"] / d["launches"]
    gbs = avg_bytes / (avg_ms * 1e-3) / 1e9
    peak = float(pk["hbm_gbs"])
    share_s, gbs_s = classes(prof_serial)
    share_o, gbs_o = classes(prof_overlap)
    return {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
            "frac": round(gbs / peak, 4), "traffic": traffic_for(dom, avg_bytes),
            "kernel": dom, "avg_launch_ms": round(avg_ms, 4),
            "algorithmic_bytes_per_launch": avg_bytes,
            "peak_source": (f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured"
                            else "fallback 6.8 TB/s"),
            "timing": "CUDA events around every fine-level launch on its stream, in one "
                      "profiled solve set run one problem at a time after the timed steps",
            "class_share": share_s, "class_gbs": gbs_s,
            "overlapped": {"note": "the same set at the timed concurrency: event pairs "
                                   "include the kernels of other problems running meanwhile",
                           "class_share": share_o, "class_gbs": gbs_o}}


def measure_extras(solver, rho, eps, phi, n, dev):
    """The two steps beside the solve set (outside the timed region): the
    field pass E = -grad phi with the relaxation time eps0 |E| / |J| (56
    algorithmic bytes per cell: phi, J and E), and one variable-coefficient
    screened solve (a diffusion factor, alpha = 1/mu with mu = 0.4 h^2 /
    max(eps)) from zero to 1e-10."""
    import torch

    pk, _ = peaks()
    E = torch.empty((3, n, n, n), dtype=torch.float64, device=dev)
    J = torch.full((3, n, n, n), 1e-9, dtype=torch.float64, device=dev)
    for _ in range(2):
        solver.efield(phi, J, E)
    torch.cuda.synchronize()
    reps = 5
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        solver.efield(phi, J, E)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    gbs = 56.0 * n ** 3 / (ms * 1e-3) / 1e9
    del E, J
    h = 1.0 / n
    alpha = float(eps.max().item()) / (0.4 * h * h)
    f = rho * (alpha / 8.8541878128e-12)
    u = torch.zeros_like(phi)
    solver.solve_screened(alpha, f, u, TOL)  # first call builds the coarse inverse
    u.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = solver.solve_screened(alpha, f, u, TOL)
    torch.cuda.synchronize()
    sms = (time.perf_counter() - t0) * 1e3
    return {"efield": {"ms": round(ms, 4), "achieved_gbs": round(gbs, 1),
                       "frac": round(gbs / float(pk["hbm_gbs"]), 4), "bytes_per_cell": 56,
                       "note": "includes the host read-back of the relaxation time"},
            "screened_solve": {"ms": round(sms, 2), "solves_per_s": round(1e3 / sms, 2),
                               "steps": st["cycles"], "rel_resid": st["rel_resid"],
                               "alpha": alpha}}


def fp64_residuals(solver, rho, phi, S, psi):
    """Relative residual ||b - A u|| / ||b|| of each answer of a set (Poisson,
    then the three Helmholtz problems), formed by the library's plain FP64
    kernel (mg_residual_norms)."""
    out = []
    rn, bn = solver.residual_norms("poisson", rho, phi)
    out.append(rn / bn)
    for p, k in zip(psi, KAPPAS):
        rn, bn = solver.residual_norms("helmholtz", S, p, k)
        out.append(rn / bn)
    return out


def measure_fp64_gpu(rho, eps, S, n, dev, phi_mixed, psi_mixed, mixed_sets_per_s, reps=2):
    """The same solve set in FP64 mode on the same GPU (plain FP64 V(2,2)
    multigrid, one problem after another, the form of the paper's solver):
    sets/s by CUDA events over `reps` sets after one untimed set, its answers'
    FP64 residuals, and the relative L2 distance of the mixed-precision
    answers from them (outside the timed region)."""
    import torch

    from paper_1809_08857_gb300 import mg

    s64 = mg.Solver((n, n, n), 1.0 / n, eps_r=eps, precision=mg.MG_PREC_FP64)
    phi = torch.zeros_like(phi_mixed)
    psi = [torch.zeros_like(phi) for _ in range(3)]
    st = None

    def one():
        nonlocal st
        phi.zero_()
        for p in psi:
            p.zero_()
        st = s64.solve_set(rho, phi, S, psi, KAPPAS, TOL)

    one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        one()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    res = fp64_residuals(s64, rho, phi, S, psi)
    s64.close()

    def rel(a, b):
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))

    dist = [rel(phi_mixed, phi)] + [rel(a, b) for a, b in zip(psi_mixed, psi)]
    del phi, psi
    torch.cuda.empty_cache()
    return {"workload": "the same set, FP64 V(2,2)-cycles on the GPU (no mixed precision, "
                        "problems one after another)",
            "ms": round(ms, 1), "sets_per_s": round(1e3 / ms, 3),
            "cycles": [x["cycles"] for x in st], "rel_resid_fp64": res,
            "mixed_over_fp64": round(mixed_sets_per_s * ms * 1e-3, 2),
            "rel_l2_mixed_vs_fp64": dist}


def measure_needle_plane(dev, n=896, reps=2):
    """The full-size needle-plane set (outside the timed region): 896^3 cells
    (719 M), a needle electrode held at phi = 1 reaching a hyperboloid tip of
    radius 5h at z = 0.8, the grounded plane z = 0, Neumann sides, charge on
    the shells of three seeded branching channels leaving the tip; the Poisson
    problem and the three Helmholtz problems (source |rho| / eps0, Psi = 0 on
    the faces and the needle) in one mixed-precision mg_solve_set from zero
    to 1e-10, after one untimed set (graphs, coarse inverses); device time
    per set by CUDA events, and each answer's plain FP64 residual.  Skipped
    when the device has less than 200 GB free."""
    import torch

    from paper_1809_08857_gb300 import mg, workloads as W

    free, _ = torch.cuda.mem_get_info()
    if free < 200e9:
        return {"skipped": f"needs about 170 GB of free device memory, {free / 1e9:.0f} GB free"}
    t_in = time.perf_counter()
    mask = torch.from_numpy(W.needle_mask(n)).to(dev)
    mv = mask.to(torch.float64)
    idx, val = W.channel_shell_cells(n, 0)
    rho = torch.zeros(n ** 3, dtype=torch.float64, device=dev)
    rho[torch.from_numpy(idx).to(dev)] = torch.from_numpy(val).to(dev)
    rho = rho.view(n, n, n)
    S = rho.abs() / W.EPS0
    t_in = time.perf_counter() - t_in
    s = mg.Solver((n, n, n), 1.0 / n, mask=mask, mask_value=mv, bc_kind=W.GAP_BC_KIND,
                  bc_value=W.GAP_BC_VALUE, precision=mg.MG_PREC_MIXED, max_cycles=400,
                  inner_cycles=2)
    del mv
    phi = torch.zeros((n, n, n), dtype=torch.float64, device=dev)
    psi = [torch.zeros_like(phi) for _ in KAPPAS]
    st = None

    def one():
        nonlocal st
        phi.zero_()
        for p in psi:
            p.zero_()
        st = s.solve_set(rho, phi, S, psi, KAPPAS, TOL)

    one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        one()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    res = fp64_residuals(s, rho, phi, S, psi)
    used = torch.cuda.max_memory_allocated()
    s.close()
    del phi, psi, rho, S, mask
    torch.cuda.empty_cache()
    return {"workload": f"needle-plane set, {n}^3 ({n ** 3 / 1e6:.0f} M cells): Poisson (needle at "
                        "phi = 1, three branching charged channels) + 3 Helmholtz, mixed, "
                        "2 inner V-cycles per refinement step",
            "ms": round(ms, 1), "sets_per_s": round(1e3 / ms, 3),
            "steps": [x["cycles"] for x in st], "rel_resid_fp64": res,
            "input_build_s": round(t_in, 1),
            "torch_peak_gb": round(used / 1e9, 1),
            "warm_start": "not used: a cold solve has no previous potential to start from"}


def measure_config3(dev, reps=3):
    """The sub-box configuration (outside the timed region): the Poisson + 3
    Helmholtz set on a 256^3 parent, face data for 16 refined sub-boxes of
    sizes drawn from {32, 48, 64, 96, 128}^3 (ratio 2) interpolated from the
    parent answers, and the 64 sub-box problems in one mg_solve_batch, all
    from zero to 1e-10 (subboxes.Config3); device time per pass by CUDA
    events after one untimed pass (contexts, graphs and inputs built
    beforehand)."""
    import torch

    from paper_1809_08857_gb300 import subboxes

    c = subboxes.Config3(n=256, count=16, seed=0)
    c.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        stp, stb = c.run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    parent_cells, box_cells = c.cells()
    out = {"workload": "256^3 Poisson + 3 Helmholtz, then 16 ratio-2 sub-boxes of sizes "
                       "{32, 48, 64, 96, 128}^3 with Dirichlet data from the parent answers, "
                       "4 problems each in one batch; mixed, 3 inner V-cycles",
           "ms": round(ms, 2), "passes_per_s": round(1e3 / ms, 2),
           "parent_steps": [x["cycles"] for x in stp],
           "subbox_steps_max": max(x["cycles"] for x in stb),
           "subbox_rel_resid_max": max(x["rel_resid"] for x in stb),
           "cells": {"parent": parent_cells, "subboxes": box_cells},
           "box_sizes": sorted(b["dims"][0] for b in c.boxes)}
    c.close()
    torch.cuda.empty_cache()
    return out


def measure_unet(dev, n=256, reps=5):
    """One warm-start U-Net forward pass (mg_unet_predict) on a 256^3 volume
    (outside the timed region): device time per pass (CUDA events) and the
    convolutions' FLOPs over that time (pooling, upsampling, head and input
    packing included in the time), as a fraction of the measured BF16 dense
    peak (burst: the pass is timed on its own)."""
    import torch

    from paper_1809_08857_gb300 import mg, workloads as W

    pk, _ = peaks()
    net = mg.UNet(seed=0)
    net.set_scales(1.0, 1.0, 1.0)
    rho = torch.from_numpy(W.streamer_shell(n, 0)).to(dev)
    prev = torch.zeros_like(rho)
    out = torch.empty_like(rho)
    for _ in range(2):
        net.predict(rho, prev, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        net.predict(rho, prev, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    net.close()
    flops = mg.unet_conv_flops(1, n, n, n)
    tf = flops / (ms * 1e-3) / 1e12
    return {"workload": f"U-Net warm-start forward, {n}^3, channels 16/32/48/64",
            "ms": round(ms, 3), "conv_tflop": round(flops / 1e12, 3),
            "achieved_tflops": round(tf, 1), "peak_tflops": float(pk["bf16_tflops"]),
            "frac": round(tf / float(pk["bf16_tflops"]), 4),
            "note": "fraction of the measured BF16 dense (cuBLAS) burst peak"}


def measure_amr(dev, n0=256, reps=3):
    """One composite AMR Poisson solve (outside the timed region): the base
    grid n0^3 with the dielectric slab and three nested refined levels around
    the streamer channel and head (workloads.streamer_amr_layout), the shell
    charge sampled on every level, from zero to 1e-10 in mixed precision with
    three inner V-cycles per box and iteration (2: 7 iterations, 3: 5, the
    fastest; 4: 5, slower); device time per solve (CUDA events), FAC
    iterations, valid cells."""
    import numpy as np
    import torch

    from paper_1809_08857_gb300 import mg, workloads as W

    h0 = 1.0 / n0
    boxes = W.streamer_amr_layout(n0)
    eps = [torch.from_numpy(W.dielectric_slab(n0)).to(dev)] + [None] * len(boxes)
    rho = [W.streamer_shell_box((n0,) * 3, h0, (0, 0, 0), 0, thickness=h0)]
    for q, b in enumerate(boxes):
        o, h = W.amr_box_origin(h0, b)
        rho.append(W.streamer_shell_box(b[2], h, o, q + 1, thickness=h0))
    rho = [torch.from_numpy(r).to(dev) for r in rho]
    A = mg.Amr((n0,) * 3, h0, boxes, eps_r=eps, bc_kind=W.GAP_BC_KIND, bc_value=W.GAP_BC_VALUE,
               precision=mg.MG_PREC_MIXED, inner_cycles=3)
    u = [torch.zeros(s, dtype=torch.float64, device=dev) for s in A.shapes]
    A.solve("poisson", rho, u, tol=TOL)  # first call builds the coarse inverses
    st = None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        for t in u:
            t.zero_()
        st = A.solve("poisson", rho, u, tol=TOL)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    A.close()
    cells = sum(int(np.prod(s)) for s in A.shapes)
    valid = cells - sum(int(np.prod(b[2])) // 8 for b in boxes)
    return {"workload": f"streamer AMR: base {n0}^3 + 3 nested ratio-2 levels, composite "
                        "Poisson (dielectric slab, shell charge) 1e-10 from zero",
            "ms": round(ms, 2), "solves_per_s": round(1e3 / ms, 2),
            "fac_iterations": st["cycles"], "rel_resid": st["rel_resid"], "cells": cells,
            "valid_cells": valid, "valid_cells_per_s": round(valid * 1e3 / ms, 1)}


# ---------------------------------------------------------------- arms


def reference_config(args):
    return {"workload": f"poisson_slab_shell_{args.n}^3 + 3x helmholtz_{args.n}^3 (kappa L = 10, 100, 1000)",
            "grid": [args.n] * 3, "tol": TOL, "implementation": "FP64 C oracle (oracle/mg_oracle.c)",
            "precision": "fp64", "smoother": "red-black Gauss-Seidel V(2,2)",
            "coarsest": "exact solve of the coarsest grid", "threads": os.cpu_count() or 1,
            "device": "host CPU cores (OpenMP)", "guess": "zero"}


# whole oracle sets of the reference arm end within this many seconds (a set
# at 512^3 takes about 45 s on 16 Arm cores)
REFERENCE_BUDGET_S = 200.0


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    inputs = workload(args.n)
    t0 = time.perf_counter()
    sec, nsets, info, cores = oracle_sets(inputs, args.n, args.steps, REFERENCE_BUDGET_S)
    wall = time.perf_counter() - t0
    value = 1.0 / sec
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": nsets, "warmup": 0, "steps_requested": args.steps,
            "warmup_requested": args.warmup, "ms_per_step": 1e3 * sec,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded streamer shell, dielectric slab, smoothed ionisation source)",
            "config": reference_config(args), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": (f"{nsets} whole oracle solve set(s) at {args.n}^3 timed "
                                        f"one after another (no warm-up: plain CPU code), "
                                        f"cycles {[c for c, _ in info]}, "
                                        f"final rel. residuals {[f'{r:.2e}' for _, r in info]}; "
                                        f"stops before a set would end after "
                                        f"{REFERENCE_BUDGET_S:.0f} s")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": round(wall, 1)}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    rank, local, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    from paper_1809_08857_gb300 import build, mg

    build.build()
    mg.load()
    n = args.n
    h = 1.0 / n
    inputs = workload(n)
    rho = torch.from_numpy(inputs["rho"]).to(dev)
    eps = torch.from_numpy(inputs["eps"]).to(dev)
    S = torch.from_numpy(inputs["S"]).to(dev)
    prec = mg.MG_PREC_MIXED if args.precision == "mixed" else mg.MG_PREC_FP64
    solver = mg.Solver((n, n, n), h, eps_r=eps, precision=prec, inner_cycles=args.inner_cycles,
                       concurrency=args.concurrency, graphs=not args.no_graphs)
    tuned = None
    if args.ir_zchunk:
        solver.set_options(ir_zchunk=args.ir_zchunk)
    if not args.no_autotune:
        import tempfile as _tf

        from paper_1809_08857_gb300 import autotune

        cache = os.path.join(_tf.gettempdir(), f"mg_autotune_rank{rank}.json")
        tuned, _ = autotune.tuned(solver, rho, S, KAPPAS, TOL, has_eps=True, precision=prec,
                                  cache_path=cache)
    if args.coarse_visits:
        solver.set_options(coarse_visits=args.coarse_visits)
    if args.stack:
        solver.set_options(stack=1)
    phi = torch.zeros((n, n, n), dtype=torch.float64, device=dev)
    psi = [torch.zeros_like(phi) for _ in range(3)]
    cycles = [0, 0, 0, 0]
    history = [[], [], [], []]

    def step():
        phi.zero_()
        for p in psi:
            p.zero_()
        st = solver.solve_set(rho, phi, S, psi, KAPPAS, TOL)
        cycles[:] = [s["cycles"] for s in st]
        history[:] = [[float(f"{x:.3e}") for x in s["hist"]] for s in st]

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    l0 = mg.launch_count()
    with Clocks(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = mg.launch_count() - l0
    # each answer of the last timed set checked in plain FP64 (not by the
    # double-float refinement pass that decided to stop)
    fp64_check = fp64_residuals(solver, rho, phi, S, psi)
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms_per_step = ms / args.steps
    value = whole_job_rate(world, ms_per_step * 1e-3)

    # end to end through host buffers (pinned), copies inside the timed
    # region: every step uploads its rho and S and downloads its four
    # answers; as in a time-stepping run, the next step's inputs upload while
    # the current step solves and the finished step's answers download while
    # the next one solves (device buffers double-buffered, the solver and the
    # two copy directions on three streams)
    rho_h = torch.from_numpy(inputs["rho"]).pin_memory()
    S_h = torch.from_numpy(inputs["S"]).pin_memory()
    out_h = [torch.empty((n, n, n), dtype=torch.float64).pin_memory() for _ in range(4)]
    bufs = [{"rho": torch.empty_like(rho), "S": torch.empty_like(S),
             "out": [torch.empty_like(phi) for _ in range(4)]} for _ in range(2)]
    s_comp, s_h2d, s_d2h = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    # each array's copy is split into slabs over several streams, so that
    # more than one copy engine can carry a direction
    s_h2d_x = [s_h2d] + [torch.cuda.Stream() for _ in range(COPY_STREAMS - 1)]
    s_d2h_x = [s_d2h] + [torch.cuda.Stream() for _ in range(COPY_STREAMS - 1)]

    def split_copy(dst, src, streams, after):
        """dst <- src in len(streams) slabs along z, slab q on streams[q]
        (each stream first waits for the event `after`, if any); returns the
        events of the slabs."""
        nz_ = src.shape[0]
        evs = []
        for q, st_ in enumerate(streams):
            a_, b_ = q * nz_ // len(streams), (q + 1) * nz_ // len(streams)
            with torch.cuda.stream(st_):
                if after is not None:
                    st_.wait_event(after)
                dst[a_:b_].copy_(src[a_:b_], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(st_)
                evs.append(ev)
        return evs
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    solver.set_stream(s_comp)

    def h2d(i):
        b = bufs[i % 2]
        # step i - 2 no longer reads these buffers once its solve is done
        after = ev_done[i % 2] if i >= 2 else None
        evs = split_copy(b["rho"], rho_h, s_h2d_x, after) + split_copy(b["S"], S_h, s_h2d_x, after)
        with torch.cuda.stream(s_h2d):
            for ev in evs:
                s_h2d.wait_event(ev)
            ev_in[i % 2].record(s_h2d)

    def solve(i):
        b = bufs[i % 2]
        with torch.cuda.stream(s_comp):
            s_comp.wait_event(ev_in[i % 2])
            if i >= 2:
                s_comp.wait_event(ev_out[i % 2])  # step i - 2's answers are out
            for t in b["out"]:
                t.zero_()
            solver.solve_set(b["rho"], b["out"][0], b["S"], b["out"][1:], KAPPAS, TOL)
            ev_done[i % 2].record(s_comp)

    def d2h(i):
        b = bufs[i % 2]
        evs = []
        for o, d in zip(out_h, b["out"]):
            evs += split_copy(o, d, s_d2h_x, ev_done[i % 2])
        with torch.cuda.stream(s_d2h):
            for ev in evs:
                s_d2h.wait_event(ev)
            ev_out[i % 2].record(s_d2h)

    def e2e_run(k):
        h2d(0)
        for i in range(k):
            if i + 1 < k:
                h2d(i + 1)
            solve(i)
            d2h(i)
        s_d2h.synchronize()

    # this box's copy rates (1 GiB each way, on the leg's own streams): the
    # leg is copy-bound where they are low
    def copy_gbs(dst, src, stream):
        with torch.cuda.stream(stream):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dst.copy_(src, non_blocking=True)
            b.record(stream)
        b.synchronize()
        return round(src.numel() * src.element_size() / (a.elapsed_time(b) * 1e-3) / 1e9, 1)

    def split_gbs(dst, src, streams):
        torch.cuda.synchronize()
        t0_ = time.perf_counter()
        split_copy(dst, src, streams, None)
        torch.cuda.synchronize()
        return round(src.numel() * src.element_size() / (time.perf_counter() - t0_) / 1e9, 1)

    copy_gbs(bufs[0]["rho"], rho_h, s_h2d)
    rates = {"h2d_gbs": copy_gbs(bufs[0]["rho"], rho_h, s_h2d),
             "d2h_gbs": copy_gbs(out_h[0], bufs[0]["rho"], s_d2h),
             "streams": COPY_STREAMS,
             "h2d_gbs_split": split_gbs(bufs[0]["rho"], rho_h, s_h2d_x),
             "d2h_gbs_split": split_gbs(out_h[0], bufs[0]["rho"], s_d2h_x)}
    e2e_run(2)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e2e_run(args.e2e_steps)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    solver.set_stream(torch.cuda.current_stream())
    del bufs
    e2e_s = max_over_ranks(e2e_s, world, dev)
    cells = n ** 3
    e2e = {"value": whole_job_rate(world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": 2 * 8 * cells,
           "d2h_bytes_per_step": 4 * 8 * cells, "box_copy_rates": rates}

    # kernel profile (outside the timed region): one set at the timed
    # concurrency, then one set with the problems run one after another
    solver.profile(True)
    step()
    torch.cuda.synchronize()
    prof_overlap = solver.profile_read(reset=True)
    conc = solver.options.concurrency
    solver.set_options(concurrency=1)
    step()
    torch.cuda.synchronize()
    prof_serial = solver.profile_read(reset=True)
    solver.set_options(concurrency=conc)
    solver.profile(False)
    if prec == mg.MG_PREC_MIXED and not args.no_fp64_leg:
        extras_fp64 = measure_fp64_gpu(rho, eps, S, n, dev, phi, psi, value)
    else:
        extras_fp64 = None
    extras = measure_extras(solver, rho, eps, phi, n, dev)
    if extras_fp64:
        extras["fp64_gpu"] = extras_fp64
    extras["unet_forward"] = measure_unet(dev)
    if not args.no_amr:
        extras["amr_solve"] = measure_amr(dev)
    if not args.no_config3:
        extras["subboxes_256"] = measure_config3(dev)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("double-float (FP32 pairs) refinement over FP32 V-cycles; FP64 data"
                      if prec else "f64"),
            "data": "synthetic (seeded streamer shell, dielectric slab, smoothed ionisation source)",
            "config": dict(config(args), autotuned=tuned, nu1=solver.options.nu1,
                           nu2=solver.options.nu2, inner_cycles=solver.options.inner_cycles,
                           ir_zchunk=solver.options.ir_zchunk,
                           sweep_zchunk=solver.options.sweep_zchunk,
                           coarse_visits=max(1, solver.options.coarse_visits),
                           stack=solver.options.stack),
            "clocks": clk.summary(), "e2e": e2e,
            "gpu_launches": launches, "cycles_per_problem": cycles,
            "residual_per_step": history,
            "rel_resid_fp64": fp64_check,
            "roofline": roofline(prof_serial, prof_overlap, n), "kernel_profile": prof_serial,
            "extras": extras}
    solver.close()
    del solver
    torch.cuda.empty_cache()
    if not args.no_needle:
        extras["needle_plane_896"] = measure_needle_plane(dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res = oracle_baseline(inputs, n)
        line["cpu_baseline"] = {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")}
    emit(line, rank)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
