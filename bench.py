#!/usr/bin/env python3
"""Benchmark of the line-list -> cross-section hot path on GB300.

Workload (default): 1e8 synthetic lines, 8 temperatures x 4 pressures = 32
(T, P) conditions, Voigt (Humlicek w4), grid 0..10000 cm^-1 step 0.01
(1 000 001 points), cut 25 cm^-1, FP32 batched kernel.  One step = load the
unsorted line list into the engine (device radix sort + gather), Q(T) for the
8 temperatures, and the batched cross sections of all 32 conditions.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import xcsynth as xs  # noqa: E402

METRIC = "line x gridpoint Voigt evals/s (FP32 batched, 32 conditions)"
UNIT = "evals/s"
# Algorithmic FP32 flops of one region-I w4 evaluation with the per-line constants
# hoisted (about 10 operations and one reciprocal per line x point): the offset
# delta = (k - n) - f (2), u = delta^2 (1), t = u + E (1), D = u t + F (2),
# q = P u + PC (2), q / D (1), accumulate (1).
ALG_FLOPS_PER_EVAL = 10
# One tcgen05.mma of the far-wing kernel: M = 128 points, N = 32 conditions, K = 8.
MMA_FLOPS = 2 * 128 * 32 * 8
# TF32 dense tensor rate relative to BF16 (nominal 1.1 vs 2.25 PFLOP/s per GPU).
TF32_PER_BF16 = 1.1 / 2.25
# DRAM bytes of one k_far_tc launch from one ncu capture on the C3 generator at 1e6
# lines (profiles/k_far_tc_c3_1e6lines_32cond.md): reads grow with the line count,
# writes are the 32-condition output; scaled to the bench's line count.
TC_DRAM_READ_PER_LINE = 37.05e6 / 1e6
TC_DRAM_WRITE_1M_PTS_32C = 197.52e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="xc", choices=["xc", "reference"])
    ap.add_argument("--workload", default="C3")
    ap.add_argument("--lines", type=int, default=0, help="override the line count (smaller test runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--fp64-compare", action="store_true", help="also time the plain FP64 form on a subset")
    ap.add_argument("--profile", default=None, help="override the workload's line profile")
    ap.add_argument("--no-extras", action="store_true", help="skip the C1/C2/C4 secondary timings")
    ap.add_argument("--step", default="forward", choices=["forward", "adjoint"],
                    help="adjoint: time the FP32 adjoint of the workload (a seeded dL/dsigma) as the step instead "
                         "of load + cross sections (for profiling the adjoint kernel)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    if args.gpus > 1 or "RANK" in os.environ:
        import torch.distributed as dist
        rank = int(os.environ.get("RANK", 0))
        world = int(os.environ.get("WORLD_SIZE", 1))
        local = int(os.environ.get("LOCAL_RANK", 0))
        backend = "nccl" if args.impl == "xc" else "gloo"
        dist.init_process_group(backend, rank=rank, world_size=world)
        return dist, rank, world, local
    return None, 0, 1, 0


def workload_config(W, n, nc):
    return {"workload": f"{W.name}: {n} lines (nu uniform in ({W.nu_lo:g},{W.nu_hi:g}]), {nc} (T,P) "
                        f"conditions, grid {W.grid_lo:g}..{W.grid_hi:g} step {W.step:g} "
                        f"({W.n_points} pts), cut {W.cutoff:g} cm-1, {W.profile}, FP32 batched",
            "l2": "inputs larger than L2 (2.8 GB line list, 256 MB output)",
            "step": "device radix sort + gather of the unsorted list, Q(T), batched cross sections"}


def make_workload(args, rank):
    W = xs.WORKLOADS[args.workload]
    n = args.lines or W.n_lines
    seed = W.seed + 1000 * rank  # each rank its own independent problem (weak scaling)
    t0 = time.time()
    lines = xs.gen_lines(seed, 0, n, W.nu_lo, W.nu_hi)
    E, g = xs.gen_states(seed, W.n_states)
    return W, n, seed, lines, E, g, time.time() - t0


# ---------------------------------------------------------------------------- reference arm
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def cpu_oracle_rate(W, lines, E, g, conds, budget_s=12.0, threads=None):
    """Time the FP64 oracle (as it stands) on a bounded sample: the first lines of the
    list, doubling until the run takes a few seconds; return evals/s."""
    import oracle
    oracle.build()
    threads = threads or (os.cpu_count() or 1)
    n_try = 500
    total = len(lines["nu"])
    best = None
    while True:
        sub = {k: v[:n_try] for k, v in lines.items()}
        c = conds[len(conds) // 2]
        Q, dQ = oracle.partition_function(E, g, c["T"])
        oc = oracle.make_condition(c["T"], c["P"], Q, dQ, mass_da=W.mass_da)
        op = oracle.make_opts(W.profile, W.cutoff, W.cutoff_width_mult, W.n_gh)
        ev = oracle.count_evals(sub, oc, W.grid_lo, W.step, W.n_points, op)
        t0 = time.perf_counter()
        oracle.cross_section(sub, oc, W.grid_lo, W.step, W.n_points, op, nthreads=threads)
        dt = time.perf_counter() - t0
        best = (ev / dt, n_try, ev, dt)
        if dt > budget_s / 4 or n_try >= total:
            break
        n_try = min(total, n_try * 4 if dt < budget_s / 40 else n_try * 2)
    return {"value": best[0], "unit": UNIT, "cores": threads, "cpu": cpu_model(), "kind": "oracle",
            "seconds": best[3],
            "sample": f"first {best[1]} lines of the {W.name} list, 1 of {len(conds)} conditions, "
                      f"full grid ({best[2]:.3g} evals in {best[3]:.1f} s)"}


# Modelled HBM traffic of the line-list sort (bytes per line): key making (read nu 8 B,
# write key 8 + index 4), one histogram pass over the keys (8), 8 LSD digit passes
# (tile histogram 8 + scatter read 12 + write 12), gather (index 4 + 28 read + 28 write).
SORT_BYTES_PER_LINE = 20 + 8 + 8 * 32 + 60
# Standalone FP64 line parameters: read nu, E'', A, g', gamma_ref, n (26 B), write I, alpha, gamma (24 B).
PARAMS_BYTES_PER_LINE = 26 + 24


def hbm_stages(eng, xc, torch, dev, n, cond, sort_ms, gather_ms):
    """The HBM-bound steps with their achieved bandwidth against the measured copy
    peak: the device sort + gather of the line list (CUDA events of the load) and a
    standalone FP64 line-parameter pass over the whole sorted list."""
    pk, basis = peaks()
    out = {"peak_gbs": pk["hbm_gbs"], "peak_basis": basis}
    sb = SORT_BYTES_PER_LINE * n
    out["sort_gather"] = {"ms": sort_ms + gather_ms, "modelled_bytes": sb,
                          "gbs": sb / ((sort_ms + gather_ms) / 1e3) / 1e9,
                          "frac": sb / ((sort_ms + gather_ms) / 1e3) / 1e9 / pk["hbm_gbs"],
                          "model": "20 + 8 + 8 x 32 + 60 B per line (keys, histogram, 8 digit passes, gather)"}
    I = torch.empty(n, dtype=torch.float64, device=dev)
    a = torch.empty_like(I)
    g = torch.empty_like(I)
    ms = _timed(torch, lambda: eng.line_params_device(cond, I, a, g))
    pb = PARAMS_BYTES_PER_LINE * n
    out["line_params_fp64"] = {"ms": ms, "bytes": pb, "gbs": pb / (ms / 1e3) / 1e9,
                               "frac": pb / (ms / 1e3) / 1e9 / pk["hbm_gbs"]}
    del I, a, g
    return out


def run_reference(args, dist, rank, world):
    if rank != 0:
        return
    W, n, seed, lines, E, g, _ = make_workload(args, rank)
    conds = xs.conditions_for(W)
    threads = os.cpu_count() or 1
    vals, secs = [], []
    for i in range(args.warmup + args.steps):
        r = cpu_oracle_rate(W, lines, E, g, conds, budget_s=8.0, threads=threads)
        if i >= args.warmup:
            vals.append(r["value"])
            secs.append(r["seconds"])
    v = statistics.median(vals)
    # evals of one full step of the workload, at the oracle's rate
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(W, n, len(conds)),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "cpu": cpu_model(), "kind": "oracle",
                         "sample": r["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------- GB300 arm
def _timed(torch, fn, reps=1):
    fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def secondary_measurements(xc, torch, dev):
    """The other workloads, one timing each (CUDA events, device-resident inputs):
    C1 (1e5 lines, FP64 plain and FP32), C2 (1e7 lines, width-limited cut, Voigt w4
    FP64 plain and FP32; GH binned, binned Gaussian and binned Lorentzian FP32; Voigt w4 FP32
    emission and with the HITRAN threshold, whose eval count still includes the lines it
    leaves out, and with a two-broadener mixture; the Vectorized Voigt with beta), C4 (1e7 lines, 2x2 conditions: FP32
    forward and FP32 adjoint).  Values are evals/s over the exact eval count."""
    out = {}
    for name in ("C1", "C2", "C4"):
        W = xs.WORKLOADS[name]
        L = {k: torch.from_numpy(v).to(dev) for k, v in xs.gen_lines(W.seed, 0, W.n_lines, W.nu_lo, W.nu_hi).items()}
        E, g = xs.gen_states(W.seed, W.n_states)
        eng = xc.Engine(dev.index or 0)
        eng.load_lines(L)
        eng.set_states(E, g)
        grid = xc.make_grid(W.grid_lo, W.step, W.n_points)
        conds = [xc.make_condition(c["T"], c["P"], mass_da=W.mass_da) for c in xs.conditions_for(W)]
        sig = torch.empty((len(conds), W.n_points), dtype=torch.float64, device=dev)
        res = {}
        cases = [("voigt_w4", "fp32", {})] if name == "C4" else [("voigt_w4", "fp64", {}), ("voigt_w4", "fp32", {})]
        if name == "C2":
            cases += [("voigt_gh_binned", "fp32", {}), ("doppler_binned", "fp32", {}), ("lorentz_binned", "fp32", {}),
                      ("voigt_w4", "fp32", {"quantity": "emission"}),
                      ("voigt_w4", "fp32", {"threshold": ("hitran", 2000.0, 1e-29)}),
                      ("voigt_vv", "fp32", {"vv_beta": True})]
        for prof, prec, kw in cases:
            o = xc.make_opts(prof, prec, W.cutoff, W.cutoff_width_mult, W.n_gh, **kw)
            ev = eng.count_evals(conds, grid, o)
            ms = _timed(torch, lambda: eng.cross_section_batched(conds, grid, o, sig))
            tag = "_emission" if kw.get("quantity") == "emission" else ("_hitran_threshold" if "threshold" in kw else
                                                                         ("_beta" if kw.get("vv_beta") else ""))
            res[f"{prof}_{prec}{tag}"] = {"ms": ms, "evals": ev, "evals_per_s": ev / (ms / 1e3)}
        if name == "C2":
            # the plain FP64 form of binned GH (20 atan2 per evaluation at the FP64 rate: about 40 s
            # over the whole grid) on the 1000 cm^-1 slice 5000..6000 with every line loaded (the
            # same line density), for the FP32 / FP64 ratio in evals/s
            o = xc.make_opts("voigt_gh_binned", "fp64", W.cutoff, W.cutoff_width_mult, W.n_gh)
            sg = xc.make_grid(W.grid_lo + 500000 * W.step, W.step, 100001)
            s1 = torch.empty((len(conds), sg.n), dtype=torch.float64, device=dev)
            ev = eng.count_evals(conds, sg, o)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            eng.cross_section_batched(conds, sg, o, s1)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            res["voigt_gh_binned_fp64_slice_5000_6000"] = {"ms": ms, "evals": ev, "evals_per_s": ev / (ms / 1e3)}
            res["voigt_gh_binned_fp32_over_fp64"] = res["voigt_gh_binned_fp32"]["evals_per_s"] / (ev / (ms / 1e3))
            del s1
            # Lorentz widths from a two-broadener mixture (an a0 table by J'' and a constant)
            a0 = {j: (0.09 - 0.001 * j, 0.75 - 0.004 * j) for j in range(0, 80)}
            eng.set_broadening([xc.make_broadener("a0", 0.8, 0.07, 0.5, a0),
                                xc.make_broadener("constant", 0.2, 0.03, 0.7)])
            o = xc.make_opts("voigt_w4", "fp32", W.cutoff, W.cutoff_width_mult, W.n_gh)
            ev = eng.count_evals(conds, grid, o)
            ms = _timed(torch, lambda: eng.cross_section_batched(conds, grid, o, sig))
            res["voigt_w4_fp32_broadener_mixture"] = {"ms": ms, "evals": ev, "evals_per_s": ev / (ms / 1e3)}
            eng.set_broadening([])
        if name == "C4":
            o = xc.make_opts("voigt_w4", "fp32", W.cutoff)
            gs = torch.ones((len(conds), W.n_points), dtype=torch.float64, device=dev)
            ev = eng.count_evals(conds, grid, o)
            ms = _timed(torch, lambda: eng.cross_section_vjp(conds, grid, o, gs, per_line=True))
            res["vjp_voigt_w4_fp32"] = {"ms": ms, "evals": ev, "evals_per_s": ev / (ms / 1e3)}
        out[name] = res
        eng.close()
        del L, sig
        torch.cuda.empty_cache()
    return out


def c5_measurement(xc, torch, dev):
    """The maximum-size workload: 1e9 lines (nu in (0, 20000], 2000 K, 1 bar), grid 0..20000
    step 0.01 (2 000 001 points), cut 25, generated on the device by the seeded generator
    and loaded (device radix sort) through the C ABI.  FP32 (the batched kernel) is timed
    over the whole grid.  The plain FP64 kernel (about 7 minutes over the whole grid) is
    timed on the 1000 cm^-1 slice 10000..11000 with every line loaded (the same line
    density; 391 FP64 windows, enough to fill the GPU), and FP32 / FP64 compares the two
    rates in evals/s; the FP32 sweep's own values on that slice are compared with the FP64
    ones (max relative difference above 1e-6 of the peak, and integrated band).  Device
    memory is the free-memory drop while the lines, the sorted copy, the sort scratch and
    the sweep's scratch are all held."""
    W = xs.WORKLOADS["C5"]
    free0, total = torch.cuda.mem_get_info(dev)
    if free0 < 140e9:
        return {"skipped": f"needs about 140 GB of free device memory ({free0 / 1e9:.0f} GB free)"}
    t0 = time.time()
    dl = xs.gen_lines_torch(W.seed, 0, W.n_lines, W.nu_lo, W.nu_hi, device=dev)
    torch.cuda.synchronize()
    t_gen = time.time() - t0
    E, g = xs.gen_states(W.seed, W.n_states)
    eng = xc.Engine(dev.index or 0)
    eng.set_timing(True)
    eng.load_lines(dl)
    tl = eng.timings()
    eng.set_states(E, g)
    c = xs.conditions_for(W)[0]
    cond = [xc.make_condition(c["T"], c["P"], mass_da=W.mass_da)]
    out = {"lines": W.n_lines, "generation_s": round(t_gen, 1), "sort_ms": tl["sort"], "gather_ms": tl["gather"]}
    grid = xc.make_grid(W.grid_lo, W.step, W.n_points)
    o32 = xc.make_opts("voigt_w4", "fp32", W.cutoff)
    o64 = xc.make_opts("voigt_w4", "fp64", W.cutoff)
    sig = torch.empty((1, W.n_points), dtype=torch.float64, device=dev)
    ev = eng.count_evals(cond, grid, o32)
    ms = _timed(torch, lambda: eng.cross_section_batched(cond, grid, o32, sig))
    out["fp32_full_grid"] = {"ms": ms, "evals": ev, "evals_per_s": ev / (ms / 1e3)}
    out["device_memory_gb"] = (free0 - torch.cuda.mem_get_info(dev)[0]) / 1e9
    k0, m = 1000000, 100001
    slice_grid = xc.make_grid(W.grid_lo + k0 * W.step, W.step, m)
    s64 = torch.empty((1, m), dtype=torch.float64, device=dev)
    evs = eng.count_evals(cond, slice_grid, o64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    eng.cross_section_batched(cond, slice_grid, o64, s64)
    e1.record()
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    a, b = sig[0, k0:k0 + m].cpu().numpy(), s64[0].cpu().numpy()
    mk = b > 1e-6 * b.max()
    r64 = evs / (ms64 / 1e3)
    out["fp64_plain_slice_10000_11000"] = {
        "evals": evs, "ms": ms64, "evals_per_s": r64,
        "fp32_vs_fp64_max_rel": float(np.max(np.abs(a[mk] - b[mk]) / b[mk])),
        "fp32_vs_fp64_band": float(abs(a.sum() - b.sum()) / b.sum())}
    out["fp32_over_fp64"] = out["fp32_full_grid"]["evals_per_s"] / r64
    eng.close()
    del dl, sig, s64
    torch.cuda.empty_cache()
    return out


def run_adjoint_step(args, eng, dlines, conds, grid, opts, torch, dev, W, n):
    """The FP32 adjoint as the timed step (lines resident and sorted; a seeded dL/dsigma):
    one JSON line with its evals/s, for profiling the adjoint kernel."""
    eng.load_lines(dlines)
    gs = torch.from_numpy(np.random.default_rng(9).standard_normal((len(conds), W.n_points))).to(dev)
    evals = eng.count_evals(conds, grid, opts)
    for _ in range(args.warmup):
        eng.cross_section_vjp(conds, grid, opts, gs, per_line=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        eng.cross_section_vjp(conds, grid, opts, gs, per_line=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"metric": "adjoint (VJP) line x gridpoint evals/s, FP32", "value": evals / (ms / 1e3),
                      "unit": UNIT, "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
                      "config": {"workload": f"{W.name}: {n} lines, {len(conds)} conditions, {W.n_points} points, "
                                             f"adjoint with per-line outputs"}}), flush=True)


def run_xc(args, dist, rank, world, local):
    import torch
    import paper_1801_09803_gb300 as xc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    xc.build.build()
    W, n, seed, lines, E, g, t_gen = make_workload(args, rank)
    conds_py = xs.conditions_for(W)
    conds = [xc.make_condition(c["T"], c["P"], mass_da=W.mass_da) for c in conds_py]
    grid = xc.make_grid(W.grid_lo, W.step, W.n_points)
    if args.profile:
        W.profile = args.profile
    opts = xc.make_opts(W.profile, "fp32", W.cutoff, W.cutoff_width_mult, W.n_gh)
    nc = len(conds)

    # inputs resident in HBM (unsorted, as generated) and pinned host copies for e2e
    dlines = {k: torch.from_numpy(v).to(dev) for k, v in lines.items()}
    sigma = torch.empty((nc, W.n_points), dtype=torch.float64, device=dev)
    eng = xc.Engine(local)
    eng.set_states(E, g)
    eng.set_timing(True)

    def step_device():
        eng.load_lines(dlines)
        eng.cross_section_batched(conds, grid, opts, sigma)

    if args.step == "adjoint":
        run_adjoint_step(args, eng, dlines, conds, grid, opts, torch, dev, W, n)
        return

    # algorithmic work: pairs (line, grid point) inside the cut, summed over conditions
    eng.load_lines(dlines)
    evals = eng.count_evals(conds, grid, opts)
    far_evals = eng.count_far_evals(conds, grid, opts)   # the tensor-core kernel's share (0 if it does not run)

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    prof_ms, core_ms, sweep_ms, launches = [], [], [], 0
    kern = []   # per step: (far-wing tensor ms, CUDA-core ms, centre-zone ms, MMA count)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step_device()
            t = eng.timings()
            prof_ms.append(t["profile"])
            core_ms.append(t["ranges_or_core"])
            sweep_ms.append(t["params_or_sweep"])
            kern.append(eng.sweep_kernels())
            launches += eng.last_launch_count()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # load_lines' own launch count is reset by the batched call; count it separately
    eng.load_lines(dlines)
    load_launches = eng.last_launch_count()
    sort_t = eng.timings()
    launches += load_launches * args.steps
    if dist:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = evals * args.steps * world / (ms / 1e3)

    # end-to-end through the public API with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        hl = {k: torch.from_numpy(v).pin_memory().numpy() for k, v in lines.items()}
        hout = torch.empty((nc, W.n_points), dtype=torch.float64).pin_memory().numpy()
        h2d = sum(v.nbytes for v in hl.values())
        d2h = hout.nbytes
        eng.load_lines(hl)
        eng.cross_section_batched(conds, grid, opts, hout)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            eng.load_lines(hl)
            eng.cross_section_batched(conds, grid, opts, hout)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if dist:
            t = torch.tensor([dt], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": evals * args.steps * world / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": dt * 1e3 / args.steps}

    # FP64 plain form on the same GPU (subset of conditions) for the FP32 vs FP64 ratio
    fp64 = None
    if args.fp64_compare:
        o64 = xc.make_opts(W.profile, "fp64", W.cutoff, W.cutoff_width_mult, W.n_gh)
        eng.load_lines(dlines)
        c1 = conds[:1]
        s1 = torch.empty((1, W.n_points), dtype=torch.float64, device=dev)
        eng.cross_section_batched(c1, grid, o64, s1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eng.cross_section_batched(c1, grid, o64, s1)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ev1 = eng.count_evals(c1, grid, o64)
        fp64 = {"value": ev1 / dt, "unit": UNIT, "conditions": 1}

    extras = None
    if not args.no_extras and rank == 0:
        extras = secondary_measurements(xc, torch, dev)
        extras["C5"] = c5_measurement(xc, torch, dev)

    if rank != 0:
        return
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or 0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    # the two profile kernels together (main region-I kernel + w4 centre-zone kernel):
    # the algorithmic eval count covers both
    prof = (statistics.mean(prof_ms) + (statistics.mean(core_ms) if core_ms else 0.0)) if prof_ms else None
    peak_max = nsm * 128 * 2 * 2070e6 / 1e12
    rl = sweep_rl = None
    if prof:
        ach = evals * ALG_FLOPS_PER_EVAL / (prof / 1e3) / 1e12
        sweep_rl = {"bound": "alu", "achieved": ach, "peak": peak_max, "unit": "TFLOP/s", "frac": ach / peak_max,
                    "traffic": None,
                    "kernel": "all profile kernels of the sweep (CUDA events inside the graph), algorithmic flops",
                    "peak_basis": f"{nsm} SMs x 128 FP32 lanes x 2 flop x 2070 MHz (max SM clock)",
                    "frac_at_sampled_clock": (ach / (nsm * 128 * 2 * sm_mhz * 1e6 / 1e12)) if sm_mhz else None,
                    "flops_per_eval": ALG_FLOPS_PER_EVAL, "kernel_ms": prof}
        rl = sweep_rl
    per_kernel = None
    if kern and kern[0][3] > 0:
        far_ms = statistics.mean(k[0] for k in kern)
        main_ms = statistics.mean(k[1] for k in kern)
        cz_ms = statistics.mean(k[2] for k in kern)
        mma = kern[-1][3]
        per_kernel = {"k_far_tc": far_ms, "k_gather_f32": main_ms, "k_core_w4_f32": cz_ms, "mma_per_launch": mma}
        pk, basis = peaks()
        tf32_peak = pk["bf16_tflops"] * TF32_PER_BF16
        nfar = far_evals
        per_kernel["far_evals_per_launch"] = nfar
        ach = nfar * ALG_FLOPS_PER_EVAL / (far_ms / 1e3) / 1e12
        issued = mma * MMA_FLOPS / (far_ms / 1e3) / 1e12
        dominant = max(("k_far_tc", "k_gather_f32", "k_core_w4_f32"), key=lambda k: per_kernel[k])
        traffic = None
        if args.workload == "C3" and not args.profile:
            traffic = TC_DRAM_READ_PER_LINE * n + TC_DRAM_WRITE_1M_PTS_32C * (nc / 32) * (W.n_points / 1e6)
        rl = {"bound": "tensor", "achieved": ach, "peak": tf32_peak, "unit": "TFLOP/s", "frac": ach / tf32_peak,
              "traffic": traffic,
              "traffic_basis": "dram read + write bytes per launch from one ncu capture at 1e6 lines, read part "
                               "scaled by the line count (profiles/k_far_tc_c3_1e6lines_32cond.md)",
              "kernel": "k_far_tc (tcgen05.mma kind::tf32, far wings)",
              "peak_basis": f"TF32 dense = {basis} BF16 burst {pk['bf16_tflops']} TFLOP/s x 1.1/2.25 (nominal ratio)",
              "flops": f"algorithmic: the far-wing kernel's evaluations ({nfar:.4g} per launch, "
                       f"{nfar / evals:.3f} of the step's evals) x {ALG_FLOPS_PER_EVAL} flops per region-I eval",
              "issued": {"value": issued, "unit": "TFLOP/s", "frac": issued / tf32_peak,
                         "flops": "executed MMA flops: MMAs per launch x 2 x 128 x 32 x 8 (operand splits and "
                                  "zero B entries included)"},
              "kernel_ms": far_ms, "dominant_kernel_of_sweep": dominant}
    cpu = None
    if not args.no_cpu:
        cpu = cpu_oracle_rate(W, lines, E, g, conds_py)
        one = cpu_oracle_rate(W, lines, E, g, conds_py, budget_s=4.0, threads=1)
        cpu["single_thread"] = {"value": one["value"], "unit": UNIT, "sample": one["sample"]}
    hbm = None
    if not args.no_extras:
        eng.load_lines(dlines)
        hbm = hbm_stages(eng, xc, torch, dev, n, conds[len(conds) // 2], sort_t["sort"], sort_t["gather"])
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(W, n, nc), evals_per_step=evals, generation_s=round(t_gen, 1)),
        "e2e": e2e, "roofline": rl, "roofline_sweep_alu": sweep_rl if rl is not sweep_rl else None,
        "hbm_stages": hbm,
        "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": int(launches),
        "stage_ms": {"sort": sort_t["sort"], "gather": sort_t["gather"],
                     "main_kernel_mean": statistics.mean(prof_ms) if prof_ms else None,
                     "centre_zone_kernel_mean": statistics.mean(core_ms) if core_ms else None,
                     "profile_kernels_mean": prof,
                     "sweep_mean": statistics.mean(sweep_ms) if sweep_ms else None,
                     "per_kernel_mean": per_kernel},
        "tuning": eng.tuning(),
    }
    if extras:
        out["other_workloads"] = extras
    if fp64:
        out["fp64_plain"] = fp64
        out["fp32_over_fp64"] = (evals / (prof / 1e3)) / fp64["value"] if prof else None
    print(json.dumps(out), flush=True)
    eng.close()


def main():
    args = parse()
    dist, rank, world, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, dist, rank, world)
    else:
        run_xc(args, dist, rank, world, local)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
