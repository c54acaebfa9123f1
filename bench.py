"""Benchmark: DOF/s to a 1e-10 relative residual on the 3D Poisson 257^3
workload (255^3 unknowns, 7-point FD, f = U[-1,1] seed 2, plain FP64 V(2,2)
red-black Gauss-Seidel, full weighting, trilinear prolongation, coarsest 3^3
solved exactly).  One step = one whole solve from u = 0.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU FP64
oracle on this host's cores on the same workload instead.
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
sys.path.insert(0, ROOT)

METRIC = "DOF/s to 1e-10 rel. residual (FP64-accurate) and HBM GB/s vs peak, per form"
D, N, SEED, RTOL = 3, 256, 2, 1e-10
WORKLOAD = ("3D Poisson -Lap u = f, 257^3 grid (255^3 = 16.58M unknowns), 7-point FD, zero "
            "Dirichlet, f = U[-1,1] i.i.d. (seed 2), plain FP64 V(2,2) red-black GS, 27-point "
            "full weighting, trilinear prolongation, coarsest 3^3 exact, to relative residual 1e-10")
# The headline solver: each FP64 V(2,2) cycle evaluated as a double-float
# V-cycle inside FP64 iterative refinement (GMG_DF_IR, one inner cycle per
# cycle): the FP64 step (residual, update, norm) after a solve's first cycle
# and then every 8 cycles, the stopping test after every cycle; the FP64
# cycle to within 1e-12 per cycle, the oracle's cycle count.
HEADLINE = dict(precision="df", inner_cycles=1)
HEADLINE_NOTE = ("each V(2,2) cycle as a double-float (2 x FP32) V-cycle inside FP64 iterative "
                 "refinement: FP64 residual, update and norm after the first cycle and then "
                 "every 8 cycles, the stopping test after every cycle; the FP64 cycle to "
                 "<= 1e-12 per cycle vs the FP64 oracle, identical cycle count")
UNKNOWNS = (N - 1) ** D
# FP64 pipe: 2 DFMA/DADD issue slots per clock per SM (GB300 nominal 1.25 TFLOP/s FP64 =
# 2 flop x 2 inst/clk x 152 SMs x 2.07 GHz), 152 SMs, 2070 MHz max SM clock.
FP64_INST_PER_CLK_SM = 2
NUM_SMS = 152
SM_MAX_MHZ = 2070.0
# DRAM bytes (read + write) per launch of the level-0 red-black half sweep of
# the 257^3 FP64 solve, from one ncu capture of the current kernel
# (dram__bytes_read.sum + dram__bytes_write.sum: 269.5 MB + 85.8 MB)
# FP64 instructions of one updated node (adds, fmas) of the FP64 level
# kernels that can dominate a solve: the diagonal-walker half sweep executes
# 4 + 1/4 adds and one fma per node
FP64_MIX = {"rb_half": (4.25, 1.0), "resnorm_red_sweep": (5.25, 2.0), "residual": (5.25, 1.0),
            # double-float step: black 3 adds; red 4.25 + 3 adds, 3 fmas (per node, both halves)
            "outer_red_update_df": (10.25, 3.0)}
# DRAM bytes (read + write) per launch at 257^3 from one ncu capture each
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by (kernel record,
# level); a kernel changed since its capture has no entry.
TRAFFIC = {
    ("rb_half", 0): 356.4e6,  # FP64 walker half sweep: 269.5 + 85.8 MB
    # double-float step's outer kernels: k_black_exact_update 331.4 + 213.1 MB,
    # k_outer_red3_walk 345.2 + 213.0 MB
    ("outer_red_update_df", 0): 1102.7e6,
    # level-0 double-float half sweep (k_rb_half_vec_df): 143.2 + 42.3 MB
    ("rb_half_df", 0): 185.5e6,
}


def fp64_bound(name: str) -> bool:
    """Kernels whose arithmetic runs on the FP64 pipe: the plain FP64 level
    kernels and every refinement form's outer residual / update."""
    if name.startswith(("outer_", "update")):
        return True
    return not name.endswith(("_df", "_f32", "_bf16"))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.monotonic(), [x.strip() for x in line.split(",")]))

    def mark(self, name):
        setattr(self, name, time.monotonic())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        """Samples taken between mark("t0") and mark("t1") (the timed region)."""
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "t0", 0.0), getattr(self, "t1", float("inf"))
        for ts, r in self.rows:
            if not (t0 <= ts <= t1 + 0.15):
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dominant(stats):
    """The (kernel, level) record with the largest summed device time: its
    kernel name, the record and its share of all kernel time."""
    rec = max(stats, key=lambda r: r["ms"])
    return rec["kernel"], rec, rec["ms"] / sum(r["ms"] for r in stats)


def time_solves(torch, S, f, u, steps, warmup, timing=True):
    """Warm-up, then `steps` solves from u = 0 bracketed by CUDA events on
    torch's stream (each solve ends with the library's stream drained),
    without per-kernel events.  With `timing`, the same `steps` solves run
    once more with per-kernel events (event nodes inside the cycle graphs,
    which lengthen each solve) for the per-kernel records; the returned
    ms/step is always the uninstrumented one."""
    stream = torch.cuda.current_stream()

    def region():
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            u.zero_()
            out = S.solve(f, u, RTOL)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, out

    S.set_timing(False)
    for _ in range(warmup):
        u.zero_()
        it, rel, conv = S.solve(f, u, RTOL)
        assert conv, "warm-up solve did not converge"
    ms, (it, rel, conv) = region()
    stats, launches = [], None
    if timing:
        S.set_timing(True)
        u.zero_()
        S.solve(f, u, RTOL)
        S.timing_reset()
        region()
        stats, launches = S.timing_report()
        S.set_timing(False)
    return ms, it, rel, stats, launches


def run_forms(torch, args):
    """The 3D 513^3 workload (3 pi^2 prod sin + 0.01 N(0,1), seed 3), RB-GS
    V(2,2): plain FP64 cycles vs FP32 and BF16-storage cycles inside FP64
    iterative refinement, each to relative residual 1e-10."""
    from paper_1208_4247_gb300 import inputs
    from paper_1208_4247_gb300.gmg import Solver
    d, n = 3, 512
    dof = (n - 1) ** d
    f = torch.from_numpy(inputs.rhs_sine_plus_gauss(d, n, 3)).cuda()
    u = torch.zeros_like(f)
    pk, _ = peaks()
    from paper_1208_4247_gb300.autotune import tune_inner_cycles
    out = {}
    tuned = {}
    for prec, ks in (("fp32", (1, 2, 3, 4, 5)), ("bf16", (1, 2, 3))):
        tuned[prec] = tune_inner_cycles(d, n, f, u, prec, ks=ks)
    for name, prec, k in [("fp64_plain", "fp64", 0), ("df_ir", "df", 1),
                          ("fp32_ir", "fp32", tuned["fp32"][0]),
                          ("bf16_ir", "bf16", tuned["bf16"][0])]:
        S = Solver(d, n, precision=prec, inner_cycles=max(k, 1))
        ms, it, rel, stats, launches = time_solves(torch, S, f, u, args.form_steps, 1)
        S.close()
        dom, rec, share = dominant(stats)
        avg_s = rec["ms"] / rec["launches"] * 1e-3
        alg = sum(r["bytes"] * r["launches"] for r in stats) / args.form_steps
        out[name] = {"value": dof / (ms * 1e-3), "unit": "DOF/s", "ms_per_step": ms,
                     "steps": args.form_steps, "outer_steps" if k else "cycles": it,
                     "inner_cycles_per_step": k or None, "relres": rel,
                     "solve_alg_gbs": alg / (ms * 1e-3) / 1e9,
                     "dominant_kernel": f"{dom} (level {rec['level']})",
                     "dominant_share": share,
                     "dominant_hbm_gbs": rec["bytes"] / avg_s / 1e9,
                     "dominant_hbm_frac": rec["bytes"] / avg_s / 1e9 / pk["hbm_gbs"],
                     "gpu_launches": launches}
    base = out["fp64_plain"]["ms_per_step"]
    for v in out.values():
        v["speedup_vs_fp64_plain"] = base / v["ms_per_step"]
    for prec, name in (("fp32", "fp32_ir"), ("bf16", "bf16_ir")):
        out[name]["autotune_ms_by_inner_cycles"] = tuned[prec][1]
    del f, u
    torch.cuda.empty_cache()
    return {"workload": "3D 513^3 (511^3 = 133.4M unknowns), f = 3 pi^2 prod sin + 0.01 N(0,1) "
                        "seed 3, RB-GS V(2,2), FW, trilinear, to relative FP64 residual 1e-10",
            "forms": out}


def run_batch(torch, args):
    """512 independent solves (seed 4): 2D (2^k+1)^2 k = 6..10 and 3D (2^k+1)^3
    k = 4..7, f = U[-1,1]; FP32 weighted-Jacobi V(1,1) cycles (omega 4/5 in 2D,
    6/7 in 3D) in FP64 refinement, one launch per level index over the batch,
    autotuned inner cycles / tile / CTAs; against the same solves one by one."""
    from paper_1208_4247_gb300 import inputs
    from paper_1208_4247_gb300.autotune import tune_batch
    from paper_1208_4247_gb300.gmg import Batch, Solver
    mix = inputs.batch_mix(512, 4)
    dims = [d for d, _ in mix]
    ns = [n for _, n in mix]
    dof = sum((n - 1) ** d for d, n in mix)
    fd = [torch.from_numpy(f).cuda() for f in inputs.batch_rhs(mix, 4)]
    ud = [torch.zeros_like(f) for f in fd]
    # weighted Jacobi with omega = 0: 4/5 for the 2D solves, 6/7 for the 3D ones
    kw = dict(smoother="wjacobi", omega=0.0, nu1=1, nu2=1, precision="fp32")
    best, tried = tune_batch(dims, ns, fd, ud, **kw)
    B = Batch(dims, ns, inner_cycles=best["inner_cycles"], chunk=best["chunk"], ctas=best["ctas"],
              **kw)
    B.set_timing(False)

    def run():
        for u in ud:
            u.zero_()
        return B.solve(fd, ud, RTOL)

    run()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(args.form_steps):
        it, rel, steps, conv = run()
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.form_steps
    # per-kernel records from an event-instrumented repeat
    B.set_timing(True)
    run()
    B.set_timing(True)
    for _ in range(args.form_steps):
        run()
    torch.cuda.synchronize()
    stats, launches = B.timing_report()
    B.close()
    hist = {}
    for v in it:
        hist[v] = hist.get(v, 0) + 1
    # the same solves one by one (same precision, smoother, sweeps, inner cycles)
    def om(d):
        return 0.8 if d == 2 else 6.0 / 7.0

    solvers = [Solver(d, n, smoother="wjacobi", omega=om(d), nu1=1, nu2=1, precision="fp32",
                      inner_cycles=best["inner_cycles"]) for d, n in mix]

    def one_by_one():
        for S, f, u in zip(solvers, fd, ud):
            u.zero_()
            S.solve(f, u, RTOL)

    one_by_one()
    torch.cuda.synchronize()
    e0.record(s)
    one_by_one()
    e1.record(s)
    torch.cuda.synchronize()
    ms1 = e0.elapsed_time(e1)
    for S in solvers:
        S.close()
    # and one by one in plain FP64 (weighted Jacobi V(1,1))
    solvers = [Solver(d, n, smoother="wjacobi", omega=om(d), nu1=1, nu2=1) for d, n in mix]
    one_by_one()
    torch.cuda.synchronize()
    e0.record(s)
    one_by_one()
    e1.record(s)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    for S in solvers:
        S.close()
    del fd, ud
    torch.cuda.empty_cache()
    dom, rec, share = dominant(stats)
    return {"workload": "512 solves, seeded mix of 2D (2^k+1)^2 k=6..10 and 3D (2^k+1)^3 k=4..7, "
                        "f = U[-1,1]; FP32 WJ V(1,1) (omega 4/5 2D, 6/7 3D) in FP64 refinement",
            "unknowns": dof, "value": dof / (ms * 1e-3), "unit": "DOF/s", "ms_per_step": ms,
            "steps": args.form_steps, "batch_steps": steps, "converged": conv,
            "max_relres": max(rel), "completion_steps_histogram": hist,
            "autotuned": best, "autotune_tried": [[p, t] for p, t in tried],
            "one_by_one_ms": ms1, "one_by_one_dof_per_s": dof / (ms1 * 1e-3),
            "speedup_vs_one_by_one": ms1 / ms, "one_by_one_fp64_ms": ms64,
            "speedup_vs_one_by_one_fp64": ms64 / ms, "dominant_kernel": dom,
            "dominant_share": share, "gpu_launches": launches}


FMG_SWEEPS = ((1, 1), (1, 2), (2, 2), (2, 3), (3, 3))


def run_fmg_vs_fft(torch, args):
    """Section 5.4's comparison at 16M unknowns (2D 4097^2, 3D 257^3): one
    FMG(nu1, nu2) pass (Algorithm 2) against the direct cuFFT DST-I solve, on
    the manufactured problem u = prod sin(pi x_m), f = d pi^2 u.  Each pass is
    timed with CUDA events around the public call (scaling of f, the FMG
    graph, the residual norm and its host read included); the L2(Omega)
    error sqrt(h^d sum (u - u*)^2) against the exact u sits beside it; the
    FFT's error is the discretisation error of the FD system itself."""
    from paper_1208_4247_gb300 import inputs
    from paper_1208_4247_gb300.gmg import FFTSolver, Solver
    stream = torch.cuda.current_stream()
    steps = max(args.form_steps, 5)
    out = {}
    for d, n in ((2, 4096), (3, 256)):
        ustar = torch.from_numpy(inputs.manufactured_u(d, n)).cuda()
        f = (d * np.pi ** 2) * ustar
        u = torch.zeros_like(f)
        h = 1.0 / n

        def l2err():
            return float(torch.sqrt(((u - ustar) ** 2).sum() * h ** d))

        def timed(call):
            for _ in range(max(args.warmup, 1)):
                call()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                call()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / steps

        F = FFTSolver(d, n)
        fft_ms = timed(lambda: F.solve(f, u))
        F.close()
        disc = l2err()
        rows = {"fft": {"ms": fft_ms, "l2_error": disc}}
        for nu1, nu2 in FMG_SWEEPS:
            S = Solver(d, n, nu1=nu1, nu2=nu2, cycle="fmg")
            ms = timed(lambda: S.cycles(f, u, 1))
            S.close()
            e = l2err()
            rows[f"fmg({nu1},{nu2})"] = {"ms": ms, "l2_error": e,
                                         "error_over_discretisation": e / disc,
                                         "speedup_vs_fft": fft_ms / ms}
        del u, f, ustar
        torch.cuda.empty_cache()
        out[f"{d}d_{n + 1}"] = {"unknowns": (n - 1) ** d, "levels": n.bit_length() - 1,
                                "passes_timed": steps, "rows": rows}
    return out


# Wall times (s) of the paper's table "Comparison of four different smoothers
# in 2D on GPU" at L = 12 (GTX 480, FP64, tol 1e-6): context only.
PAPER_SMOOTHER_L12 = {"wj_0.667": (22, 1.02), "wj_0.8": (19, 0.888), "gs_2colour": (16, 0.682),
                      "gs_4colour": (11, 0.485)}


def run_paper_variant(torch, args):
    """The paper's own variant (its 4/8-colour Gauss-Seidel with the colour
    order reversed in post-smoothing, 7/15-point restriction, diagonal-linear
    prolongation), V(1,1): the smoother comparison at 2D 4097^2 (f = sin sin,
    tol 1e-6, as the paper's table) and the 3D 257^3 workload input to 1e-10
    beside the plain red-black V(2,2)."""
    from paper_1208_4247_gb300 import inputs
    from paper_1208_4247_gb300.gmg import Solver
    stream = torch.cuda.current_stream()
    steps = max(args.form_steps, 3)

    def timed(S, f, u, rtol):
        for _ in range(max(args.warmup, 1)):
            u.zero_()
            S.solve(f, u, rtol)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            u.zero_()
            it, rel, conv = S.solve(f, u, rtol)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, it, rel, conv

    out = {}
    n = 4096
    x = np.arange(n + 1) / n
    sx = np.sin(np.pi * x)
    sx[0] = sx[-1] = 0.0
    f = torch.from_numpy(np.ascontiguousarray(sx[:, None] * sx[None, :])).cuda()
    u = torch.zeros_like(f)
    rows = {}
    for name, sm, om, tr in (("wj_0.667", "wjacobi", 2.0 / 3.0, "paper"),
                             ("wj_0.8", "wjacobi", 0.8, "paper"),
                             ("gs_2colour_rb", "rbgs", 0.8, "paper"),
                             ("gs_4colour", "mcgs", 0.8, "paper")):
        with Solver(2, n, smoother=sm, omega=om, nu1=1, nu2=1, transfer=tr) as S:
            ms, it, rel, conv = timed(S, f, u, 1e-6)
        rows[name] = {"ms": ms, "cycles": it, "relres": rel, "converged": conv}
    out["2d_4097_tol1e-6"] = {"rows": rows, "paper_gtx480_L12": PAPER_SMOOTHER_L12,
                              "note": "gs_2colour_rb keeps red-black order in both sweeps "
                                      "(the paper's reverses it: 16 cycles)"}
    del f, u
    d, n = 3, 256
    f = torch.from_numpy(inputs.rhs_uniform(d, n, 2)).cuda()
    u = torch.zeros_like(f)
    rows = {}
    for name, sm, tr, nu in (("gs_8colour_paper_v11", "mcgs", "paper", 1),
                             ("gs_8colour_paper_v22", "mcgs", "paper", 2),
                             ("rb_fw_v22", "rbgs", "fw", 2)):
        with Solver(d, n, smoother=sm, nu1=nu, nu2=nu, transfer=tr) as S:
            ms, it, rel, conv = timed(S, f, u, 1e-10)
        rows[name] = {"ms": ms, "cycles": it, "relres": rel, "converged": conv,
                      "dof_per_s": (n - 1) ** d / (ms * 1e-3)}
    out["3d_257_tol1e-10"] = rows
    del f, u
    torch.cuda.empty_cache()
    return out


def run_sweeps(torch, args, full=True):
    """Smoother x sweeps x inner-cycle sweeps of the refinement forms (3D
    513^3 workload input) and of the batched form (the 512-solve mix, default
    tile and CTAs): time to 1e-10 for every combination.  full = False: the
    reduced default set -- red-black GS, nu = 1..3, FP32 with k = 2..4 and
    BF16 with k = 1, no batch sweep."""
    from paper_1208_4247_gb300 import inputs
    from paper_1208_4247_gb300.autotune import sweep_batch, sweep_refinement
    out = {}
    d, n = 3, 512
    f = torch.from_numpy(inputs.rhs_sine_plus_gauss(d, n, 3)).cuda()
    u = torch.zeros_like(f)
    sms = (("rbgs", 0.8), ("wjacobi", 6.0 / 7.0)) if full else (("rbgs", 0.8),)
    plan = (("fp32", (1, 2, 3, 4)), ("bf16", (1, 2))) if full else (("fp32", (2, 3, 4)),
                                                                     ("bf16", (1,)))
    for prec, ks in plan:
        rows, best = sweep_refinement(d, n, f, u, prec, sms, (1, 2, 3), ks=ks)
        out[f"{prec}_513"] = {"rows": rows, "best": best}
    del f, u
    torch.cuda.empty_cache()
    if not full:
        return out
    mix = inputs.batch_mix(512, 4)
    fd = [torch.from_numpy(x).cuda() for x in inputs.batch_rhs(mix, 4)]
    ud = [torch.zeros_like(x) for x in fd]
    rows, best = sweep_batch([a for a, _ in mix], [b for _, b in mix], fd, ud, "fp32",
                             (("wjacobi", 0.8), ("rbgs", 0.8)), (1, 2), ks=(1, 2, 3))
    out["batch_512_fp32"] = {"rows": rows, "best": best}
    del fd, ud
    torch.cuda.empty_cache()
    return out


def run_learned(torch, args):
    """3D 257^3 GRF workload (power ~|k|^-2, seed 5): V(1,1) cycles with the
    learned smoother (trained here on the GPU on 10k error samples from plain
    V-cycles on 65^3 and 129^3 grids, kept per level only where it beats
    red-black GS) vs plain FP64 red-black V(1,1) and V(2,2)."""
    from paper_1208_4247_gb300 import inputs
    from paper_1208_4247_gb300 import learned_setup as ls
    from paper_1208_4247_gb300.gmg import Solver, jacobi_weights
    d, n = 3, 256
    dof = (n - 1) ** d
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sizes = ((64, args.train_steps65, 8), (128, args.train_steps129, 8))
    weights, hist = ls.train_weights(d, sizes=sizes)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    f = torch.from_numpy(inputs.rhs_grf(d, n, 5)).cuda()
    u = torch.zeros_like(f)
    levels = 8
    cand = {l: weights[128] if l < 2 else weights[64] for l in range(6)}
    S = Solver(d, n, smoother="learned", nu1=1, nu2=1)
    kept, rho_rb, rho_learned = ls.select_levels(S, f, u, cand, levels)
    for l in kept:
        S.set_learned_weights(l, jacobi_weights(d, 6.0 / 7.0))
    rho_untrained = ls.contraction(S, f, u) if kept else None
    for l in kept:
        S.set_learned_weights(l, cand[l])
    out = {"workload": "3D 257^3, f = Gaussian random field (power ~|k|^-2, unit RMS, seed 5), "
                       "FP64 V(1,1), learned smoother on the kept levels, to relative residual 1e-10",
           "training": {"pairs": sum(st * b for _, st, b in sizes), "grids": [s_[0] for s_ in sizes],
                        "seconds": train_s,
                        "loss_first_last": {str(k): [float(np.mean(v[:10])), float(np.mean(v[-10:]))]
                                            for k, v in hist.items()}},
           "levels_kept": kept,
           "contraction": {"rbgs_v11": rho_rb, "learned_v11": rho_learned,
                           "untrained_jacobi_start_v11": rho_untrained}}
    runs = {}
    for name, solver in (("learned_v11", S), ("rbgs_v11", Solver(d, n, nu1=1, nu2=1)),
                         ("rbgs_v22", Solver(d, n, nu1=2, nu2=2))):
        ms, it, rel, stats, launches = time_solves(torch, solver, f, u, args.form_steps, 1)
        res = solver.residual_norm(f, u)
        top = sorted(stats, key=lambda r: -r["ms"])[:6]
        runs[name] = {"value": dof / (ms * 1e-3), "unit": "DOF/s", "ms_per_step": ms,
                      "cycles": it, "relres": rel, "fp64_residual_norm": res,
                      "dominant_kernel": dominant(stats)[0],
                      "top_kernels_ms_per_step": [[r["kernel"], r["level"],
                                                   r["ms"] / args.form_steps] for r in top]}
        solver.close()
    out["runs"] = runs
    out["speedup_learned_vs_rbgs_v22"] = runs["rbgs_v22"]["ms_per_step"] / runs["learned_v11"]["ms_per_step"]
    del f, u
    torch.cuda.empty_cache()
    return out


def config_of(cycles, ws):
    """The workload's config (the same dict on both arms of the benchmark)."""
    return {"workload": WORKLOAD, "cycles": cycles,
            "l2": "inputs larger than L2 (u, q, r: 3 x 136 MB at level 0)",
            "parallelism": "replicas" if ws > 1 else "single GPU"}


def _r(x, digits=4):
    """x rounded to `digits` significant digits (None passes through)."""
    if x is None:
        return None
    if isinstance(x, bool) or not isinstance(x, (int, float)):
        return x
    return float(f"{x:.{digits}g}")


def summarise(line):
    """Compact per-form results: time per solve (ms), DOF/s, cycles or outer
    steps, final relative residual and speed-up against the plain FP64 solve
    of the same workload."""
    out = {"plain_fp64_257": {"ms": _r(line["ms_per_step"]), "dofs": _r(line["value"]),
                              "cyc": line["config"]["cycles"]}}
    if line.get("e2e"):
        out["e2e_257"] = {"ms": _r(line["e2e"]["ms_per_step"]), "dofs": _r(line["e2e"]["value"])}
    nat = line.get("fp64_native_257")
    if nat:
        out["fp64_native_257"] = {"ms": _r(nat["ms_per_step"]), "cyc": nat["cycles"],
                                  "x_headline": _r(nat["headline_speedup"], 3)}
    rf = line.get("roofline") or {}
    out["roofline"] = {"kernel": rf.get("kernel"), "frac": _r(rf.get("frac"), 3),
                       "hbm_frac": _r(rf.get("hbm_frac"), 3), "bound": rf.get("bound")}
    fft = line.get("cufft_dst_257")
    if fft:
        out["cufft_257"] = {"ms": _r(fft["ms_per_step"]), "rel": _r(fft["relres"], 2),
                            "gmg_x": _r(fft["gmg_speedup_vs_fft"], 3)}
    forms = (line.get("mixed_precision_513") or {}).get("forms") or {}
    for name, v in forms.items():
        out[name + "_513"] = {"ms": _r(v["ms_per_step"]), "dofs": _r(v["value"]),
                              "it": v.get("outer_steps") or v.get("cycles"),
                              "k": v.get("inner_cycles_per_step"), "rel": _r(v["relres"], 2),
                              "x": _r(v.get("speedup_vs_fp64_plain"), 3)}
    b = line.get("batched_512")
    if b:
        out["batch_512"] = {"ms": _r(b["ms_per_step"]), "dofs": _r(b["value"]),
                            "maxrel": _r(b["max_relres"], 2),
                            "x_1by1": _r(b["speedup_vs_one_by_one"], 3),
                            "x_1by1_fp64": _r(b["speedup_vs_one_by_one_fp64"], 3),
                            "tuned": b.get("autotuned")}
    lr = line.get("learned_257")
    if lr:
        runs = lr["runs"]
        out["learned_257"] = {"ms": _r(runs["learned_v11"]["ms_per_step"]),
                              "cyc": runs["learned_v11"]["cycles"],
                              "rho": _r(lr["contraction"]["learned_v11"], 3),
                              "rho_rb_v11": _r(lr["contraction"]["rbgs_v11"], 3),
                              "kept": lr["levels_kept"],
                              "rb_v22_ms": _r(runs["rbgs_v22"]["ms_per_step"]),
                              "x_rb_v22": _r(lr["speedup_learned_vs_rbgs_v22"], 3)}
    fm = line.get("fmg_257") or {}
    for k, v in fm.items():
        out[k + "_257"] = {"ms": _r(v["ms_per_step"]), "cyc": v["cycles"],
                           "x": _r(v["speedup_vs_plain_v22"], 3)}
    cpu = line.get("cpu_baseline")
    if cpu:
        out["oracle_cpu_257"] = {"dofs": _r(cpu["value"]), "cores": cpu["cores"]}
    return out


def reduce_max_ms(ms: float, ws: int, device) -> float:
    """Max of a per-rank time over all ranks (the job's time); identity at N=1."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, ws: int, ms_per_step: float) -> float:
    """Whole-job throughput: the units all ranks processed / the max time."""
    return units_per_rank * ws / (ms_per_step * 1e-3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_solve_timed(f, cores_note):
    import oracle
    cfg = oracle.make_cfg(D, N, 0, oracle.RBGS, 0.8, 2, 2, 1)
    u = np.zeros_like(f)
    t0 = time.perf_counter()
    it, hist = oracle.solve(cfg, f, u, RTOL, 100)
    dt = time.perf_counter() - t0
    return it, dt


ORACLE_CORES_SCRIPT = r"""
import json, time
import numpy as np
import oracle
from paper_1208_4247_gb300 import inputs
oracle.build()
out = {}
f = inputs.rhs_sine_plus_uniform(2, 256, 1)
cfg = oracle.make_cfg(2, 256, 0, oracle.WJACOBI, 0.8, 2, 2, 1)
u = np.zeros_like(f)
t0 = time.perf_counter()
it, hist = oracle.solve(cfg, f, u, 1e-10, 100)
out["2d_257_wj"] = {"s_per_solve": time.perf_counter() - t0, "cycles": it}
for key, n, seed in (("3d_257_rb", 256, 2), ("3d_513_rb", 512, 3)):
    f = inputs.rhs_uniform(3, n, seed) if n == 256 else inputs.rhs_sine_plus_gauss(3, n, seed)
    b = oracle.scale_rhs(f)
    u = np.zeros_like(f)
    cfg = oracle.make_cfg(3, n, 0, oracle.RBGS, 0.8, 2, 2, 1)
    t0 = time.perf_counter()
    oracle.vcycle(cfg, b, u)
    out[key] = {"s_per_cycle": time.perf_counter() - t0}
print(json.dumps(out))
"""


def run_oracle_cores(cycles_257, cycles_513):
    """The CPU oracle on all host cores and on one core (OpenMP threads set in
    a child process): the 2D 257^2 weighted-Jacobi V(2,2) workload as a full
    solve; 3D 257^3 and 513^3 red-black V(2,2) as one timed V-cycle each,
    converted to DOF/s to 1e-10 with the cycle counts of the same solves on
    the GPU (the oracle takes the same counts: parity tests)."""
    import subprocess
    out = {}
    for label, threads in (("all_cores", cores()), ("one_core", 1)):
        env = dict(os.environ, OMP_NUM_THREADS=str(threads))
        r = subprocess.run([sys.executable, "-c", ORACLE_CORES_SCRIPT], env=env,
                           capture_output=True, text=True, cwd=os.path.dirname(os.path.abspath(__file__)))
        if r.returncode != 0:
            out[label] = {"error": r.stderr.strip().splitlines()[-1] if r.stderr else "failed"}
            continue
        m = json.loads(r.stdout.strip().splitlines()[-1])
        w = m["2d_257_wj"]
        out[label] = {
            "threads": threads,
            "2d_257_wj_v22": {"dof_per_s": 255 ** 2 / w["s_per_solve"], "s": w["s_per_solve"],
                              "cycles": w["cycles"], "sample": "one full solve"},
            "3d_257_rb_v22": {"dof_per_s": 255 ** 3 / (m["3d_257_rb"]["s_per_cycle"] * cycles_257),
                              "s_per_cycle": m["3d_257_rb"]["s_per_cycle"], "cycles": cycles_257,
                              "sample": "one V-cycle (no norm), times the cycle count"},
            "3d_513_rb_v22": {"dof_per_s": 511 ** 3 / (m["3d_513_rb"]["s_per_cycle"] * cycles_513),
                              "s_per_cycle": m["3d_513_rb"]["s_per_cycle"], "cycles": cycles_513,
                              "sample": "one V-cycle (no norm), times the cycle count"}}
    return out


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args, rank, ws):
    """The CPU FP64 oracle on this host's cores, same workload and metric."""
    if rank != 0:
        return
    from paper_1208_4247_gb300 import inputs
    import oracle
    oracle.build()
    f = inputs.rhs_uniform(D, N, SEED)
    for _ in range(args.warmup):
        oracle_solve_timed(f, None)
    times, its = [], []
    for _ in range(args.steps):
        it, dt = oracle_solve_timed(f, None)
        times.append(dt)
        its.append(it)
    t = sum(times) / len(times)
    value = UNKNOWNS / t
    c = cores()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(its[-1], ws),
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": c, "kind": "oracle",
                             "sample": "full 257^3 solve to 1e-10 per step (OpenMP, all cores)"},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, ws, local):
    import torch
    from paper_1208_4247_gb300 import build as _b
    from paper_1208_4247_gb300 import inputs
    from paper_1208_4247_gb300.gmg import Solver

    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0 or ws == 1:
        _b.build()
    if ws > 1:
        torch.distributed.barrier()
    dev = torch.device("cuda", torch.cuda.current_device())
    f_np = inputs.rhs_uniform(D, N, SEED)
    f = torch.from_numpy(f_np).to(dev)
    u = torch.zeros_like(f)
    S = Solver(D, N, **HEADLINE)
    S.set_timing(False)
    cycles = None

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            u.zero_()
            cycles, rel, conv = S.solve(f, u, RTOL)
            assert conv, "warm-up solve did not converge"
        S.timing_reset()
        time.sleep(0.5)  # let the sampler start
        barrier()
        clk.mark("t0")
        ev0.record(stream)
        for _ in range(args.steps):
            u.zero_()
            cycles, rel, conv = S.solve(f, u, RTOL)
        ev1.record(stream)
        barrier()
        clk.mark("t1")
    ms_total = ev0.elapsed_time(ev1)
    ms_total = reduce_max_ms(ms_total, ws, dev)
    ms_step = ms_total / args.steps
    value = job_value(UNKNOWNS, ws, ms_step)

    # per-kernel records: the same steps once more with an event node around
    # every kernel of the cycle graph (they add ~15% to a solve, so the
    # headline above is timed without them)
    S.set_timing(True)
    u.zero_()
    S.solve(f, u, RTOL)
    S.timing_reset()
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        u.zero_()
        S.solve(f, u, RTOL)
    ev1.record(stream)
    barrier()
    ms_instr = reduce_max_ms(ev0.elapsed_time(ev1), ws, dev) / args.steps
    stats, launches = S.timing_report()
    S.set_timing(False)

    # dominant kernel: largest summed device time; achieved = its per-launch
    # FP64 instruction count / its average launch time (level 0 record)
    clocks = clk.summary()
    pk, pk_kind = peaks()
    alg_bytes = sum(r["bytes"] * r["launches"] for r in stats) / args.steps
    # the FP64 pipe's rate measured in this run (independent DFMA / DADD
    # chains), weighted by a kernel's add : fma mix
    from paper_1208_4247_gb300.gmg import measure_fp64_rate
    r_fma, r_add = measure_fp64_rate(0) / 1e12, measure_fp64_rate(1) / 1e12
    nominal_inst = FP64_INST_PER_CLK_SM * NUM_SMS * SM_MAX_MHZ * 1e6 / 1e12  # T inst/s
    total_ms = sum(r["ms"] for r in stats)

    def roofline_of(rec):
        """The roofline record of one (kernel, level): FP64-pipe bound for the
        FP64 kernels, HBM bound for the double-float / FP32 / BF16 ones."""
        name = rec["kernel"]
        avg_s = rec["ms"] / rec["launches"] * 1e-3
        gbs = rec["bytes"] / avg_s / 1e9
        common = {"kernel": f"{name} (level {rec['level']})", "alg_bytes_per_launch": rec["bytes"],
                  "traffic": TRAFFIC.get((name, rec["level"])),
                  "traffic_unit": "bytes per launch (ncu dram read + write)",
                  "kernel_share": rec["ms"] / total_ms, "avg_launch_us": avg_s * 1e6,
                  "hbm_gbs": gbs, "hbm_frac": gbs / pk["hbm_gbs"]}
        if fp64_bound(name):
            n_add, n_fma = FP64_MIX.get(name, (1.0, 0.0))
            peak = (n_add + n_fma) / (n_add / r_add + n_fma / r_fma)
            ach = rec["dp_ops"] / avg_s / 1e12
            return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "T FP64-pipe inst/s",
                    "frac": ach / peak,
                    "peak_note": (f"measured in this run: {r_fma:.4f} T DFMA/s, {r_add:.4f} T "
                                  f"DADD/s (gmg_measure_fp64_rate), weighted {n_add}:{n_fma} "
                                  "add:fma"), **common}
        return {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / pk["hbm_gbs"], "peak_note": f"{pk_kind} copy bandwidth", **common}

    dom_rec = max(stats, key=lambda r: r["ms"])  # the largest (kernel, level) record
    roof = roofline_of(dom_rec)
    roof.update({"peak_measured_fp64": {"dfma": r_fma, "dadd": r_add},
                 "peak_nominal_fp64": nominal_inst, "hbm_peak_gbs": pk["hbm_gbs"],
                 "hbm_peak_kind": pk_kind,
                 "timing": "per-kernel CUDA events (event nodes in the cycle graph on the "
                           "library's stream) over a repeat of the timed steps",
                 "instrumented_ms_per_step": ms_instr})
    hbm_recs = [r for r in stats if not fp64_bound(r["kernel"])]
    if hbm_recs:
        roof["hbm_kernel"] = roofline_of(max(hbm_recs, key=lambda r: r["ms"]))
    hbm = {"solve_alg_bytes": alg_bytes, "achieved_gbs": alg_bytes / (ms_step * 1e-3) / 1e9,
           "peak_gbs": pk["hbm_gbs"], "peak_kind": pk_kind,
           "frac": alg_bytes / (ms_step * 1e-3) / 1e9 / pk["hbm_gbs"],
           "frac_of_nominal_8000": alg_bytes / (ms_step * 1e-3) / 1e9 / 8000.0}

    # the paper's comparison point: direct cuFFT DST-I solve of the same system
    from paper_1208_4247_gb300.gmg import FFTSolver
    F = FFTSolver(D, N)
    uf = torch.zeros_like(f)
    for _ in range(max(args.warmup, 1)):
        F.solve(f, uf)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.form_steps):
        F.solve(f, uf)
    e1.record(stream)
    torch.cuda.synchronize()
    fft_ms = e0.elapsed_time(e1) / args.form_steps
    F.close()
    S.set_timing(False)
    fft_res = S.residual_norm(f, uf) / S.residual_norm(f, torch.zeros_like(f))
    fft = {"value": UNKNOWNS / (fft_ms * 1e-3), "unit": "DOF/s", "ms_per_step": fft_ms,
           "relres": fft_res, "method": "DST-I by length-2n cuFFT D2Z per axis, exact eigenvalues",
           "gmg_speedup_vs_fft": fft_ms / ms_step}
    del uf

    # the paper's FMG (Algorithm 2) as the first cycle, then V(2,2) cycles
    # the same cycles with FP64 arithmetic throughout (the plain kernels)
    S64 = Solver(D, N)
    ms64, it64, rel64, stats64, _ = time_solves(torch, S64, f, u, args.form_steps,
                                                max(args.warmup, 1))
    S64.close()
    dom64, rec64, share64 = dominant(stats64)
    fp64_native = {"value": UNKNOWNS / (ms64 * 1e-3), "unit": "DOF/s", "ms_per_step": ms64,
                   "cycles": it64, "relres": rel64,
                   "dominant_kernel": f"{dom64} (level {rec64['level']})",
                   "dominant_share": share64,
                   "headline_speedup": ms64 / ms_step}

    fmg_runs = {}
    for nu in (2, 3):
        Sf = Solver(D, N, nu1=nu, nu2=nu, cycle="fmg")
        ms_f, it_f, rel_f, _, _ = time_solves(torch, Sf, f, u, args.form_steps,
                                              max(args.warmup, 1), timing=False)
        Sf.close()
        fmg_runs[f"fmg_v{nu}{nu}"] = {"value": UNKNOWNS / (ms_f * 1e-3), "unit": "DOF/s",
                                      "ms_per_step": ms_f, "cycles": it_f, "relres": rel_f,
                                      "speedup_vs_plain_v22": ms_step / ms_f}

    # end to end through the public API: pinned host f, u; H2D + solve + D2H
    e2e = None
    if not args.no_e2e:
        fh = torch.empty(f_np.shape, dtype=torch.float64, pin_memory=True).numpy()
        fh[...] = f_np
        uh = torch.empty(f_np.shape, dtype=torch.float64, pin_memory=True).numpy()
        S.set_timing(False)
        uh[...] = 0.0
        S.solve_host(fh, uh, RTOL)
        # each call bracketed by its own pair of events (gmg_solve_host returns
        # with the copies and the solve done); resetting the host initial
        # guess between calls is host work outside the call and is not timed
        pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.steps)]
        barrier()
        for a, b in pairs:
            uh[...] = 0.0
            a.record(stream)
            S.solve_host(fh, uh, RTOL)
            b.record(stream)
        barrier()
        e_ms = reduce_max_ms(sum(a.elapsed_time(b) for a, b in pairs), ws, dev) / args.steps
        e2e = {"value": UNKNOWNS * ws / (e_ms * 1e-3), "unit": "DOF/s", "ms_per_step": e_ms,
               "h2d_bytes_per_step": 2 * fh.nbytes, "d2h_bytes_per_step": uh.nbytes}
    S.close()

    if rank != 0:
        return
    forms = batch = learned = fmg_fft = paper_variant = None
    if not args.no_forms:
        fmg_fft = run_fmg_vs_fft(torch, args)
        paper_variant = run_paper_variant(torch, args)
        forms = run_forms(torch, args)
        batch = run_batch(torch, args)
        learned = run_learned(torch, args)
    sweeps = None if args.no_forms else run_sweeps(torch, args, full=args.sweeps)
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        times = []
        while sum(times) < args.cpu_seconds:
            it_o, dt = oracle_solve_timed(f_np, None)
            times.append(dt)
        dt = sum(times) / len(times)
        cpu = {"value": UNKNOWNS / dt, "unit": "DOF/s", "cores": cores(), "kind": "oracle",
               "sample": f"{len(times)} full 257^3 solves to 1e-10 ({it_o} cycles, "
                         f"{dt:.2f} s each, {sum(times):.1f} s total, OpenMP on all cores)"}
        c513 = (forms or {}).get("forms", {}).get("fp64_plain", {}).get("cycles") or 11
        cpu["by_cores"] = run_oracle_cores(cycles, c513)
    line = {"metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+df32x2",
            "data": "synthetic",
            "config": config_of(cycles, ws),
            "evaluation": HEADLINE_NOTE, "fp64_native_257": fp64_native,
            "roofline": roof, "hbm": hbm, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks, "cufft_dst_257": fft,
            "fmg_257": fmg_runs, "fmg_pass_vs_fft": fmg_fft, "paper_variant": paper_variant,
            "sweeps": sweeps,
            "mixed_precision_513": forms, "batched_512": batch,
            "learned_257": learned}
    if args.kernels:
        line["kernels"] = stats
    # last key: the per-form results in a few hundred bytes, so that a reader
    # of only the end of the line still sees every form's number
    line["summary"] = summarise(line)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernels", action="store_true", help="add per-kernel records")
    ap.add_argument("--no-forms", action="store_true", help="skip the 513^3 precision forms")
    ap.add_argument("--sweeps", action="store_true",
                    help="the full smoother x sweeps x inner-cycle sweeps (default: a reduced set)")
    ap.add_argument("--form-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--train-steps65", type=int, default=1000)
    ap.add_argument("--train-steps129", type=int, default=250)
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, ws)
    else:
        run_ours(args, rank, ws, local)


if __name__ == "__main__":
    main()
