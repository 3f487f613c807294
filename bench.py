#!/usr/bin/env python3
"""Benchmark of the odd-even Wilson-clover hot path on one GB300 (or N replicas).

Workload (the metric's configuration): a 32^3 x 64 lattice, periodic space /
antiperiodic time, SU(3) links U = exp(i 0.25 sum_k a_k lambda_k) with
a_k ~ N(0,1) (seed 1001), c_sw = 1.0, m0 = 0.02, Gaussian complex source
(seed 2001).  One step is one pass of the whole path through the C ABI:

  1. lq_set_gauge      link import, clover build, D_oo^{-1} (LDL)        (a1-a3)
  2. lq_estimate_norm  10 FP32 power iterations on D_S^+ D_S -> omega     (a8)
  3. lq_smooth         odd-even Richardson(5, delta = 0.8) smoother M_5 r (a6, a7)
  4. lq_solve          odd-even FGMRES(10) in df64 (FP64-accurate double-float),
                       right-preconditioned by GMRES(8) in FP32 to 1e-5, to a
                       1e-10 residual                                      (a4-a6, a9-a11)

value = algorithmic bytes of every library kernel in the timed steps (the
library counts them per launch) / device time of the steps, in GB/s, summed
over ranks.  Beside it, as named fields of the same line:

  ds_f32   the FP32 D_S (K1 + K2) on 32^3 x 64, 48^3 x 96 and 8^4 against the
           measured HBM bandwidth (the operator half of the metric);
  solve    the mixed solve against plain FP64 GMRES(30) to 1e-10 on the same
           lattices: times, speed-up, true residuals, and the relative
           difference of the two solutions;
  batched, force, sap, bf16   the other workloads, summarised.

--detail PATH writes the per-kernel-class profile and every section's full
record to a JSON file.

--impl reference runs the FP64 CPU oracle instead (the test oracle, as it
stands) on the host cores: each step applies the oracle's D_S (Eq. 3) to a
bounded sample of the workload (a 16^3 x 32 lattice with the same parameters).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "odd-even Wilson-clover op GB/s vs HBM peak; mixed vs FP64 solve time @1e-10"
L_WORK = (32, 32, 32, 64)
EPS, M0, CSW, TBC = 0.25, 0.02, 1.0, -1
LINK_SEED, SRC_SEED = 1001, 2001
L_SAMPLE = (16, 16, 16, 32)
BYTES_DS_F64 = 4416.0   # algorithmic bytes per even site of one FP64 D_S (18-real links)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-force", action="store_true")
    ap.add_argument("--no-sap", action="store_true")
    ap.add_argument("--no-bf16", action="store_true")
    ap.add_argument("--no-48x96", action="store_true")
    ap.add_argument("--no-8x4", action="store_true")
    ap.add_argument("--detail", default=None,
                    help="write the per-kernel-class profile and every section's full record to this JSON file")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "src": "fallback"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
_SAMPLE = {}


def oracle_ds_sample(seconds: float, min_apps: int = 3):
    """Time the FP64 oracle's D_S (Eq. 3) on the 16^3 x 32 sample lattice."""
    import numpy as np

    import oracle
    from paper_2407_08092_gb300 import synth
    if "lat" not in _SAMPLE:
        U = synth.gauge_links(L_SAMPLE, EPS, LINK_SEED)
        lat = oracle.Lattice(L_SAMPLE, U, m0=M0, csw=CSW, t_bc=TBC)
        _ = lat.C, lat.Cinv                  # clover and inverse: setup, not timed
        _SAMPLE["lat"] = lat
        _SAMPLE["x"] = synth.gaussian_spinor(lat.Vh, SRC_SEED)
        lat.schur(_SAMPLE["x"])              # warm
    lat, x = _SAMPLE["lat"], _SAMPLE["x"]
    n, t0 = 0, time.perf_counter()
    while n < min_apps or time.perf_counter() - t0 < seconds:
        x = lat.schur(x)
        x /= np.sqrt(np.vdot(x, x).real)
        n += 1
    dt = time.perf_counter() - t0
    gbs = n * lat.Vh * BYTES_DS_F64 / dt / 1e9
    return gbs, n, dt, oracle.threads()


def oracle_c0_solves():
    """The oracle's odd-even solves of the 8^4 workload (eps 0.25, m0 0.05, c_sw 1,
    link seed 1000, Gaussian source seed 2000) to 1e-10 on the host cores: plain
    GMRES(30) and FGMRES(30) right-preconditioned by Richardson(5, delta 0.8),
    omega from 30 power iterations (not timed)."""
    import numpy as np

    import oracle
    from paper_2407_08092_gb300 import synth
    L = (8, 8, 8, 8)
    lat = oracle.Lattice(L, synth.gauge_links(L, EPS, 1000), m0=0.05, csw=CSW, t_bc=TBC)
    _ = lat.C, lat.Cinv
    b = synth.gaussian_spinor(lat.V, 2000)
    norm = oracle.power_norm(lat.schur, lat.schur_dag, b[:lat.Vh], 30)
    out = {}
    for name, kw in (("gmres30", {"solver": "gmres", "restart": 30}),
                     ("fgmres30_rich5", {"solver": "fgmres", "restart": 30, "precond": "richardson",
                                         "smooth_n": 5, "omega": 0.8 / norm})):
        t0 = time.perf_counter()
        _, info = oracle.solve(lat, b, tol=1e-10, max_restarts=200, **kw)
        out[name] = {"s": round(time.perf_counter() - t0, 3), "iters": info["iters"],
                     "rres": float(f"{info['rel_resid_true']:.3g}")}
    del np
    return out


def cpu_baseline(seconds: float):
    """The oracle as it stands on the host cores: its D_S on the 16^3 x 32 sample
    with every core and with one core, and its two 8^4 solves with every core."""
    import oracle
    g, n, dt, cores = oracle_ds_sample(seconds)
    oracle.set_threads(1)
    try:
        g1, n1, dt1, _ = oracle_ds_sample(max(2.0, seconds / 4))
    finally:
        oracle.set_threads(cores)
    c0 = oracle_c0_solves()
    return {"value": round(g, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle FP64 D_S x{n} ({dt:.0f} s; 1 core x{n1}, {dt1:.0f} s), 16^3x32, this workload's "
                      f"parameters; c0: its 8^4 solves",
            "single_core": {"value": round(g1, 3), "cores": 1}, "c0": c0}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    per_step = max(1.0, min(10.0, 100.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_ds_sample(per_step, 1)
    vals, apps, secs = [], 0, 0.0
    for _ in range(args.steps):
        g, n, dt, cores = oracle_ds_sample(per_step, 1)
        vals.append(g)
        apps += n
        secs += dt
    value = apps * (L_SAMPLE[0] * L_SAMPLE[1] * L_SAMPLE[2] * L_SAMPLE[3] // 2) * BYTES_DS_F64 / secs / 1e9
    sample = (f"FP64 oracle D_S (Eq. 3) applied {apps} times on a 16^3x32 lattice with the 32^3x64 "
              f"workload's parameters (eps 0.25, m0 0.02, csw 1, antiperiodic t); clover precomputed")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "odd-even Wilson-clover D_S, FP64 CPU oracle on a bounded sample",
                       "lattice": list(L_SAMPLE), "eps": EPS, "m0": M0, "csw": CSW, "t_bc": TBC},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def traffic_per_launch(cls_name: str, V: int):
    """DRAM bytes per launch of a kernel class from the committed ncu summary
    (profiles/traffic.txt), or None when the kernel's source file changed since
    the capture."""
    return table_per_launch("traffic.txt", cls_name, V)


# Kernel classes whose roof is arithmetic, not HBM: native FP64 runs on the
# FP64 pipe (GB300: 2 FMA/clk/SM -> 152 * 2 * 2 flop * 2.07 GHz = 1.26 TFLOP/s,
# the nominal 1.25 TFLOP/s), df64 on the FP32 pipe.  A df64 class is measured by
# instruction issue: the warp instructions one launch executes (ncu
# sm__inst_executed.sum per unit site, profiles/issue.txt) over its duration,
# against the SMs' issue ceiling of 152 SMs x 4 schedulers x 1 warp instruction
# per clock at 2.07 GHz = 1258.6 G warp instructions/s.  Beside it stays the
# flop model: 15 FP32 instructions per df64 FMA (2prod 2, cross terms 2, 2sum
# 6, low-part adds 2, fast2sum 3): 152 * 128 lanes * 2.07 GHz / 15 * 2 flop =
# 5.37 TFLOP/s FP64-equivalent.
ALU_F64 = {"hop_k1_f64", "hop_k2_f64"}
ALU_DF64 = {"hop_k1_df64", "hop_k2_df64", "hop_other", "clover", "clover_field", "force"}
# FP32 kernels whose data sit in L2 for most of their work (the SAP block solves
# re-read each block's links and clover on every half-step): their DRAM traffic
# is near their algorithmic bytes but far below the bandwidth, so they are
# reported against the same issue ceiling, with the HBM fraction beside it.
ISSUE_F32 = {"sap"}
SM_MHZ_MAX = 2070.0
ISSUE_PEAK_G = 152 * 4 * SM_MHZ_MAX / 1e3   # G warp instructions per second


def table_per_launch(fname: str, cls_name: str, V: int):
    """Per-launch value of a kernel class from a committed ncu table
    (profiles/<fname>: class, value per unit site, unit V or Vh, source file,
    sha256[:16] of that file at capture), or None when the kernel's source file
    changed since the capture."""
    path = os.path.join(ROOT, "profiles", fname)
    try:
        for ln in open(path):
            parts = ln.split()
            if ln.startswith("#") or len(parts) < 5 or parts[0] != cls_name:
                continue
            src = os.path.join(ROOT, "paper_2407_08092_gb300", "csrc", parts[3])
            if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == parts[4]:
                return float(parts[1]) * (V if parts[2] == "V" else V // 2)
    except OSError:
        pass
    return None


def roofline_of(name, d, pk, V):
    t = d["ms"] / 1e3
    base = {"kernel": name, "avg_launch_us": round(1e3 * d["ms"] / d["launches"], 2),
            "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
            "algorithmic_flops_per_launch": d["flops"] / d["launches"],
            "gbs": round(d["bytes"] / t / 1e9, 1), "hbm_frac": round(d["bytes"] / t / 1e9 / pk["hbm_gbs"], 4)}
    inst = table_per_launch("issue.txt", name, V) if name in ALU_DF64 or name in ISSUE_F32 else None
    if inst is not None:
        # instructions per launch over the launch's average duration, against the issue ceiling
        ach = inst / (d["ms"] / d["launches"] / 1e3) / 1e9
        base.update({"bound": "issue", "achieved": round(ach, 1), "peak": round(ISSUE_PEAK_G, 1),
                     "unit": "Gwarp-inst/s", "frac": round(ach / ISSUE_PEAK_G, 4),
                     "traffic": traffic_per_launch(name, V),
                     "peak_src": f"hardware issue ceiling: 152 SMs x 4 schedulers x {SM_MHZ_MAX:.0f} MHz; "
                                 "instructions from ncu sm__inst_executed.sum (profiles/issue.txt)"})
        if name in ALU_DF64:
            model = d["flops"] / t / 1e12 / (152 * 128 * SM_MHZ_MAX * 1e6 / 15 * 2 / 1e12)
            base["df64_model_frac"] = round(model, 4)
    elif name in ALU_F64 or name in ALU_DF64:
        peak = (152 * 2 * 2 * SM_MHZ_MAX * 1e6 if name in ALU_F64 else 152 * 128 * SM_MHZ_MAX * 1e6 / 15 * 2) / 1e12
        ach = d["flops"] / t / 1e12
        base.update({"bound": "alu", "achieved": round(ach, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
                     "frac": round(ach / peak, 4), "traffic": traffic_per_launch(name, V),
                     "peak_src": "derived: " + ("FP64 pipe, 2 FMA/clk/SM" if name in ALU_F64
                                                else "FP32 pipe, 15 instructions per df64 FMA")
                                 + f" at {SM_MHZ_MAX:.0f} MHz"})
    else:
        ach = d["bytes"] / t / 1e9
        base.update({"bound": "hbm", "achieved": round(ach, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": round(ach / pk["hbm_gbs"], 4), "traffic": traffic_per_launch(name, V),
                     "peak_src": f"{pk['src']} hbm_gbs (STREAM-style copy)"})
    return base


BATCH_LATTICES = [((24, 24, 24, 48), 1103), ((8, 8, 8, 8), 1101), ((16, 16, 16, 16), 1102), ((16, 16, 16, 32), 1104)]


def run_batched(lqdd, synth, torch, stream, dev):
    """The batched workload: 12 spin-colour point sources (at the origin) on each
    of 24^3 x 48, 8^4, 16^4 and 16^3 x 32, each lattice with its own links (eps
    0.25, m0 0.05, c_sw 1), all solved to 1e-10 by one lq_solve_group (df64
    defect correction around one batched FP32 GMRES(8) whose operator launches
    are single persistent grids over every lattice and right-hand side, cycles
    replayed from CUDA graphs, launch shapes autotuned), against one
    lq_solve_batch per lattice, 48 single mixed solves, and 48 plain FP64
    GMRES(30) solves, all on the same GPU."""
    import numpy as np
    n = 12
    ctxs, bs, xs = [], [], []
    try:
        for L, seed in BATCH_LATTICES:
            V = int(np.prod(L))
            ctx = lqdd.lq_create(lqdd.make_lattice(L, TBC, 0.05, CSW), stream.cuda_stream)
            ctxs.append(ctx)
            lqdd.lq_set_gauge(ctx, torch.from_numpy(synth.gauge_links(L, EPS, seed)).to(dev))
            b = torch.zeros((n, V, 4, 3), dtype=torch.complex128, device=dev)
            for r in range(n):
                b[r, 0, r % 4, r // 4] = 1.0        # point source at the origin, spin r%4, colour r//4
            bs.append(b)
            xs.append(torch.zeros_like(b))
        grp = lqdd.lq_group_create(ctxs, stream.cuda_stream)
        bp = lqdd.make_batch_params(tol=1e-10, restart=8, max_restarts=10, smooth_n=16, smooth_tol=1e-5)
        single = lqdd.make_params(solver=lqdd.LQ_SOLVER_FGMRES, prec=lqdd.LQ_DF64, tol=1e-10, restart=10,
                                  max_restarts=20, smoother=lqdd.LQ_SMOOTH_GMRES, smooth_n=40, smooth_m=8,
                                  smooth_tol=1e-5, inner_prec=lqdd.LQ_F32)
        fp64 = lqdd.make_params(tol=1e-10, restart=30, max_restarts=200)

        def run(name):
            worst, ok = 0.0, "LQ_OK"
            for x in xs:
                x.zero_()
            if name == "group":
                s, st = lqdd.lq_solve_group(grp, ctxs[0], bp, bs, xs)
                worst = max(q.rel_resid_true for q in st)
                ok = lqdd.lq_status_string(s)
                return worst, ok
            for ctx, b, x in zip(ctxs, bs, xs):
                if name == "per_lattice":
                    s, st = lqdd.lq_solve_batch(ctx, bp, n, b, x)
                    worst = max([worst] + [q.rel_resid_true for q in st])
                else:
                    for r in range(n):
                        s, q = lqdd.lq_solve(ctx, single if name == "sequential" else fp64, b[r], x[r])
                        worst = max(worst, q.rel_resid_true)
                if s != lqdd.LQ_OK:
                    ok = lqdd.lq_status_string(s)
            return worst, ok

        res = {}
        x_group = None
        for name, reps in (("group", 3), ("per_lattice", 3), ("sequential", 2), ("fp64_sequential", 1)):
            run(name)                                   # warm-up: workspace, tuning, graph capture
            times = []
            for _ in range(reps):
                torch.cuda.synchronize()
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                worst, ok = run(name)
                z.record(stream)
                torch.cuda.synchronize()
                times.append(a.elapsed_time(z))
            res[name] = {"ms": round(sorted(times)[len(times) // 2], 2), "worst_rel_resid_true": worst, "status": ok}
            if name == "group":
                x_group = [x.clone() for x in xs]
        # the group's solutions against the plain FP64 ones (left in xs by the last run)
        res["xdiff_vs_fp64"] = max(max(rel_diff(torch, xg[r], xf[r]) for r in range(n))
                                   for xg, xf in zip(x_group, xs))
        spt, rpt, grid, blas, hop_ms, blas_ms = lqdd.lq_group_tuning(grp)
        res["tuning"] = {"sites_per_tile": spt, "rhs_per_thread": rpt,
                         "rhs_per_tile": rpt * 128 // spt if rpt else "all (staged links and clover)",
                         "grid": grid, "blas_blocks": blas, "hop_pair_ms": round(hop_ms, 4),
                         "blas_pair_ms": round(blas_ms, 4)}
        res["speedup_vs_per_lattice"] = round(res["per_lattice"]["ms"] / res["group"]["ms"], 2)
        res["speedup_vs_sequential"] = round(res["sequential"]["ms"] / res["group"]["ms"], 2)
        res["speedup_vs_fp64"] = round(res["fp64_sequential"]["ms"] / res["group"]["ms"], 2)
        res["config"] = ("12 spin-colour point sources on each of 24^3x48, 8^4, 16^4, 16^3x32 (own links, eps 0.25, "
                         "m0 0.05, csw 1), 48 systems, all to 1e-10; group: one lq_solve_group; per_lattice: "
                         "lq_solve_batch per lattice; sequential: 48 x FGMRES(10) df64 / GMRES(8) FP32; "
                         "fp64_sequential: 48 x plain FP64 GMRES(30); medians")
        lqdd.lq_group_destroy(grp)
        return res
    finally:
        for ctx in ctxs:
            lqdd.lq_destroy(ctx)


def run_sap(lqdd, torch, stream, ctx, db, x, pk_peaks, V, omega):
    """SAP(3, 4) and Richardson(5) smoother calls (medians of 5) and the FGMRES(10)
    df64 solve to 1e-10 preconditioned by SAP(3, 4), on the benchmark lattice."""
    sap = lqdd.make_params(smoother=lqdd.LQ_SMOOTH_SAP, smooth_n=3, smooth_m=4, inner_prec=lqdd.LQ_F32,
                           prec=lqdd.LQ_DF64)
    rich = lqdd.make_params(smoother=lqdd.LQ_SMOOTH_RICHARDSON, smooth_n=5, omega=omega, inner_prec=lqdd.LQ_F32,
                            prec=lqdd.LQ_DF64)
    solve = lqdd.make_params(solver=lqdd.LQ_SOLVER_FGMRES, prec=lqdd.LQ_DF64, tol=1e-10, restart=10,
                             max_restarts=20, smoother=lqdd.LQ_SMOOTH_SAP, smooth_n=3, smooth_m=4,
                             inner_prec=lqdd.LQ_F32)
    e = torch.empty_like(db)

    def med(fn, reps=5):
        fn()
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out = fn()
            z.record(stream)
            torch.cuda.synchronize()
            ts.append((a.elapsed_time(z), out))
        return sorted(ts, key=lambda t: t[0])[len(ts) // 2]

    lqdd.lq_profile(ctx, 1)
    t_sap, _ = med(lambda: lqdd.lq_smooth(ctx, sap, db, e))
    prof = read_profile(lqdd, ctx)
    lqdd.lq_profile(ctx, 0)
    t_rich, _ = med(lambda: lqdd.lq_smooth(ctx, rich, db, e))

    def solve_once():
        x.zero_()
        return lqdd.lq_solve(ctx, solve, db, x)
    t_solve, (status, st) = med(solve_once, reps=3)
    res = {"sap_3_4_ms": round(t_sap, 3), "richardson_5_ms": round(t_rich, 3), "blocks": [4, 4, 4, 4],
           "fgmres_sap_ms": round(t_solve, 2), "fgmres_sap": st.as_dict(), "status": lqdd.lq_status_string(status)}
    if "sap" in prof:
        res["roofline"] = roofline_of("sap", prof["sap"], pk_peaks, V)
    return res


def ds_rate(lqdd, ctx, prec, xe, ye, pk, reps=10):
    """D_S = K1 + K2 in precision prec: device time of the two hopping kernels per
    apply (CUDA events around each launch), algorithmic GB/s and fraction of the
    measured HBM bandwidth."""
    name = {lqdd.LQ_F32: "f32", lqdd.LQ_F64: "f64", lqdd.LQ_DF64: "df64", lqdd.LQ_BF16: "bf16"}[prec]
    lqdd.lq_apply(ctx, lqdd.LQ_OP_SCHUR, prec, xe, ye)
    lqdd.lq_profile(ctx, 1)
    for _ in range(reps):
        lqdd.lq_apply(ctx, lqdd.LQ_OP_SCHUR, prec, xe, ye)
    prof = read_profile(lqdd, ctx)
    lqdd.lq_profile(ctx, 0)
    k1, k2 = f"hop_k1_{name}", f"hop_k2_{name}"
    ms = (prof[k1]["ms"] + prof[k2]["ms"]) / reps
    by = (prof[k1]["bytes"] + prof[k2]["bytes"]) / reps
    gbs = by / (ms / 1e3) / 1e9
    return {"us": round(1e3 * ms, 1), "gbs": round(gbs, 1), "frac": round(gbs / pk["hbm_gbs"], 4)}


def timed_solves(lqdd, torch, stream, ctx, b, cases):
    """Each (name, params, reps) solve from zero: the median device time, its
    stats, and the solution of the last run."""
    res, xs = {}, {}
    x = torch.zeros_like(b)
    for name, prm, reps in cases:
        x.zero_()
        lqdd.lq_solve(ctx, prm, b, x)                 # workspace
        runs = []
        for _ in range(reps):
            x.zero_()
            torch.cuda.synchronize()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            status, st = lqdd.lq_solve(ctx, prm, b, x)
            z.record(stream)
            torch.cuda.synchronize()
            runs.append((a.elapsed_time(z), st.as_dict(), lqdd.lq_status_string(status)))
        ms, st, status = sorted(runs, key=lambda r: r[0])[len(runs) // 2]
        res[name] = {"ms": round(ms, 2), "status": status, **st}
        xs[name] = x.clone()
    return res, xs


def rel_diff(torch, a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def mixed_params(lqdd):
    """The mixed-precision solve: FGMRES(10) in df64 right-preconditioned by
    GMRES(8) in FP32 to 1e-5, to a 1e-10 relative residual of D x = b."""
    return lqdd.make_params(solver=lqdd.LQ_SOLVER_FGMRES, prec=lqdd.LQ_DF64, tol=1e-10, restart=10,
                            max_restarts=20, smoother=lqdd.LQ_SMOOTH_GMRES, smooth_n=40, smooth_m=8,
                            smooth_tol=1e-5, inner_prec=lqdd.LQ_F32)


def solve_summary(res, xs, torch, keys=("mixed", "fp64")):
    """Compact record of a mixed-vs-FP64 comparison: times, ratio, true residuals
    and the relative difference of the two solutions."""
    m, f = keys
    return {"mixed_ms": res[m]["ms"], "fp64_ms": res[f]["ms"], "x": round(res[f]["ms"] / res[m]["ms"], 2),
            "rres": [float(f"{res[m]['rel_resid_true']:.3g}"), float(f"{res[f]['rel_resid_true']:.3g}")],
            "xdiff": float(f"{rel_diff(torch, xs[m], xs[f]):.3g}"),
            "ok": res[m]["status"] == "LQ_OK" and res[f]["status"] == "LQ_OK"}


def run_48x96(lqdd, synth, torch, stream, dev, pk):
    """The 48^3 x 96 workload (eps 0.2, m0 0.01, c_sw 1, antiperiodic t, link
    seed 1002, Gaussian source seed 2002): the FP32 and FP64 D_S against the
    measured HBM bandwidth, and the mixed solve against plain FP64 GMRES(30),
    both to 1e-10, with the relative difference of their solutions."""
    import numpy as np
    L = (48, 48, 48, 96)
    V = int(np.prod(L))
    ctx = lqdd.lq_create(lqdd.make_lattice(L, TBC, 0.01, CSW), stream.cuda_stream)
    try:
        lqdd.lq_set_gauge(ctx, torch.from_numpy(synth.gauge_links(L, 0.2, 1002)).to(dev))
        b = torch.from_numpy(synth.gaussian_spinor(V, 2002)).to(dev)
        xe = b[:V // 2].contiguous()
        ye = torch.empty_like(xe)
        res = {"lattice": list(L), "ds_f32": ds_rate(lqdd, ctx, lqdd.LQ_F32, xe, ye, pk),
               "ds_f64": ds_rate(lqdd, ctx, lqdd.LQ_F64, xe, ye, pk)}
        fp64 = lqdd.make_params(tol=1e-10, restart=30, max_restarts=200)
        sol, xs = timed_solves(lqdd, torch, stream, ctx, b, (("mixed", mixed_params(lqdd), 3), ("fp64", fp64, 1)))
        res["solves"] = sol
        res["solve"] = solve_summary(sol, xs, torch)
        return res
    finally:
        lqdd.lq_destroy(ctx)


def run_c0(lqdd, synth, torch, stream, dev, pk):
    """The 8^4 workload (eps 0.25, m0 0.05, c_sw 1, link seed 1000, Gaussian
    source seed 2000): the D_S apply (its 4 MB working set sits in L2, so its
    GB/s is no HBM figure), plain FP64 GMRES(30), FGMRES(30) in FP64 with
    Richardson(5, delta 0.8) in FP32, and the mixed solve, all to 1e-10."""
    import numpy as np
    L = (8, 8, 8, 8)
    V = int(np.prod(L))
    ctx = lqdd.lq_create(lqdd.make_lattice(L, TBC, 0.05, CSW), stream.cuda_stream)
    try:
        lqdd.lq_set_gauge(ctx, torch.from_numpy(synth.gauge_links(L, EPS, 1000)).to(dev))
        b = torch.from_numpy(synth.gaussian_spinor(V, 2000)).to(dev)
        xe = b[:V // 2].contiguous()
        ye = torch.empty_like(xe)
        res = {"lattice": list(L), "ds_f32": ds_rate(lqdd, ctx, lqdd.LQ_F32, xe, ye, pk, reps=50),
               "ds_f64": ds_rate(lqdd, ctx, lqdd.LQ_F64, xe, ye, pk, reps=50)}
        norm = lqdd.lq_estimate_norm(ctx, lqdd.LQ_F64, 30, xe)
        fp64 = lqdd.make_params(tol=1e-10, restart=30, max_restarts=200)
        rich = lqdd.make_params(solver=lqdd.LQ_SOLVER_FGMRES, tol=1e-10, restart=30, max_restarts=100,
                                smoother=lqdd.LQ_SMOOTH_RICHARDSON, smooth_n=5, omega=0.8 / norm,
                                inner_prec=lqdd.LQ_F32)
        sol, xs = timed_solves(lqdd, torch, stream, ctx, b, (("mixed", mixed_params(lqdd), 5), ("fp64", fp64, 5),
                                                              ("fgmres_rich5", rich, 5)))
        res["solves"] = sol
        res["solve"] = solve_summary(sol, xs, torch)
        res["solve"]["fgmres_rich5_ms"] = sol["fgmres_rich5"]["ms"]
        return res
    finally:
        lqdd.lq_destroy(ctx)


def run_bf16(lqdd, torch, stream, ctx, db, x, pk, V, omega):
    """BF16 storage on the benchmark lattice: the D_S apply (1200 algorithmic
    bytes per site) against FP32 (1824), its relative error against the FP64
    apply, and FGMRES(10) df64 to 1e-10 preconditioned by Richardson(5) with
    BF16 against FP32 storage."""
    Vh = V // 2
    xe = db[:Vh].contiguous()
    out = {p: torch.empty_like(xe) for p in (lqdd.LQ_F64, lqdd.LQ_F32, lqdd.LQ_BF16)}
    res = {}
    for prec, name in ((lqdd.LQ_F32, "f32"), (lqdd.LQ_BF16, "bf16")):
        lqdd.lq_apply(ctx, lqdd.LQ_OP_SCHUR, prec, xe, out[prec])
        lqdd.lq_profile(ctx, 1)
        for _ in range(20):
            lqdd.lq_apply(ctx, lqdd.LQ_OP_SCHUR, prec, xe, out[prec])
        prof = read_profile(lqdd, ctx)
        lqdd.lq_profile(ctx, 0)
        k1, k2 = ("hop_k1_f32", "hop_k2_f32") if name == "f32" else ("hop_k1_bf16", "hop_k2_bf16")
        ms = (prof[k1]["ms"] + prof[k2]["ms"]) / 20
        by = (prof[k1]["bytes"] + prof[k2]["bytes"]) / 20
        res[name] = {"ds_us": round(1e3 * ms, 1), "ds_gbs": round(by / (ms / 1e3) / 1e9, 1),
                     "ds_frac": round(by / (ms / 1e3) / 1e9 / pk["hbm_gbs"], 4),
                     "bytes_per_site": round(by / Vh, 1)}
    lqdd.lq_apply(ctx, lqdd.LQ_OP_SCHUR, lqdd.LQ_F64, xe, out[lqdd.LQ_F64])
    ref = out[lqdd.LQ_F64]
    for prec, name in ((lqdd.LQ_F32, "f32"), (lqdd.LQ_BF16, "bf16")):
        res[name]["rel_err_vs_fp64"] = float(torch.linalg.vector_norm(out[prec] - ref) / torch.linalg.vector_norm(ref))
    for prec, name in ((lqdd.LQ_F32, "f32"), (lqdd.LQ_BF16, "bf16")):
        prm = lqdd.make_params(solver=lqdd.LQ_SOLVER_FGMRES, prec=lqdd.LQ_DF64, tol=1e-10, restart=10,
                               max_restarts=50, smoother=lqdd.LQ_SMOOTH_RICHARDSON, smooth_n=5, omega=omega,
                               inner_prec=prec)
        x.zero_()
        lqdd.lq_solve(ctx, prm, db, x)
        ts = []
        for _ in range(3):
            x.zero_()
            torch.cuda.synchronize()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            status, st = lqdd.lq_solve(ctx, prm, db, x)
            z.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(z))
        res[name]["fgmres_richardson5_ms"] = round(sorted(ts)[1], 2)
        res[name]["fgmres_richardson5_iters"] = st.iters
        res[name]["fgmres_richardson5_rel_resid_true"] = st.rel_resid_true
    return res


def read_profile(lqdd, ctx):
    """Per-class launches, device ms, algorithmic bytes and flops since lq_profile(ctx, 1)."""
    prof = {}
    for c in range(lqdd.LQ_K_COUNT):
        nl, cms, cb, cf = lqdd.lq_profile_read(ctx, c)
        if nl or cms:
            prof[lqdd.lq_kernel_class_name(c)] = {"launches": nl, "ms": round(cms, 4), "bytes": cb, "flops": cf}
    return prof


def run_force(lqdd, synth, torch, stream, dev, pk):
    """The fermion force of S = phi^+ (D^+ D)^{-1} phi on 24^3 x 48 (eps 0.25,
    m0 0.05, c_sw 1, Gaussian phi): the whole lq_fermion_force (two mixed
    odd-even solves to 1e-10 and the df64 gradient kernel) and the gradient
    kernel alone (lq_force), median of 5, with its per-class roofline."""
    import numpy as np
    L = (24, 24, 24, 48)
    V = int(np.prod(L))
    ctx = lqdd.lq_create(lqdd.make_lattice(L, TBC, 0.05, CSW), stream.cuda_stream)
    try:
        lqdd.lq_set_gauge(ctx, torch.from_numpy(synth.gauge_links(L, EPS, 1004)).to(dev))
        phi = torch.from_numpy(synth.gaussian_spinor(V, 2004)).to(dev)
        G = torch.empty((V, 4, 3, 3), dtype=torch.complex128, device=dev)
        prm = lqdd.make_params(solver=lqdd.LQ_SOLVER_FGMRES, prec=lqdd.LQ_DF64, tol=1e-10, restart=10,
                               max_restarts=20, smoother=lqdd.LQ_SMOOTH_GMRES, smooth_n=40, smooth_m=8,
                               smooth_tol=1e-5, inner_prec=lqdd.LQ_F32)
        X, Y = torch.empty_like(phi), torch.empty_like(phi)
        lqdd.lq_fermion_force(ctx, prm, phi, G)                      # workspace
        lqdd.lq_fermion_action(ctx, prm, phi, X, Y)

        def timed(fn):
            runs = []
            for _ in range(5):
                torch.cuda.synchronize()
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                out = fn()
                z.record(stream)
                torch.cuda.synchronize()
                runs.append((a.elapsed_time(z), out))
            return sorted(runs, key=lambda r: r[0])[2]

        t_full, (status, S, st) = timed(lambda: lqdd.lq_fermion_force(ctx, prm, phi, G))
        lqdd.lq_profile(ctx, 1)
        t_kernel, _ = timed(lambda: lqdd.lq_force(ctx, X, Y, G, coef=-2.0))
        prof = read_profile(lqdd, ctx)
        lqdd.lq_profile(ctx, 0)
        res = {"lattice": list(L), "S": S, "status": lqdd.lq_status_string(status),
               "fermion_force_ms": round(t_full, 2), "force_call_ms": round(t_kernel, 3),
               "solves": [s.as_dict() for s in st]}
        if "force" in prof:
            res["roofline"] = roofline_of("force", prof["force"], pk, V)
        return res
    finally:
        lqdd.lq_destroy(ctx)


def combine_ranks(dist, torch, device, ms, tot_bytes, e2e_ms):
    """Replicas: the timed region of the whole job is the slowest rank's (max
    over ranks), the work is every rank's (bytes summed over ranks)."""
    t = torch.tensor([ms, tot_bytes, e2e_ms], device=device, dtype=torch.float64)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t.clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[1]), float(tmax[2])


def run_ours(args):
    import numpy as np
    import torch

    from paper_2407_08092_gb300 import build as libbuild
    libbuild.build()
    from paper_2407_08092_gb300 import lqdd, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    V = int(np.prod(L_WORK))
    Vh = V // 2
    U = synth.gauge_links(L_WORK, EPS, LINK_SEED + rank)
    b = synth.gaussian_spinor(V, SRC_SEED + rank)
    stream = torch.cuda.current_stream()
    ctx = lqdd.lq_create(lqdd.make_lattice(L_WORK, TBC, M0, CSW), stream.cuda_stream)
    dU = torch.from_numpy(U).to(dev)
    db = torch.from_numpy(b).to(dev)
    dbe = db[:Vh].contiguous()
    x = torch.zeros_like(db)
    e = torch.empty_like(db)
    mixed = mixed_params(lqdd)
    info = {}

    def step(Ud, bd, bed, xd, ed):
        lqdd.lq_set_gauge(ctx, Ud)
        nrm = lqdd.lq_estimate_norm(ctx, lqdd.LQ_F32, 10, bed)
        rich = lqdd.make_params(prec=lqdd.LQ_DF64, smoother=lqdd.LQ_SMOOTH_RICHARDSON, smooth_n=5,
                                omega=0.8 / nrm, inner_prec=lqdd.LQ_F32)
        lqdd.lq_smooth(ctx, rich, bd, ed)
        xd.zero_()
        status, st = lqdd.lq_solve(ctx, mixed, bd, xd)
        if status != lqdd.LQ_OK:
            raise RuntimeError(f"solve: {lqdd.lq_status_string(status)} {st.as_dict()}")
        info["solve"] = st.as_dict()
        info["omega"] = 0.8 / nrm

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(dU, db, dbe, x, e)
    barrier()

    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    time.sleep(1.5)   # nvidia-smi's start-up queries disturb the GPU: let it settle first
    step_ms = {}

    def timed_steps(tag):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier()
        torch.cuda.nvtx.range_push(tag)
        for i in range(args.steps):
            ev[i][0].record(stream)
            step(dU, db, dbe, x, e)
            ev[i][1].record(stream)
        barrier()
        torch.cuda.nvtx.range_pop()
        step_ms[tag] = [round(a.elapsed_time(z), 3) for a, z in ev]
        return sum(step_ms[tag])

    # the timed region: K steps, CUDA events around each step on the library's stream
    n0, b0 = lqdd.lq_counters(ctx)
    ms = timed_steps("timed")
    n1, b1 = lqdd.lq_counters(ctx)
    step_bytes = (b1 - b0) / args.steps
    # the per-kernel-class device times (roofline, op): the same K steps again with
    # a pair of CUDA events around every launch on the library's stream (those
    # events cost about 2 us per launch, so the timed region above runs without them)
    lqdd.lq_profile(ctx, True)
    ms_profiled = timed_steps("profiled")
    prof = read_profile(lqdd, ctx)
    lqdd.lq_profile(ctx, False)

    # e2e: host (pinned) inputs and result, copies inside the timed region.  The
    # inputs are buffered four deep: an upload stream copies step i+3's gauge
    # field and source while step i computes, and a download stream reads step
    # i's solution after it.  Three steps of slack absorb the occasional
    # host-device transfer that takes many times its usual 7.6 ms (measured on
    # these shared hosts: single uploads of 70-139 ms and downloads of 30-43 ms,
    # a few times per 20 steps, with or without the clock sampler running).
    e2e = None
    if not args.no_e2e:
        NB = 4
        Uh = torch.from_numpy(U).pin_memory()
        bh = torch.from_numpy(b).pin_memory()
        xh = torch.empty_like(bh).pin_memory()
        bufs = [(torch.empty_like(dU), torch.empty_like(db), torch.zeros_like(db)) for _ in range(NB)]
        cu, cd = torch.cuda.Stream(), torch.cuda.Stream()
        ready = [torch.cuda.Event() for _ in range(NB)]   # inputs of the buffer set uploaded
        done = [torch.cuda.Event() for _ in range(NB)]    # the step using the set has finished
        read = [torch.cuda.Event() for _ in range(NB)]    # the set's solution has been downloaded
        ea, ez = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ea.record(stream)
        cu.wait_stream(stream)
        cd.wait_stream(stream)

        # where the time goes: each upload and download, and each step's span on
        # the compute stream (from the end of its wait for its inputs)
        tev = {k: [] for k in ("up", "down", "comp")}

        def span(st):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            return a, z

        def upload(i):
            k = i % NB
            if i >= NB:
                cu.wait_event(done[k])   # step i - NB, which used this set, has finished
            with torch.cuda.stream(cu):
                a, z = span(cu)
                bufs[k][0].copy_(Uh, non_blocking=True)
                bufs[k][1].copy_(bh, non_blocking=True)
                z.record(cu)
                tev["up"].append((a, z))
                ready[k].record(cu)

        for i in range(min(NB - 1, args.steps)):
            upload(i)
        t0s = []
        for i in range(args.steps):
            k = i % NB
            t0 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            t0s.append(t0)
            stream.wait_event(ready[k])
            if i >= NB:
                stream.wait_event(read[k])   # step i - NB's solution has left this set's x
            if i + NB - 1 < args.steps:
                upload(i + NB - 1)
            Ud, bd, xd = bufs[k]
            a, z = span(stream)
            step(Ud, bd, bd[:Vh].contiguous(), xd, e)
            z.record(stream)
            tev["comp"].append((a, z))
            done[k].record(stream)
            cd.wait_event(done[k])
            with torch.cuda.stream(cd):
                a, z = span(cd)
                xh.copy_(xd, non_blocking=True)
                z.record(cd)
                tev["down"].append((a, z))
                read[k].record(cd)
        stream.wait_stream(cu)
        stream.wait_stream(cd)
        ez.record(stream)
        barrier()
        e2e_ms = ea.elapsed_time(ez) / args.steps
        e2e_split = {k + "_ms": round(statistics.median(a.elapsed_time(z) for a, z in v), 3) for k, v in tev.items()}
        # per-step spans for the detail record: the interval between consecutive
        # step starts on the compute stream (waits included), and each part
        e2e_steps = {"start_to_start_ms": [round(a.elapsed_time(z), 3) for a, z in zip(t0s, t0s[1:] + [ez])]}
        e2e_steps.update({k + "_ms": [round(a.elapsed_time(z), 3) for a, z in v] for k, v in tev.items()})
        e2e = {"ms_per_step": e2e_ms, "h2d_bytes_per_step": int(Uh.numel() * 16 + bh.numel() * 16),
               "d2h_bytes_per_step": int(xh.numel() * 16), "step_bytes": step_bytes,
               "overlap": "inputs buffered four deep: step i+3's upload and step i's download on their own streams",
               "split_median": e2e_split, "per_step": e2e_steps}
        lqdd.lq_set_gauge(ctx, dU)

    clk = clocks.stop()

    # the operator the metric names: FP32 D_S on this lattice against measured HBM
    pk = peaks()
    ds_c1 = ds_rate(lqdd, ctx, lqdd.LQ_F32, dbe, torch.empty_like(dbe), pk, reps=20)

    # the plain FP64 GMRES(30) solve of the same system (native FP64 and df64),
    # timed beside the mixed one, medians of 5
    fp64 = lqdd.make_params(tol=1e-10, restart=30, max_restarts=200)
    df64 = lqdd.make_params(prec=lqdd.LQ_DF64, tol=1e-10, restart=30, max_restarts=200)
    solves, xsol = timed_solves(lqdd, torch, stream, ctx, db, (("fp64", fp64, 5), ("df64", df64, 5),
                                                              ("mixed", mixed, 5)))
    solve_c1 = solve_summary(solves, xsol, torch)
    solve_c1["df64_ms"] = solves["df64"]["ms"]
    del xsol

    # smoothers on the benchmark lattice: one SAP(3, 4) call (the paper's Table 2
    # smoother call; 4^4 blocks, FP32) against one odd-even Richardson(5) call,
    # and the FGMRES solve preconditioned by SAP(3, 4) against the mixed solve
    sap = None
    if not args.no_sap:
        sap = run_sap(lqdd, torch, stream, ctx, db, x, pk_peaks=pk, V=V, omega=info["omega"])

    # BF16 storage of spinors and links against FP32
    bf16 = None
    if not args.no_bf16:
        bf16 = run_bf16(lqdd, torch, stream, ctx, db, x, pk, V, info["omega"])

    # batched: 12 spin-colour point sources on each of four lattices
    batched = None
    if not args.no_batch:
        batched = run_batched(lqdd, synth, torch, stream, dev)

    big = None
    if not args.no_48x96 and world == 1:
        big = run_48x96(lqdd, synth, torch, stream, dev, pk)

    c0 = None
    if not args.no_8x4 and world == 1:
        c0 = run_c0(lqdd, synth, torch, stream, dev, pk)

    force = None
    if not args.no_force:
        force = run_force(lqdd, synth, torch, stream, dev, pk)

    # max over ranks of the timed region, bytes summed over ranks
    tot_bytes = step_bytes * args.steps
    if dist:
        ms, tot_bytes, e2e_ms = combine_ranks(dist, torch, dev, ms, tot_bytes, (e2e or {}).get("ms_per_step", 0.0))
        if e2e:
            e2e["ms_per_step"] = e2e_ms
    lqdd.lq_destroy(ctx)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    value = tot_bytes / (ms / 1e3) / 1e9
    # dominant kernel class by device time
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"]) if prof else None
    roofline = None
    if dom:
        r = roofline_of(dom[0], dom[1], pk, V)
        roofline = {k: r[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel",
                                      "avg_launch_us", "algorithmic_bytes_per_launch")}
        roofline["share_of_step"] = round(dom[1]["ms"] / ms_profiled, 4)
        roofline["peak_src"] = "measured"
        roofline["timing"] = f"events per launch, 2nd pass of the K steps ({ms_profiled / args.steps:.1f} ms/step)"
    ops = {k: roofline_of(k, prof[k], pk, V) for k in sorted(prof) if prof[k]["ms"] > 0 and prof[k]["launches"]}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)

    def pick(d, *keys):
        return None if d is None else {k: d[k] for k in keys if k in d}

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+df64", "data": "synthetic",
        "config": {"workload": "32^3x64 step: set_gauge, 10 FP32 power its, Richardson(5) FP32, "
                               "FGMRES(10) df64 / GMRES(8) FP32 to 1e-10",
                   "eps": EPS, "m0": M0, "csw": CSW, "t_bc": TBC,
                   "l2": "inputs larger than L2; no flush",
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": None if e2e is None else {
            "value": round(e2e["step_bytes"] * world / (e2e["ms_per_step"] / 1e3) / 1e9, 1), "unit": "GB/s",
            "h2d_bytes_per_step": e2e["h2d_bytes_per_step"], "d2h_bytes_per_step": e2e["d2h_bytes_per_step"],
            "ms_per_step": round(e2e["ms_per_step"], 3)},
        "gpu_launches": int(n1 - n0),
        "clocks": clk,
        # the metric's two halves, named: FP32 D_S against measured HBM, and the
        # mixed solve against plain FP64 GMRES(30) (x = speed-up, rres = true
        # residuals, xdiff = ||x_mixed - x_fp64|| / ||x_fp64||)
        "ds_f32": {"32^3x64": ds_c1, "48^3x96": None if big is None else big["ds_f32"],
                   "8^4_in_L2": None if c0 is None else c0["ds_f32"]},
        "solve": {"32^3x64": solve_c1, "48^3x96": None if big is None else big["solve"],
                  "8^4": None if c0 is None else c0["solve"]},
        "batched": None if batched is None else {
            "group_ms": batched["group"]["ms"], "per_lattice_ms": batched["per_lattice"]["ms"],
            "seq_mixed_ms": batched["sequential"]["ms"], "seq_fp64_ms": batched["fp64_sequential"]["ms"],
            "x_fp64": batched["speedup_vs_fp64"], "worst_rres": float(f"{batched['group']['worst_rel_resid_true']:.3g}"),
            "xdiff": float(f"{batched['xdiff_vs_fp64']:.3g}"),
            "hop_pair_ms": batched["tuning"]["hop_pair_ms"]},
        "force": None if force is None else {
            "ms": force["fermion_force_ms"], "kernel_ms": force["force_call_ms"],
            "frac": (force.get("roofline") or {}).get("frac")},
        "sap": None if sap is None else {
            "sap34_ms": sap["sap_3_4_ms"], "rich5_ms": sap["richardson_5_ms"], "fgmres_sap_ms": sap["fgmres_sap_ms"],
            "bound": (sap.get("roofline") or {}).get("bound"), "frac": (sap.get("roofline") or {}).get("frac"),
            "hbm_frac": (sap.get("roofline") or {}).get("hbm_frac")},
        "bf16": None if bf16 is None else pick(bf16["bf16"], "ds_us", "ds_frac", "rel_err_vs_fp64"),
        # df64 classes against the SMs' instruction-issue ceiling (ncu-counted
        # instructions per launch over the live launch time); the 15-instruction
        # flop model beside it
        "df64_issue": {k: {"frac": v["frac"], "model_frac": v["df64_model_frac"]}
                       for k, v in ops.items() if v.get("bound") == "issue"},
        "detail": args.detail,
    }
    print(json.dumps(line), flush=True)
    if args.detail:
        detail = {"line": line, "kernels": prof, "op": ops, "step_bytes": step_bytes, "step_ms": step_ms,
                  "solve_32x64": solves, "sap": sap, "bf16": bf16, "batched": batched, "lattice_48x96": big,
                  "lattice_8x4": c0, "force": force, "e2e": e2e}
        os.makedirs(os.path.dirname(os.path.abspath(args.detail)), exist_ok=True)
        with open(args.detail, "w") as f:
            json.dump(detail, f, indent=1, default=str)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
