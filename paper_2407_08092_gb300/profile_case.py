"""A small, self-contained case of the library's kernels for profiler captures.

Builds a context on a seeded lattice (default 24^3 x 48, whose per-launch
working set is larger than L2 but whose device footprint stays within a few
GB) and then either applies D_S (K1 + K2) `--apps` times in one precision
through the C ABI (printing per-class device times), runs `--apps`
mixed-precision solves (FGMRES(10) in df64 preconditioned by GMRES(8) in
FP32), a batched solve of `--nrhs` point sources through a one-member group
(printing the autotuner's choice), SAP(3, 4) smoother calls, the
fermion-force kernel, or lq_set_gauge (the clover build), e.g.
``python -m paper_2407_08092_gb300.profile_case --lattice 24,24,24,48 --prec 1 --apps 3``.
"""
import argparse

import numpy as np
import torch

from paper_2407_08092_gb300 import lqdd, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lattice", default="24,24,24,48")
    ap.add_argument("--prec", type=int, default=1, help="0 FP64, 1 FP32, 2 df64")
    ap.add_argument("--apps", type=int, default=3)
    ap.add_argument("--op", type=int, default=lqdd.LQ_OP_SCHUR)
    ap.add_argument("--mode", default="apply", choices=["apply", "solve", "batch", "force", "sap", "gauge"])
    ap.add_argument("--nrhs", type=int, default=12)
    ap.add_argument("--shape", default=None,
                    help="batch mode: pin the batched hop's launch shape 'sites_per_tile,rhs_per_thread,grid_factor' "
                         "instead of autotuning it")
    a = ap.parse_args()
    L = tuple(int(v) for v in a.lattice.split(","))
    V = int(np.prod(L))
    ctx = lqdd.lq_create(lqdd.make_lattice(L, -1, 0.05, 1.0), torch.cuda.current_stream().cuda_stream)
    lqdd.lq_set_gauge(ctx, torch.from_numpy(synth.gauge_links(L, 0.25, 1003)).cuda())
    if a.mode == "apply":
        n = V if a.op == lqdd.LQ_OP_FULL else V // 2
        x = torch.from_numpy(synth.gaussian_spinor(n, 2003)).cuda()
        y = torch.empty_like(x)
        lqdd.lq_apply(ctx, a.op, a.prec, x, y)
        lqdd.lq_profile(ctx, 1)
        for _ in range(a.apps):
            lqdd.lq_apply(ctx, a.op, a.prec, x, y)
        torch.cuda.synchronize()
        for c in range(lqdd.LQ_K_COUNT):
            nl, ms, by, fl = lqdd.lq_profile_read(ctx, c)
            if nl:
                print(f"{lqdd.lq_kernel_class_name(c):14s} {nl:5d} launches {1e3 * ms / nl:9.2f} us/launch "
                      f"{by / (ms * 1e6):8.1f} GB/s")
        lqdd.lq_profile(ctx, 0)
        out = float(y.abs().sum())
    elif a.mode == "batch":
        n = a.nrhs
        b = torch.zeros((n, V, 4, 3), dtype=torch.complex128, device="cuda")
        for r in range(n):
            b[r, 0, r % 4, (r // 4) % 3] = 1.0
        x = torch.zeros_like(b)
        grp = lqdd.lq_group_create([ctx], torch.cuda.current_stream().cuda_stream)
        if a.shape:
            lqdd.lq_group_set_shape(grp, *(int(v) for v in a.shape.split(",")))
        for _ in range(a.apps):
            x.zero_()
            status, st = lqdd.lq_solve_group(grp, ctx, lqdd.make_batch_params(), [b], [x])
            assert status == lqdd.LQ_OK, lqdd.lq_status_string(status)
        out = max(s.rel_resid_true for s in st)
        print("outer corrections", [s.iters for s in st], "inner steps", [s.inner_iters for s in st],
              "ms", round(st[0].time_ms, 2))
        print("tuning (sites/tile, rhs/thread, grid, blas blocks, hop pair ms, blas pair ms)", lqdd.lq_group_tuning(grp))
        lqdd.lq_group_destroy(grp)
    elif a.mode == "sap":
        r = torch.from_numpy(synth.gaussian_spinor(V, 2003)).cuda()
        e = torch.empty_like(r)
        prm = lqdd.make_params(smoother=lqdd.LQ_SMOOTH_SAP, smooth_n=3, smooth_m=4, inner_prec=lqdd.LQ_F32,
                               prec=lqdd.LQ_DF64)
        lqdd.lq_smooth(ctx, prm, r, e)
        lqdd.lq_profile(ctx, 1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(a.apps):
            lqdd.lq_smooth(ctx, prm, r, e)
        ev[1].record()
        torch.cuda.synchronize()
        print("SAP(3,4)", round(ev[0].elapsed_time(ev[1]) / a.apps, 3), "ms per call")
        for c in range(lqdd.LQ_K_COUNT):
            nl, ms, by, fl = lqdd.lq_profile_read(ctx, c)
            if nl:
                print(f"{lqdd.lq_kernel_class_name(c):14s} {nl:5d} launches {1e3 * ms / nl:9.2f} us/launch "
                      f"{by / (ms * 1e6):8.1f} GB/s")
        lqdd.lq_profile(ctx, 0)
        out = float(e.abs().sum())
    elif a.mode == "gauge":   # lq_set_gauge: layout, clover field, assembly and inverse
        U = torch.from_numpy(synth.gauge_links(L, 0.25, 1003)).cuda()
        lqdd.lq_profile(ctx, 1)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(a.apps):
            lqdd.lq_set_gauge(ctx, U)
        ev[1].record()
        torch.cuda.synchronize()
        print("set_gauge", round(ev[0].elapsed_time(ev[1]) / a.apps, 3), "ms per call")
        for c in range(lqdd.LQ_K_COUNT):
            nl, ms, by, fl = lqdd.lq_profile_read(ctx, c)
            if nl:
                print(f"{lqdd.lq_kernel_class_name(c):14s} {nl:5d} launches {1e3 * ms / nl:9.2f} us/launch "
                      f"{by / (ms * 1e6):8.1f} GB/s {fl / (ms * 1e9):8.3f} TFLOP/s")
        lqdd.lq_profile(ctx, 0)
        out = 0.0
    elif a.mode == "force":
        X = torch.from_numpy(synth.gaussian_spinor(V, 71)).cuda()
        Y = torch.from_numpy(synth.gaussian_spinor(V, 72)).cuda()
        G = torch.empty((V, 4, 3, 3), dtype=torch.complex128, device="cuda")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(a.apps):
            lqdd.lq_force(ctx, X, Y, G, coef=-2.0)
        ev[1].record()
        torch.cuda.synchronize()
        print("force kernel pair", round(ev[0].elapsed_time(ev[1]) / a.apps, 3), "ms per call")
        out = float(G.abs().max())
    else:
        b = torch.from_numpy(synth.gaussian_spinor(V, 2003)).cuda()
        x = torch.zeros_like(b)
        p = lqdd.make_params(solver=lqdd.LQ_SOLVER_FGMRES, prec=lqdd.LQ_DF64, tol=1e-10, restart=10,
                             max_restarts=20, smoother=lqdd.LQ_SMOOTH_GMRES, smooth_n=40, smooth_m=8,
                             smooth_tol=1e-5, inner_prec=lqdd.LQ_F32)
        lqdd.lq_solve(ctx, p, b, x)
        lqdd.lq_profile(ctx, 1)
        for _ in range(a.apps):
            x.zero_()
            status, st = lqdd.lq_solve(ctx, p, b, x)
            assert status == lqdd.LQ_OK, lqdd.lq_status_string(status)
        torch.cuda.synchronize()
        print("mixed solve", round(st.time_ms, 2), "ms", st.iters, "outer", st.inner_iters, "inner")
        for c in range(lqdd.LQ_K_COUNT):
            nl, ms, by, fl = lqdd.lq_profile_read(ctx, c)
            if nl:
                print(f"{lqdd.lq_kernel_class_name(c):14s} {nl:5d} launches {1e3 * ms / nl:9.2f} us/launch "
                      f"{by / (ms * 1e6):8.1f} GB/s")
        lqdd.lq_profile(ctx, 0)
        out = st.rel_resid_true
    torch.cuda.synchronize()
    print("ok", L, a.mode, "prec", a.prec, "apps", a.apps, out)
    lqdd.lq_destroy(ctx)


if __name__ == "__main__":
    main()
