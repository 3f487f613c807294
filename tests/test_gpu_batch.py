"""Batched (multi right-hand side) solve against the FP64 oracle.

lq_solve_batch applies D_S to all right-hand sides in each launch (each
site's links and clover read once), runs batched FP32 GMRES cycles with the
Givens least squares on the device (replayed as a CUDA graph), and corrects in
df64.  Each right-hand side's solution must meet the 1e-10 target on the true
residual recomputed by the oracle, and agree with the oracle's own solution.
"""
import numpy as np
import pytest

import oracle
from paper_2407_08092_gb300 import synth

from .gpu_util import Pair, rel

pytestmark = pytest.mark.gpu


def sources(lat, n, seed):
    """A mix of spin-colour point sources and Gaussian sources."""
    out = []
    for r in range(n):
        if r % 2 == 0:
            site = (r * 7919) % lat.V
            out.append(synth.point_source(lat.L, site, (r // 2) % 4, (r // 8) % 3))
        else:
            out.append(synth.gaussian_spinor(lat.V, seed + r))
    return np.stack(out)


@pytest.mark.parametrize("L,n", [((4, 4, 4, 4), 3), ((6, 4, 2, 4), 5), ((8, 8, 8, 8), 12)],
                         ids=["4^4x3", "6x4x2x4x5", "8^4x12"])
def test_solve_batch_against_oracle(L, n):
    from paper_2407_08092_gb300 import lqdd
    p = Pair(L, eps=0.25, seed=1100 + sum(L), m0=0.05, csw=1.0)
    try:
        b = sources(p.lat, n, 300)
        db = p.dev(b)
        x = p.torch.zeros_like(db)
        status, stats = lqdd.lq_solve_batch(p.ctx, lqdd.make_batch_params(tol=1e-10, restart=16), n, db, x)
        assert status == lqdd.LQ_OK, (lqdd.lq_status_string(status), [s.as_dict() for s in stats])
        xs = p.host(x)
        for r in range(n):
            r_true = np.linalg.norm(b[r] - p.lat.dirac(xs[r])) / np.linalg.norm(b[r])
            assert r_true <= 1e-10, (r, r_true)
            assert abs(r_true - stats[r].rel_resid_true) <= 1e-3 * r_true + 1e-15
            assert stats[r].rel_resid <= 1e-10
        # the solutions themselves against the oracle's odd-even GMRES
        for r in (0, n - 1):
            xo, _ = oracle.solve(p.lat, b[r], tol=1e-12, restart=30, max_restarts=200)
            assert rel(xs[r], xo) < 1e-8
    finally:
        p.close()


def test_solve_batch_matches_single_solves():
    """The same systems solved one at a time and as one batch agree to the
    solves' tolerance; a zero right-hand side gives x = 0."""
    from paper_2407_08092_gb300 import lqdd
    p = Pair((8, 4, 4, 8), eps=0.25, seed=77)
    try:
        b = sources(p.lat, 4, 400)
        b[2] = 0.0
        db = p.dev(b)
        xb = p.torch.zeros_like(db)
        status, _ = lqdd.lq_solve_batch(p.ctx, lqdd.make_batch_params(tol=1e-11), 4, db, xb)
        assert status == lqdd.LQ_OK
        xbh = p.host(xb)
        assert np.abs(xbh[2]).max() == 0.0
        for r in (0, 1, 3):
            xs = p.torch.zeros_like(db[r])
            st, _ = lqdd.lq_solve(p.ctx, lqdd.make_params(tol=1e-11, restart=30, max_restarts=200),
                                  db[r].contiguous(), xs)
            assert st == lqdd.LQ_OK
            assert rel(xbh[r], p.host(xs)) < 1e-9
    finally:
        p.close()


def test_solve_batch_status_codes():
    from paper_2407_08092_gb300 import lqdd
    p = Pair((4, 4, 4, 4))
    try:
        b = sources(p.lat, 2, 500)
        db = p.dev(b)
        x = p.torch.zeros_like(db)
        bad = lqdd.make_batch_params()
        bad.inner_prec = lqdd.LQ_F64
        with pytest.raises(lqdd.LqError) as ei:
            lqdd.lq_solve_batch(p.ctx, bad, 2, db, x)
        assert ei.value.status == lqdd.LQ_ERR_ARG
        # one correction step cannot reach 1e-12: NOT_CONVERGED with stats filled
        status, stats = lqdd.lq_solve_batch(p.ctx, lqdd.make_batch_params(tol=1e-12, max_restarts=1,
                                                                          smooth_tol=1e-3), 2, db, x)
        assert status == lqdd.LQ_ERR_NOT_CONVERGED
        assert all(s.rel_resid > 1e-12 for s in stats)
        b[1, 0, 0, 0] = np.nan
        with pytest.raises(lqdd.LqError) as ei:
            lqdd.lq_solve_batch(p.ctx, lqdd.make_batch_params(), 2, p.dev(b), x)
        assert ei.value.status == lqdd.LQ_ERR_NAN
    finally:
        p.close()


def test_solve_group_uneven_lattices():
    """Right-hand sides of four lattices of different sizes (each with its own
    links) solved together: every system meets the target on the oracle's true
    residual, and the launch shapes the autotuner chose are valid; with the
    autotuner off the fixed shapes give converged solutions as well."""
    from paper_2407_08092_gb300 import lqdd
    specs = [((8, 8, 8, 8), 3), ((6, 4, 2, 4), 2), ((4, 4, 4, 4), 4), ((16, 8, 8, 8), 2)]
    pairs = [Pair(L, eps=0.25, seed=1101 + i, m0=0.05, csw=1.0) for i, (L, _) in enumerate(specs)]
    grp = lqdd.lq_group_create([p.ctx for p in pairs], pairs[0].torch.cuda.current_stream().cuda_stream)
    try:
        bs = [sources(p.lat, n, 400 + 10 * i) for i, (p, (_, n)) in enumerate(zip(pairs, specs))]
        db = [p.dev(b) for p, b in zip(pairs, bs)]
        for autotune in (True, False):
            lqdd.lq_group_set_autotune(grp, autotune)
            xs = [p.torch.zeros_like(d) for p, d in zip(pairs, db)]
            status, stats = lqdd.lq_solve_group(grp, pairs[0].ctx, lqdd.make_batch_params(tol=1e-10, restart=16),
                                                db, xs)
            assert status == lqdd.LQ_OK, lqdd.lq_status_string(status)
            assert len(stats) == sum(n for _, n in specs)
            k = 0
            for p, b, x in zip(pairs, bs, xs):
                xh = p.host(x)
                for r in range(b.shape[0]):
                    r_true = np.linalg.norm(b[r] - p.lat.dirac(xh[r])) / np.linalg.norm(b[r])
                    assert r_true <= 1e-10, (p.L, r, r_true)
                    assert abs(r_true - stats[k].rel_resid_true) <= 1e-3 * r_true + 1e-15
                    k += 1
            spt, rpt, grid, blas, hop_ms, blas_ms = lqdd.lq_group_tuning(grp)
            assert spt in (16, 32, 64, 128) and rpt in (0, 1, 2) and grid >= 1 and blas >= 1
            assert rpt != 0 or spt in (32, 64)
            if autotune:
                assert hop_ms > 0 and blas_ms > 0
            else:
                assert (spt, rpt, hop_ms, blas_ms) == (32, 1, 0.0, 0.0)
        # every pinned launch shape (two right-hand sides per thread with odd counts
        # included, and the staged form whose tiles cover every right-hand side)
        # gives converged solutions
        for spt, rpt, fac in [(32, 2, 1), (128, 2, 0), (16, 1, 2), (64, 2, 2), (32, 0, 1), (64, 0, 2), (32, 0, 0)]:
            lqdd.lq_group_set_shape(grp, spt, rpt, fac)
            xs2 = [p.torch.zeros_like(d) for p, d in zip(pairs, db)]
            status, stats = lqdd.lq_solve_group(grp, pairs[0].ctx, lqdd.make_batch_params(tol=1e-10), db, xs2)
            assert status == lqdd.LQ_OK
            assert lqdd.lq_group_tuning(grp)[:2] == (spt, rpt)
            for p, b, x in zip(pairs, bs, xs2):
                xh = p.host(x)
                for r in range(b.shape[0]):
                    assert np.linalg.norm(b[r] - p.lat.dirac(xh[r])) / np.linalg.norm(b[r]) <= 1e-10
        # the same systems one member at a time (lq_solve_batch) give the same solutions
        for p, d, x in zip(pairs, db, xs):
            x1 = p.torch.zeros_like(d)
            status, _ = lqdd.lq_solve_batch(p.ctx, lqdd.make_batch_params(tol=1e-10, restart=16), d.shape[0], d, x1)
            assert status == lqdd.LQ_OK
            assert rel(p.host(x1), p.host(x)) < 1e-8
    finally:
        lqdd.lq_group_destroy(grp)
        for p in pairs:
            p.close()


def test_solve_group_status_codes():
    from paper_2407_08092_gb300 import lqdd
    a = Pair((4, 4, 4, 4), seed=7)
    b = Pair((6, 4, 2, 4), seed=8)
    try:
        with pytest.raises(lqdd.LqError):
            lqdd.lq_group_create([a.ctx, a.ctx])            # a context twice
        grp = lqdd.lq_group_create([a.ctx, b.ctx])
        try:
            with pytest.raises(lqdd.LqError):
                lqdd.lq_group_tuning(grp)                   # no solve yet
            with pytest.raises(lqdd.LqError) as ei:          # the staged form takes 32 or 64 sites per tile
                lqdd.lq_group_set_shape(grp, 16, 0, 1)
            assert ei.value.status == lqdd.LQ_ERR_ARG
            da = a.dev(sources(a.lat, 2, 11))
            dbb = b.dev(sources(b.lat, 1, 12))
            xa, xb = a.torch.zeros_like(da), b.torch.zeros_like(dbb)
            with pytest.raises(lqdd.LqError) as ei:          # the batch runs in df64 / FP32 only
                lqdd.lq_solve_group(grp, a.ctx, lqdd.make_params(tol=1e-10), [da, dbb], [xa, xb])
            assert ei.value.status == lqdd.LQ_ERR_ARG
            status, stats = lqdd.lq_solve_group(grp, a.ctx, lqdd.make_batch_params(tol=1e-13, max_restarts=1,
                                                                                     smooth_n=1),
                                                [da, dbb], [xa, xb])
            assert status == lqdd.LQ_ERR_NOT_CONVERGED and len(stats) == 3
        finally:
            lqdd.lq_group_destroy(grp)
    finally:
        a.close()
        b.close()


def test_full_size_batched_workload():
    """The full batched workload: 12 spin-colour point sources at the origin on
    each of 24^3 x 48, 8^4, 16^4 and 16^3 x 32 (own links, eps 0.25, m0 0.05,
    c_sw 1; link seeds 1103, 1101, 1102, 1104), 48 systems in one lq_solve_group
    with the benchmark's parameters (inner batched GMRES(8) to 1e-5).  Every
    solution's true residual, recomputed by one oracle application of the full
    D, meets 1e-10, and agrees with the library's own report."""
    from paper_2407_08092_gb300 import lqdd
    specs = [((24, 24, 24, 48), 1103), ((8, 8, 8, 8), 1101), ((16, 16, 16, 16), 1102), ((16, 16, 16, 32), 1104)]
    n = 12
    pairs = [Pair(L, eps=0.25, seed=seed, m0=0.05, csw=1.0) for L, seed in specs]
    torch = pairs[0].torch
    grp = lqdd.lq_group_create([p.ctx for p in pairs], torch.cuda.current_stream().cuda_stream)
    try:
        db, xs = [], []
        for p in pairs:
            b = torch.zeros((n, p.V, 4, 3), dtype=torch.complex128, device="cuda")
            for r in range(n):
                b[r, 0, r % 4, r // 4] = 1.0
            db.append(b)
            xs.append(torch.zeros_like(b))
        status, stats = lqdd.lq_solve_group(grp, pairs[0].ctx, lqdd.make_batch_params(), db, xs)
        assert status == lqdd.LQ_OK, lqdd.lq_status_string(status)
        k = 0
        worst = 0.0
        for p, b, x in zip(pairs, db, xs):
            bh, xh = p.host(b), p.host(x)
            for r in range(n):
                r_true = np.linalg.norm(bh[r] - p.lat.dirac(xh[r])) / np.linalg.norm(bh[r])
                assert r_true <= 1e-10, (p.L, r, r_true)
                assert abs(r_true - stats[k].rel_resid_true) <= 1e-3 * r_true + 1e-15
                worst = max(worst, r_true)
                k += 1
        assert k == 4 * n and worst > 0
    finally:
        lqdd.lq_group_destroy(grp)
        for p in pairs:
            p.close()
