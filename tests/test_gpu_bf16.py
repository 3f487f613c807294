"""BF16 storage (spinors and 12-real links in BF16, FP32 clover and arithmetic)
against the FP64 oracle.

BF16 keeps 8 significand bits: one rounding has a relative error up to 2^-9
(about 2e-3).  A D_S apply rounds its input, every link and its output, so
its error against the FP64 oracle is a few 1e-3 in the norm; the tests bound
it by 1e-2 and report it.  The FGMRES solve with a BF16 Richardson
preconditioner must still reach 1e-10 on the oracle's true residual: the FP64
(df64) outer iteration corrects the low-precision preconditioner.
"""
import numpy as np
import pytest

from paper_2407_08092_gb300 import synth

from .gpu_util import Pair, rel

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4, 4), (8, 6, 4, 10), (16, 16, 16, 8)]


@pytest.mark.parametrize("L", SHAPES, ids=lambda L: "x".join(map(str, L)))
def test_bf16_schur_against_oracle(L):
    from paper_2407_08092_gb300 import lqdd
    p = Pair(L, eps=0.25, seed=1300 + sum(L), m0=0.05, csw=1.0)
    try:
        x = synth.gaussian_spinor(p.Vh, 51)
        got = p.apply(lqdd.LQ_OP_SCHUR, lqdd.LQ_BF16, x)
        want = p.lat.schur(x)
        err = rel(got, want)
        assert err < 1e-2, err
        # it is BF16, not FP32: the FP32 apply is far closer
        assert rel(p.apply(lqdd.LQ_OP_SCHUR, lqdd.LQ_F32, x), want) < 1e-5 < err
        got_dag = p.apply(lqdd.LQ_OP_SCHUR_DAG, lqdd.LQ_BF16, x)
        assert rel(got_dag, p.lat.schur_dag(x)) < 1e-2
    finally:
        p.close()


def test_bf16_richardson_smoother_against_oracle():
    import oracle
    from paper_2407_08092_gb300 import lqdd
    L = (8, 8, 8, 8)
    p = Pair(L, eps=0.25, seed=1000, m0=0.05, csw=1.0)
    try:
        r = synth.gaussian_spinor(p.V, 61)
        omega = 0.8 / 5.2
        prm = lqdd.make_params(prec=lqdd.LQ_DF64, smoother=lqdd.LQ_SMOOTH_RICHARDSON, smooth_n=5, omega=omega,
                               inner_prec=lqdd.LQ_BF16)
        out = p.torch.empty_like(p.dev(r))
        lqdd.lq_smooth(p.ctx, prm, p.dev(r), out)
        want = oracle.smoother(p.lat, r, "richardson", 5, omega=omega)
        assert rel(p.host(out), want) < 1e-2
    finally:
        p.close()


def test_fgmres_with_bf16_richardson_reaches_1e10():
    from paper_2407_08092_gb300 import lqdd
    L = (8, 8, 8, 8)
    p = Pair(L, eps=0.25, seed=1000, m0=0.05, csw=1.0)
    try:
        b = synth.gaussian_spinor(p.V, 2000)
        db = p.dev(b)
        nrm = lqdd.lq_estimate_norm(p.ctx, lqdd.LQ_F32, 20, db[:p.Vh].contiguous())
        x = p.torch.zeros_like(db)
        prm = lqdd.make_params(solver=lqdd.LQ_SOLVER_FGMRES, prec=lqdd.LQ_DF64, tol=1e-10, restart=10,
                               max_restarts=50, smoother=lqdd.LQ_SMOOTH_RICHARDSON, smooth_n=5, omega=0.8 / nrm,
                               inner_prec=lqdd.LQ_BF16)
        status, st = lqdd.lq_solve(p.ctx, prm, db, x)
        assert status == lqdd.LQ_OK
        r_true = np.linalg.norm(b - p.lat.dirac(p.host(x))) / np.linalg.norm(b)
        assert r_true <= 1e-10
    finally:
        p.close()


def test_bf16_argument_errors():
    from paper_2407_08092_gb300 import lqdd
    p = Pair((4, 4, 4, 4), seed=3)
    try:
        v = p.dev(synth.gaussian_spinor(p.V, 1))
        out = p.torch.empty_like(v)
        with pytest.raises(lqdd.LqError) as ei:
            lqdd.lq_apply(p.ctx, lqdd.LQ_OP_FULL, lqdd.LQ_BF16, v, out)
        assert ei.value.status == lqdd.LQ_ERR_ARG
        with pytest.raises(lqdd.LqError) as ei:     # BF16 is offered for Richardson only
            lqdd.lq_smooth(p.ctx, lqdd.make_params(prec=lqdd.LQ_DF64, smoother=lqdd.LQ_SMOOTH_GMRES, smooth_n=1,
                                                   smooth_m=4, inner_prec=lqdd.LQ_BF16), v, out)
        assert ei.value.status == lqdd.LQ_ERR_ARG
    finally:
        p.close()
