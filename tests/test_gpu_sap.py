"""SAP(n, m) on the GPU (FP32 block solves, one CTA per block) against the
FP64 oracle of Algorithm 1.

* lq_smooth with the SAP smoother against oracle/sap.py on lattices with
  several blocks per colour, blocks spanning a whole direction, both time
  boundary conditions: relative error <= 1e-5 (FP32);
* the FGMRES solve preconditioned by SAP reaches 1e-10 on the oracle's true
  residual;
* at the benchmark size 32^3 x 64, with exact block solves, the residual left
  by SAP(1, many) vanishes on the blocks of the last colour swept (black), a
  property of Algorithm 1 at any size (checked with the FP64 operator);
* argument errors.
"""
import numpy as np
import pytest

from oracle import sap as osap
from paper_2407_08092_gb300 import synth

from .gpu_util import Pair, rel

pytestmark = pytest.mark.gpu


def sap_params(lqdd, n, m, block=(0, 0, 0, 0)):
    return lqdd.make_params(smoother=lqdd.LQ_SMOOTH_SAP, smooth_n=n, smooth_m=m, inner_prec=lqdd.LQ_F32,
                            prec=lqdd.LQ_DF64, sap_block=block)


@pytest.mark.parametrize("L,block,t_bc,nm", [
    ((8, 8, 4, 4), (4, 4, 2, 2), -1, (3, 4)),
    ((4, 4, 4, 4), (2, 2, 2, 2), 1, (2, 3)),
    ((8, 4, 4, 8), (4, 4, 4, 4), -1, (3, 4)),       # y and z: one block spanning the direction
    ((4, 4, 2, 4), (4, 2, 2, 4), -1, (1, 6)),       # x, z, t spanned: the time wrap stays inside a block
    ((8, 8, 8, 8), (4, 4, 4, 4), -1, (3, 4)),
], ids=["8x8x4x4/4x4x2x2", "4^4/2^4-periodic", "8x4x4x8/4^4", "4x4x2x4/4x2x2x4", "8^4/4^4"])
def test_sap_smoother_matches_oracle(L, block, t_bc, nm):
    from paper_2407_08092_gb300 import lqdd
    p = Pair(L, eps=0.25, seed=1200 + sum(L), m0=0.05, csw=1.0, t_bc=t_bc)
    try:
        n, m = nm
        r = synth.gaussian_spinor(p.V, 91)
        out = p.torch.empty_like(p.dev(r))
        lqdd.lq_smooth(p.ctx, sap_params(lqdd, n, m, block), p.dev(r), out)
        got = p.host(out)
        want = osap.sap(p.lat, r, n, m, block)
        assert rel(got, want) < 1e-5
    finally:
        p.close()


def test_fgmres_with_sap_preconditioner():
    from paper_2407_08092_gb300 import lqdd
    L = (8, 8, 8, 8)
    p = Pair(L, eps=0.25, seed=1000, m0=0.05, csw=1.0)
    try:
        b = synth.gaussian_spinor(p.V, 2000)
        db = p.dev(b)
        x = p.torch.zeros_like(db)
        prm = lqdd.make_params(solver=lqdd.LQ_SOLVER_FGMRES, prec=lqdd.LQ_DF64, tol=1e-10, restart=10,
                               max_restarts=20, smoother=lqdd.LQ_SMOOTH_SAP, smooth_n=3, smooth_m=4,
                               inner_prec=lqdd.LQ_F32)
        status, st = lqdd.lq_solve(p.ctx, prm, db, x)
        assert status == lqdd.LQ_OK
        r_true = np.linalg.norm(b - p.lat.dirac(p.host(x))) / np.linalg.norm(b)
        assert r_true <= 1e-10
        # SAP(3, 4) is a strong preconditioner: far fewer outer steps than plain GMRES needs
        assert st.iters <= 20, st.iters
    finally:
        p.close()


def test_full_size_exact_block_solves_zero_the_black_residual():
    from paper_2407_08092_gb300 import lqdd
    L = (32, 32, 32, 64)
    torch = pytest.importorskip("torch")
    V = int(np.prod(L))
    ctx = lqdd.lq_create(lqdd.make_lattice(L, -1, 0.02, 1.0), torch.cuda.current_stream().cuda_stream)
    try:
        lqdd.lq_set_gauge(ctx, torch.from_numpy(synth.gauge_links(L, 0.25, 1001)).cuda())
        b = torch.from_numpy(synth.gaussian_spinor(V, 2001)).cuda()
        x = torch.empty_like(b)
        lqdd.lq_smooth(ctx, sap_params(lqdd, 1, 60), b, x)
        Dx = torch.empty_like(b)
        lqdd.lq_apply(ctx, lqdd.LQ_OP_FULL, lqdd.LQ_F64, x, Dx)
        r = (b - Dx).cpu().numpy()
        bn = np.abs(b.cpu().numpy()).max()
        blk = osap.Blocks(L, (4, 4, 4, 4))
        rng = np.random.default_rng(3)
        black = blk.of_colour(osap.BLACK)
        red = blk.of_colour(osap.RED)
        for k in rng.choice(black, 6, replace=False):
            assert np.abs(r[blk.sites(k)]).max() < 1e-4 * bn
        # the red blocks' residual does not vanish (the black sweep changed it)
        assert max(np.abs(r[blk.sites(k)]).max() for k in red[:4]) > 1e-2 * bn
    finally:
        lqdd.lq_destroy(ctx)


def test_sap_argument_errors():
    from paper_2407_08092_gb300 import lqdd
    p = Pair((8, 8, 8, 8), seed=7)
    try:
        r = p.dev(synth.gaussian_spinor(p.V, 1))
        out = p.torch.empty_like(r)
        with pytest.raises(lqdd.LqError) as ei:       # SAP runs in FP32
            lqdd.lq_smooth(p.ctx, lqdd.make_params(smoother=lqdd.LQ_SMOOTH_SAP, smooth_n=1, smooth_m=2,
                                                   inner_prec=lqdd.LQ_F64, prec=lqdd.LQ_DF64), r, out)
        assert ei.value.status == lqdd.LQ_ERR_ARG
        for block in [(3, 4, 4, 4), (8, 8, 4, 4), (4, 4, 4, 6)]:   # odd extent, > 256 sites, does not divide
            with pytest.raises(lqdd.LqError) as ei:
                lqdd.lq_smooth(p.ctx, sap_params(lqdd, 1, 2, block), r, out)
            assert ei.value.status == lqdd.LQ_ERR_ARG
    finally:
        p.close()
