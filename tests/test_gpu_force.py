"""Fermion force on the GPU against the FP64 oracle.

* ``lq_force`` (the df64 gradient kernel of Re(Y^+ D X)) element by element
  against the oracle's autograd gradient, for Gaussian X, Y, at sizes that
  span several blocks and a ragged tail, and on sampled links of 24^3 x 48;
* ``lq_fermion_force`` (two odd-even solves plus the kernel) against the
  oracle's force, and at 24^3 x 48 against the oracle's force from its own
  solves on sampled links, plus the gauge-invariance identity at sampled
  sites;
* the ``torch.autograd.Function`` wrapper: autograd gradient = the library's
  force, and its directional derivative = central differences of S.

Tolerances: the kernel is FP64-accurate (df64), so 1e-12 relative to the
largest gradient entry; the full force inherits the solves' tolerance.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import force as of
from paper_2407_08092_gb300 import synth

from .gpu_util import Pair

pytestmark = pytest.mark.gpu


def maxrel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def force_params(lqdd, tol):
    return lqdd.make_params(solver=lqdd.LQ_SOLVER_FGMRES, prec=lqdd.LQ_DF64, tol=tol, restart=10, max_restarts=50,
                            smoother=lqdd.LQ_SMOOTH_GMRES, smooth_n=20, smooth_m=16, smooth_tol=1e-5,
                            inner_prec=lqdd.LQ_F32)


@pytest.mark.parametrize("L,t_bc,csw", [((2, 2, 2, 2), -1, 1.0), ((4, 4, 4, 4), -1, 1.0), ((6, 2, 2, 2), 1, 1.3),
                                        ((6, 4, 2, 4), -1, 0.0), ((8, 6, 4, 10), -1, 1.0), ((16, 16, 16, 8), -1, 1.0)],
                         ids=["2^4", "4^4", "6x2x2x2-periodic", "6x4x2x4-wilson", "8x6x4x10", "16^3x8"])
def test_force_kernel_matches_oracle(L, t_bc, csw):
    p = Pair(L, eps=0.4, seed=500 + sum(L), m0=0.07, csw=csw, t_bc=t_bc)
    try:
        X = synth.gaussian_spinor(p.V, 61)
        Y = synth.gaussian_spinor(p.V, 62)
        G = p.torch.empty_like(p.dU)
        p.lqdd.lq_force(p.ctx, p.dev(X), p.dev(Y), G, coef=1.0)
        got = p.host(G)
        want = of.bilinear_grad(L, p.U, X, Y, p.lat.m0, p.lat.csw, p.lat.t_bc)
        assert maxrel(got, want) < 1e-12
        # the coefficient scales the result exactly
        p.lqdd.lq_force(p.ctx, p.dev(X), p.dev(Y), G, coef=-2.0)
        assert np.array_equal(p.host(G), -2.0 * got)
    finally:
        p.close()


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (8, 8, 8, 8)], ids=["4^4", "8^4"])
def test_fermion_force_matches_oracle(L):
    p = Pair(L, eps=0.25, seed=1004, m0=0.05, csw=1.0)
    try:
        phi = synth.gaussian_spinor(p.V, 2004)
        G = p.torch.empty_like(p.dU)
        status, S, st = p.lqdd.lq_fermion_force(p.ctx, force_params(p.lqdd, 1e-12), p.dev(phi), G)
        assert status == p.lqdd.LQ_OK
        S_o, F_o = of.force(p.lat, phi, tol=1e-12)
        assert abs(S - S_o) < 1e-10 * S_o
        assert maxrel(p.host(G), F_o) < 1e-9
        assert all(s.rel_resid_true < 1e-11 for s in st)
    finally:
        p.close()


def test_force_status_codes():
    from paper_2407_08092_gb300 import lqdd
    torch = pytest.importorskip("torch")
    ctx = lqdd.lq_create(lqdd.make_lattice((4, 4, 4, 4), -1, 0.05, 1.0), torch.cuda.current_stream().cuda_stream)
    try:
        X = torch.zeros((256, 4, 3), dtype=torch.complex128, device="cuda")
        G = torch.zeros((256, 4, 3, 3), dtype=torch.complex128, device="cuda")
        with pytest.raises(lqdd.LqError) as ei:          # no gauge field yet
            lqdd.lq_force(ctx, X, X, G)
        assert ei.value.status == lqdd.LQ_ERR_STATE
        lqdd.lq_set_gauge(ctx, torch.from_numpy(synth.gauge_links((4, 4, 4, 4), 0.25, 9)).cuda())
        assert lqdd.library().lq_force(ctx, 0, 0, 1.0, 0) == lqdd.LQ_ERR_ARG
        phi = torch.from_numpy(synth.gaussian_spinor(256, 3)).cuda()
        status, S, st = lqdd.lq_fermion_force(ctx, lqdd.make_params(tol=1e-14, restart=4, max_restarts=1), phi, G)
        assert status == lqdd.LQ_ERR_NOT_CONVERGED and S > 0
    finally:
        lqdd.lq_destroy(ctx)


def test_autograd_function_gradient_and_central_difference():
    torch = pytest.importorskip("torch")
    from paper_2407_08092_gb300.autograd import FermionAction
    L = (4, 2, 2, 4)
    U0 = synth.gauge_links(L, 0.4, 77)
    phi = torch.from_numpy(synth.gaussian_spinor(int(np.prod(L)), 78)).cuda()
    act = FermionAction(L, m0=0.1, csw=1.0, t_bc=-1)
    act.params.tol = 1e-13
    try:
        U = torch.from_numpy(U0).cuda().requires_grad_(True)
        S = act(U, phi)
        (g,) = torch.autograd.grad(S, U)
        g = g.cpu().numpy()
        # the same as the library's force and the oracle's
        lat = oracle.Lattice(L, U0, 0.1, 1.0, -1)
        S_o, F_o = of.force(lat, phi.cpu().numpy(), dense=True)
        assert abs(float(S.detach()) - S_o) < 1e-11 * S_o
        assert maxrel(g, F_o) < 1e-10
        # directional derivatives along su(3) generators = central differences of S
        T = synth.gell_mann() / 2.0
        h = 1e-4
        for site, mu, a in [(3, 0, 1), (37, 3, 6), (60, 2, 7)]:
            Ue = [U0.copy(), U0.copy()]
            Ue[0][site, mu] = scipy.linalg.expm(1j * h * T[a]) @ U0[site, mu]
            Ue[1][site, mu] = scipy.linalg.expm(-1j * h * T[a]) @ U0[site, mu]
            Sp, Sm = (float(act(torch.from_numpy(u).cuda(), phi)) for u in Ue)
            fd = (Sp - Sm) / (2 * h)
            an = of.generator_derivative(g, U0, site, mu, T[a])
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (site, mu, a, fd, an)
    finally:
        act.close()


def test_full_size_force_24x48():
    """24^3 x 48 (eps 0.25, c_sw 1, m0 0.05, Gaussian phi), as the benchmark
    launches it: the kernel on sampled links against the oracle's autograd
    gradient for Gaussian X, Y; then the whole force against the oracle's force
    from its own solves, on sampled links, and the gauge-invariance identity at
    sampled sites."""
    L = (24, 24, 24, 48)
    p = Pair(L, eps=0.25, seed=1004, m0=0.05, csw=1.0)
    rng = np.random.default_rng(5)
    links = rng.integers(0, p.V, 48)
    try:
        X = synth.gaussian_spinor(p.V, 71)
        Y = synth.gaussian_spinor(p.V, 72)
        G = p.torch.empty_like(p.dU)
        p.lqdd.lq_force(p.ctx, p.dev(X), p.dev(Y), G, coef=1.0)
        got = p.host(G)[links]
        want = of.bilinear_grad(L, p.U, X, Y, p.lat.m0, p.lat.csw, p.lat.t_bc)[links]
        assert maxrel(got, want) < 1e-12

        phi = synth.gaussian_spinor(p.V, 2004)
        dphi = p.dev(phi)
        dX, dY = p.torch.empty_like(dphi), p.torch.empty_like(dphi)
        status, S, st = p.lqdd.lq_fermion_action(p.ctx, force_params(p.lqdd, 1e-11), dphi, dX, dY)
        assert status == p.lqdd.LQ_OK
        p.lqdd.lq_force(p.ctx, dX, dY, G, coef=-2.0)
        F = p.host(G)
        Xh = p.host(dX)
        S_o, F_o = of.force(p.lat, phi, tol=1e-11)
        assert abs(S - S_o) < 1e-9 * S_o
        assert maxrel(F[links], F_o[links]) < 1e-8
        # gauge invariance at sampled sites (exact up to the solves' tolerance)
        T = synth.gell_mann() / 2.0
        scale = np.abs(F).max()
        for x in links[:8]:
            c = [x % L[0], (x // L[0]) % L[1], (x // (L[0] * L[1])) % L[2], x // (L[0] * L[1] * L[2])]
            for a in range(8):
                tot = 2.0 * np.vdot(np.einsum("ab,sb->sa", 1j * T[a], phi[x]), Xh[x]).real
                for mu in range(4):
                    cm = list(c)
                    cm[mu] = (cm[mu] - 1) % L[mu]
                    xm = cm[0] + L[0] * (cm[1] + L[1] * (cm[2] + L[2] * cm[3]))
                    tot += np.sum(np.conj(F[x, mu]) * (1j * T[a] @ p.U[x, mu])).real
                    tot -= np.sum(np.conj(F[xm, mu]) * (p.U[xm, mu] @ (1j * T[a]))).real
                assert abs(tot) < 1e-8 * scale, (x, a, tot, scale)
    finally:
        p.close()
