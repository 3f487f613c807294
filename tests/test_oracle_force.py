"""Pins of the fermion-force oracle (``oracle/force.py``).

The paper has no force; the pins are what the mathematics fixes:

* the plain-PyTorch operator equals the independent C operator of the oracle
  (so every operator pin carries over to it);
* the autograd gradient of the bilinear form Re(Y^+ D(U) X) equals central
  differences of that form along random complex directions;
* the force dS/dU of S = phi^+ (D^+ D)^{-1} phi equals central differences of
  S (dense LU solves) along the su(3) generators T_a = lambda_a / 2, on links
  in the bulk and across the antiperiodic time boundary;
* gauge invariance of S: the force satisfies the lattice Gauss law at every
  site;
* the iterative (odd-even GMRES) force equals the dense-solve force.

A dropped factor 2, a swapped X and Y, a missing boundary sign, a wrong
leaf or a wrong sign of the clover term fails at least one of these.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import force as of
from paper_2407_08092_gb300 import synth


def lattice(L, seed=11, eps=0.4, m0=0.1, csw=1.0, t_bc=-1):
    return oracle.Lattice(L, synth.gauge_links(L, eps, seed), m0=m0, csw=csw, t_bc=t_bc)


def lex(L, x, y, z, t):
    return x + L[0] * (y + L[1] * (z + L[2] * t))


@pytest.mark.parametrize("L,t_bc,csw", [((4, 4, 4, 4), -1, 1.0), ((4, 2, 2, 4), 1, 1.3), ((2, 2, 2, 2), -1, 0.0),
                                        ((6, 4, 2, 2), -1, 1.0)])
def test_torch_dirac_equals_c_oracle(L, t_bc, csw):
    lat = lattice(L, seed=3, t_bc=t_bc, csw=csw)
    psi = synth.gaussian_spinor(lat.V, 5)
    a = of.dirac(L, lat.U, psi, lat.m0, lat.csw, lat.t_bc)
    b = lat.dirac(psi)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-14


def test_bilinear_grad_central_difference():
    L = (4, 2, 2, 4)
    lat = lattice(L)
    X = synth.gaussian_spinor(lat.V, 21)
    Y = synth.gaussian_spinor(lat.V, 22)
    G = of.bilinear_grad(L, lat.U, X, Y, lat.m0, lat.csw, lat.t_bc)
    rng = np.random.default_rng(4)

    def b(U):
        return np.vdot(Y, oracle.Lattice(L, U, lat.m0, lat.csw, lat.t_bc).dirac(X)).real

    h = 1e-5
    for trial in range(3):
        d = rng.standard_normal(lat.U.shape) + 1j * rng.standard_normal(lat.U.shape)
        if trial == 2:                       # a single link across the time boundary
            mask = np.zeros(lat.U.shape)
            mask[lex(L, 1, 0, 1, L[3] - 1), 3] = 1.0
            d = d * mask
        fd = (b(lat.U + h * d) - b(lat.U - h * d)) / (2 * h)
        an = np.sum(np.conj(G) * d).real
        assert abs(fd - an) < 1e-7 * max(1.0, abs(an)), (trial, fd, an)


def _perturbed(U, site, mu, T, h):
    U2 = U.copy()
    U2[site, mu] = scipy.linalg.expm(1j * h * T) @ U[site, mu]
    return U2


@pytest.mark.parametrize("L,links", [
    ((2, 2, 2, 2), [(0, 0), (5, 1), (9, 2), (lex((2, 2, 2, 2), 1, 0, 1, 1), 3)]),
    ((4, 2, 2, 4), [(lex((4, 2, 2, 4), 3, 1, 0, 2), 0), (lex((4, 2, 2, 4), 2, 0, 1, 3), 3),
                    (lex((4, 2, 2, 4), 1, 1, 1, 0), 2)]),
])
def test_force_central_difference_along_generators(L, links):
    lat = lattice(L, seed=17)
    phi = synth.gaussian_spinor(lat.V, 23)
    S, F = of.force(lat, phi, dense=True)
    assert S > 0
    T = synth.gell_mann() / 2.0
    h = 1e-6
    worst = 0.0
    scale = max(abs(of.generator_derivative(F, lat.U, s, m, T[a])) for s, m in links for a in range(8))
    for site, mu in links:
        for a in range(8):
            Sp = of.action(oracle.Lattice(L, _perturbed(lat.U, site, mu, T[a], h), lat.m0, lat.csw, lat.t_bc),
                           phi, dense=True)
            Sm = of.action(oracle.Lattice(L, _perturbed(lat.U, site, mu, T[a], -h), lat.m0, lat.csw, lat.t_bc),
                           phi, dense=True)
            fd = (Sp - Sm) / (2 * h)
            an = of.generator_derivative(F, lat.U, site, mu, T[a])
            worst = max(worst, abs(fd - an) / scale)
    assert worst < 1e-6, worst


def test_force_obeys_gauss_law():
    """S(U, phi) is invariant under the gauge transformation U_mu(x) ->
    W(x) U_mu(x) W(x+mu)^+, phi(x) -> W(x) phi(x).  Taking W = exp(i h T_a) at
    one site x and differentiating at h = 0 gives, with X = (D^+ D)^{-1} phi,
      sum_mu [Re tr(G_mu(x)^+ i T_a U_mu(x)) - Re tr(G_mu(x-mu)^+ U_mu(x-mu) i T_a)]
        + 2 Re((i T_a phi(x))^+ X(x)) = 0
    at every site and for every generator."""
    L = (4, 2, 2, 4)
    lat = lattice(L, seed=29)
    phi = synth.gaussian_spinor(lat.V, 31)
    _, F = of.force(lat, phi, dense=True)
    X, _ = of.solve_pair(lat, phi, dense=True)
    T = synth.gell_mann() / 2.0
    c = np.stack([np.arange(lat.V) % L[0], (np.arange(lat.V) // L[0]) % L[1],
                  (np.arange(lat.V) // (L[0] * L[1])) % L[2], np.arange(lat.V) // (L[0] * L[1] * L[2])], axis=1)

    def gauss(F, x, a):
        tot = 2.0 * np.vdot(np.einsum("ab,sb->sa", 1j * T[a], phi[x]), X[x]).real
        for mu in range(4):
            cm = c[x].copy()
            cm[mu] = (cm[mu] - 1) % L[mu]
            xm = lex(L, *cm)
            tot += np.sum(np.conj(F[x, mu]) * (1j * T[a] @ lat.U[x, mu])).real
            tot -= np.sum(np.conj(F[xm, mu]) * (lat.U[xm, mu] @ (1j * T[a]))).real
        return tot

    scale = np.abs(F).max()
    worst = max(abs(gauss(F, x, a)) for x in range(lat.V) for a in range(8))
    assert worst < 1e-11 * scale, (worst, scale)
    # a force that is not the gradient of this action fails it
    bad = F.copy()
    bad[:, 3] *= 1.001
    assert max(abs(gauss(bad, x, a)) for x in range(4) for a in range(8)) > 1e-6 * scale


def test_iterative_force_equals_dense_force():
    L = (4, 2, 2, 4)
    lat = lattice(L, seed=37)
    phi = synth.gaussian_spinor(lat.V, 41)
    S1, F1 = of.force(lat, phi, tol=1e-13)
    S2, F2 = of.force(lat, phi, dense=True)
    assert abs(S1 - S2) < 1e-11 * S2
    assert np.abs(F1 - F2).max() < 1e-10 * np.abs(F2).max()
    # S = phi^+ X as well as ||Y||^2
    X, Y = of.solve_pair(lat, phi, dense=True)
    assert abs(np.vdot(phi, X) - S2) < 1e-12 * S2
