"""Pins of the SAP oracle (``oracle/sap.py``) against what the mathematics fixes.

* Minimal Residual: the one-step closed form, the orthogonality of each new
  residual to A times the old one, and convergence to A^{-1} b for a matrix with
  a positive definite Hermitian part;
* the block decomposition: the blocks partition the lattice, and no two blocks
  that touch share a colour;
* the block operator equals the dense D restricted to the block's rows and
  columns, and the block solve with many Minimal Residual steps equals the
  dense solve of that restriction;
* an exact red sweep leaves a zero residual on every red block, and the red
  blocks' solves do not depend on their order;
* one block covering the lattice turns SAP(1, many) into D^{-1} b;
* SAP lowers the residual as n grows;
* after a colour's block solves (inexact, m MR steps), the whole operator's
  residual on a block of that colour is the MR residual of the block's Schur
  system on the even sites and zero on the odd sites, and on the other
  colour's blocks it changed only by the hops of the correction across the
  block faces -- the identities that let the GPU path keep the residual block
  by block instead of applying D to the whole lattice before every colour.
"""
import numpy as np
import pytest

import oracle
from oracle import sap as osap
from paper_2407_08092_gb300 import synth


def lattice(L, seed=5, eps=0.3, m0=0.2, csw=1.0, t_bc=-1):
    return oracle.Lattice(L, synth.gauge_links(L, eps, seed), m0=m0, csw=csw, t_bc=t_bc)


def dense_D(lat):
    n = lat.V * 12
    A = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1.0
        A[:, j] = lat.dirac(e.reshape(lat.V, 4, 3)).reshape(-1)
    return A


def test_minimal_residual_closed_form_and_orthogonality():
    rng = np.random.default_rng(1)
    n = 12
    A = np.eye(n) * 3 + 0.4 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    op = lambda v: A @ v  # noqa: E731
    x1 = osap.minimal_residual(op, b, 1)
    Ab = A @ b
    assert np.allclose(x1, (np.vdot(Ab, b) / np.vdot(Ab, Ab)) * b, atol=1e-14)
    x, r = np.zeros(n, complex), b.copy()
    for _ in range(5):
        p = A @ r
        x2 = osap.minimal_residual(op, b, 1, x0=x)
        r2 = b - A @ x2
        assert abs(np.vdot(p, r2)) < 1e-12 * np.linalg.norm(p) * np.linalg.norm(r2)
        x, r = x2, r2
    # A + A^+ positive definite: MR converges to the solution
    H = A + A.conj().T
    assert np.linalg.eigvalsh(H).min() > 0
    xs = osap.minimal_residual(op, b, 400)
    assert np.linalg.norm(xs - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(xs)


@pytest.mark.parametrize("L,block", [((8, 8, 4, 4), (4, 4, 2, 2)), ((4, 4, 4, 8), (2, 4, 4, 2)), ((8, 4, 4, 4), (4, 4, 4, 4))])
def test_blocks_partition_and_colouring(L, block):
    blk = osap.Blocks(L, block)
    V = int(np.prod(L))
    seen = np.zeros(V, dtype=int)
    for k in range(blk.count):
        s = blk.sites(k)
        assert len(s) == int(np.prod(block))
        seen[s] += 1
    assert np.all(seen == 1)
    # neighbouring sites in different blocks lie in blocks of different colours
    x = np.arange(V)
    c = np.stack([x % L[0], (x // L[0]) % L[1], (x // (L[0] * L[1])) % L[2], x // (L[0] * L[1] * L[2])], axis=1)
    for mu in range(4):
        cn = c.copy()
        cn[:, mu] = (cn[:, mu] + 1) % L[mu]
        nb = cn[:, 0] + L[0] * (cn[:, 1] + L[1] * (cn[:, 2] + L[2] * cn[:, 3]))
        a, b = blk.block_of[x], blk.block_of[nb]
        diff = a != b
        assert np.all(blk.colour[a[diff]] != blk.colour[b[diff]])
    with pytest.raises(ValueError):
        osap.Blocks((12, 4, 4, 4), (4, 4, 4, 4))        # three blocks along x: no red-black colouring


def test_block_operator_is_the_restricted_dense_matrix():
    L = (4, 4, 2, 4)
    lat = lattice(L)
    blk = osap.Blocks(L, (2, 2, 2, 2))
    A = dense_D(lat)
    rng = np.random.default_rng(3)
    for k in (0, 5, blk.count - 1):
        op = osap.BlockOperator(lat, blk, k)
        idx = (blk.sites(k)[:, None] * 12 + np.arange(12)[None, :]).ravel()
        Ak = A[np.ix_(idx, idx)]
        v = np.zeros((lat.V, 4, 3), dtype=np.complex128)
        v[blk.sites(k)] = rng.standard_normal((len(blk.sites(k)), 4, 3)) + 1j * rng.standard_normal((len(blk.sites(k)), 4, 3))
        got = op.D(v)
        assert np.abs(got.reshape(-1)[idx] - Ak @ v.reshape(-1)[idx]).max() < 1e-13
        outside = np.setdiff1d(np.arange(lat.V), blk.sites(k))
        assert np.abs(got[outside]).max() == 0.0
        # the odd-even block solve with many MR steps is the dense block solve
        r = synth.gaussian_spinor(lat.V, 7 + k)
        e = op.solve(r, 300)
        want = np.linalg.solve(Ak, r.reshape(-1)[idx])
        assert np.abs(e.reshape(-1)[idx] - want).max() < 1e-10 * np.abs(want).max()
        assert np.abs(e[outside]).max() == 0.0


def test_exact_red_sweep_zeroes_red_residual_and_is_order_free():
    L = (8, 4, 4, 4)
    lat = lattice(L, seed=9)
    blk = osap.Blocks(L, (4, 2, 2, 2))
    b = synth.gaussian_spinor(lat.V, 11)
    ops = [osap.BlockOperator(lat, blk, k) for k in range(blk.count)]
    red = blk.of_colour(osap.RED)
    x = np.zeros_like(b)
    for k in red:
        x = x + ops[k].solve(b, 300)
    r = b - lat.dirac(x)
    for k in red:
        assert np.abs(r[blk.sites(k)]).max() < 1e-9 * np.abs(b).max()
    # the red blocks do not talk to each other within the sweep
    x2 = np.zeros_like(b)
    for k in reversed(red):
        x2 = x2 + ops[k].solve(b, 4)
    x1 = np.zeros_like(b)
    for k in red:
        x1 = x1 + ops[k].solve(b, 4)
    assert np.abs(x1 - x2).max() < 1e-14


def test_single_block_sap_is_the_inverse():
    L = (4, 2, 2, 4)
    lat = lattice(L, seed=13)
    b = synth.gaussian_spinor(lat.V, 17)
    x = osap.sap(lat, b, 1, 400, L)
    want = np.linalg.solve(dense_D(lat), b.reshape(-1)).reshape(lat.V, 4, 3)
    assert np.abs(x - want).max() < 1e-9 * np.abs(want).max()


def test_single_block_schur_preconditioner_is_the_schur_inverse():
    L = (4, 2, 2, 4)
    lat = lattice(L, seed=29)
    M = osap.sap_schur_preconditioner(lat, 1, 400, L)
    ve = synth.gaussian_spinor(lat.Vh, 31)
    got = M(ve)
    S = np.zeros((lat.Vh * 12, lat.Vh * 12), dtype=np.complex128)
    for j in range(lat.Vh * 12):
        e = np.zeros(lat.Vh * 12, dtype=np.complex128)
        e[j] = 1.0
        S[:, j] = lat.schur(e.reshape(lat.Vh, 4, 3)).reshape(-1)
    want = np.linalg.solve(S, ve.reshape(-1)).reshape(lat.Vh, 4, 3)
    assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()


def test_sap_reduces_the_residual():
    L = (8, 8, 4, 4)
    lat = lattice(L, seed=19, eps=0.25, m0=0.05)
    b = synth.gaussian_spinor(lat.V, 23)
    res = []
    for n in (1, 2, 3):
        x = osap.sap(lat, b, n, 4, (4, 4, 2, 2))
        res.append(np.linalg.norm(b - lat.dirac(x)) / np.linalg.norm(b))
    assert res[0] < 0.5 and res[1] < res[0] and res[2] < res[1], res


@pytest.mark.parametrize("L,block", [((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 4, 4, 4), (4, 2, 4, 2))])
def test_colour_sweep_residual_is_blockwise(L, block):
    lat = lattice(L, seed=11)
    blocks = osap.Blocks(L, block)
    ops = [osap.BlockOperator(lat, blocks, k) for k in range(blocks.count)]
    b = synth.gaussian_spinor(lat.V, 12).reshape(lat.V, 4, 3)
    x0 = 0.1 * synth.gaussian_spinor(lat.V, 13).reshape(lat.V, 4, 3)   # an earlier iterate
    r = b - lat.dirac(x0)
    e = np.zeros_like(b)
    for k in blocks.of_colour(osap.RED):
        e = e + ops[k].solve(r, 3)
    r1 = b - lat.dirac(x0 + e)
    tol = 1e-12 * np.abs(b).max()
    for k in blocks.of_colour(osap.RED):
        op = ops[k]
        rhat = op.even * r - op.D_eo(op.D_oo_inv(op.odd * r))
        mr_residual = rhat - op.schur(op.even * e)
        assert np.abs(op.even * r1 - mr_residual).max() < tol
        assert np.abs(op.odd * r1).max() < tol
    black = np.isin(blocks.block_of, blocks.of_colour(osap.BLACK))[:, None, None]
    # e vanishes on the black sites, so D e there is the hop term alone: -1/2 hop(e)
    assert np.abs(black * (r1 - (r + 0.5 * lat.hop(e)))).max() < tol
    # and only sites with a red neighbour across a face change
    assert np.abs(black * (r1 - r)).max() > 1e-3 * np.abs(b).max()
