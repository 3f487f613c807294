"""SAP(n, m), the Schwarz alternating procedure of Algorithm 1 -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the product never does.

What it computes (arxiv 2407.08092, Sec. 2.4.1 and Sec. 2.4.5), in complex
double precision:

* the decomposition of the lattice into 4D blocks, numbered and coloured red /
  black so that no two blocks that touch share a colour (``Blocks``);
* the block operator D_k: D with every hop that leaves block k dropped, i.e.
  D restricted to the rows and columns of block k (Dirichlet boundary);
* the block solve of Algorithm 1 with odd-even preconditioning inside the
  block (Sec. 2.4.5): r_hat_e = r_e - D_eo D_oo^{-1} r_o, m steps of Minimal
  Residual on the block Schur complement S_k = D_ee - D_eo D_oo^{-1} D_oe from
  zero, e_o = D_oo^{-1}(r_o - D_oe e_e);
* Minimal Residual (the block solver the paper names): per step p = A r,
  alpha = (p, r) / (p, p), x += alpha r, r -= alpha p;
* SAP(n, m): n times, r = b - D x then every red block's solve added to x,
  r = b - D x then every black block's (Algorithm 1 as listed, from x = 0 when
  used as a smoother).

Readings where the paper is silent: the block extents are a parameter (every
extent even and dividing the lattice, and the number of blocks along each
direction even or 1, so that the red / black colouring by the parity of the
block coordinates is valid); the colour of block (B_x, B_y, B_z, B_t) is the
parity of B_x + B_y + B_z + B_t, red = 0 first; the convergence check of the
listing is skipped for the smoother (fixed n).
"""
from __future__ import annotations

import numpy as np

from . import EVEN, ODD, Lattice

RED, BLACK = 0, 1


def minimal_residual(A, b, m: int, x0=None):
    """m steps of Minimal Residual for A x = b (x0 = 0 by default)."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - A(x) if x0 is not None else b.copy()
    floor = 1e-60 * np.vdot(b, b).real
    for _ in range(m):
        if np.vdot(r, r).real <= floor:     # converged to roundoff: further steps add nothing
            break
        p = A(r)
        pp = np.vdot(p, p).real
        if pp == 0.0:
            break
        alpha = np.vdot(p, r) / pp
        x = x + alpha * r
        r = r - alpha * p
    return x


class Blocks:
    """The block decomposition of a lattice into blocks of extents ``block``."""

    def __init__(self, L, block):
        self.L = tuple(int(v) for v in L)
        self.b = tuple(int(v) for v in block)
        for mu in range(4):
            if self.b[mu] < 2 or self.b[mu] % 2 or self.L[mu] % self.b[mu]:
                raise ValueError("block extents must be even and divide the lattice")
        self.n = tuple(self.L[mu] // self.b[mu] for mu in range(4))
        for mu in range(4):
            if self.n[mu] != 1 and self.n[mu] % 2:
                raise ValueError("the number of blocks along each direction must be even or 1")
        V = int(np.prod(self.L))
        x = np.arange(V)
        c = np.stack([x % self.L[0], (x // self.L[0]) % self.L[1], (x // (self.L[0] * self.L[1])) % self.L[2],
                      x // (self.L[0] * self.L[1] * self.L[2])], axis=1)
        B = c // np.asarray(self.b)
        self.block_of = B[:, 0] + self.n[0] * (B[:, 1] + self.n[1] * (B[:, 2] + self.n[2] * B[:, 3]))
        nblk = int(np.prod(self.n))
        bc = np.stack([np.arange(nblk) % self.n[0], (np.arange(nblk) // self.n[0]) % self.n[1],
                       (np.arange(nblk) // (self.n[0] * self.n[1])) % self.n[2],
                       np.arange(nblk) // (self.n[0] * self.n[1] * self.n[2])], axis=1)
        self.coords = bc
        self.colour = bc.sum(axis=1) % 2
        self.count = nblk

    def sites(self, k: int) -> np.ndarray:
        return np.flatnonzero(self.block_of == k)

    def of_colour(self, colour: int):
        return [k for k in range(self.count) if self.colour[k] == colour]


class BlockOperator:
    """D restricted to block k (hops leaving the block dropped) and its odd-even
    pieces, on full-lattice vectors that vanish outside the block."""

    def __init__(self, lat: Lattice, blocks: Blocks, k: int):
        self.lat = lat
        inside = blocks.block_of == k
        self.mask = inside[:, None, None].astype(np.float64)
        self.even = (inside & (lat.parity == EVEN))[:, None, None].astype(np.float64)
        self.odd = (inside & (lat.parity == ODD))[:, None, None].astype(np.float64)

    def D(self, v):
        """D_k v = P_k D P_k v."""
        return self.mask * self.lat.dirac(self.mask * v)

    def D_ee(self, v):
        return self.even * self.lat.block(self.lat.C, self.even * v)

    def D_oo_inv(self, v):
        return self.odd * self.lat.block(self.lat.Cinv, self.odd * v)

    def D_eo(self, v):          # odd sites of the block -> even sites of the block
        return self.even * (-0.5 * self.lat.hop(self.odd * v))

    def D_oe(self, v):          # even sites of the block -> odd sites of the block
        return self.odd * (-0.5 * self.lat.hop(self.even * v))

    def schur(self, ve):
        """S_k v_e = D_ee v_e - D_eo D_oo^{-1} D_oe v_e."""
        return self.D_ee(ve) - self.D_eo(self.D_oo_inv(self.D_oe(ve)))

    def solve(self, r, m: int):
        """e ~ D_k^{-1} r_k: odd-even inside the block with m Minimal Residual steps."""
        re, ro = self.even * r, self.odd * r
        rhat = re - self.D_eo(self.D_oo_inv(ro))
        ee = minimal_residual(self.schur, rhat, m)
        eo = self.D_oo_inv(ro - self.D_oe(ee))
        return ee + eo


def sap(lat: Lattice, b, n: int, m: int, block, x0=None, blocks: Blocks | None = None):
    """SAP(n, m) for D x = b (Algorithm 1): full-lattice vectors [V, 4, 3]."""
    b = np.asarray(b, dtype=np.complex128).reshape(lat.V, 4, 3)
    blocks = blocks or Blocks(lat.L, block)
    ops = [BlockOperator(lat, blocks, k) for k in range(blocks.count)]
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128).reshape(lat.V, 4, 3)
    for _ in range(n):
        for colour in (RED, BLACK):
            r = b - lat.dirac(x)
            for k in blocks.of_colour(colour):
                x = x + ops[k].solve(r, m)
    return x


def sap_schur_preconditioner(lat: Lattice, n: int, m: int, block):
    """v_e -> the even half of SAP(n, m) applied to (v_e, 0): since the even-even
    block of D^{-1} is D_S^{-1}, this approximates D_S^{-1} (the preconditioner
    of the odd-even FGMRES when SAP is the smoother)."""
    blocks = Blocks(lat.L, block)

    def M(ve):
        return lat.restrict(sap(lat, lat.embed(ve, EVEN), n, m, block, blocks=blocks), EVEN)
    return M
