"""Seeded synthetic inputs for the odd-even Wilson-clover path.

This module only draws inputs: gauge links, spinor sources and gauge
transformations.  It holds none of the operator's arithmetic and is the one
module shared by the CUDA path's callers (tests, ``bench.py``) and by the FP64
oracle's tests, so both sides see bit-identical inputs.

Conventions (the same on both sides of every comparison):

* A lattice is ``L = (Lx, Ly, Lz, Lt)``; the natural site index is
  lexicographic with x fastest: ``lex = x + Lx*(y + Ly*(z + Lz*t))``.
* A gauge field is a complex128 array ``U[V, 4, 3, 3]``; ``U[s, mu]`` is the
  SU(3) link leaving site ``s`` in direction ``mu`` (0..3 = x, y, z, t), stored
  row-major (``U[s, mu, a, b]`` = row a, column b).
* A spinor field is complex128 ``psi[V, 4, 3]`` (spin, then colour).

The gauge field stands in for the thermalised 96x48^3 configuration of the
paper's Table 5, which is not available: near-unit random links
``U = exp(i * eps * sum_k a_k lambda_k)`` with ``a_k ~ N(0, 1)`` drawn per site
(lexicographic order) and per direction, eight draws in the order k = 1..8.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "volume", "gell_mann", "su3_from_algebra", "gauge_links", "gaussian_spinor",
    "point_source", "random_gauge_transform", "unit_links",
]


def volume(L) -> int:
    Lx, Ly, Lz, Lt = (int(v) for v in L)
    return Lx * Ly * Lz * Lt


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, normalised so that tr(l_a l_b) = 2 delta_ab."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1.0, 1.0, -2.0]) / np.sqrt(3.0)
    return lam


def su3_from_algebra(a: np.ndarray, eps: float, chunk: int = 1 << 20) -> np.ndarray:
    """exp(i*eps*sum_k a[..., k] lambda_k) for an array of coefficient 8-vectors.

    The Hermitian generator H = eps*sum_k a_k lambda_k is diagonalised
    (H = W diag(w) W^dagger, batched LAPACK) and U = W diag(exp(i w)) W^dagger,
    which is unitary with det U = exp(i tr H) = 1.  Work is chunked to bound
    host memory on large lattices.
    """
    lam = gell_mann()
    flat = a.reshape(-1, 8)
    out = np.empty((flat.shape[0], 3, 3), dtype=np.complex128)
    for lo in range(0, flat.shape[0], chunk):
        hi = min(lo + chunk, flat.shape[0])
        H = eps * np.einsum("nk,kab->nab", flat[lo:hi], lam)
        w, W = np.linalg.eigh(H)
        out[lo:hi] = np.einsum("nab,nb,ncb->nac", W, np.exp(1j * w), W.conj())
    return out.reshape(a.shape[:-1] + (3, 3))


def gauge_links(L, eps: float, seed: int) -> np.ndarray:
    """Seeded SU(3) gauge field U[V, 4, 3, 3] (complex128, natural order)."""
    V = volume(L)
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal((V, 4, 8))
    return su3_from_algebra(a, eps)


def unit_links(L) -> np.ndarray:
    """The free field U = 1 on every link."""
    V = volume(L)
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    U[:, :, 0, 0] = U[:, :, 1, 1] = U[:, :, 2, 2] = 1.0
    return U


def gaussian_spinor(n_sites: int, seed: int) -> np.ndarray:
    """Complex Gaussian spinor psi[n_sites, 4, 3]: Re and Im i.i.d. N(0, 1).

    Draw order: for each site, spin, colour the real part then the imaginary
    part.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal((int(n_sites), 4, 3, 2))
    return z[..., 0] + 1j * z[..., 1]


def point_source(L, site: int, spin: int, colour: int) -> np.ndarray:
    """delta_{x,site} delta_{s,spin} delta_{c,colour} as psi[V, 4, 3]."""
    psi = np.zeros((volume(L), 4, 3), dtype=np.complex128)
    psi[site, spin, colour] = 1.0
    return psi


def random_gauge_transform(L, seed: int, eps: float = 1.0) -> np.ndarray:
    """Seeded SU(3) matrices Omega[V, 3, 3] for gauge-covariance checks."""
    V = volume(L)
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal((V, 8))
    return su3_from_algebra(a, eps)
