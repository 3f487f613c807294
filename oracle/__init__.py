"""FP64 CPU oracle for the odd-even Wilson-clover path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
Python binding) never imports, loads or calls anything here, and shares no
code with it: no kernels, headers, helpers, tables or constants.  The only
common module is ``paper_2407_08092_gb300.synth``, which draws seeded inputs
and holds none of the method's arithmetic.

What it computes, in complex double precision, each function citing the
passage it follows (arxiv 2407.08092):

* the Wilson-clover operator D and its hopping and clover parts
  (Sec. 2.3; formula in ``oracle.c``), written site by site in C with full
  4x4 gamma and 12x12 clover matrices;
* the odd-even blocks of Eq. 1, the Schur complement D_S of Eq. 3 and the
  factorised inverse of Eq. 2 (prepare / reconstruct), composed literally
  from those blocks;
* Richardson(n, delta) (Algorithm 4), restarted GMRES(n, m) with modified
  Gram-Schmidt (Algorithm 2), flexible GMRES (Sec. 2.3, the outer solver of
  every level), the power-iteration norm estimate behind Richardson's omega
  (Sec. 2.4.4) and the odd-even smoother M_n (Sec. 2.4.5, Fig. 1);
* dense matrices of any of these operators on tiny lattices (for the pins).

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants and brute-force dense linear algebra.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_liboracle.so`` with gcc (-O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            lib.orc_gamma.argtypes = [ctypes.c_int, P]
            lib.orc_parity.argtypes = [P, ctypes.c_long]
            lib.orc_parity.restype = ctypes.c_int
            lib.orc_hop.argtypes = [P, ctypes.c_int, P, P, P, ctypes.c_int]
            lib.orc_clover.argtypes = [P, P, ctypes.c_double, ctypes.c_double, P]
            lib.orc_clover_sites.argtypes = [P, P, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_long, P, P]
            lib.orc_invert.argtypes = [ctypes.c_long, ctypes.c_int, P, P]
            lib.orc_invert.restype = ctypes.c_long
            lib.orc_block.argtypes = [P, P, P, P, ctypes.c_int]
            lib.orc_schur_sites.argtypes = [P, ctypes.c_int, P, ctypes.c_double, ctypes.c_double,
                                            P, ctypes.c_long, P, P, P]
            lib.orc_schur_sites.restype = ctypes.c_long
            lib.orc_threads.restype = ctypes.c_int
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def threads() -> int:
    """OpenMP threads the oracle's site loops use."""
    return int(_load().orc_threads())


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def gamma(mu: int) -> np.ndarray:
    """The 4x4 gamma matrix gamma_{mu+1} (mu = 0..3) or gamma_5 (mu = 4), chiral basis."""
    g = np.zeros((4, 4), dtype=np.complex128)
    _load().orc_gamma(int(mu), _p(g))
    return g


# ---------------------------------------------------------------------------
# the lattice operator
# ---------------------------------------------------------------------------

EVEN, ODD = 0, 1


class Lattice:
    """A 4D lattice with its gauge field and clover parameters.

    Vectors are natural-order complex128 arrays: full fields ``[V, 4, 3]`` and
    single-parity fields ``[V/2, 4, 3]`` listing that parity's sites in
    lexicographic order.
    """

    def __init__(self, L, U, m0: float, csw: float, t_bc: int = -1):
        self.L = tuple(int(v) for v in L)
        if any(v % 2 for v in self.L):
            raise ValueError("all lattice extents must be even")
        self.V = int(np.prod(self.L))
        self.Vh = self.V // 2
        self.U = _c128(U).reshape(self.V, 4, 3, 3)
        self.m0 = float(m0)
        self.csw = float(csw)
        self.t_bc = int(t_bc)
        self._L = np.asarray(self.L, dtype=np.int32)
        # Sec. 2.4.5: a site is even iff x1 + x2 + x3 + x4 is even
        x = np.arange(self.V)
        c = [x % self.L[0], (x // self.L[0]) % self.L[1],
             (x // (self.L[0] * self.L[1])) % self.L[2], x // (self.L[0] * self.L[1] * self.L[2])]
        self.parity = (c[0] + c[1] + c[2] + c[3]) % 2
        self.sites = (np.flatnonzero(self.parity == EVEN), np.flatnonzero(self.parity == ODD))
        self._C = None
        self._Cinv = None

    # -- pieces of D ------------------------------------------------------
    @property
    def C(self) -> np.ndarray:
        """Clover matrices C(x) as [V, 12, 12] (index spin*3 + colour)."""
        if self._C is None:
            C = np.zeros((self.V, 12, 12), dtype=np.complex128)
            _load().orc_clover(_p(self._L), _p(self.U), self.csw, self.m0, _p(C))
            self._C = C
        return self._C

    @property
    def Cinv(self) -> np.ndarray:
        """C(x)^{-1} at every site (Gauss-Jordan with partial pivoting)."""
        if self._Cinv is None:
            self._Cinv = invert(self.C)
        return self._Cinv

    def clover_sites(self, sites) -> np.ndarray:
        sites = np.ascontiguousarray(sites, dtype=np.int64)
        C = np.zeros((len(sites), 12, 12), dtype=np.complex128)
        _load().orc_clover_sites(_p(self._L), _p(self.U), self.csw, self.m0,
                                 len(sites), _p(sites), _p(C))
        return C

    def hop(self, psi, parity: int = -1) -> np.ndarray:
        """(H psi)(x) = sum_mu [(1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^+ psi(x-mu)]
        at the sites of ``parity`` (-1: all), zero elsewhere."""
        psi = _c128(psi).reshape(self.V, 4, 3)
        out = np.empty_like(psi)
        _load().orc_hop(_p(self._L), self.t_bc, _p(self.U), _p(psi), _p(out), int(parity))
        return out

    def block(self, M, psi, parity: int = -1) -> np.ndarray:
        """(M psi)(x) = M(x) psi(x) for site matrices M[V, 12, 12]."""
        psi = _c128(psi).reshape(self.V, 4, 3)
        out = np.empty_like(psi)
        _load().orc_block(_p(self._L), _p(_c128(M)), _p(psi), _p(out), int(parity))
        return out

    def dirac(self, psi) -> np.ndarray:
        """D psi = C psi - 1/2 H psi on the full lattice."""
        return self.block(self.C, psi) - 0.5 * self.hop(psi)

    # -- odd-even blocks, Eq. 1 -------------------------------------------
    def embed(self, v, parity: int) -> np.ndarray:
        full = np.zeros((self.V, 4, 3), dtype=np.complex128)
        full[self.sites[parity]] = np.asarray(v).reshape(self.Vh, 4, 3)
        return full

    def restrict(self, full, parity: int) -> np.ndarray:
        return np.ascontiguousarray(np.asarray(full).reshape(self.V, 4, 3)[self.sites[parity]])

    def D_pp(self, v, parity: int) -> np.ndarray:          # D_ee or D_oo
        return self.restrict(self.block(self.C, self.embed(v, parity), parity), parity)

    def D_pp_inv(self, v, parity: int) -> np.ndarray:      # D_ee^{-1} or D_oo^{-1}
        return self.restrict(self.block(self.Cinv, self.embed(v, parity), parity), parity)

    def D_hop(self, v, src: int) -> np.ndarray:            # D_oe (src even) or D_eo (src odd)
        dst = 1 - src
        return self.restrict(-0.5 * self.hop(self.embed(v, src), dst), dst)

    # -- Eq. 3 and Eq. 2 --------------------------------------------------
    def schur(self, xe) -> np.ndarray:
        """D_S x_e = D_ee x_e - D_eo D_oo^{-1} D_oe x_e (Eq. 3)."""
        t = self.D_pp_inv(self.D_hop(xe, EVEN), ODD)
        return self.D_pp(xe, EVEN) - self.D_hop(t, ODD)

    def g5(self, v) -> np.ndarray:
        g = gamma(4)
        return np.einsum("st,nta->nsa", g, np.asarray(v).reshape(-1, 4, 3))

    def schur_dag(self, xe) -> np.ndarray:
        """D_S^+ = g5 D_S g5 (gamma5-hermiticity, pinned by the tests)."""
        return self.g5(self.schur(self.g5(xe)))

    def prepare(self, b) -> np.ndarray:
        """b_hat_e = b_e - D_eo D_oo^{-1} b_o (right factor of Eq. 2)."""
        b = _c128(b).reshape(self.V, 4, 3)
        be, bo = self.restrict(b, EVEN), self.restrict(b, ODD)
        return be - self.D_hop(self.D_pp_inv(bo, ODD), ODD)

    def reconstruct(self, b, xe) -> np.ndarray:
        """x_o = D_oo^{-1} (b_o - D_oe x_e) (left factor of Eq. 2); returns the full x."""
        b = _c128(b).reshape(self.V, 4, 3)
        xo = self.D_pp_inv(self.restrict(b, ODD) - self.D_hop(xe, EVEN), ODD)
        return self.embed(xe, EVEN) + self.embed(xo, ODD)

    def schur_sites(self, xe, sites_e) -> np.ndarray:
        """(D_S x_e) at the listed positions of the even half-vector only; every
        ingredient (hops, clover, inverse) is evaluated just where those outputs
        need it, so this works on lattices too large for the full oracle."""
        sites_e = np.asarray(sites_e, dtype=np.int64)
        lex = np.ascontiguousarray(self.sites[EVEN][sites_e], dtype=np.int64)
        xfull = self.embed(xe, EVEN)
        scratch = np.zeros_like(xfull)
        out = np.zeros((len(lex), 4, 3), dtype=np.complex128)
        bad = _load().orc_schur_sites(_p(self._L), self.t_bc, _p(self.U), self.csw, self.m0,
                                      _p(xfull), len(lex), _p(lex), _p(out), _p(scratch))
        if bad:
            raise ArithmeticError("singular clover block")
        return out


def invert(M) -> np.ndarray:
    """Inverse of every n x n matrix of a stack [..., n, n]."""
    M = _c128(M)
    n = M.shape[-1]
    out = np.empty_like(M)
    count = int(np.prod(M.shape[:-2])) if M.ndim > 2 else 1
    bad = _load().orc_invert(count, n, _p(M), _p(out))
    if bad:
        raise ArithmeticError(f"{bad} singular matrices")
    return out


# ---------------------------------------------------------------------------
# iterative methods (generic in the operator; vectors of any shape)
# ---------------------------------------------------------------------------

def _norm(v) -> float:
    return float(np.sqrt(np.vdot(v, v).real))


def richardson(A, b, omega: float, n: int, x0=None):
    """Richardson(n, delta), Algorithm 4, with omega = delta/|lambda_max| given.

    Every sweep recomputes r = b - A x and adds omega*r, exactly as listed.
    """
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    for _ in range(n):
        r = b - A(x)
        x = x + omega * r
    return x


def _lsq(H, beta):
    """y = argmin ||beta e1 - H y|| (library least squares) and its residual norm."""
    rhs = np.zeros(H.shape[0], dtype=np.complex128)
    rhs[0] = beta
    y = np.linalg.lstsq(H, rhs, rcond=None)[0]
    return y, float(np.linalg.norm(rhs - H @ y))


def gmres(A, b, m: int, n_cycles: int, tol: float, x0=None, breakdown: float = 1e-14):
    """Restarted GMRES(n, m), Algorithm 2.

    Each cycle: r = b - A x, beta = ||r||, stop if beta <= tol*||b||;
    Arnoldi with modified Gram-Schmidt (h_jk = (v_j, w), w -= h_jk v_j) and
    h_{k+1,k} = ||w||; then y = argmin ||beta e1 - H y|| and x += V y.
    Readings where the listing is garbled or silent: v_1 = r/beta and
    v_{k+1} = w/h_{k+1,k}; a cycle also ends early when the least-squares
    residual reaches tol*||b|| (tol > 0) or on a lucky breakdown
    (h_{k+1,k} <= 1e-14 ||A v_k||).  tol = 0 runs exactly n cycles of m steps.
    """
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = _norm(b)
    info = {"cycles": 0, "iters": 0, "converged": False}
    for _ in range(n_cycles):
        r = b - A(x)
        beta = _norm(r)
        if beta <= tol * bnorm or beta == 0.0:
            info["converged"] = True
            break
        info["cycles"] += 1
        V = [r / beta]
        H = np.zeros((m + 1, m), dtype=np.complex128)
        k_used = 0
        for k in range(m):
            w = A(V[k])
            wnorm0 = _norm(w)
            for j in range(k + 1):
                H[j, k] = np.vdot(V[j], w)
                w = w - H[j, k] * V[j]
            H[k + 1, k] = _norm(w)
            k_used = k + 1
            info["iters"] += 1
            _, est = _lsq(H[:k + 2, :k + 1], beta)
            if H[k + 1, k].real <= breakdown * wnorm0 or (tol > 0 and est <= tol * bnorm):
                break
            V.append(w / H[k + 1, k])
        y, _ = _lsq(H[:k_used + 1, :k_used], beta)
        for j in range(k_used):
            x = x + y[j] * V[j]
    r = b - A(x)
    info["rel_resid"] = _norm(r) / bnorm if bnorm > 0 else 0.0
    info["converged"] = info["rel_resid"] <= tol if tol > 0 else info["converged"]
    return x, info


def fgmres(A, b, M, m: int, n_cycles: int, tol: float, x0=None, breakdown: float = 1e-14):
    """Flexible GMRES (right preconditioning by a variable M), the outer solver
    of every level in Sec. 2.3: as GMRES, but z_k = M(v_k), w = A z_k and
    x += Z y.  Same readings as ``gmres``."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = _norm(b)
    info = {"cycles": 0, "iters": 0, "converged": False}
    for _ in range(n_cycles):
        r = b - A(x)
        beta = _norm(r)
        if beta <= tol * bnorm or beta == 0.0:
            info["converged"] = True
            break
        info["cycles"] += 1
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m), dtype=np.complex128)
        k_used = 0
        for k in range(m):
            Z.append(M(V[k]))
            w = A(Z[k])
            wnorm0 = _norm(w)
            for j in range(k + 1):
                H[j, k] = np.vdot(V[j], w)
                w = w - H[j, k] * V[j]
            H[k + 1, k] = _norm(w)
            k_used = k + 1
            info["iters"] += 1
            _, est = _lsq(H[:k + 2, :k + 1], beta)
            if H[k + 1, k].real <= breakdown * wnorm0 or (tol > 0 and est <= tol * bnorm):
                break
            V.append(w / H[k + 1, k])
        y, _ = _lsq(H[:k_used + 1, :k_used], beta)
        for j in range(k_used):
            x = x + y[j] * Z[j]
    r = b - A(x)
    info["rel_resid"] = _norm(r) / bnorm if bnorm > 0 else 0.0
    info["converged"] = info["rel_resid"] <= tol
    return x, info


def power_norm(A, Adag, v0, iters: int) -> float:
    """Estimate of ||A||_2 by power iteration on A^+ A (Sec. 2.4.4: lambda_max is
    computed approximately with a few power iterations).

    v = v0/||v0||; repeat: w = A^+ A v, lam = ||w||, v = w/lam; return sqrt(lam).
    """
    v = np.asarray(v0, dtype=np.complex128)
    v = v / _norm(v)
    lam = 0.0
    for _ in range(iters):
        w = Adag(A(v))
        lam = _norm(w)
        v = w / lam
    return float(np.sqrt(lam))


def smoother(lat: Lattice, r, kind: str, n: int, m: int = 0, omega: float = 0.0):
    """The odd-even smoother M_n r of Sec. 2.4.5 / Fig. 1: Eq. 2 with D_S^{-1}
    replaced by n Richardson sweeps (``kind='richardson'``, weight omega) or by
    GMRES(n, m) (``kind='gmres'``), both started from zero."""
    rhat = lat.prepare(r)
    if kind == "richardson":
        ee = richardson(lat.schur, rhat, omega, n)
    elif kind == "gmres":
        ee, _ = gmres(lat.schur, rhat, m, n, 0.0)
    else:
        raise ValueError(kind)
    return lat.reconstruct(r, ee)


def solve(lat: Lattice, b, tol: float = 1e-10, restart: int = 30, max_restarts: int = 1000,
          solver: str = "gmres", precond: str | None = None, smooth_n: int = 5,
          smooth_m: int = 4, omega: float = 0.0):
    """Odd-even solve of D x = b: prepare (Eq. 2), solve D_S x_e = b_hat_e with
    GMRES(restart) or FGMRES(restart) right-preconditioned by a Richardson or
    GMRES smoother on D_S, reconstruct, and report the true full residual.

    ``tol`` is the relative residual of the full system, ||b - D x|| <= tol ||b||
    (the paper's level-1 (F)GMRES acts on D x = b itself with a relative residual
    tolerance of 1e-10: Sec. 3 and the appendix table of solver parameters).  After the reconstruction
    the odd residual is zero and the even one is b_hat_e - D_S x_e, so the Schur
    solve runs to the relative tolerance tol ||b|| / ||b_hat_e||."""
    b = _c128(b).reshape(lat.V, 4, 3)
    bhat = lat.prepare(b)
    nbh = _norm(bhat)
    tol_s = tol * _norm(b) / nbh if nbh > 0 else tol
    if solver == "gmres":
        xe, info = gmres(lat.schur, bhat, restart, max_restarts, tol_s)
    elif solver == "fgmres":
        if precond == "richardson":
            M = lambda v: richardson(lat.schur, v, omega, smooth_n)  # noqa: E731
        elif precond == "gmres":
            M = lambda v: gmres(lat.schur, v, smooth_m, smooth_n, 0.0)[0]  # noqa: E731
        else:
            M = lambda v: v  # noqa: E731
        xe, info = fgmres(lat.schur, bhat, M, restart, max_restarts, tol_s)
    else:
        raise ValueError(solver)
    x = lat.reconstruct(b, xe)
    info["rel_resid_true"] = _norm(b - lat.dirac(x)) / _norm(b)
    return x, info


def dense(op, n_in: int, shape_in) -> np.ndarray:
    """The dense matrix of a linear operator, column j = op(e_j)."""
    cols = []
    for j in range(n_in):
        e = np.zeros(n_in, dtype=np.complex128)
        e[j] = 1.0
        cols.append(np.asarray(op(e.reshape(shape_in))).reshape(-1))
    return np.stack(cols, axis=1)
