"""FP64 CPU oracle of the fermion force -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the product never does.

The paper has no fermion force: this is the differentiation workload built on
its operator.  For the pseudofermion action

    S(U) = phi^+ (D^+ D)^{-1} phi

(D the Wilson-clover operator of Sec. 2.3 on the full lattice), with
X = (D^+ D)^{-1} phi and Y = D X = D^{-+} phi, varying U gives

    dS = -2 Re( Y^+ dD X ),

so the gradient of S is -2 times the gradient of the bilinear form
b(U) = Re(Y^+ D(U) X) at fixed X, Y.

Everything here is the plain definition:

* ``dirac`` applies D written out with ``torch.roll`` shifts on the
  lattice-shaped field: the hopping term with the fermion time-boundary sign,
  and C = (4 + m0) + c_sw (i/4) sum_{mu != nu} sigma_mu_nu F_mu_nu with
  F = (Q - Q^+)/8 and Q the four same-orientation plaquette leaves at x.  It is
  a second, independent implementation of the operator in ``oracle.c``; the
  pins require the two to agree.
* ``bilinear_grad`` is the gradient of b(U) taken by ``torch.autograd`` through
  ``dirac`` (one pass for the hopping term and one per plane of the clover
  term, to bound memory).  Gradients use torch's convention for a real
  function of a complex matrix: G = dS/dRe U + i dS/dIm U, so that
  dS = Re sum conj(G) dU.
* ``action`` and ``force`` solve for X and Y with the oracle's own odd-even
  solves (or dense LU on tiny lattices) and return S and -2 G.

The pins (``tests/test_oracle_force.py``) compare ``dirac`` with ``oracle.c``,
the bilinear gradient with central differences of b, and the force with
central differences of S along the su(3) generators T_a = lambda_a / 2.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Lattice, gamma, solve


def _tensor(a) -> torch.Tensor:
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.complex128)


class TorchDirac:
    """The Wilson-clover D of Sec. 2.3 on fields shaped [Lt, Lz, Ly, Lx, ...].

    Direction mu = 0..3 (x, y, z, t) is tensor dimension 3 - mu; the natural
    order lex = x + Lx (y + Ly (z + Lz t)) is the row-major order of that shape.
    """

    def __init__(self, L, m0: float, csw: float, t_bc: int = -1):
        self.L = tuple(int(v) for v in L)
        self.shape = (self.L[3], self.L[2], self.L[1], self.L[0])
        self.m0, self.csw, self.t_bc = float(m0), float(csw), int(t_bc)
        self.g = [_tensor(gamma(mu)) for mu in range(4)]
        one = torch.eye(4, dtype=torch.complex128)
        self.pm = [one - g for g in self.g]      # 1 - gamma_mu (forward hop)
        self.pp = [one + g for g in self.g]      # 1 + gamma_mu (backward hop)
        # sigma_mu_nu = (i/2) [gamma_mu, gamma_nu]
        self.sigma = [[0.5j * (self.g[m] @ self.g[n] - self.g[n] @ self.g[m]) for n in range(4)] for m in range(4)]
        # fermion boundary sign of a hop that wraps around in time, by t
        sgn = torch.ones(self.L[3], dtype=torch.complex128)
        self.sign_fwd = sgn.clone()
        self.sign_fwd[-1] = self.t_bc                # psi(x + t) read at t = Lt - 1 wraps
        self.sign_bwd = sgn.clone()
        self.sign_bwd[0] = self.t_bc                 # psi(x - t) read at t = 0 wraps

    # -- shifts ------------------------------------------------------------
    @staticmethod
    def fwd(f, mu):
        """f(x + mu) at x."""
        return torch.roll(f, shifts=-1, dims=3 - mu)

    @staticmethod
    def bwd(f, mu):
        """f(x - mu) at x."""
        return torch.roll(f, shifts=1, dims=3 - mu)

    def reshape_links(self, U):
        return U.reshape(*self.shape, 4, 3, 3)

    def reshape_field(self, psi):
        return psi.reshape(*self.shape, 4, 3)

    # -- hopping term ----------------------------------------------------------
    def hop(self, U, psi):
        """H psi = sum_mu [(1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu)]
        with the time-boundary sign on the hops that wrap around in t."""
        out = torch.zeros_like(psi)
        for mu in range(4):
            Um = U[..., mu, :, :]
            f = torch.einsum("...ab,...sb->...sa", Um, self.fwd(psi, mu))
            Ub = self.bwd(Um, mu).conj().transpose(-1, -2)
            b = torch.einsum("...ab,...sb->...sa", Ub, self.bwd(psi, mu))
            if mu == 3:
                f = f * self.sign_fwd.view(-1, 1, 1, 1, 1, 1)
                b = b * self.sign_bwd.view(-1, 1, 1, 1, 1, 1)
            out = out + torch.einsum("rs,...sa->...ra", self.pm[mu], f)
            out = out + torch.einsum("rs,...sa->...ra", self.pp[mu], b)
        return out

    # -- clover term -------------------------------------------------------------
    def leaves(self, U, mu, nu):
        """Q_mu_nu(x): the four plaquettes in the (mu, nu) plane that start and end
        at x, all with the orientation mu -> nu."""
        Um, Un = U[..., mu, :, :], U[..., nu, :, :]
        dag = lambda M: M.conj().transpose(-1, -2)  # noqa: E731
        f, b = self.fwd, self.bwd
        q = Um @ f(Un, mu) @ dag(f(Um, nu)) @ dag(Un)
        q = q + Un @ dag(b(f(Um, nu), mu)) @ dag(b(Un, mu)) @ b(Um, mu)
        q = q + dag(b(Um, mu)) @ dag(b(b(Un, mu), nu)) @ b(b(Um, mu), nu) @ b(Un, nu)
        q = q + dag(b(Un, nu)) @ b(Um, nu) @ f(b(Un, nu), mu) @ dag(Um)
        return q

    def field_strength(self, U, mu, nu):
        """F_mu_nu = (Q_mu_nu - Q_mu_nu^+) / 8."""
        Q = self.leaves(U, mu, nu)
        return (Q - Q.conj().transpose(-1, -2)) / 8.0

    def clover_plane(self, U, psi, mu, nu):
        """c_sw (i/4) sigma_mu_nu F_mu_nu psi for one ordered pair (mu, nu)."""
        F = self.field_strength(U, mu, nu)
        return (0.25j * self.csw) * torch.einsum("rs,...ab,...sb->...ra", self.sigma[mu][nu], F, psi)

    def clover(self, U, psi):
        """C psi = (4 + m0) psi + c_sw (i/4) sum_{mu != nu} sigma_mu_nu F_mu_nu psi."""
        out = (4.0 + self.m0) * psi
        for mu in range(4):
            for nu in range(4):
                if mu != nu:
                    out = out + self.clover_plane(U, psi, mu, nu)
        return out

    def dirac(self, U, psi):
        """D psi = C psi - (1/2) H psi."""
        return self.clover(U, psi) - 0.5 * self.hop(U, psi)


def dirac(L, U, psi, m0: float, csw: float, t_bc: int = -1) -> np.ndarray:
    """D psi in natural order ([V, 4, 3] complex128) by ``TorchDirac``."""
    op = TorchDirac(L, m0, csw, t_bc)
    with torch.no_grad():
        out = op.dirac(op.reshape_links(_tensor(U)), op.reshape_field(_tensor(psi)))
    return out.reshape(-1, 4, 3).numpy()


def bilinear_grad(L, U, X, Y, m0: float, csw: float, t_bc: int = -1) -> np.ndarray:
    """G = grad_U Re(Y^+ D(U) X) at fixed X, Y: [V, 4, 3, 3] complex128 with
    G = d/dRe U + i d/dIm U.  The hopping term and each plane of the clover
    term are differentiated in separate autograd passes and summed."""
    op = TorchDirac(L, m0, csw, t_bc)
    Xt = op.reshape_field(_tensor(X))
    Yt = op.reshape_field(_tensor(Y))
    U0 = op.reshape_links(_tensor(U))
    G = torch.zeros_like(U0)

    def add(fn):
        Ut = U0.clone().requires_grad_(True)
        b = torch.sum(Yt.conj() * fn(Ut)).real
        (g,) = torch.autograd.grad(b, Ut)
        G.add_(g)

    add(lambda Ut: -0.5 * op.hop(Ut, Xt))
    for mu in range(4):
        for nu in range(mu + 1, 4):
            add(lambda Ut, mu=mu, nu=nu: op.clover_plane(Ut, Xt, mu, nu) + op.clover_plane(Ut, Xt, nu, mu))
    return G.reshape(-1, 4, 3, 3).numpy()


def solve_pair(lat: Lattice, phi, tol: float = 1e-12, dense: bool = False):
    """X = (D^+ D)^{-1} phi and Y = D X = D^{-+} phi.

    D^+ = g5 D g5, so Y = g5 D^{-1} g5 phi and X = D^{-1} Y: two odd-even solves
    (Eq. 2, GMRES to ``tol``), or dense LU when ``dense``."""
    phi = np.asarray(phi, dtype=np.complex128).reshape(lat.V, 4, 3)
    if dense:
        n = lat.V * 12
        A = np.zeros((n, n), dtype=np.complex128)
        for j in range(n):
            e = np.zeros(n, dtype=np.complex128)
            e[j] = 1.0
            A[:, j] = lat.dirac(e.reshape(lat.V, 4, 3)).reshape(-1)
        Y = np.linalg.solve(A.conj().T, phi.reshape(-1))
        X = np.linalg.solve(A, Y)
        return X.reshape(lat.V, 4, 3), Y.reshape(lat.V, 4, 3)
    W, _ = solve(lat, lat.g5(phi), tol=tol)
    Y = lat.g5(W)
    X, _ = solve(lat, Y, tol=tol)
    return X, Y


def action(lat: Lattice, phi, tol: float = 1e-12, dense: bool = False) -> float:
    """S = phi^+ (D^+ D)^{-1} phi = ||D^{-+} phi||^2."""
    _, Y = solve_pair(lat, phi, tol, dense)
    return float(np.vdot(Y, Y).real)


def force(lat: Lattice, phi, tol: float = 1e-12, dense: bool = False):
    """(S, dS/dU) with dS/dU = -2 grad_U Re(Y^+ D X), [V, 4, 3, 3] complex128."""
    X, Y = solve_pair(lat, phi, tol, dense)
    G = bilinear_grad(lat.L, lat.U, X, Y, lat.m0, lat.csw, lat.t_bc)
    return float(np.vdot(Y, Y).real), -2.0 * G


def generator_derivative(G, U, site: int, mu: int, T) -> float:
    """dS/dh of S(exp(i h T) U_mu(x) at x = site) at h = 0 from a gradient G:
    Re sum conj(G) (i T U)."""
    dU = 1j * T @ U[site, mu]
    return float(np.sum(np.conj(G[site, mu]) * dU).real)
