"""The pseudofermion action as a differentiable PyTorch function.

``PseudofermionAction.apply(U, phi, action)`` returns S = phi^+ (D^+ D)^{-1} phi
for the gauge field U ([V, 4, 3, 3] complex128, CUDA) and backpropagates
dS/dU.  Forward is ``lq_fermion_action`` (two odd-even solves through the C
ABI, the adjoint one with D^+ = g5 D g5); backward is ``lq_force``, the
hand-written df64 gradient kernel, applied to the saved X and Y.  Gradients
follow torch's convention for complex inputs, dS/dRe U + i dS/dIm U.  phi is
treated as a constant (no gradient flows to it).

The wrapper only marshals arguments: every step runs in the library's kernels.
"""
from __future__ import annotations

import torch

from . import lqdd


class FermionAction:
    """A lattice context plus solver parameters for the pseudofermion action.

    The context holds one gauge field at a time; ``ensure_gauge`` re-imports U
    (and rebuilds the clover term) only when a different tensor, or the same
    tensor after an in-place change, is passed."""

    def __init__(self, L, m0: float, csw: float, t_bc: int = -1, params=None, stream=None):
        self.L = tuple(int(v) for v in L)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = lqdd.lq_create(lqdd.make_lattice(self.L, t_bc, m0, csw), s.cuda_stream)
        self.params = params if params is not None else lqdd.make_params(
            solver=lqdd.LQ_SOLVER_FGMRES, prec=lqdd.LQ_DF64, tol=1e-12, restart=10, max_restarts=50,
            smoother=lqdd.LQ_SMOOTH_GMRES, smooth_n=40, smooth_m=8, smooth_tol=1e-5, inner_prec=lqdd.LQ_F32)
        self._key = None
        self._ref = None
        self.last_stats = None

    def ensure_gauge(self, U: torch.Tensor):
        # the reference kept in _ref stops the allocator from handing the same
        # address to another tensor while the key is in use
        key = (U.data_ptr(), U._version, tuple(U.shape))
        if key != self._key:
            lqdd.lq_set_gauge(self.ctx, U)
            self._key, self._ref = key, U

    def close(self):
        if self.ctx is not None:
            lqdd.lq_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __call__(self, U: torch.Tensor, phi: torch.Tensor) -> torch.Tensor:
        return PseudofermionAction.apply(U, phi, self)


class PseudofermionAction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, U, phi, action: FermionAction):
        U = U.detach().contiguous()
        phi = phi.detach().contiguous()
        action.ensure_gauge(U)
        X = torch.empty_like(phi)
        Y = torch.empty_like(phi)
        status, S, stats = lqdd.lq_fermion_action(action.ctx, action.params, phi, X, Y)
        if status != lqdd.LQ_OK:
            raise lqdd.LqError(status, lqdd.lq_last_error(action.ctx))
        action.last_stats = stats
        fctx.action = action
        fctx.save_for_backward(U, X, Y)
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(fctx, grad_S):
        U, X, Y = fctx.saved_tensors
        action = fctx.action
        action.ensure_gauge(U)
        G = torch.empty_like(U)
        lqdd.lq_force(action.ctx, X, Y, G, coef=-2.0)
        return grad_S.to(G.real.dtype) * G, None, None
