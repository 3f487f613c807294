"""Helpers shared by the GPU parity tests (device plumbing only)."""
import numpy as np

import oracle
from paper_2407_08092_gb300 import synth


def rel(a, b) -> float:
    a, b = np.ravel(np.asarray(a)), np.ravel(np.asarray(b))
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


class Pair:
    """The same lattice on the GPU (through the C ABI) and in the oracle."""

    def __init__(self, L, eps=0.25, seed=1000, m0=0.05, csw=1.0, t_bc=-1, U=None):
        import torch

        from paper_2407_08092_gb300 import lqdd
        self.lqdd = lqdd
        self.torch = torch
        self.L = tuple(L)
        self.U = synth.gauge_links(L, eps, seed) if U is None else U
        self.lat = oracle.Lattice(L, self.U, m0=m0, csw=csw, t_bc=t_bc)
        self.V, self.Vh = self.lat.V, self.lat.Vh
        self.ctx = lqdd.lq_create(lqdd.make_lattice(L, t_bc, m0, csw), torch.cuda.current_stream().cuda_stream)
        self.dU = torch.from_numpy(self.U).cuda()
        lqdd.lq_set_gauge(self.ctx, self.dU)

    def dev(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()

    def host(self, t):
        self.torch.cuda.synchronize()
        return t.cpu().numpy()

    def apply(self, op, prec, x):
        dx = self.dev(x)
        out = self.torch.empty_like(dx)
        self.lqdd.lq_apply(self.ctx, op, prec, dx, out)
        return self.host(out)

    def close(self):
        self.lqdd.lq_destroy(self.ctx)
