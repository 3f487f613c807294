"""A small, self-contained case of the hopping kernels for profiler captures.

Builds a context on a seeded lattice (default 24^3 x 48, whose per-launch
working set is larger than L2 but whose device footprint stays near 1.5 GB)
and applies D_S (K1 + K2) `--apps` times in one precision through the C ABI:
``python -m paper_2407_08092_gb300.profile_case --lattice 24,24,24,48 --prec 1 --apps 3``.
"""
import argparse

import numpy as np
import torch

from paper_2407_08092_gb300 import lqdd, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lattice", default="24,24,24,48")
    ap.add_argument("--prec", type=int, default=1)
    ap.add_argument("--apps", type=int, default=3)
    ap.add_argument("--op", type=int, default=lqdd.LQ_OP_SCHUR)
    a = ap.parse_args()
    L = tuple(int(v) for v in a.lattice.split(","))
    V = int(np.prod(L))
    ctx = lqdd.lq_create(lqdd.make_lattice(L, -1, 0.05, 1.0), torch.cuda.current_stream().cuda_stream)
    lqdd.lq_set_gauge(ctx, torch.from_numpy(synth.gauge_links(L, 0.25, 1003)).cuda())
    n = V if a.op == lqdd.LQ_OP_FULL else V // 2
    x = torch.from_numpy(synth.gaussian_spinor(n, 2003)).cuda()
    y = torch.empty_like(x)
    for _ in range(a.apps):
        lqdd.lq_apply(ctx, a.op, a.prec, x, y)
    torch.cuda.synchronize()
    print("ok", L, "prec", a.prec, "apps", a.apps, float(y.abs().sum()))
    lqdd.lq_destroy(ctx)


if __name__ == "__main__":
    main()
