"""Child process of test_gpu_bounds: loads the index-checked library (the
LQ_LIBRARY environment variable names it), runs the hopping kernels K1 and K2
in every precision, the full operator, the SAP smoother, the batched hop in
every launch form and the fermion-force kernels on small lattices, with every
caller field surrounded by canary values, compares the operators with the
oracle, and prints one JSON line: the index-check report of the library, the
canaries that changed, and the largest parity errors."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from paper_2407_08092_gb300 import lqdd, synth  # noqa: E402

PAD = 4096                      # complex values of canary on each side of a field
CANARY = complex(1234.5, -6789.25)
SHAPES = [((2, 2, 2, 2), (2, 2, 2, 2)), ((4, 4, 4, 4), (4, 4, 4, 4)), ((6, 4, 2, 4), (6, 4, 2, 4)),
          ((8, 8, 8, 8), (4, 4, 4, 4))]


class Padded:
    """A device field of `shape` complex doubles inside a buffer with PAD
    canary values before and after it."""

    def __init__(self, shape, init=None):
        n = int(np.prod(shape))
        self.buf = torch.full((n + 2 * PAD,), CANARY, dtype=torch.complex128, device="cuda")
        self.t = self.buf[PAD:PAD + n].view(shape)
        if init is not None:
            self.t.copy_(torch.from_numpy(np.ascontiguousarray(init)).reshape(shape))
        else:
            self.t.zero_()

    def intact(self):
        torch.cuda.synchronize()
        return bool((self.buf[:PAD] == CANARY).all() and (self.buf[-PAD:] == CANARY).all())


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def main():
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    bad_canaries, errs = [], {}
    fields = []
    for L, blk in SHAPES:
        name = "x".join(map(str, L))
        U = synth.gauge_links(L, 0.25, 1000 + sum(L))
        lat = oracle.Lattice(L, U, m0=0.05, csw=1.0, t_bc=-1)
        V, Vh = lat.V, lat.Vh
        ctx = lqdd.lq_create(lqdd.make_lattice(L, -1, 0.05, 1.0), stream)
        try:
            dU = Padded((V, 4, 3, 3), U)
            fields.append((name + ":U", dU))
            lqdd.lq_set_gauge(ctx, dU.t)                   # layout, clover field, assembly, inverse
            xe_h = synth.gaussian_spinor(Vh, 11)
            xe = Padded((Vh, 4, 3), xe_h)
            ye = Padded((Vh, 4, 3))
            fields += [(name + ":xe", xe), (name + ":ye", ye)]
            ref = lat.schur(xe_h)
            for prec, tol in ((lqdd.LQ_F64, 1e-12), (lqdd.LQ_F32, 1e-5), (lqdd.LQ_DF64, 1e-12),
                              (lqdd.LQ_BF16, 1e-2)):
                lqdd.lq_apply(ctx, lqdd.LQ_OP_SCHUR, prec, xe.t, ye.t)   # K1 + K2
                e = rel(ye.t.cpu().numpy(), ref)
                errs[f"{name}:schur{prec}"] = e
                if e > tol:
                    errs.setdefault("failed", []).append(f"{name}:schur{prec}")
            b_h = synth.gaussian_spinor(V, 12)
            b = Padded((V, 4, 3), b_h)
            y = Padded((V, 4, 3))
            fields += [(name + ":b", b), (name + ":y", y)]
            lqdd.lq_apply(ctx, lqdd.LQ_OP_FULL, lqdd.LQ_F64, b.t, y.t)
            errs[f"{name}:full"] = rel(y.t.cpu().numpy(), lat.dirac(b_h))
            # SAP(2, 4) on the full lattice (block-local hops, faces, global indices)
            sap = lqdd.make_params(smoother=lqdd.LQ_SMOOTH_SAP, smooth_n=2, smooth_m=4, inner_prec=lqdd.LQ_F32,
                                   prec=lqdd.LQ_DF64, sap_block=blk)
            lqdd.lq_smooth(ctx, sap, b.t, y.t)
            # fermion force kernels (clover insertion, per-link gradient)
            G = Padded((V, 4, 3, 3))
            fields.append((name + ":G", G))
            lqdd.lq_force(ctx, b.t, y.t, G.t)
            # the batched hop in every launch form (3 right-hand sides)
            nb = 3
            B = Padded((nb, V, 4, 3), np.stack([synth.gaussian_spinor(V, 20 + r) for r in range(nb)]))
            X = Padded((nb, V, 4, 3))
            fields += [(name + ":B", B), (name + ":X", X)]
            grp = lqdd.lq_group_create([ctx], stream)
            try:
                for spt, rpt, fac in [(32, 1, 1), (16, 2, 0), (32, 0, 1), (64, 0, 2), (128, 1, 2)]:
                    lqdd.lq_group_set_shape(grp, spt, rpt, fac)
                    X.t.zero_()
                    st, _ = lqdd.lq_solve_group(grp, ctx, lqdd.make_batch_params(tol=1e-8, restart=8), [B.t], [X.t])
                    if st != lqdd.LQ_OK:
                        errs.setdefault("failed", []).append(f"{name}:group{spt},{rpt}")
            finally:
                lqdd.lq_group_destroy(grp)
        finally:
            lqdd.lq_destroy(ctx)
    for fname, f in fields:
        if not f.intact():
            bad_canaries.append(fname)
    status, checked, violations, first = lqdd.lq_bounds_check()
    print(json.dumps({"checked": checked, "status": status, "violations": violations, "first_code": first,
                      "bad_canaries": bad_canaries, "failed": errs.get("failed", []),
                      "max_err": {k: v for k, v in errs.items() if k != "failed"}}), flush=True)


if __name__ == "__main__":
    main()
