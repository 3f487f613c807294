"""lq_norm2_noalloc: the no-allocation variant of the norm reduction.

Some callers cannot allocate device memory (they run inside a fixed memory
budget owned by another framework, where a cudaMalloc could fail or
synchronise the device at the wrong moment).  For them the library offers
lq_norm2_noalloc, which keeps its reduction scratch in a static device array
and needs no context.  This test calls it through the C ABI and compares it
with the context-based lq_norm2 on two calls in a row: a large field that
fills many scratch slots, then a small one that must not pick up the first
call's leftovers.  It also checks that a call after the first one on the device
leaves the device's free memory unchanged, and runs once at the largest size
the scratch array allows.  It lives in a file pytest collects last, so a run
that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_norm2_noalloc_matches_norm2_two_calls_in_a_row():
    import torch

    from paper_2407_08092_gb300 import lqdd, synth

    stream = torch.cuda.current_stream().cuda_stream
    ctx = lqdd.lq_create(lqdd.make_lattice((8, 8, 8, 8), -1, 0.05, 1.0), stream)
    try:
        big = torch.from_numpy(synth.gaussian_spinor(600_000, 11)).cuda()      # 880 scratch slots
        small = torch.from_numpy(synth.gaussian_spinor(1_000, 12)).cuda()      # 2 scratch slots
        out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        for v in (big, small):
            n = v.shape[0]
            lqdd.lq_norm2_noalloc(v, n, out, stream)
            torch.cuda.synchronize()
            got = float(out.item())
            ref = lqdd.lq_norm2(ctx, v, n)
            assert abs(got - ref) <= 1e-12 * ref, (n, got, ref)
            host = float(np.vdot(v.cpu().numpy(), v.cpu().numpy()).real)
            assert abs(got - host) <= 1e-12 * host
        # once the first call has run on this device, a call allocates nothing:
        # neither the driver's free memory nor torch's allocator changes
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        lqdd.lq_norm2_noalloc(big, big.shape[0], out, stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_allocated() == alloc0
        # exactly the largest field: all 4096 scratch slots in use
        n_max = lqdd.LQ_NORM2_NOALLOC_MAX_SITES
        g = torch.Generator(device="cuda")
        g.manual_seed(13)
        full = torch.randn((n_max, 4, 3), dtype=torch.complex128, device="cuda", generator=g)
        lqdd.lq_norm2_noalloc(full, n_max, out, stream)
        torch.cuda.synchronize()
        got = float(out.item())
        ref = lqdd.lq_norm2(ctx, full, n_max)
        assert abs(got - ref) <= 1e-12 * ref, (n_max, got, ref)
        del full
        # an empty field gives zero
        lqdd.lq_norm2_noalloc(None, 0, out, stream)
        torch.cuda.synchronize()
        assert float(out.item()) == 0.0
        # a size beyond the stated maximum is rejected before any launch
        with pytest.raises(lqdd.LqError) as ei:
            lqdd.lq_norm2_noalloc(big, lqdd.LQ_NORM2_NOALLOC_MAX_SITES + 1, out, stream)
        assert ei.value.status == lqdd.LQ_ERR_ARG
    finally:
        lqdd.lq_destroy(ctx)
