"""The allocation-free inner Jacobi-PCG entry point (pfk_pc_apply_inner_pcg_noalloc).

It serves callers that cannot allocate device memory when they apply the
preconditioner (their memory belongs to another pool allocator, or they cannot
afford the synchronisation an allocation may cause).  Its scratch is a static
device array, so these checks call it through the C ABI twice in a row on
preallocated buffers and compare with the ordinary, allocating preconditioner
of the same kind.  This file is collected last on purpose: a failure here must
not stop the rest of the GPU suite from running first.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_twice(lib):
    import torch
    from paper_1511_07226_gb300 import pfk
    ctx = pfk.Context(0)
    dims = (48, 40, 36)
    c = W.poisson3d_gaussian(dims=dims, ell=4.0, log_contrast=3.0, config_id=2, item_id=31)
    op = pfk.Operator.stencil(ctx, dims, c["eta"])
    assert op.n <= pfk.NOALLOC_MAX_N
    pc = pfk.Preconditioner(ctx, op, "inner_pcg", inner_iters=4, precision="fp64")
    y = torch.empty(op.n, dtype=torch.float64, device="cuda")
    for call in range(2):
        v = torch.from_numpy(W.random_vector(op.n, 40 + call)).cuda()
        ref = pc.apply(v).cpu().numpy()
        st = lib.pfk_pc_apply_inner_pcg_noalloc(ctx.h, op.h, 4, C.c_void_p(v.data_ptr()),
                                                C.c_void_p(y.data_ptr()))
        assert st == 0, lib.pfk_last_error(ctx.h)
        got = y.cpu().numpy()
        # the tolerance of the inner-PCG parity tests
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    import torch
    from paper_1511_07226_gb300 import pfk
    ctx = pfk.Context(0)
    dims = (72, 64, 64)
    assert 72 * 64 * 64 > pfk.NOALLOC_MAX_N
    op = pfk.Operator.stencil(ctx, dims, np.ones(72 * 64 * 64))
    v = torch.zeros(op.n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(v)
    st = lib.pfk_pc_apply_inner_pcg_noalloc(ctx.h, op.h, 4, C.c_void_p(v.data_ptr()), C.c_void_p(y.data_ptr()))
    assert st == -1
    assert b"PFK_NOALLOC_MAX_N" in lib.pfk_last_error(ctx.h)
