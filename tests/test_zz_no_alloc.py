"""hisq_deflate_noalloc: the deflated guess for callers that may not allocate
device memory (for example code that runs inside a memory budget owned by
another allocator).  Called through the C ABI on device buffers, twice in a
row with different sources, it must give the same result as hisq_deflate.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest
import torch

from gpu_common import make, rel
from oracle.oracle import project_parity
from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _to_even_layout(dims, field):
    """Host full-lattice field -> even-site device layout [colour][Vh] complex
    (even site s has index s // 2)."""
    par = (np.indices(dims[::-1]).sum(axis=0) & 1).reshape(-1)  # parity of s = x + X(y + Y(z + Z t))
    even = np.nonzero(par == 0)[0]
    return torch.from_numpy(np.ascontiguousarray(field[even].T)).cuda(), even


def test_noalloc_matches_hisq_deflate_twice():
    dims = (6, 6, 6, 8)
    m = 0.01
    ctx, o = make(dims, seed=21, eps=0.3, mass=m)
    try:
        lam, vecs = o.eig_dense(0.0, 24)
        H.hisq_set_eigvecs(ctx, vecs, lam, 32)
        for seed in (31, 32):  # two calls in a row, different sources
            b = project_parity(dims, I.gaussian_field(dims, seed), 0)
            ref = H.hisq_deflate(ctx, b)  # the existing entry point (context scratch)
            b_dev, even = _to_even_layout(dims, b)
            x_dev = torch.full_like(b_dev, complex(np.nan, np.nan))  # output is overwritten
            H.hisq_deflate_noalloc(ctx, b_dev, x_dev)
            torch.cuda.synchronize()
            x = np.zeros_like(b)
            x[even] = x_dev.cpu().numpy().T
            assert rel(x, ref) <= 1e-12
    finally:
        ctx.close()


def test_noalloc_rejects_state_errors():
    dims = (4, 4, 4, 4)
    ctx, o = make(dims, mass=0.1)
    try:
        b = torch.zeros(3 * I.volume(dims) // 2, dtype=torch.complex128, device="cuda")
        with pytest.raises(H.HisqError) as e:
            H.hisq_deflate_noalloc(ctx, b, torch.zeros_like(b))
        assert e.value.status == H.HISQ_ERR_STATE  # no eigenpairs stored yet
    finally:
        ctx.close()
