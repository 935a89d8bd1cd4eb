"""hisq_deflate_noalloc: the deflated guess of Eq. 4 for callers that may not
allocate device memory, for example code running inside a memory budget that
another allocator owns.  It uses a fixed scratch array that is reserved when a
context is created.

The tests call the entry point through the C ABI on caller-owned device
buffers:
  * twice in a row with different sources, for every eigenvector storage
    format, against the FP64 oracle's Eq. 4 evaluated on the values the
    storage format holds (within FP32 accumulation), and against hisq_deflate;
  * in a fresh process, where the first call must leave the device's free
    memory and the context's device bytes unchanged.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

from gpu_common import make, orthonormal_even_set, rel, stored_vectors
from oracle.oracle import deflation_guess, project_parity
from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _to_even_layout(dims, field):
    """Host full-lattice field -> even-site device layout [colour][Vh] complex
    (even site s has index s // 2)."""
    par = (np.indices(dims[::-1]).sum(axis=0) & 1).reshape(-1)  # parity of s = x + X(y + Y(z + Z t))
    even = np.nonzero(par == 0)[0]
    return torch.from_numpy(np.ascontiguousarray(field[even].T)).cuda(), even


@pytest.mark.parametrize("storage", [32, 16, H.HISQ_PREC_BF16, H.HISQ_PREC_HALF_EV])
def test_noalloc_matches_oracle_twice(storage):
    """12^3 x 16 (Vh = 13,824: four projection chunks, the last one ragged),
    40 orthonormal even-site fields with chosen eigenvalues."""
    dims = (12, 12, 12, 16)
    m = 0.01
    n = 40
    ctx, _ = make(dims, seed=21, eps=0.3, mass=m)
    try:
        lam, vecs = orthonormal_even_set(dims, n, seed=5)
        H.hisq_set_eigvecs(ctx, vecs, lam, storage)
        vs = stored_vectors(vecs, storage, I.volume(dims) // 2)
        for seed in (31, 32):  # two calls in a row, different sources
            b = project_parity(dims, I.gaussian_field(dims, seed), 0)
            ref = deflation_guess(vs, lam + 4 * m * m, b)
            b_dev, even = _to_even_layout(dims, b)
            x_dev = torch.full_like(b_dev, complex(np.nan, np.nan))  # the output is overwritten
            H.hisq_deflate_noalloc(ctx, b_dev, x_dev)
            torch.cuda.synchronize()
            x = np.zeros_like(b)
            x[even] = x_dev.cpu().numpy().T
            # FP32 accumulation over 40 vectors and the site sums of the projection
            assert rel(x, ref) <= 2e-6, (storage, seed, rel(x, ref))
            # the same guess as the allocating entry point
            assert rel(x, H.hisq_deflate(ctx, b)) <= 1e-12
    finally:
        ctx.close()


_FRESH = textwrap.dedent(r"""
    import json, sys
    import numpy as np, torch
    sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
    from gpu_common import make, orthonormal_even_set
    from oracle.oracle import project_parity
    from paper_2502_00152_gb300 import hisq as H
    from paper_2502_00152_gb300 import inputs as I
    dims = (8, 8, 8, 8)
    ctx, _ = make(dims, seed=4, eps=0.3, mass=0.02)
    lam, vecs = orthonormal_even_set(dims, 16, seed=6)
    H.hisq_set_eigvecs(ctx, vecs, lam, 32)
    b = project_parity(dims, I.gaussian_field(dims, 7), 0)
    H.hisq_deflate(ctx, b)  # loads the code of the deflation kernels
    par = (np.indices(dims[::-1]).sum(axis=0) & 1).reshape(-1)
    b_dev = torch.from_numpy(np.ascontiguousarray(b[par == 0].T)).cuda()
    x_dev = torch.zeros_like(b_dev)
    torch.cuda.synchronize()
    free0, bytes0 = torch.cuda.mem_get_info()[0], H.hisq_device_bytes(ctx)
    H.hisq_deflate_noalloc(ctx, b_dev, x_dev)
    torch.cuda.synchronize()
    free1, bytes1 = torch.cuda.mem_get_info()[0], H.hisq_device_bytes(ctx)
    H.hisq_deflate_noalloc(ctx, b_dev, x_dev)
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    print(json.dumps(dict(free=[free0, free1, free2], bytes=[bytes0, bytes1])))
    ctx.close()
""")


def test_noalloc_first_call_allocates_nothing():
    """The defining property, in a process of its own: the device's free memory
    and the context's device bytes are the same before and after the first
    (and a second) call."""
    code = _FRESH.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    import json

    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["free"][0] == d["free"][1] == d["free"][2], d
    assert d["bytes"][0] == d["bytes"][1], d


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
