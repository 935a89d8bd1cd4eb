"""The batched operator of the multi-RHS solve (Section 4 outlook: several
right-hand sides per pass over the links) against the FP64 oracle's D, for every
launch shape: the register kernel (each thread loads its site's links) with and
without the L2 link prefetch, the same with the right-hand sides in pairs on
packed two-wide FP32 FMAs, and the TMA-fed kernel (links of each site group and
direction bulk-copied into a shared-memory ring) at its three occupancies, with
2, 3 and 4 right-hand sides per thread.

14^3 x 18 has Vh = 24,696 = 771 full site groups of 32 and a ragged one of 24,
enough groups that every block walks several of them (the TMA ring wraps
around); 12-real long links (the only format of the TMA kernel)."""
import numpy as np
import pytest

from gpu_common import dslash_ref, make, rel
from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DIMS = (14, 14, 14, 18)


@pytest.fixture(scope="module")
def lat():
    ctx, o = make(DIMS, seed=8, eps=0.3, recon=12, mass=0.01)
    fields = np.stack([I.gaussian_field(DIMS, 300 + j) for j in range(12)])
    refs = {par: [dslash_ref(o, DIMS, fields[j], par) for j in range(12)] for par in (0, 1)}
    yield ctx, fields, refs
    ctx.close()


SHAPES = ([(1, R, b) for R in (4, 3, 2) for b in (0, 1)] + [(2, R, b) for R in (4, 3, 2) for b in (2, 3, 4)]
          + [(3, R, b) for R in (4, 2) for b in (0, 1)])


@pytest.mark.parametrize("kind,R,budget", SHAPES)
@pytest.mark.parametrize("prec,tol", [(32, 1e-6), (16, 5e-3)])
def test_batched_dslash_shapes_match_oracle(lat, kind, R, budget, prec, tol):
    ctx, fields, refs = lat
    H.hisq_set_batched_kernel(ctx, kind, R, budget)
    try:
        for k, par in ((12, 1), (5, 0)):  # a full batch and a partial last chunk
            out = H.hisq_apply_dslash_batch(ctx, par, prec, fields[:k])
            for j in range(k):
                assert rel(out[j], refs[par][j]) <= tol, (kind, R, budget, prec, k, j, rel(out[j], refs[par][j]))
    finally:
        H.hisq_set_batched_kernel(ctx, 0)


def test_batched_dslash_autotuned(lat):
    ctx, fields, refs = lat
    out = H.hisq_apply_dslash_batch(ctx, 1, 16, fields)
    for j in range(12):
        assert rel(out[j], refs[1][j]) <= 5e-3


def test_missing_shape_is_refused(lat):
    ctx, fields, refs = lat
    H.hisq_set_batched_kernel(ctx, 1, 2, 0)
    try:
        # 64 right-hand sides at 2 per thread would need 32 warps per site group
        with pytest.raises(H.HisqError) as e:
            H.hisq_apply_dslash_batch(ctx, 1, 32, np.concatenate([fields] * 6)[:64])
        assert e.value.status == H.HISQ_ERR_INVALID_ARG
    finally:
        H.hisq_set_batched_kernel(ctx, 0)
