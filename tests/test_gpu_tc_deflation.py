"""Tensor-core batched deflation (tcgen05 GEMMs) against the FP64 oracle's
deflated guess of Eq. 4, for several right-hand sides at once:
x_j = V Lambda^-1 V^dag b_j and r_j = b_j - V V^dag b_j.  The FP16 high/low
split with FP32 accumulation carries about 22 significant bits."""
import numpy as np
import pytest

from gpu_common import make, rel
from oracle.oracle import deflation_guess, project_parity
from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,n,k", [((6, 6, 6, 6), 32, 3), ((6, 6, 6, 8), 40, 7), ((6, 6, 6, 8), 130, 24)])
def test_tc_deflation_matches_oracle(dims, n, k):
    m = 0.01
    ctx, o = make(dims, seed=21, eps=0.3, mass=m)
    try:
        lam, vecs = o.eig_dense(0.0, n)
        H.hisq_set_eigvecs(ctx, vecs, lam, 32)
        bs = np.stack([project_parity(dims, I.gaussian_field(dims, 40 + j), 0) for j in range(k)])
        x, r = H.hisq_deflate_batch(ctx, bs)
        for j in range(k):
            ref = deflation_guess(vecs, lam + 4 * m * m, bs[j])
            assert rel(x[j], ref) <= 1e-5, (j, rel(x[j], ref))
            Vm = vecs.reshape(n, -1)
            rref = bs[j] - (Vm.T @ (Vm.conj() @ bs[j].reshape(-1))).reshape(bs[j].shape)
            assert rel(r[j], rref) <= 1e-5, (j, rel(r[j], rref))
            # the tensor-core result agrees with the CUDA-core deflation
            assert rel(x[j], H.hisq_deflate(ctx, bs[j])) <= 1e-5
    finally:
        ctx.close()


def test_batched_solve_uses_tc_deflation():
    dims = (6, 6, 6, 8)
    m = 0.01
    ctx, o = make(dims, seed=21, eps=0.3, mass=m)
    try:
        lam, vecs = o.eig_dense(0.0, 48)
        H.hisq_set_eigvecs(ctx, vecs, lam, 32)
        etas = np.stack([I.gaussian_source(dims, 9, j) for j in range(6)])
        launches0 = H.hisq_kernel_launches(ctx)
        psi, st, status = H.hisq_solve(ctx, etas, H.hisq_default_solve_params(batch=1, deflate=1, precision_sloppy=16))
        assert status == H.HISQ_OK
        for j in range(6):
            assert o.full_residual(m, psi[j], etas[j]) <= 1e-10
        assert H.hisq_kernel_launches(ctx) > launches0
    finally:
        ctx.close()


def test_tc_wait_timeout_is_reported_and_recovered():
    """The bounded waits of the tensor-core GEMM: with the producer told to issue
    nothing and a short spin limit (host-set, one-shot), the MMA warp's wait for
    its operands runs out with no copy and no MMA in flight; the call returns
    HISQ_ERR_TIMEOUT with a message, and the same context then deflates
    correctly."""
    dims = (6, 6, 6, 8)
    m = 0.01
    ctx, o = make(dims, seed=21, eps=0.3, mass=m)
    try:
        lam, vecs = o.eig_dense(0.0, 40)
        H.hisq_set_eigvecs(ctx, vecs, lam, 32)
        bs = np.stack([project_parity(dims, I.gaussian_field(dims, 50 + j), 0) for j in range(5)])
        H.hisq_inject_wait_timeout(ctx, True)
        with pytest.raises(H.HisqError) as e:
            H.hisq_deflate_batch(ctx, bs)
        assert e.value.status == H.HISQ_ERR_TIMEOUT
        assert "ran out" in str(e.value)
        x, r = H.hisq_deflate_batch(ctx, bs)  # the injection was one-shot
        for j in range(5):
            assert rel(x[j], deflation_guess(vecs, lam + 4 * m * m, bs[j])) <= 1e-5
    finally:
        ctx.close()
