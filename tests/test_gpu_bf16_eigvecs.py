"""BF16 eigenvector storage (12 B per site): the stored values are the
round-to-nearest-even BF16 of the FP32 vectors (bit-exact), and every deflation
path -- the CUDA-core projection/expansion, the tensor-core BF16 GEMMs of a
batch and the batched deflated solve -- agrees with the FP64 oracle's deflated
guess of Eq. 4 evaluated on those same rounded vectors."""
import os
import tempfile

import numpy as np
import pytest

from gpu_common import make, rel
from oracle.oracle import deflation_guess, project_parity
from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def bf16_round(x):
    """FP64 complex -> FP32 -> BF16 (round to nearest even) -> FP64 complex."""
    def one(a):
        f = np.ascontiguousarray(a, dtype=np.float32)
        u = f.view(np.uint32).astype(np.uint64)
        u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
        return u.astype(np.uint32).view(np.float32).astype(np.float64)
    x = np.asarray(x)
    return one(x.real) + 1j * one(x.imag)


def _setup(dims, n, m=0.01):
    ctx, o = make(dims, seed=21, eps=0.3, mass=m)
    lam, vecs = o.eig_dense(0.0, n)
    H.hisq_set_eigvecs(ctx, vecs, lam, H.HISQ_PREC_BF16)
    return ctx, o, lam, vecs, bf16_round(vecs)


def test_bf16_storage_is_round_to_nearest_even():
    dims = (4, 4, 4, 6)
    ctx, o, lam, vecs, vr = _setup(dims, 12)
    try:
        for i in range(12):
            got = H.hisq_get_eigvec(ctx, i)
            assert np.array_equal(got, vr[i])
        assert np.allclose(H.hisq_get_eigvals(ctx), lam, rtol=0, atol=0)
        # save / load keeps the stored bytes
        with tempfile.TemporaryDirectory() as d:
            path = os.path.join(d, "ev.bin")
            H.hisq_save_eigvecs(ctx, path)
            H.hisq_set_eigvecs(ctx, vecs[:2], lam[:2], 32)
            H.hisq_load_eigvecs(ctx, path)
            for i in (0, 5, 11):
                assert np.array_equal(H.hisq_get_eigvec(ctx, i), vr[i])
    finally:
        ctx.close()


@pytest.mark.parametrize("dims,n,k", [((6, 6, 6, 6), 32, 3), ((6, 6, 6, 8), 130, 24)])
def test_bf16_deflation_matches_oracle(dims, n, k):
    m = 0.01
    ctx, o, lam, vecs, vr = _setup(dims, n, m)
    try:
        bs = np.stack([project_parity(dims, I.gaussian_field(dims, 40 + j), 0) for j in range(k)])
        x, r = H.hisq_deflate_batch(ctx, bs)  # tensor-core BF16 GEMMs
        Vm = vr.reshape(n, -1)
        for j in range(k):
            ref = deflation_guess(vr, lam + 4 * m * m, bs[j])
            assert rel(H.hisq_deflate(ctx, bs[j]), ref) <= 1e-5  # CUDA-core path
            assert rel(x[j], ref) <= 1e-4, (j, rel(x[j], ref))
            rref = bs[j] - (Vm.T @ (Vm.conj() @ bs[j].reshape(-1))).reshape(bs[j].shape)
            assert rel(r[j], rref) <= 1e-4, (j, rel(r[j], rref))
    finally:
        ctx.close()


def test_bf16_batched_deflated_solve_meets_tolerance():
    dims = (6, 6, 6, 8)
    m = 0.01
    ctx, o, lam, vecs, vr = _setup(dims, 48, m)
    try:
        etas = np.stack([I.gaussian_source(dims, 9, j) for j in range(6)])
        prm = H.hisq_default_solve_params(batch=1, deflate=1, precision_sloppy=16)
        psi, st, status = H.hisq_solve(ctx, etas, prm)
        assert status == H.HISQ_OK
        for j in range(6):
            assert o.full_residual(m, psi[j], etas[j]) <= 1e-10
        # single right-hand side (CUDA-core deflation, exact FP64 residual after each step)
        psi1, st1, status1 = H.hisq_solve(ctx, etas[0], H.hisq_default_solve_params(deflate=1))
        assert status1 == H.HISQ_OK and o.full_residual(m, psi1, etas[0]) <= 1e-10
    finally:
        ctx.close()


def test_bf16_eigensolve_storage():
    dims = (6, 6, 6, 6)
    m = 0.01
    ctx, o = make(dims, seed=21, eps=0.3, mass=m)
    try:
        eps, nconv = H.hisq_eigensolve(ctx, H.hisq_default_eig_params(n_ev=16, n_kr=48, tol=1e-8, max_restarts=200,
                                                                     storage_precision=H.HISQ_PREC_BF16))
        lam = o.eig_dense(0.0, 20)[0]
        assert nconv == 16
        assert np.allclose(eps, lam[:16], rtol=1e-8, atol=0)
        for i in (0, 7, 15):
            v = H.hisq_get_eigvec(ctx, i)
            assert np.array_equal(v, bf16_round(v))  # representable in BF16
            assert abs(np.linalg.norm(v) - 1.0) <= 4e-3
    finally:
        ctx.close()
