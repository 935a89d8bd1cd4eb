"""Batched multi right-hand-side solves (the paper's outlook, Section 4):
several right-hand sides through one batched operator per CG iteration, each
with its own CG, FP64 reliable updates and re-deflations.  Every solution is
checked with the FP64 oracle operator: |eta - M psi| / |eta| <= 1e-10."""
import numpy as np
import pytest

from gpu_common import make, rel
from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("k,prec", [(2, 32), (5, 16), (9, 32)])
def test_batched_matches_oracle_residual(k, prec):
    dims = (6, 6, 6, 8)
    m = 0.02
    ctx, o = make(dims, seed=13, eps=0.4, mass=m)
    try:
        etas = np.stack([I.gaussian_source(dims, 21, j) for j in range(k)])
        prm = H.hisq_default_solve_params(precision_sloppy=prec, batch=1)
        psi, st, status = H.hisq_solve(ctx, etas, prm)
        assert status == H.HISQ_OK
        for j in range(k):
            assert st[j]["converged"] == 1
            res = o.full_residual(m, psi[j], etas[j])
            assert res <= 1e-10
            assert abs(st[j]["full_residual"] - res) <= 0.1 * res + 1e-15
        # the batched and the one-by-one solver reach the same solutions
        psi1, st1, s1 = H.hisq_solve(ctx, etas, H.hisq_default_solve_params(precision_sloppy=prec, batch=0))
        assert s1 == H.HISQ_OK
        for j in range(k):
            assert rel(psi[j], psi1[j]) <= 1e-6
            assert abs(st[j]["iterations"] - st1[j]["iterations"]) <= 0.1 * st1[j]["iterations"] + 5
    finally:
        ctx.close()


def test_batched_masking_with_mixed_difficulty():
    """Right-hand sides of very different difficulty (a zero source, a point
    source, Gaussian sources) leave the batch at different iterations."""
    dims = (6, 6, 6, 8)
    m = 0.01
    ctx, o = make(dims, seed=3, eps=0.4, mass=m)
    try:
        V = I.volume(dims)
        etas = np.stack([np.zeros((V, 3), np.complex128), I.point_source(dims, 1), I.gaussian_source(dims, 4, 0),
                         I.z2_wall_source(dims, 5, 2, 0), I.gaussian_source(dims, 4, 1)])
        psi, st, status = H.hisq_solve(ctx, etas, H.hisq_default_solve_params(batch=1))
        assert status == H.HISQ_OK
        assert np.all(psi[0] == 0) and st[0]["iterations"] == 0
        for j in range(1, 5):
            assert o.full_residual(m, psi[j], etas[j]) <= 1e-10
        assert len({s["iterations"] for s in st[1:]}) > 1
    finally:
        ctx.close()


def test_batched_deflated_with_redeflation():
    dims = (6, 6, 6, 6)
    m = 0.01
    ctx, o = make(dims, seed=21, eps=0.3, mass=m)
    try:
        lam, vecs = o.eig_dense(0.0, 32)
        H.hisq_set_eigvecs(ctx, vecs, lam, 16)
        etas = np.stack([I.gaussian_source(dims, 8, j) for j in range(4)])
        psi, st, status = H.hisq_solve(ctx, etas, H.hisq_default_solve_params(batch=1, deflate=1, precision_sloppy=16))
        assert status == H.HISQ_OK
        for j in range(4):
            assert o.full_residual(m, psi[j], etas[j]) <= 1e-10
            assert st[j]["redeflations"] >= 1
    finally:
        ctx.close()


def test_batched_full_size_z2_walls():
    """24 Z2 wall sources (8 timeslices x 3 colours) on the 32^3x64 lattice,
    one batched solve, plain and deflated (64 eigenpairs from the library's
    block thick-restart Lanczos, BF16 storage as in the batched benchmark, so the
    tensor-core deflation with its re-deflations runs at full size); every
    solution meets 1e-10 under the oracle operator, and deflation removes
    iterations from every right-hand side (a wrong deflation would still
    converge, but only with more iterations)."""
    c = I.lattice_config("c3")
    dims, m = c["dims"], c["mass"]
    ctx, o = make(dims, seed=c["seed"], eps=c["eps"], mass=m)
    try:
        etas = np.stack([I.z2_wall_source(dims, 7, s, col) for s in range(8) for col in range(3)])
        psi, st, status = H.hisq_solve(ctx, etas, H.hisq_default_solve_params(batch=1, precision_sloppy=16))
        assert status == H.HISQ_OK
        for j in (0, 7, 13, 23):
            assert o.full_residual(m, psi[j], etas[j]) <= 1e-10
        plain_it = [s["iterations"] for s in st]
        eps, nconv = H.hisq_eigensolve(ctx, H.hisq_default_eig_params(
            n_ev=64, n_kr=192, tol=1e-6, max_restarts=100, cheby_degree=60, a_min=-2.0,
            storage_precision=H.HISQ_PREC_BF16, seed=5, block_size=32))
        assert nconv == 64
        psi, st, status = H.hisq_solve(ctx, etas, H.hisq_default_solve_params(batch=1, deflate=1,
                                                                             precision_sloppy=16))
        assert status == H.HISQ_OK
        for j in (0, 5, 11, 16, 23):
            assert o.full_residual(m, psi[j], etas[j]) <= 1e-10
        for j in range(24):
            assert st[j]["iterations"] <= 0.9 * plain_it[j], (j, st[j]["iterations"], plain_it[j])
    finally:
        ctx.close()


def test_host_solve_into_caller_buffer():
    """hisq_solve writes into a caller-provided (e.g. pinned) output array: the
    same solutions as with an array of its own."""
    import torch

    dims = (6, 6, 6, 8)
    m = 0.01
    ctx, o = make(dims, seed=21, eps=0.3, mass=m)
    try:
        etas = np.stack([I.gaussian_source(dims, 5, j) for j in range(3)])
        prm = H.hisq_default_solve_params(batch=1, precision_sloppy=16)
        psi, _, status = H.hisq_solve(ctx, etas, prm)
        out = torch.full((3, I.volume(dims), 3), complex(np.nan, np.nan), dtype=torch.complex128).pin_memory()
        psi2, _, status2 = H.hisq_solve(ctx, etas, prm, out=out.numpy())
        assert status == status2 == H.HISQ_OK
        assert np.array_equal(psi, out.numpy()) and np.shares_memory(psi2, out.numpy())
        for j in range(3):
            assert o.full_residual(m, out.numpy()[j], etas[j]) <= 1e-10
    finally:
        ctx.close()


def test_fp64_operator_profiling():
    """hisq_profiled_fp64 counts and times the FP64 Dslash launches made while
    profiling is on: at least two per reliable update of every right-hand side
    and one for each one's source preparation; switching profiling on again
    restarts the sums, and nothing is counted while it is off."""
    dims = (6, 6, 6, 8)
    m = 0.01
    ctx, o = make(dims, seed=21, eps=0.3, mass=m)
    try:
        etas = np.stack([I.gaussian_source(dims, 6, j) for j in range(3)])
        prm = H.hisq_default_solve_params(batch=1, precision_sloppy=16)
        H.hisq_set_profiling(ctx, True)
        psi, st, status = H.hisq_solve(ctx, etas, prm)
        H.hisq_set_profiling(ctx, False)
        assert status == H.HISQ_OK
        sec, n = H.hisq_profiled_fp64(ctx)
        assert n >= 2 * sum(s["reliable_updates"] for s in st) + len(st), (n, st)
        assert 0 < sec < sum(s["seconds_total"] for s in st) + 1.0
        H.hisq_solve(ctx, etas, prm)  # profiling off: the sums stay
        assert H.hisq_profiled_fp64(ctx) == (sec, n)
        H.hisq_set_profiling(ctx, True)
        assert H.hisq_profiled_fp64(ctx) == (0.0, 0)
        H.hisq_set_profiling(ctx, False)
        for j in range(3):
            assert o.full_residual(m, psi[j], etas[j]) <= 1e-10
    finally:
        ctx.close()
