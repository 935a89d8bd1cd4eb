"""The persistent form of the batched CG (one cooperative launch per stretch of
sloppy iterations between host interventions, grid-wide phases separated by
bounded barriers) against the FP64 oracle: every solution meets the 1e-10 true
residual under the oracle's operator, with and without deflation, FP16 and
FP32 sloppy vectors, 12- and 18-real long links; iteration counts agree with
the launch-per-phase form (both hand a right-hand side to the host two
iterations after it reaches a reliable-update threshold).  The bounded
barrier's timeout path is taken on purpose with a zero time limit (host-set,
one-shot): the solve reports HISQ_ERR_TIMEOUT and the same context then solves
normally."""
import numpy as np
import pytest

from gpu_common import make, orthonormal_even_set
from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 16)  # Vh = 4096: 128 site groups, several per block


@pytest.mark.parametrize("recon,sloppy,deflate", [(12, 16, 0), (12, 16, 1), (18, 32, 0), (12, 32, 1)])
def test_persistent_batched_solve(recon, sloppy, deflate):
    m = 0.01
    ctx, o = make(DIMS, seed=13, eps=0.3, recon=recon, mass=m)
    try:
        if deflate:
            lam, vecs = orthonormal_even_set(DIMS, 24, seed=3)
            # Rayleigh quotients recomputed by the library (eps = None): the
            # guess is then a projection onto an arbitrary subspace, which CG
            # corrects; only the solution is checked
            H.hisq_set_eigvecs(ctx, vecs, None, H.HISQ_PREC_HALF_EV)
        etas = np.stack([I.gaussian_source(DIMS, 21, j) for j in range(7)])
        etas[3] = 0  # a zero right-hand side is done before the first iteration
        runs = {}
        for persistent in (0, 1):
            prm = H.hisq_default_solve_params(batch=1, deflate=deflate, precision_sloppy=sloppy,
                                              persistent=persistent)
            psi, st, status = H.hisq_solve(ctx, etas, prm)
            assert status == H.HISQ_OK
            for j in range(7):
                if j == 3:
                    assert np.all(psi[j] == 0)
                    continue
                assert o.full_residual(m, psi[j], etas[j]) <= 1e-10, (persistent, j)
            runs[persistent] = [s["iterations"] for s in st]
        for j in range(7):
            a, b = runs[0][j], runs[1][j]
            assert abs(a - b) <= max(4, 0.05 * a), (j, a, b)
    finally:
        ctx.close()


def test_persistent_barrier_timeout_is_reported_and_recovered():
    m = 0.01
    ctx, o = make(DIMS, seed=13, eps=0.3, recon=12, mass=m)
    try:
        etas = np.stack([I.gaussian_source(DIMS, 22, j) for j in range(4)])
        prm = H.hisq_default_solve_params(batch=1, precision_sloppy=16, persistent=1)
        H.hisq_inject_wait_timeout(ctx, True)
        with pytest.raises(H.HisqError) as e:
            H.hisq_solve(ctx, etas, prm)
        assert e.value.status == H.HISQ_ERR_TIMEOUT
        assert "grid barrier ran out" in str(e.value)
        psi, st, status = H.hisq_solve(ctx, etas, prm)  # the injection was one-shot
        assert status == H.HISQ_OK
        for j in range(4):
            assert o.full_residual(m, psi[j], etas[j]) <= 1e-10
    finally:
        ctx.close()


def test_persistent_full_size():
    """32^3 x 64 (Vh = 1,048,576: every block of the cooperative grid walks many
    site groups), the batched benchmark's lattice and mass, 12 Gaussian
    right-hand sides with FP16 sloppy vectors, 12-real links and FP64 reliable
    updates: every solution of the persistent form meets 1e-10 under the
    oracle's operator, with iteration counts within a few of the
    launch-per-phase form's."""
    c = I.lattice_config("c2")
    dims, m = c["dims"], c["mass"]
    ctx, o = make(dims, seed=c["seed"], eps=c["eps"], recon=12, mass=m)
    try:
        etas = np.stack([I.gaussian_source(dims, 23, j) for j in range(12)])
        runs = {}
        for persistent in (0, 1):
            prm = H.hisq_default_solve_params(batch=1, precision_sloppy=16, persistent=persistent)
            psi, st, status = H.hisq_solve(ctx, etas, prm)
            assert status == H.HISQ_OK
            for j in range(12):
                assert o.full_residual(m, psi[j], etas[j]) <= 1e-10, (persistent, j)
            runs[persistent] = [s["iterations"] for s in st]
        for j in range(12):
            a, b = runs[0][j], runs[1][j]
            assert abs(a - b) <= max(4, 0.02 * a), (j, a, b)
    finally:
        ctx.close()
