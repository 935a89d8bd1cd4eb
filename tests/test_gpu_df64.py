"""Double-float (HISQ_PREC_DF64) reliable-update residuals against the FP64 oracle.

The operator: every real is the sum hi + lo of two FP32 numbers; a product of
two such numbers carries a relative error of at most about 5 * 2^-48 (split
errors of both factors, the dropped lo*lo term, the rounding of the low part),
and each output component sums 96 terms whose two-sum errors are collected in
FP32, so |D_df x - D x| <= about (5 + 96) * 2^-48 * sum |terms| ~ 4e-13 of the
sum of term magnitudes; with the cancellation of a Gaussian field the relative
error bound is taken as 2e-12 (FP64: 1e-13 in the Dslash parity tests, FP32:
1e-6).  The solves: the oracle's FP64 operator confirms |eta - M psi| / |eta|
<= 1e-10 on the downloaded psi, as for FP64 reliable updates (Section 3)."""
import numpy as np
import pytest

from gpu_common import dslash_ref, make, rel
from oracle.oracle import project_parity
from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DF = H.HISQ_PREC_DF64
TOL_DF = 2e-12

# the Naik-distinct minimum, L = 4 (x+3 == x-1 aliasing), ragged half-volumes
# below one 256-thread block, and several blocks
LATTICES = [(6, 6, 6, 6), (4, 4, 4, 4), (4, 6, 4, 10), (8, 8, 8, 12)]


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("antip", [True, False])
def test_df64_dslash_matches_oracle(dims, antip):
    ctx, o = make(dims, antip=antip)
    try:
        src = I.gaussian_field(dims, 23)
        for par in (0, 1):
            ref = dslash_ref(o, dims, src, par)
            out = H.hisq_apply_dslash(ctx, par, DF, src)
            e_df = rel(out, ref)
            assert e_df <= TOL_DF, (par, e_df)
            assert np.all(project_parity(dims, out, 1 - par) == 0)
            # far below the FP32 operator's error: the low parts are used
            e32 = rel(H.hisq_apply_dslash(ctx, par, 32, src), ref)
            assert e_df <= 1e-4 * e32, (e_df, e32)
    finally:
        ctx.close()


@pytest.mark.parametrize("recon", [18, 12])
def test_df64_normal_op_matches_oracle(recon):
    """(M^dag M)_ee = 4m^2 - D_eo D_oe (Eq. 1); the double-float operator always
    uses all 18 reals of the FP64 links, whatever the sloppy long-link format."""
    dims, m = (6, 6, 6, 8), 0.02
    ctx, o = make(dims, recon=recon, mass=m)
    try:
        x = project_parity(dims, I.gaussian_field(dims, 31), 0)
        ref = project_parity(dims, o.apply_Aee(m, x), 0)
        out = H.hisq_apply_normal_op(ctx, DF, x)
        assert rel(out, ref) <= TOL_DF
        assert np.all(project_parity(dims, out, 1) == 0)
    finally:
        ctx.close()


def test_df64_precision_arguments_are_checked():
    dims = (4, 4, 4, 4)
    ctx, o = make(dims, mass=0.1)
    try:
        src = I.gaussian_field(dims, 1)
        for vp, lp in ((DF, 32), (32, DF), (64, DF), (DF, 64)):
            with pytest.raises(H.HisqError):
                H.hisq_apply_dslash(ctx, 0, vp, src, link_precision=lp)
        with pytest.raises(H.HisqError):
            H.hisq_solve(ctx, src, H.hisq_default_solve_params(precision_reliable=32))
    finally:
        ctx.close()


@pytest.mark.parametrize("prec,lprec", [(32, 32), (16, 32), (64, 64)])
def test_df64_reliable_updates_solve(prec, lprec):
    """Same tolerance as FP64 reliable updates; about the same iteration count."""
    c = I.lattice_config("c1")
    dims, m, tol = c["dims"], c["mass"], c["tol"]
    ctx, o = make(dims, seed=c["seed"], eps=c["eps"], mass=m)
    try:
        eta = I.gaussian_source(dims, 5, 0)
        its = {}
        for rp in (64, DF):
            prm = H.hisq_default_solve_params(tol=tol, precision_sloppy=prec, link_precision_sloppy=lprec,
                                              precision_reliable=rp)
            psi, st, status = H.hisq_solve(ctx, eta, prm)
            assert status == H.HISQ_OK and st[0]["converged"] == 1
            assert o.full_residual(m, psi, eta) <= tol
            its[rp] = st[0]["iterations"]
        assert abs(its[DF] - its[64]) <= max(3, 0.05 * its[64]), its
    finally:
        ctx.close()


@pytest.mark.parametrize("eig_prec", [32, H.HISQ_PREC_BF16])
def test_df64_deflated_batched_and_single(eig_prec):
    """Deflation with re-deflation, batched (tensor-core deflation) and single
    right-hand-side paths, FP32 and BF16 eigenvectors."""
    dims, m = (6, 6, 6, 8), 0.01
    ctx, o = make(dims, seed=21, eps=0.3, mass=m)
    try:
        lam, vecs = o.eig_dense(0.0, 48)
        H.hisq_set_eigvecs(ctx, vecs, lam, eig_prec)
        etas = np.stack([I.gaussian_source(dims, 9, j) for j in range(6)])
        for batch in (1, 0):
            prm = H.hisq_default_solve_params(batch=batch, deflate=1, precision_sloppy=16, precision_reliable=DF)
            psi, st, status = H.hisq_solve(ctx, etas, prm)
            assert status == H.HISQ_OK
            for j in range(6):
                assert st[j]["converged"] == 1
                assert o.full_residual(m, psi[j], etas[j]) <= 1e-10
    finally:
        ctx.close()


def test_df64_full_size_solve_true_residual():
    """32^3 x 64, m = 0.002: the double-float reliable updates reach the same
    FP64-confirmed residual as the FP64 ones, in about as many iterations."""
    c = I.lattice_config("c2")
    dims, m = c["dims"], c["mass"]
    ctx, o = make(dims, seed=c["seed"], eps=c["eps"], mass=m)
    try:
        eta = I.gaussian_source(dims, 11, 0)
        psi, st, status = H.hisq_solve(ctx, eta, H.hisq_default_solve_params(precision_sloppy=16,
                                                                             precision_reliable=DF))
        assert status == H.HISQ_OK
        assert o.full_residual(m, psi, eta) <= 1e-10
        assert st[0]["reliable_updates"] >= 5
    finally:
        ctx.close()


@pytest.mark.parametrize("nrhs", [2, 3, 6, 9])
def test_df64_batched_residuals_match_oracle(nrhs):
    """A batched solve stopped by max_iter takes one reliable update of every
    right-hand side in the same round: the double-float residuals of the whole
    group come from one batched launch pair (1, 2, 3 or 4 fields per thread and
    ragged warps).  The reported even residual |y_e - A psi_e| / |y_e| matches
    the oracle's FP64 residual of the returned psi_e."""
    dims, m = (6, 6, 6, 8), 0.02
    ctx, o = make(dims, seed=5, eps=0.3, mass=m)
    try:
        etas = np.stack([I.gaussian_source(dims, 13, j) for j in range(nrhs)])
        for rp in (64, DF):
            prm = H.hisq_default_solve_params(batch=1, max_iter=3, tol=1e-14, precision_sloppy=32,
                                              precision_reliable=rp, compute_full_residual=0)
            psi, st, status = H.hisq_solve(ctx, etas, prm)
            assert status == H.HISQ_ERR_NOT_CONVERGED
            for j in range(nrhs):
                y = project_parity(dims, o.prepare_source(m, etas[j]), 0)
                ref = o.even_residual(m, project_parity(dims, psi[j], 0), y)
                assert abs(st[j]["even_residual"] - ref) <= 1e-9 * ref, (rp, j, st[j]["even_residual"], ref)
    finally:
        ctx.close()


def test_df64_link_allocation_failure_leaves_no_half_built_state():
    """The double-float links are built on first use.  Refused allocations
    (host-side injection) of the first parity, then of the second, give
    HISQ_ERR_OOM and keep neither; the next call builds both and applies the
    operator to the parity tolerance."""
    dims = (6, 6, 6, 6)
    ctx, o = make(dims)
    try:
        src = I.gaussian_field(dims, 23)
        ref = dslash_ref(o, dims, src, 0)
        assert rel(H.hisq_apply_dslash(ctx, 0, 64, src), ref) <= 1e-13  # scratch fields exist from here
        # 1st: the double-float scratch field is allocated, the first link parity refused
        # 2nd: the scratch field exists, the first parity is allocated, the second refused
        for _ in range(2):
            H.hisq_inject_alloc_failure(ctx, 1)
            with pytest.raises(H.HisqError):
                H.hisq_apply_dslash(ctx, 0, DF, src)
        H.hisq_inject_alloc_failure(ctx, -1)
        assert rel(H.hisq_apply_dslash(ctx, 0, DF, src), ref) <= TOL_DF
        assert rel(H.hisq_apply_dslash(ctx, 1, DF, src), dslash_ref(o, dims, src, 1)) <= TOL_DF
    finally:
        ctx.close()
