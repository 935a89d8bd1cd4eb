"""GPU propagator solves against the FP64 oracle (Sections 2 and 3).

Bar: the full-system true residual |eta - M psi| / |eta| computed by the
oracle's FP64 operator on the downloaded psi is <= the tolerance (1e-10), and
psi agrees with the oracle's own solution within the conditioning bound."""
import numpy as np
import pytest
import torch

from gpu_common import make, rel
from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _kappa_bound(m, lam_max=30.0):
    # |psi - psi*| / |psi*| <= kappa * residual with kappa <= lam_max / (4 m^2)
    return lam_max / (4 * m * m)


@pytest.mark.parametrize("prec,lprec", [(64, 64), (32, 32), (16, 32), (16, 16)])
def test_c1_solve_matches_oracle(prec, lprec):
    """8^4, m = 0.05, point source: plain even-odd CG (FP64) and the
    mixed-precision variants with FP64 reliable updates."""
    c = I.lattice_config("c1")
    dims, m, tol = c["dims"], c["mass"], c["tol"]
    ctx, o = make(dims, seed=c["seed"], eps=c["eps"], mass=m)
    try:
        eta = I.point_source(dims, 0)
        prm = H.hisq_default_solve_params(tol=tol, precision_sloppy=prec, link_precision_sloppy=lprec)
        psi, st, status = H.hisq_solve(ctx, eta, prm)
        assert status == H.HISQ_OK and st[0]["converged"] == 1
        res = o.full_residual(m, psi, eta)
        assert res <= tol
        assert abs(st[0]["full_residual"] - res) <= 0.1 * res + 1e-15
        ref, ost = o.solve(m, eta, tol)
        assert rel(psi, ref) <= 2 * tol * _kappa_bound(m)
        if prec == 64:
            # FP64 CG takes about as many iterations as the oracle's CG
            assert abs(st[0]["iterations"] - ost["iterations"]) <= 3
        else:
            assert st[0]["reliable_updates"] >= 1
    finally:
        ctx.close()


def test_multi_rhs_host_and_device_paths():
    dims = (6, 6, 6, 8)
    m = 0.03
    ctx, o = make(dims, seed=9, eps=0.4, mass=m)
    try:
        etas = np.stack([I.gaussian_source(dims, 3, k) for k in range(3)])
        prm = H.hisq_default_solve_params(tol=1e-10, precision_sloppy=32)
        psi, st, status = H.hisq_solve(ctx, etas, prm)
        assert status == H.HISQ_OK
        for k in range(3):
            assert o.full_residual(m, psi[k], etas[k]) <= 1e-10
        # device pointers (torch tensors) give the same result
        e_dev = torch.from_numpy(etas).cuda()
        p_dev = torch.zeros_like(e_dev)
        st2, status2 = H.hisq_solve_device(ctx, e_dev, p_dev, 3, prm)
        torch.cuda.synchronize()
        assert status2 == H.HISQ_OK
        assert np.array_equal(p_dev.cpu().numpy(), psi)  # deterministic reductions
    finally:
        ctx.close()


def test_z2_wall_source_and_recon12():
    dims = (6, 6, 6, 8)
    m = 0.02
    ctx, o = make(dims, seed=5, eps=0.3, mass=m, recon=12)
    try:
        eta = I.z2_wall_source(dims, 7, 3, 1)
        for lp in (32, 16):
            psi, st, status = H.hisq_solve(ctx, eta, H.hisq_default_solve_params(precision_sloppy=16,
                                                                                link_precision_sloppy=lp))
            assert status == H.HISQ_OK
            assert o.full_residual(m, psi, eta) <= 1e-10
    finally:
        ctx.close()


def test_recon8_solves_single_and_batched():
    dims = (6, 6, 6, 8)
    m = 0.02
    ctx, o = make(dims, seed=5, eps=0.3, mass=m, recon=8)
    try:
        etas = np.stack([I.z2_wall_source(dims, 7, 3, c) for c in range(3)])
        psi, st, status = H.hisq_solve(ctx, etas[0], H.hisq_default_solve_params(precision_sloppy=16))
        assert status == H.HISQ_OK and o.full_residual(m, psi, etas[0]) <= 1e-10
        psi, st, status = H.hisq_solve(ctx, etas, H.hisq_default_solve_params(precision_sloppy=16, batch=1))
        assert status == H.HISQ_OK
        for j in range(3):
            assert o.full_residual(m, psi[j], etas[j]) <= 1e-10
    finally:
        ctx.close()


def test_zero_source():
    dims = (4, 4, 4, 4)
    ctx, o = make(dims, mass=0.1)
    try:
        psi, st, status = H.hisq_solve(ctx, np.zeros((I.volume(dims), 3), np.complex128))
        assert status == H.HISQ_OK and np.all(psi == 0)
    finally:
        ctx.close()


def test_not_converged_returns_best_iterate():
    dims = (6, 6, 6, 8)
    m = 0.01
    ctx, o = make(dims, seed=2, eps=0.4, mass=m)
    try:
        eta = I.gaussian_source(dims, 1, 0)
        prm = H.hisq_default_solve_params(tol=1e-12, max_iter=20)
        psi, st, status = H.hisq_solve(ctx, eta, prm)
        assert status == H.HISQ_ERR_NOT_CONVERGED and st[0]["converged"] == 0
        assert st[0]["iterations"] == 20
        r = o.full_residual(m, psi, eta)
        assert np.isfinite(r) and r < 1.0
        assert abs(st[0]["full_residual"] - r) <= 1e-6 * r
    finally:
        ctx.close()


def test_state_errors():
    dims = (4, 4, 4, 4)
    ctx = H.hisq_create(dims)
    try:
        eta = I.point_source(dims)
        with pytest.raises(H.HisqError) as e:
            H.hisq_solve(ctx, eta)
        assert e.value.status == H.HISQ_ERR_STATE
        with pytest.raises(H.HisqError) as e:
            H.hisq_set_mass(ctx, -1.0)
        assert e.value.status == H.HISQ_ERR_INVALID_ARG
    finally:
        ctx.close()


def test_full_size_solve_true_residual():
    """32^3 x 64 (the benchmark lattice), m = 0.002, Gaussian source, FP32/FP16
    mixed precision: the oracle's FP64 operator confirms |eta - M psi|/|eta| <= 1e-10."""
    c = I.lattice_config("c2")
    dims, m = c["dims"], c["mass"]
    ctx, o = make(dims, seed=c["seed"], eps=c["eps"], mass=m)
    try:
        eta = I.gaussian_source(dims, 11, 0)
        for prec, lp in ((32, 32), (16, 32)):
            psi, st, status = H.hisq_solve(ctx, eta, H.hisq_default_solve_params(precision_sloppy=prec,
                                                                                 link_precision_sloppy=lp))
            assert status == H.HISQ_OK
            assert o.full_residual(m, psi, eta) <= 1e-10
    finally:
        ctx.close()


def test_fp16_links_stagnation_is_reported():
    """FP16 link storage perturbs the operator by ~5e-4 * lambda_max, more than
    the smallest eigenvalue of the light-mass 32^3x64 workload; the solve must
    then stop with HISQ_ERR_NOT_CONVERGED (stagnation), not run to max_iter."""
    c = I.lattice_config("c2")
    dims, m = c["dims"], c["mass"]
    ctx, o = make(dims, seed=c["seed"], eps=c["eps"], mass=m)
    try:
        eta = I.gaussian_source(dims, 11, 0)
        prm = H.hisq_default_solve_params(precision_sloppy=16, link_precision_sloppy=16, max_iter=20000)
        psi, st, status = H.hisq_solve(ctx, eta, prm)
        if status == H.HISQ_OK:
            assert o.full_residual(m, psi, eta) <= 1e-10
        else:
            assert status == H.HISQ_ERR_NOT_CONVERGED
            assert st[0]["iterations"] < 20000
            assert "stagnation" in H.hisq_last_error(ctx)
    finally:
        ctx.close()


def test_injected_allocation_failure_is_reported_and_recovered():
    """Host-side fault injection: allocations refused mid-solve give
    HISQ_ERR_OOM with a message; with the injection off the same context
    solves to the tolerance."""
    dims = (6, 6, 6, 8)
    ctx, o = make(dims, seed=5, eps=0.3, mass=0.05)
    try:
        eta = I.gaussian_source(dims, 3, 0)
        H.hisq_inject_alloc_failure(ctx, 0)
        with pytest.raises(H.HisqError) as ei:
            H.hisq_solve(ctx, eta, H.hisq_default_solve_params())
        assert "injected" in str(ei.value)
        H.hisq_inject_alloc_failure(ctx, 2)  # fails part-way through buffer set-up
        with pytest.raises(H.HisqError):
            H.hisq_solve(ctx, eta, H.hisq_default_solve_params())
        H.hisq_inject_alloc_failure(ctx, -1)
        psi, st, status = H.hisq_solve(ctx, eta, H.hisq_default_solve_params())
        assert status == H.HISQ_OK and o.full_residual(0.05, psi, eta) <= 1e-10
    finally:
        ctx.close()
