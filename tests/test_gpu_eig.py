"""GPU thick-restart Lanczos and deflation against the FP64 oracle (Section 2:
eigenvectors of the squared massless operator; Eq. 3 mass shift; Eq. 4
deflated guess; Section 3: re-deflation with single-precision eigenvectors).
Eigenvalues agree with dense diagonalisation to 1e-8 relative."""
import numpy as np
import pytest

from gpu_common import make, rel
from oracle.oracle import deflation_guess, project_parity
from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lat():
    dims = (6, 6, 6, 6)
    m = 0.01
    ctx, o = make(dims, seed=21, eps=0.3, mass=m)
    w, vecs = o.eig_dense(0.0, 40)
    yield dims, m, ctx, o, w, vecs
    ctx.close()


def _clusters_ok(w, n):
    """indices i < n whose eigenvalue is not degenerate with the cut at n"""
    gap = 1e-9 * w[n - 1]
    return [i for i in range(n) if abs(w[i] - w[n]) > gap]


@pytest.mark.parametrize("cheby", [0, 12])
def test_trlm_eigenvalues_match_dense(lat, cheby):
    dims, m, ctx, o, w, vecs = lat
    n_ev = 16
    prm = H.hisq_default_eig_params(n_ev=n_ev, n_kr=48, tol=1e-6, max_restarts=300, cheby_degree=cheby,
                                    a_min=float(w[30]) if cheby else 0.0, a_max=0.0, seed=7)
    eps, nconv = H.hisq_eigensolve(ctx, prm)
    assert nconv == n_ev
    ok = _clusters_ok(w, n_ev)
    assert np.max(np.abs(eps[ok] - w[ok]) / w[ok]) <= 1e-8
    # each stored vector is an eigenvector of the oracle's operator
    for i in range(n_ev):
        v = H.hisq_get_eigvec(ctx, i)
        th, res = o.rayleigh(0.0, v)
        assert abs(th - eps[i]) <= 1e-8 * eps[i]
        assert res <= 1e-4 * w[-1]
        assert np.all(project_parity(dims, v, 1) == 0)


@pytest.mark.parametrize("block,cheby", [(4, 0), (8, 12), (16, 12)])
def test_block_trlm_eigenvalues_match_dense(lat, block, cheby):
    """Block thick-restart Lanczos (the operator applied to `block` fields at a
    time with the batched Dslash): same eigenpairs as dense diagonalisation."""
    dims, m, ctx, o, w, vecs = lat
    n_ev = 16
    prm = H.hisq_default_eig_params(n_ev=n_ev, n_kr=64, tol=1e-6, max_restarts=300, cheby_degree=cheby,
                                    a_min=float(w[30]) if cheby else 0.0, a_max=0.0, seed=11, block_size=block)
    eps, nconv = H.hisq_eigensolve(ctx, prm)
    assert nconv == n_ev
    ok = _clusters_ok(w, n_ev)
    assert np.max(np.abs(eps[ok] - w[ok]) / w[ok]) <= 1e-8
    for i in range(n_ev):
        v = H.hisq_get_eigvec(ctx, i)
        th, res = o.rayleigh(0.0, v)
        assert abs(th - eps[i]) <= 1e-8 * eps[i]
        assert res <= 1e-4 * w[-1]
        assert np.all(project_parity(dims, v, 1) == 0)


def test_block_size_adapts_to_small_basis(lat):
    """The block shrinks to (n_kr - n_ev) / 2 when the Krylov space is small,
    and a space with no room for two blocks is refused."""
    dims, m, ctx, o, w, vecs = lat
    eps, nconv = H.hisq_eigensolve(ctx, H.hisq_default_eig_params(n_ev=8, n_kr=20, block_size=16, tol=1e-6,
                                                                  max_restarts=500, cheby_degree=12,
                                                                  a_min=float(w[30]), seed=3))
    ok = _clusters_ok(w, 8)
    assert nconv == 8 and np.max(np.abs(eps[ok] - w[ok]) / w[ok]) <= 1e-8
    with pytest.raises(H.HisqError):
        H.hisq_eigensolve(ctx, H.hisq_default_eig_params(n_ev=8, n_kr=11, block_size=8))


def test_mass_shift_of_stored_eigenvalues(lat):
    """lambda_i = eps_i + 4 m^2 (Eq. 3): deflating with the stored pairs equals
    the oracle's deflation with the dense eigenvectors of A_ee(m)."""
    dims, m, ctx, o, w, vecs = lat
    n = 24
    H.hisq_set_eigvecs(ctx, vecs[:n], None, 32)
    eps = H.hisq_get_eigvals(ctx)
    assert np.max(np.abs(eps - w[:n]) / w[:n]) <= 1e-8  # FP64 Rayleigh quotients on load
    b = project_parity(dims, I.gaussian_field(dims, 4), 0)
    x = H.hisq_deflate(ctx, b)
    ref = deflation_guess(vecs[:n], w[:n] + 4 * m * m, b)
    assert rel(x, ref) <= 1e-5  # FP32 storage and accumulation


def test_fp16_eigvecs_deflate(lat):
    dims, m, ctx, o, w, vecs = lat
    n = 24
    H.hisq_set_eigvecs(ctx, vecs[:n], w[:n], 16)
    b = project_parity(dims, I.gaussian_field(dims, 6), 0)
    x = H.hisq_deflate(ctx, b)
    ref = deflation_guess(vecs[:n], w[:n] + 4 * m * m, b)
    assert rel(x, ref) <= 5e-3


@pytest.mark.parametrize("vprec,sloppy,lprec", [(32, 32, 32), (16, 16, 16), (32, 64, 64), (32, 16, 32)])
def test_deflated_solve_and_redeflation(lat, vprec, sloppy, lprec):
    dims, m, ctx, o, w, vecs = lat
    n = 32
    H.hisq_set_eigvecs(ctx, vecs[:n], w[:n], vprec)
    eta = I.gaussian_source(dims, 8, 0)
    kw = dict(precision_sloppy=sloppy, link_precision_sloppy=lprec)
    plain, st0, s0 = H.hisq_solve(ctx, eta, H.hisq_default_solve_params(**kw))
    defl, st1, s1 = H.hisq_solve(ctx, eta, H.hisq_default_solve_params(deflate=1, **kw))
    assert s0 == H.HISQ_OK and s1 == H.HISQ_OK
    assert o.full_residual(m, plain, eta) <= 1e-10
    assert o.full_residual(m, defl, eta) <= 1e-10
    assert st1[0]["iterations"] < st0[0]["iterations"]
    assert st1[0]["redeflations"] >= 1
    assert st1[0]["seconds_deflate"] > 0


def test_save_load_roundtrip(lat, tmp_path):
    dims, m, ctx, o, w, vecs = lat
    H.hisq_set_eigvecs(ctx, vecs[:8], None, 32)
    before = [H.hisq_get_eigvec(ctx, i) for i in range(8)]
    eps0 = H.hisq_get_eigvals(ctx)
    path = str(tmp_path / "ev.bin")
    H.hisq_save_eigvecs(ctx, path)
    H.hisq_set_eigvecs(ctx, vecs[8:10], None, 32)
    H.hisq_load_eigvecs(ctx, path)
    assert np.array_equal(H.hisq_get_eigvals(ctx), eps0)
    for i in range(8):
        assert np.array_equal(H.hisq_get_eigvec(ctx, i), before[i])
    # a corrupted file is rejected
    raw = bytearray(open(path, "rb").read())
    raw[-5] ^= 0xFF
    open(path, "wb").write(bytes(raw))
    with pytest.raises(H.HisqError):
        H.hisq_load_eigvecs(ctx, path)
