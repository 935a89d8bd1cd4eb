"""GPU parity of the HISQ Dslash and of the even-odd normal operator against the
FP64 oracle (Section 2: M = D + 2m; Eq. 1).  Tolerances: relative error
<= 1e-13 in FP64, <= 1e-6 in FP32, <= 5e-3 with FP16 vector storage."""
import numpy as np
import pytest

from gpu_common import dslash_ref, make, rel
from oracle.oracle import project_parity
from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {64: 1e-13, 32: 1e-6, 16: 5e-3}
# (vector storage, link storage); FP16 anywhere means the FP16 tolerance
COMBOS = [(64, 64), (32, 32), (16, 32), (32, 16), (16, 16)]


def tol(vp, lp):
    return TOL[min(vp, lp)]

# lattices: the Naik-distinct minimum, L = 4 (x+3 == x-1 aliasing), ragged
# half-volumes that do not fill a 256-thread block, and several tiles
LATTICES = [(6, 6, 6, 6), (4, 4, 4, 4), (4, 6, 4, 10), (8, 4, 6, 6), (8, 8, 8, 12)]


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("antip", [True, False])
def test_dslash_all_precisions(dims, antip):
    ctx, o = make(dims, antip=antip)
    try:
        src = I.gaussian_field(dims, 17)
        for par in (0, 1):
            ref = dslash_ref(o, dims, src, par)
            for vp, lp in COMBOS:
                out = H.hisq_apply_dslash(ctx, par, vp, src, link_precision=lp)
                assert rel(out, ref) <= tol(vp, lp), (par, vp, lp, rel(out, ref))
                # the other parity of the output is exactly zero
                assert np.all(project_parity(dims, out, 1 - par) == 0)
    finally:
        ctx.close()


@pytest.mark.parametrize("dims", [(6, 6, 6, 6), (4, 6, 4, 10)])
def test_dslash_long_recon12(dims):
    """12-real long links (two rows + SU(3) third row, c3 and signs rebuilt)."""
    ctx, o = make(dims, recon=12)
    try:
        src = I.gaussian_field(dims, 18)
        for par in (0, 1):
            ref = dslash_ref(o, dims, src, par)
            for vp, lp in COMBOS:
                assert rel(H.hisq_apply_dslash(ctx, par, vp, src, link_precision=lp), ref) <= tol(vp, lp)
    finally:
        ctx.close()


@pytest.mark.parametrize("dims,eps", [((6, 6, 6, 6), 0.4), ((4, 6, 4, 10), 0.3), ((8, 8, 8, 12), 0.1)])
def test_dslash_long_recon8(dims, eps):
    """8-real long links: (a2, a3, b1, arg a1, arg c1) of the SU(3) factor, the
    rest rebuilt from unitarity with FP32 arithmetic.  The rebuilt entries
    carry the FP32 rounding amplified by 1/N, N = |a2|^2 + |a3|^2 (the links
    here are near the identity, N ~ 0.05 at eps 0.1), hence 1e-5 for FP32
    vectors; FP16 storage dominates otherwise."""
    fat, lng = I.hisq_links(dims, 3, eps)
    from oracle.oracle import Oracle

    o = Oracle(dims, fat, lng)
    ctx = H.hisq_create(dims)
    try:
        H.hisq_load_links(ctx, fat, lng, long_recon=8, long_scale=I.C3_NAIK)
        src = I.gaussian_field(dims, 18)
        for par in (0, 1):
            ref = dslash_ref(o, dims, src, par)
            assert rel(H.hisq_apply_dslash(ctx, par, 64, src, link_precision=64), ref) <= TOL[64]
            assert rel(H.hisq_apply_dslash(ctx, par, 32, src, link_precision=32), ref) <= 1e-5
            assert rel(H.hisq_apply_dslash(ctx, par, 16, src, link_precision=32), ref) <= TOL[16]
        with pytest.raises(H.HisqError):  # FP16 links are not offered with 8-real long links
            H.hisq_apply_dslash(ctx, 0, 16, src, link_precision=16)
    finally:
        ctx.close()


def test_recon12_rejects_non_su3_links():
    dims = (4, 4, 4, 6)
    fat, lng = I.hisq_links(dims, 1, 0.3)
    ctx = H.hisq_create(dims)
    try:
        with pytest.raises(H.HisqError) as e:
            H.hisq_load_links(ctx, fat, lng * 1.01, long_recon=12, long_scale=I.C3_NAIK)
        assert e.value.status == H.HISQ_ERR_INVALID_ARG
    finally:
        ctx.close()


def test_nonfinite_links_rejected():
    dims = (4, 4, 4, 4)
    fat, lng = I.hisq_links(dims, 1, 0.3)
    fat[7, 2, 1, 1] = np.nan
    ctx = H.hisq_create(dims)
    try:
        with pytest.raises(H.HisqError) as e:
            H.hisq_load_links(ctx, fat, lng)
        assert e.value.status == H.HISQ_ERR_NUMERICAL
    finally:
        ctx.close()


@pytest.mark.parametrize("vp,lp", COMBOS)
def test_normal_operator(vp, lp):
    dims = (6, 4, 6, 8)
    m = 0.02
    ctx, o = make(dims, mass=m)
    try:
        x = project_parity(dims, I.gaussian_field(dims, 19), 0)
        ref = o.apply_Aee(m, x)
        out = H.hisq_apply_normal_op(ctx, vp, x, link_precision=lp)
        assert rel(out, ref) <= tol(vp, lp) * (10 if min(vp, lp) == 16 else 1)
    finally:
        ctx.close()


def test_gauge_covariance_on_gpu():
    """D[U^g] g psi = g D[U] psi, both sides from the GPU FP64 operator."""
    dims = (6, 6, 4, 8)
    V = I.volume(dims)
    fat, lng = I.hisq_links(dims, 4, 0.4)
    g = I.random_su3(V, seed=2)

    def shift(f, mu, n):
        X, Y, Z, T = dims
        return np.roll(f.reshape((T, Z, Y, X) + f.shape[1:]), -n, axis=3 - mu).reshape(f.shape)

    fg, lgk = np.empty_like(fat), np.empty_like(lng)
    for mu in range(4):
        fg[:, mu] = g @ fat[:, mu] @ np.conj(np.swapaxes(shift(g, mu, 1), -1, -2))
        lgk[:, mu] = g @ lng[:, mu] @ np.conj(np.swapaxes(shift(g, mu, 3), -1, -2))
    psi = I.gaussian_field(dims, 7)
    c1 = H.hisq_create(dims)
    c2 = H.hisq_create(dims)
    try:
        H.hisq_load_links(c1, fat, lng)
        H.hisq_load_links(c2, fg, lgk)
        a = H.hisq_apply_dslash(c2, 1, 64, np.einsum("sij,sj->si", g, psi))
        b = np.einsum("sij,sj->si", g, H.hisq_apply_dslash(c1, 1, 64, psi))
        assert rel(a, b) <= 1e-13
    finally:
        c1.close()
        c2.close()


@pytest.mark.parametrize("cfg", ["c2"])
def test_dslash_full_size(cfg):
    """The benchmark lattice (32^3 x 64) in the launch configuration the
    benchmark uses, every output site compared with the oracle."""
    c = I.lattice_config(cfg)
    dims = c["dims"]
    ctx, o = make(dims, seed=c["seed"], eps=c["eps"])
    try:
        src = I.gaussian_field(dims, 5)
        ref = dslash_ref(o, dims, src, 1)
        for vp, lp in COMBOS:
            assert rel(H.hisq_apply_dslash(ctx, 1, vp, src, link_precision=lp), ref) <= tol(vp, lp)
    finally:
        ctx.close()
