"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each checks a property that a
plausible slip in the oracle (a dropped hop, a wrong sign, phase, link index or
boundary factor, a transposed link, a wrong mass term, a broken even-odd split)
would violate.

Paper: "Improving HISQ propagator solves using deflation".
  Section 2: M = D + 2m, D anti-Hermitian; normal equation (Eq. 1);
             lambda_max about 23; lambda_min = eps_min + (2am)^2 (Eq. 3);
             even-odd solve with odd reconstruction; deflated guess (Eq. 4).
"""
import os

import numpy as np
import pytest

from oracle.oracle import Oracle, deflation_guess, even_sites, project_parity, site_parity
from paper_2502_00152_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_links(dims, seed=7, eps=0.4):
    return I.hisq_links(dims, seed, eps)


def _coords(dims):
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    return [a.reshape(-1) for a in (x, y, z, t)]


def _shift_site_field(dims, f, mu, n):
    """g(x) = f(x + n mu) with periodic wrap, f shaped (V, ...)."""
    X, Y, Z, T = dims
    g = f.reshape((T, Z, Y, X) + f.shape[1:])
    return np.roll(g, -n, axis=3 - mu).reshape(f.shape)


# ---------------------------------------------------------------- operator D
@pytest.mark.parametrize("dims,antip", [((6, 6, 6, 6), True), ((4, 6, 4, 8), False)])
def test_D_anti_hermitian(dims, antip):
    """<x, D y> = -<D x, y> (Section 2: D is anti-Hermitian)."""
    fat, lng = _rand_links(dims)
    o = Oracle(dims, fat, lng, antip)
    x = I.gaussian_field(dims, 1)
    y = I.gaussian_field(dims, 2)
    lhs = np.vdot(x, o.dslash(y))
    rhs = -np.vdot(o.dslash(x), y)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_D_connects_opposite_parities():
    """D maps even-site fields to odd-site fields and vice versa (the structure
    behind the even-odd preconditioning of Section 2)."""
    dims = (6, 4, 6, 8)
    o = Oracle(dims, *_rand_links(dims))
    par = site_parity(dims)
    for p in (0, 1):
        x = project_parity(dims, I.gaussian_field(dims, 3), p)
        y = o.dslash(x)
        assert np.all(y[par == p] == 0)
        assert np.linalg.norm(y[par != p]) > 0


@pytest.mark.parametrize("antip", [True, False])
def test_D_gauge_covariant(antip):
    """D[U^g](g psi) = g D[U] psi with U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag for the
    one-hop links and g(x) L_mu(x) g(x+3mu)^dag for the three-hop links."""
    dims = (6, 6, 4, 8)
    V = I.volume(dims)
    fat, lng = _rand_links(dims)
    g = I.random_su3(V, seed=9)
    fat_g = np.empty_like(fat)
    lng_g = np.empty_like(lng)
    for mu in range(4):
        g1 = _shift_site_field(dims, g, mu, 1)
        g3 = _shift_site_field(dims, g, mu, 3)
        fat_g[:, mu] = g @ fat[:, mu] @ np.conj(np.swapaxes(g1, -1, -2))
        lng_g[:, mu] = g @ lng[:, mu] @ np.conj(np.swapaxes(g3, -1, -2))
    psi = I.gaussian_field(dims, 4)
    a = Oracle(dims, fat_g, lng_g, antip).dslash(np.einsum("sij,sj->si", g, psi))
    b = np.einsum("sij,sj->si", g, Oracle(dims, fat, lng, antip).dslash(psi))
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)


def test_D_point_source_golden():
    """Free-field D on a point source against the hand-worked values in
    tests/golden (pins the hop signs, phases and time boundary factor)."""
    dims = (8, 8, 8, 8)
    o = Oracle(dims, *I.unit_links(dims), t_antiperiodic=True)
    src = I.point_source(dims, 0, (1, 0, 1, 0))
    out = o.dslash(src)
    expect = np.zeros_like(out)
    X, Y, Z, T = dims
    rows = np.loadtxt(os.path.join(GOLDEN, "point_source_free_field_8888.txt"))
    assert rows.shape == (16, 7)
    for x, y, z, t, c, re, im in rows:
        s = int(x) + X * (int(y) + Y * (int(z) + Z * int(t)))
        expect[s, int(c)] = re + 1j * im
    assert np.max(np.abs(out - expect)) <= 1e-15


# --------------------------------------------------- free field closed form
def _free_field_even_spectrum(dims, m, antip, c1=I.C1_NAIK, c3=I.C3_NAIK):
    """Eigenvalues of (M^dag M)_ee on unit links from the closed form:
    -D^2 = sum_mu Delta_mu^2 (the phases anticommute across odd hops), and a
    plane wave e^{ipx} gives Delta_mu -> 2i f(p_mu), f(p) = c1 sin p + c3 sin 3p.
    So M^dag M = 4m^2 + 4 sum_mu f(p_mu)^2, three colours per momentum; the even
    block holds half of that multiset (p and p + (pi,pi,pi,pi) give the same
    value and the same even-site vector)."""
    ps = []
    for mu, L in enumerate(dims):
        n = np.arange(L)
        if mu == 3 and antip:
            ps.append((2 * n + 1) * np.pi / L)
        else:
            ps.append(2 * n * np.pi / L)
    f2 = [(c1 * np.sin(p) + c3 * np.sin(3 * p)) ** 2 for p in ps]
    tot = (f2[0][:, None, None, None] + f2[1][None, :, None, None]
           + f2[2][None, None, :, None] + f2[3][None, None, None, :])
    lam = np.sort(np.repeat(4 * m * m + 4 * tot.reshape(-1), 3))
    return lam[::2]


@pytest.mark.parametrize("dims,antip", [((6, 6, 6, 6), True), ((4, 4, 6, 8), False), ((8, 4, 4, 4), True)])
def test_free_field_spectrum(dims, antip):
    m = 0.05
    o = Oracle(dims, *I.unit_links(dims), t_antiperiodic=antip)
    w = np.linalg.eigvalsh(o.dense_Aee(m))
    expect = _free_field_even_spectrum(dims, m, antip)
    assert w.shape == expect.shape
    assert np.max(np.abs(w - expect)) <= 1e-12


def test_free_field_lambda_max_normalisation():
    """With no factor 1/2 in D, the free-field lambda_max is 16 (7/6)^2 = 21.8,
    the paper's "lambda_max about 23" (Section 2); with a factor 1/2 it would be
    5.4.  On a lattice with p = pi/2 available the maximum is reached exactly."""
    dims = (4, 4, 4, 8)
    o = Oracle(dims, *I.unit_links(dims), t_antiperiodic=False)
    w = np.linalg.eigvalsh(o.dense_Aee(0.0))
    assert abs(w[-1] - 16 * (7 / 6) ** 2) <= 1e-12
    assert 0.85 * 23 < w[-1] < 23


def test_disordered_lambda_max_near_23():
    """On disordered SU(3) links the top of the spectrum of the squared operator
    stays near the paper's empirical lambda_max of about 23 (Section 2), and
    inside the rigorous bound |D| <= 8 (|c1| + |c3|) (each of the 16 hops is a
    unitary times its coefficient), i.e. lambda_max <= (8 * 7/6)^2 = 87.1.
    The spectrum is non-negative (M^dag M is positive semi-definite at m = 0)."""
    dims = (6, 6, 6, 6)
    o = Oracle(dims, *_rand_links(dims, eps=0.4))
    w = np.linalg.eigvalsh(o.dense_Aee(0.0))
    assert 0.8 * 23 < w[-1] < 1.2 * 23
    assert w[-1] <= (8 * 7 / 6) ** 2
    assert w[0] > -1e-12


def test_mass_shift_exact():
    """lambda(m) = lambda(0) + (2m)^2 for every eigenvalue (Section 2, Eq. 3)."""
    dims = (4, 4, 4, 6)
    o = Oracle(dims, *_rand_links(dims))
    m = 0.037
    w0 = np.linalg.eigvalsh(o.dense_Aee(0.0))
    wm = np.linalg.eigvalsh(o.dense_Aee(m))
    assert np.max(np.abs(wm - w0 - 4 * m * m)) <= 1e-12


def test_Aee_equals_even_block_of_MdagM():
    """(M^dag M)_ee, taken from M = D + 2m and D^dag = -D applied on the full
    lattice, equals the oracle's even-odd operator 4m^2 - D_eo D_oe."""
    dims = (6, 4, 4, 6)
    o = Oracle(dims, *_rand_links(dims))
    m = 0.1
    x = project_parity(dims, I.gaussian_field(dims, 5), 0)
    Mx = o.apply_M(m, x)
    MdagMx = -o.dslash(Mx) + 2 * m * Mx  # M^dag = -D + 2m
    a = project_parity(dims, MdagMx, 0)
    b = o.apply_Aee(m, x)
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(a)


# --------------------------------------------------------------- solve
def test_solve_true_residual_c1():
    """The plain FP64 even-odd CG on the 8^4 workload reaches the full-system
    true residual |eta - M psi|/|eta| <= 1e-10 (computed with M = D + 2m)."""
    cfg = I.lattice_config("c1")
    dims = cfg["dims"]
    o = Oracle(dims, *I.hisq_links(dims, cfg["seed"], cfg["eps"]))
    eta = I.point_source(dims, 0)
    psi, st = o.solve(cfg["mass"], eta, cfg["tol"])
    assert st["converged"]
    assert o.full_residual(cfg["mass"], psi, eta) <= cfg["tol"]
    assert st["even_residual"] <= cfg["tol"]


def test_solve_matches_dense_solve():
    """Even-odd CG + reconstruction equals numpy's dense solve of M psi = eta,
    M built column by column from D + 2m (brute force on a 4^3 x 6 lattice)."""
    dims = (4, 4, 4, 6)
    V = I.volume(dims)
    o = Oracle(dims, *_rand_links(dims, eps=0.5))
    m = 0.08
    M = np.zeros((3 * V, 3 * V), dtype=np.complex128)
    e = np.zeros((V, 3), dtype=np.complex128)
    for j in range(3 * V):
        e.reshape(-1)[j] = 1
        M[:, j] = o.apply_M(m, e).reshape(-1)
        e.reshape(-1)[j] = 0
    eta = I.gaussian_field(dims, 6)
    ref = np.linalg.solve(M, eta.reshape(-1)).reshape(V, 3)
    psi, st = o.solve(m, eta, 1e-12)
    assert st["converged"]
    assert np.linalg.norm(psi - ref) <= 1e-10 * np.linalg.norm(ref)


def test_prepare_source_is_even_part_of_Mdag_eta():
    """y_e = (M^dag eta)_e with M^dag = -D + 2m (Section 2)."""
    dims = (6, 6, 4, 4)
    o = Oracle(dims, *_rand_links(dims))
    m = 0.02
    eta = I.gaussian_field(dims, 8)
    ref = project_parity(dims, -o.dslash(eta) + 2 * m * eta, 0)
    y = o.prepare_source(m, eta)
    assert np.linalg.norm(y - ref) <= 1e-14 * np.linalg.norm(ref)


def test_full_residual_after_reconstruction_is_schur_residual():
    """With the odd sites reconstructed exactly, psi_o = (eta_o - D_oe psi_e) / 2m
    (Section 2), the odd rows of eta - M psi vanish for ANY psi_e and the even
    rows equal (y_e - A_ee psi_e) / 2m: a wrong sign of the hop term, a wrong
    mass factor or a wrong reconstruction breaks one of the two.  (The solver's
    FP64 confirmation forms the even-system residual this way.)"""
    dims = (6, 4, 6, 4)
    o = Oracle(dims, *_rand_links(dims, seed=11))
    m = 0.07
    eta = I.gaussian_field(dims, 21)
    psi_e = project_parity(dims, I.gaussian_field(dims, 22), 0)
    psi = o.reconstruct(m, psi_e, eta)
    assert np.array_equal(project_parity(dims, psi, 0), psi_e)
    r = eta - o.apply_M(m, psi)
    assert np.linalg.norm(project_parity(dims, r, 1)) <= 1e-13 * np.linalg.norm(eta)
    schur = project_parity(dims, o.prepare_source(m, eta) - o.apply_Aee(m, psi_e), 0) / (2 * m)
    re = project_parity(dims, r, 0)
    assert np.linalg.norm(re - schur) <= 1e-12 * np.linalg.norm(schur)


# ---------------------------------------------------------- eigenpairs
def test_lanczos_matches_dense():
    """Plain Lanczos with full reorthogonalisation finds the same lowest
    eigenvalues of A_ee as dense eigh (6^4)."""
    dims = (6, 6, 6, 6)
    o = Oracle(dims, *_rand_links(dims, eps=0.3))
    m = 0.01
    w = np.linalg.eigvalsh(o.dense_Aee(m))
    th, vecs = o.lanczos(m, 8, 600, I.gaussian_field(dims, 21, I.STREAM_START))
    assert np.max(np.abs(th - w[:8]) / w[:8]) <= 1e-10
    for i in range(8):
        t, res = o.rayleigh(m, vecs[i])
        assert abs(t - w[i]) <= 1e-10 * w[i]
        assert res <= 1e-6


def test_deflated_guess_and_solve():
    """With exact low eigenpairs, the deflated guess of Eq. 4 leaves a residual
    with no component along the deflation space, and CG from it reaches the
    same solution as CG from zero in fewer iterations."""
    dims = (6, 6, 6, 6)
    o = Oracle(dims, *_rand_links(dims, eps=0.3))
    m = 0.005
    lam, vecs = o.eig_dense(m, 32)
    eta = I.gaussian_field(dims, 12)
    y = o.prepare_source(m, eta)
    x0 = deflation_guess(vecs, lam, y)
    r0 = y - o.apply_Aee(m, x0)
    proj = vecs.reshape(32, -1).conj() @ r0.reshape(-1)
    assert np.max(np.abs(proj)) <= 1e-12 * np.linalg.norm(y)
    tgt = 1e-11 * np.linalg.norm(y)
    xa, ita, _, oka = o.cg(m, y, None, tgt)
    xb, itb, _, okb = o.cg(m, y, x0, tgt)
    assert oka and okb and itb < ita
    assert np.linalg.norm(xa - xb) <= 1e-8 * np.linalg.norm(xa)
    # the deflated guess solves the low-mode part exactly
    ev = even_sites(dims)
    assert np.all(x0.reshape(I.volume(dims), 3)[np.setdiff1d(np.arange(I.volume(dims)), ev)] == 0)
