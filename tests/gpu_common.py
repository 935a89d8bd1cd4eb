"""Shared helpers of the GPU parity tests (inputs and oracle objects only)."""
import numpy as np

from oracle.oracle import Oracle, even_sites, project_parity
from paper_2502_00152_gb300 import hisq as H
from paper_2502_00152_gb300 import inputs as I


def make(dims, seed=3, eps=0.4, antip=True, recon=18, mass=None):
    fat, lng = I.hisq_links(dims, seed, eps)
    o = Oracle(dims, fat, lng, t_antiperiodic=antip)
    ctx = H.hisq_create(dims, t_antiperiodic=antip, device=0)
    H.hisq_load_links(ctx, fat, lng, long_recon=recon, long_scale=I.C3_NAIK if recon != 18 else 1.0)
    if mass is not None:
        H.hisq_set_mass(ctx, mass)
    return ctx, o


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def dslash_ref(o, dims, field, out_parity):
    return project_parity(dims, o.dslash(project_parity(dims, field, 1 - out_parity)), out_parity)


def orthonormal_even_set(dims, n, seed, lam_lo=5e-3, lam_hi=0.2):
    """n orthonormal even-site fields (host QR of seeded Gaussian columns) and n
    chosen massless eigenvalues, ascending.  Eq. 4 is a plain formula, so the
    oracle's deflated guess is exact for any orthonormal set: these stand in for
    eigenvectors where dense diagonalisation is out of reach."""
    ev = even_sites(dims)
    rng = np.random.default_rng(seed)
    L = 3 * len(ev)
    G = rng.standard_normal((L, n)) + 1j * rng.standard_normal((L, n))
    Q, _ = np.linalg.qr(G)
    V = np.zeros((n, int(np.prod(dims)), 3), dtype=np.complex128)
    V[:, ev, :] = Q.T.reshape(n, len(ev), 3)
    return np.geomspace(lam_lo, lam_hi, n), V


def stored_vectors(vecs, prec, Vh):
    """The values a deflation kernel reads back for eigenvectors stored at
    `prec`, simulated on the host: FP64 -> FP32, then the storage rounding
    (32: none; 15: BF16 round to nearest even; 16: FP16 with one FP32 scale per
    site, the largest of its six components; 14: FP16 of v * 2^e, 4^e >= 3 Vh)."""
    v = np.asarray(vecs)
    re = v.real.astype(np.float32)
    im = v.imag.astype(np.float32)
    if prec == 32:
        return re.astype(np.float64) + 1j * im.astype(np.float64)
    if prec == 15:
        def bf(a):
            u = np.ascontiguousarray(a).view(np.uint32).astype(np.uint64)
            u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
            return u.astype(np.uint32).view(np.float32).astype(np.float64)
        return bf(re) + 1j * bf(im)
    if prec == 14:
        e = 0
        while 4 ** e < 3 * Vh:
            e += 1
        s, inv = np.float32(2.0 ** e), np.float32(2.0 ** -e)
        q = lambda a: ((a * s).astype(np.float16).astype(np.float32) * inv).astype(np.float64)
        return q(re) + 1j * q(im)
    if prec == 16:
        m = np.maximum(np.abs(re).max(axis=-1), np.abs(im).max(axis=-1))[..., None]
        with np.errstate(divide="ignore"):
            inv = np.where(m > 0, np.float32(1.0) / m, np.float32(0.0)).astype(np.float32)
        q = lambda a: ((a * inv).astype(np.float16).astype(np.float32) * m).astype(np.float64)
        return q(re) + 1j * q(im)
    raise ValueError(prec)
