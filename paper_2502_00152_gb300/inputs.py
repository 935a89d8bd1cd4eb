"""Seeded synthetic inputs: gauge links, sources and random colour vectors.

This module is the one piece shared by the FP64 oracle tests and the CUDA path.
It holds no arithmetic of the solve itself (no Dirac operator, no solver, no
projection): it only draws random numbers and builds the synthetic stand-ins for
the paper's gauge ensembles (Section 2, Table 1), whose real MILC HISQ
configurations are not available.

Host layouts (FP64, the C-ABI's layouts):
  * site index   s = x + X*(y + Y*(z + Z*t))
  * links        [s][mu][row][col] complex128, mu order x, y, z, t
  * colour field [s][colour] complex128 over the full lattice

Random numbers come from a counter-based generator: the splitmix64 output
function (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to a key built from (seed, stream, index),
followed by the Box-Muller transform for normal deviates.  Any element can be
regenerated on its own, so large lattices are produced in chunks.

Link recipe (synthetic HISQ-like links):
  thin links  U_mu(x) = exp(i * eps * A),  A = sum_a omega_a lambda_a / 2,
              omega_a ~ N(0, 1), lambda_a the Gell-Mann matrices;
  fat links   F_mu(x) = c1 * U_mu(x)                                (c1 = 9/8)
  long links  L_mu(x) = c3 * U_mu(x) U_mu(x+mu) U_mu(x+2mu)          (c3 = -1/24)
with periodic wrap of the thin links.  Staggered phases and the time boundary
condition are NOT folded in: they belong to the operator.
"""
from __future__ import annotations

import numpy as np

C1_NAIK = 9.0 / 8.0
C3_NAIK = -1.0 / 24.0

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers of the counter-based generator
STREAM_LINK = 1
STREAM_GAUSS_SOURCE = 2
STREAM_Z2 = 3
STREAM_SPINOR = 4
STREAM_GAUGE_XFORM = 5
STREAM_START = 6


def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def random_u64(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """64 random bits for each counter in `index` (uint64 array)."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([seed], dtype=np.uint64) * _GOLDEN + np.uint64(stream))[0]
        idx = np.asarray(index, dtype=np.uint64)
        return _mix64(key + (idx + np.uint64(1)) * _GOLDEN)


def random_uniform(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """Uniform doubles in the open interval (0, 1)."""
    bits = random_u64(seed, stream, index) >> np.uint64(11)
    return (bits.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def random_normal(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """`count` standard normal deviates with counters start .. start+count-1.

    Deviate k uses uniforms with counters 2k and 2k+1 (Box-Muller, cosine branch).
    """
    k = np.arange(start, start + count, dtype=np.uint64)
    u1 = random_uniform(seed, stream, np.uint64(2) * k)
    u2 = random_uniform(seed, stream, np.uint64(2) * k + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def volume(dims) -> int:
    X, Y, Z, T = dims
    return X * Y * Z * T


def check_dims(dims) -> None:
    if len(dims) != 4 or any(int(d) < 2 or int(d) % 2 for d in dims):
        raise ValueError(f"lattice extents must be 4 even integers >= 2, got {dims}")


def _gell_mann() -> np.ndarray:
    g = np.zeros((8, 3, 3), dtype=np.complex128)
    g[0, 0, 1] = g[0, 1, 0] = 1
    g[1, 0, 1], g[1, 1, 0] = -1j, 1j
    g[2, 0, 0], g[2, 1, 1] = 1, -1
    g[3, 0, 2] = g[3, 2, 0] = 1
    g[4, 0, 2], g[4, 2, 0] = -1j, 1j
    g[5, 1, 2] = g[5, 2, 1] = 1
    g[6, 1, 2], g[6, 2, 1] = -1j, 1j
    g[7] = np.diag([1, 1, -2]) / np.sqrt(3.0)
    return g


_LAMBDA = _gell_mann()


def _reunitarise(u: np.ndarray) -> np.ndarray:
    """Project (n,3,3) near-SU(3) matrices back onto SU(3): Gram-Schmidt on rows
    0 and 1, row 2 = conj(row0 x row1)."""
    r0 = u[:, 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=1, keepdims=True)
    r1 = u[:, 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=1)


def _workers() -> int:
    import os

    return max(1, min(16, os.cpu_count() or 1))


def thin_links(dims, seed: int, eps: float, chunk: int = 1 << 20) -> np.ndarray:
    """Thin SU(3) links U_mu(x) = exp(i eps A), layout [s][mu][3][3].  Chunks of
    links are independent (counter-based deviates), so they are computed on a
    pool of threads; the result does not depend on the number of threads."""
    from concurrent.futures import ThreadPoolExecutor

    import torch

    check_dims(dims)
    n = volume(dims) * 4
    out = np.empty((n, 3, 3), dtype=np.complex128)

    def one(c0):
        c1 = min(n, c0 + chunk)
        om = random_normal(seed, STREAM_LINK, 8 * c0, 8 * (c1 - c0)).reshape(c1 - c0, 8)
        a = np.einsum("na,aij->nij", om, _LAMBDA) * 0.5
        u = torch.linalg.matrix_exp(torch.from_numpy(1j * eps * a)).numpy()
        out[c0:c1] = _reunitarise(u)

    with ThreadPoolExecutor(max_workers=_workers()) as ex:
        list(ex.map(one, range(0, n, chunk)))
    return out.reshape(volume(dims), 4, 3, 3)


def _shift_forward(field: np.ndarray, dims, mu: int, n: int) -> np.ndarray:
    """g(x) = field(x + n*mu_hat) with periodic wrap; field shaped [s][...]."""
    X, Y, Z, T = dims
    f = field.reshape((T, Z, Y, X) + field.shape[1:])
    axis = 3 - mu
    return np.roll(f, -n, axis=axis).reshape(field.shape)


def hisq_links(dims, seed: int, eps: float, c1: float = C1_NAIK, c3: float = C3_NAIK):
    """Fat and long links of the synthetic recipe: (fat, long), each [s][mu][3][3].
    The products of three thin links are batched 3x3 complex matrix products
    (torch.bmm on the host, in chunks)."""
    import torch

    u = thin_links(dims, seed, eps)
    fat = c1 * u
    lng = np.empty_like(u)
    chunk = 1 << 20
    for mu in range(4):
        umu = np.ascontiguousarray(u[:, mu])
        u1 = _shift_forward(umu, dims, mu, 1)
        u2 = _shift_forward(umu, dims, mu, 2)
        for s0 in range(0, len(umu), chunk):
            s1 = min(len(umu), s0 + chunk)
            p = torch.bmm(torch.bmm(torch.from_numpy(umu[s0:s1]), torch.from_numpy(u1[s0:s1])),
                          torch.from_numpy(u2[s0:s1]))
            lng[s0:s1, mu] = c3 * p.numpy()
        del umu, u1, u2
    return fat, lng


def unit_links(dims, c1: float = C1_NAIK, c3: float = C3_NAIK):
    """Free-field links: F = c1 * 1, L = c3 * 1."""
    V = volume(dims)
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3))
    return c1 * eye.copy(), c3 * eye.copy()


def gaussian_field(dims, seed: int, stream: int = STREAM_SPINOR, index0: int = 0) -> np.ndarray:
    """Complex colour field with re, im ~ N(0,1) on every site: [s][3]."""
    V = volume(dims)
    r = random_normal(seed, stream, index0, 6 * V).reshape(V, 3, 2)
    return r[..., 0] + 1j * r[..., 1]


def point_source(dims, colour: int = 0, site=(0, 0, 0, 0)) -> np.ndarray:
    X, Y, Z, T = dims
    eta = np.zeros((volume(dims), 3), dtype=np.complex128)
    x, y, z, t = site
    eta[x + X * (y + Y * (z + Z * t)), colour] = 1.0
    return eta


def z2_wall_source(dims, seed: int, source: int, colour: int, n_sources: int = 8) -> np.ndarray:
    """Z2 wall source `source` (0..n_sources-1): +-1 (real) on every site of
    timeslice t = source*T/n_sources, colour `colour` only."""
    X, Y, Z, T = dims
    vs = X * Y * Z
    t0 = (source * T) // n_sources
    u = random_uniform(seed, STREAM_Z2, np.arange(source * vs, (source + 1) * vs, dtype=np.uint64))
    eta = np.zeros((volume(dims), 3), dtype=np.complex128)
    eta[t0 * vs:(t0 + 1) * vs, colour] = np.where(u < 0.5, -1.0, 1.0)
    return eta


def gaussian_source(dims, seed: int, source: int) -> np.ndarray:
    """Gaussian complex source number `source` (re, im ~ N(0,1) on every site)."""
    return gaussian_field(dims, seed, STREAM_GAUSS_SOURCE, index0=source * 6 * volume(dims))


def gaussian_colour_source(dims, seed: int, source: int, colour: int) -> np.ndarray:
    """Colour-diluted Gaussian source: the colour-`colour` component of Gaussian
    source `source` on every site, the other two colours zero."""
    eta = np.zeros((volume(dims), 3), dtype=np.complex128)
    eta[:, colour] = gaussian_source(dims, seed, source)[:, colour]
    return eta


def random_su3(n: int, seed: int, stream: int = STREAM_GAUGE_XFORM) -> np.ndarray:
    """n Haar-random SU(3) matrices: QR of a complex Gaussian matrix, with the
    phases of R's diagonal moved into Q (Mezzadri, Notices AMS 54 (2007) 592),
    then the determinant divided out."""
    r = random_normal(seed, stream, 0, 18 * n).reshape(n, 3, 3, 2)
    z = (r[..., 0] + 1j * r[..., 1]) / np.sqrt(2.0)
    q, rr = np.linalg.qr(z)
    d = np.diagonal(rr, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[:, None, None]


def lattice_config(name: str) -> dict:
    """Synthetic workloads shaped like the paper's runs (Section 3, Table 2)."""
    cfgs = {
        # plain method, small: FP64 even-odd CG, point source
        "c1": dict(dims=(8, 8, 8, 8), seed=1, eps=0.4, mass=0.05, tol=1e-10),
        # deflated mixed-precision CG, single right-hand side
        "c2": dict(dims=(32, 32, 32, 64), seed=2, eps=0.3, mass=0.002, tol=1e-10, n_ev=256),
        # batched multi right-hand sides (Z2 wall sources)
        "c3": dict(dims=(32, 32, 32, 64), seed=2, eps=0.3, mass=0.002, tol=1e-10, n_ev=512),
        # learned initial guess
        "c4": dict(dims=(24, 24, 24, 48), seed=3, eps=0.3, mass=0.003, tol=1e-10, n_ev=128),
        # small lattice for profiler captures (a few GB on the device at most)
        "s16": dict(dims=(16, 16, 16, 32), seed=6, eps=0.3, mass=0.01, tol=1e-10, n_ev=64),
        # largest single-GPU lattice
        "c5": dict(dims=(64, 64, 64, 96), seed=4, eps=0.25, mass=0.0008, tol=1e-10, n_ev=200),
    }
    return dict(cfgs[name])
