"""The seeded input generators are reproducible: the thin links are computed in
independent chunks from counter-based deviates, so they do not depend on how
many threads compute them nor on the chunk size, and every link is SU(3)."""
import numpy as np

from paper_2502_00152_gb300 import inputs as I


def test_thin_links_independent_of_threads_and_chunks(monkeypatch):
    dims = (4, 4, 6, 8)
    ref = I.thin_links(dims, 7, 0.3)  # one chunk (768 links < 2^20)
    for workers, chunk in ((1, 64), (4, 64), (3, 100), (8, 1 << 20)):
        monkeypatch.setattr(I, "_workers", lambda w=workers: w)
        u = I.thin_links(dims, 7, 0.3, chunk=chunk)
        assert np.array_equal(u, ref), (workers, chunk)
    # unitary with unit determinant
    m = ref.reshape(-1, 3, 3)
    assert np.max(np.abs(m @ np.conj(np.swapaxes(m, 1, 2)) - np.eye(3))) < 1e-13
    assert np.max(np.abs(np.linalg.det(m) - 1)) < 1e-13


def test_long_links_are_products_of_three_thin_links():
    """The long link is c3 U(x) U(x+mu) U(x+2mu), checked at a few sites by
    explicit coordinate arithmetic against the chunked batched products."""
    dims = (4, 6, 4, 8)
    X, Y, Z, T = dims
    u = I.thin_links(dims, 3, 0.4)
    fat, lng = I.hisq_links(dims, 3, 0.4)
    assert np.array_equal(fat, I.C1_NAIK * u)
    rng = np.random.default_rng(0)
    for _ in range(20):
        x = [int(rng.integers(0, d)) for d in dims]
        mu = int(rng.integers(0, 4))

        def site(c):
            return c[0] + X * (c[1] + Y * (c[2] + Z * c[3]))

        def step(c, n):
            c = list(c)
            c[mu] = (c[mu] + n) % dims[mu]
            return c

        want = I.C3_NAIK * u[site(x), mu] @ u[site(step(x, 1)), mu] @ u[site(step(x, 2)), mu]
        assert np.allclose(lng[site(x), mu], want, rtol=0, atol=1e-14)
