"""Pins of the oracle of the learned-guess network (CPU, FP64): its one-hop
transports reproduce the fat-link part of the (pinned) Dirac operator, it is
gauge covariant, its weight gradient matches finite differences, and the
adjoint-weight formula used by the GPU backward pass is the true adjoint."""
import numpy as np
import pytest

from oracle.oracle import Oracle, net_forward, net_layer, net_wgrad
from paper_2502_00152_gb300 import inputs as I


def _rng_c(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def _adjoint_weights(w):
    """w'[a, b, 0] = conj(w[b, a, 0]); w'[a, b, 1+2mu+d] = -conj(w[b, a, 1+2mu+(1-d)])."""
    cout, cin, _ = w.shape
    wa = np.zeros((cin, cout, 9), dtype=np.complex128)
    for a in range(cin):
        for b in range(cout):
            wa[a, b, 0] = np.conj(w[b, a, 0])
            for mu in range(4):
                for d in range(2):
                    wa[a, b, 1 + 2 * mu + d] = -np.conj(w[b, a, 1 + 2 * mu + (1 - d)])
    return wa


@pytest.mark.parametrize("antip", [True, False])
def test_unit_hops_give_fat_part_of_D(antip):
    dims = (6, 4, 6, 8)
    fat, lng = I.hisq_links(dims, 3, 0.4)
    o = Oracle(dims, fat, np.zeros_like(lng), antip)
    psi = I.gaussian_field(dims, 2)
    w = np.zeros((1, 1, 9), dtype=np.complex128)
    w[0, 0, 1:] = 1.0
    out = net_layer(dims, fat, w, [psi], antip)[0]
    ref = o.dslash(psi)
    assert np.linalg.norm(out - ref) <= 1e-13 * np.linalg.norm(ref)


def test_network_gauge_covariant():
    dims = (4, 6, 4, 6)
    V = I.volume(dims)
    fat, _ = I.hisq_links(dims, 4, 0.4)
    g = I.random_su3(V, seed=8)
    X, Y, Z, T = dims

    def sh(f, mu, n):
        return np.roll(f.reshape((T, Z, Y, X) + f.shape[1:]), -n, axis=3 - mu).reshape(f.shape)

    fg = np.empty_like(fat)
    for mu in range(4):
        fg[:, mu] = g @ fat[:, mu] @ np.conj(np.swapaxes(sh(g, mu, 1), -1, -2))
    ws = [_rng_c((4, 2, 9), 1), _rng_c((2, 4, 9), 2)]
    ins = [I.gaussian_field(dims, 5), I.gaussian_field(dims, 6)]
    gins = [np.einsum("sij,sj->si", g, f) for f in ins]
    a = net_forward(dims, fg, ws, gins)
    b = [np.einsum("sij,sj->si", g, f) for f in net_forward(dims, fat, ws, ins)]
    for x, y in zip(a, b):
        assert np.linalg.norm(x - y) <= 1e-12 * np.linalg.norm(y)


def test_adjoint_weight_formula():
    dims = (4, 4, 6, 6)
    fat, _ = I.hisq_links(dims, 5, 0.4)
    w = _rng_c((3, 2, 9), 3)
    v = [I.gaussian_field(dims, 7), I.gaussian_field(dims, 8)]
    u = [I.gaussian_field(dims, 9), I.gaussian_field(dims, 10), I.gaussian_field(dims, 11)]
    lv = net_layer(dims, fat, w, v)
    lu = net_layer(dims, fat, _adjoint_weights(w), u)
    lhs = sum(np.vdot(u[b], lv[b]) for b in range(3))
    rhs = sum(np.vdot(lu[a], v[a]) for a in range(2))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_weight_gradient_finite_differences():
    """dL/dRe(w) + i dL/dIm(w) for L = sum_b |out_b - t_b|^2 equals
    net_wgrad(ins, 2 (out - t)) (gradient of a real loss w.r.t. conj(w), times 2)."""
    dims = (4, 4, 4, 6)
    fat, _ = I.hisq_links(dims, 6, 0.4)
    w = _rng_c((2, 2, 9), 4) * 0.3
    ins = [I.gaussian_field(dims, 12), I.gaussian_field(dims, 13)]
    t = [I.gaussian_field(dims, 14), I.gaussian_field(dims, 15)]

    def loss(ww):
        out = net_layer(dims, fat, ww, ins)
        return sum(np.linalg.norm(out[b] - t[b]) ** 2 for b in range(2))

    out = net_layer(dims, fat, w, ins)
    G = net_wgrad(dims, fat, ins, [2 * (out[b] - t[b]) for b in range(2)])
    for (b, a, h) in [(0, 0, 0), (1, 0, 3), (0, 1, 8), (1, 1, 5)]:
        d = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[b, a, h] += d
        wm[b, a, h] -= d
        gre = (loss(wp) - loss(wm)) / (2 * d)
        wp, wm = w.copy(), w.copy()
        wp[b, a, h] += 1j * d
        wm[b, a, h] -= 1j * d
        gim = (loss(wp) - loss(wm)) / (2 * d)
        assert abs(complex(gre, gim) - G[b, a, h]) <= 1e-6 * max(1.0, abs(G[b, a, h]))
