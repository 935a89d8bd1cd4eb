"""Python face of the FP64 CPU oracle -- TEST INFRASTRUCTURE.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this module.  The heavy loops (the Dirac operator, CG) are the plain C in
hisq_oracle.c; the small dense steps here use numpy library routines (eigh,
matrix products) as single steps, without any blocking or reordering.

Paper: "Improving HISQ propagator solves using deflation".
  Section 2, Eq. 1 ........ normal equation M^dag M psi = M^dag eta
  Section 2, Eq. 3 ........ lambda_min = eps_min + (2 a m)^2 (mass shift)
  Section 2, Eq. 4 ........ deflated initial guess x = sum_i v_i lambda_i^-1 v_i^dag b
  Section 2 (last para.) .. eigenvectors of the squared operator on even sites by
                            Lanczos (the paper uses thick-restart Lanczos; the
                            oracle uses plain Lanczos with full
                            reorthogonalisation, which reaches the same
                            eigenpairs without restarts)

Fields are full-lattice complex arrays shaped (V, 3); "even-site" vectors have
zero odd sites.  Links are (V, 4, 3, 3) complex arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_dslash.argtypes = [ip, ctypes.c_int, dp, dp, dp, dp]
        lib.oracle_apply_M.argtypes = [ip, ctypes.c_int, dp, dp, ctypes.c_double, dp, dp]
        lib.oracle_apply_Aee.argtypes = [ip, ctypes.c_int, dp, dp, ctypes.c_double, dp, dp]
        lib.oracle_prepare_source.argtypes = [ip, ctypes.c_int, dp, dp, ctypes.c_double, dp, dp]
        lib.oracle_reconstruct.argtypes = [ip, ctypes.c_int, dp, dp, ctypes.c_double, dp, dp, dp]
        lib.oracle_cg.argtypes = [ip, ctypes.c_int, dp, dp, ctypes.c_double, dp, dp,
                                  ctypes.c_double, ctypes.c_int, ip, dp]
        lib.oracle_cg.restype = ctypes.c_int
        lib.oracle_solve.argtypes = [ip, ctypes.c_int, dp, dp, ctypes.c_double, dp, dp,
                                     ctypes.c_double, ctypes.c_int, dp, dp]
        lib.oracle_solve.restype = ctypes.c_int
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return _load().oracle_num_threads()


def _dp(a: np.ndarray):
    assert a.dtype == np.complex128 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _field(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def site_parity(dims) -> np.ndarray:
    """(x+y+z+t) mod 2 for every site s = x + X(y + Y(z + Z t))."""
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    return ((x + y + z + t) & 1).reshape(-1)


def even_sites(dims) -> np.ndarray:
    """Indices of the even sites in lexicographic order (the oracle's own
    even-site numbering)."""
    return np.nonzero(site_parity(dims) == 0)[0]


def project_parity(dims, field: np.ndarray, parity: int) -> np.ndarray:
    out = np.array(field, dtype=np.complex128, copy=True)
    out[site_parity(dims) != parity] = 0
    return out


class Oracle:
    """The operator and solver on one gauge field."""

    def __init__(self, dims, fat, lng, t_antiperiodic: bool = True):
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.fat = _field(fat).reshape(self.V, 4, 3, 3)
        self.lng = _field(lng).reshape(self.V, 4, 3, 3)
        self.antip = 1 if t_antiperiodic else 0
        self._L = (ctypes.c_int * 4)(*self.dims)
        self._lib = _load()

    def _new(self):
        return np.zeros((self.V, 3), dtype=np.complex128)

    # ---- operator (Section 2) ---------------------------------------------
    def dslash(self, psi):
        psi = _field(psi).reshape(self.V, 3)
        out = self._new()
        self._lib.oracle_dslash(self._L, self.antip, _dp(self.fat), _dp(self.lng), _dp(psi), _dp(out))
        return out

    def apply_M(self, m, psi):
        psi = _field(psi).reshape(self.V, 3)
        out = self._new()
        self._lib.oracle_apply_M(self._L, self.antip, _dp(self.fat), _dp(self.lng), m, _dp(psi), _dp(out))
        return out

    def apply_Aee(self, m, x):
        x = _field(x).reshape(self.V, 3)
        out = self._new()
        self._lib.oracle_apply_Aee(self._L, self.antip, _dp(self.fat), _dp(self.lng), m, _dp(x), _dp(out))
        return out

    def prepare_source(self, m, eta):
        eta = _field(eta).reshape(self.V, 3)
        out = self._new()
        self._lib.oracle_prepare_source(self._L, self.antip, _dp(self.fat), _dp(self.lng), m, _dp(eta), _dp(out))
        return out

    def reconstruct(self, m, psi_e, eta):
        psi_e = _field(psi_e).reshape(self.V, 3)
        eta = _field(eta).reshape(self.V, 3)
        out = self._new()
        self._lib.oracle_reconstruct(self._L, self.antip, _dp(self.fat), _dp(self.lng), m,
                                     _dp(psi_e), _dp(eta), _dp(out))
        return out

    # ---- solvers -----------------------------------------------------------
    def cg(self, m, b, x0=None, rtarget=1e-10, maxiter=100000):
        """FP64 CG on A_ee from x0; returns (x, iterations, |b - A x|, converged)."""
        b = _field(b).reshape(self.V, 3)
        x = self._new() if x0 is None else _field(x0).reshape(self.V, 3).copy()
        it = ctypes.c_int(0)
        res = ctypes.c_double(0)
        st = self._lib.oracle_cg(self._L, self.antip, _dp(self.fat), _dp(self.lng), m, _dp(b), _dp(x),
                                 rtarget, maxiter, ctypes.byref(it), ctypes.byref(res))
        return x, it.value, res.value, st == 0

    def solve(self, m, eta, tol=1e-10, x0_e=None, maxiter=100000):
        """psi = M^-1 eta by even-odd CG; returns (psi, stats dict)."""
        eta = _field(eta).reshape(self.V, 3)
        psi = self._new()
        stats = np.zeros(3)
        x0 = None
        if x0_e is not None:
            x0 = _field(x0_e).reshape(self.V, 3)
        st = self._lib.oracle_solve(self._L, self.antip, _dp(self.fat), _dp(self.lng), m, _dp(eta),
                                    None if x0 is None else _dp(x0), tol, maxiter, _dp(psi),
                                    stats.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return psi, dict(iterations=int(stats[0]), even_residual=float(stats[1]),
                         full_residual=float(stats[2]), converged=(st == 0))

    def full_residual(self, m, psi, eta) -> float:
        """|eta - M psi| / |eta| in FP64 (Section 3's |r|/|b| on the full system)."""
        r = _field(eta).reshape(self.V, 3) - self.apply_M(m, psi)
        return float(np.linalg.norm(r) / np.linalg.norm(eta))

    def even_residual(self, m, x_e, b_e) -> float:
        r = _field(b_e).reshape(self.V, 3) - self.apply_Aee(m, x_e)
        return float(np.linalg.norm(r) / np.linalg.norm(b_e))

    # ---- eigenpairs (Section 2, last paragraph; Eq. 3) ---------------------
    def dense_Aee(self, m) -> np.ndarray:
        """Dense matrix of A_ee on the even sites (oracle numbering), built
        column by column by applying the operator to unit vectors."""
        ev = even_sites(self.dims)
        n = 3 * len(ev)
        A = np.zeros((n, n), dtype=np.complex128)
        e = self._new()
        for j in range(n):
            s, c = ev[j // 3], j % 3
            e[s, c] = 1.0
            col = self.apply_Aee(m, e)
            A[:, j] = col[ev].reshape(-1)
            e[s, c] = 0.0
        return A

    def eig_dense(self, m, n_ev=None):
        """All (or the lowest n_ev) eigenpairs of A_ee by dense eigh; the
        vectors are returned as full-lattice fields (n, V, 3)."""
        A = self.dense_Aee(m)
        w, U = np.linalg.eigh(A)
        k = len(w) if n_ev is None else n_ev
        return w[:k], self._even_to_fields(U[:, :k])

    def _even_to_fields(self, U: np.ndarray) -> np.ndarray:
        ev = even_sites(self.dims)
        k = U.shape[1]
        out = np.zeros((k, self.V, 3), dtype=np.complex128)
        out[:, ev, :] = U.T.reshape(k, len(ev), 3)
        return out

    def lanczos(self, m, n_ev: int, n_steps: int, v0):
        """Lowest n_ev eigenpairs of A_ee by plain Lanczos with full
        reorthogonalisation (Golub & Van Loan, Matrix Computations, Sec. 10.1)
        over n_steps steps from the start field v0 (its even sites are used);
        Ritz values and vectors from numpy's eigh of the tridiagonal matrix."""
        ev = even_sites(self.dims)
        n = 3 * len(ev)
        n_steps = min(n_steps, n)
        Q = np.zeros((n_steps + 1, n), dtype=np.complex128)
        alpha = np.zeros(n_steps)
        beta = np.zeros(n_steps)
        q = _field(v0).reshape(self.V, 3)[ev].reshape(-1)
        Q[0] = q / np.linalg.norm(q)
        field = self._new()
        k_done = n_steps
        for j in range(n_steps):
            field[ev] = Q[j].reshape(-1, 3)
            w = self.apply_Aee(m, field)[ev].reshape(-1)
            alpha[j] = np.real(np.vdot(Q[j], w))
            # full reorthogonalisation against all basis vectors, applied twice
            for _ in range(2):
                w = w - Q[: j + 1].T @ (Q[: j + 1].conj() @ w)
            beta[j] = np.linalg.norm(w)
            if beta[j] < 1e-13 * max(1.0, abs(alpha[j])):
                k_done = j + 1
                break
            Q[j + 1] = w / beta[j]
        T = np.diag(alpha[:k_done]) + np.diag(beta[: k_done - 1], 1) + np.diag(beta[: k_done - 1], -1)
        th, Y = np.linalg.eigh(T)
        Z = Q[:k_done].T @ Y[:, :n_ev]
        return th[:n_ev], self._even_to_fields(Z)

    def rayleigh(self, m, v):
        """Rayleigh quotient theta = <v, A v> / <v, v> and residual |A v - theta v| / |v|."""
        v = _field(v).reshape(self.V, 3)
        Av = self.apply_Aee(m, v)
        vv = np.real(np.vdot(v, v))
        th = np.real(np.vdot(v, Av)) / vv
        return th, float(np.linalg.norm(Av - th * v) / np.sqrt(vv))


def deflation_guess(evecs: np.ndarray, evals: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x = sum_i v_i lambda_i^-1 v_i^dag b (Section 2, Eq. 4), for orthonormal v_i
    given as (n, V, 3) fields and the eigenvalues lambda_i of A_ee."""
    Vm = evecs.reshape(evecs.shape[0], -1)
    c = Vm.conj() @ np.asarray(b, dtype=np.complex128).reshape(-1)
    return (Vm.T @ (c / np.asarray(evals))).reshape(b.shape)



# ------------------------------------------------------------------------
# Learned initial guess: gauge-covariant parallel-transport network (the paper
# has none; the oracle states the network's definition plainly).
#   out_b(x) = sum_a sum_h w[b, a, h] (T_h in_a)(x)
#   T_0 = 1,  T_{mu,fwd} f(x) =  eta_mu(x) bc(x) F_mu(x) f(x + mu),
#             T_{mu,bwd} f(x) = -eta_mu(x) bc(x - mu) F_mu(x - mu)^dag f(x - mu)
# hop index h = 1 + 2 mu + d (d = 0 fwd, 1 bwd).  With all hop weights 1 and
# identity weight 0 one layer is the one-hop (fat-link) part of D.
def _coords(dims):
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    return [a.reshape(-1) for a in (x, y, z, t)]


def _shift(dims, f, mu, n):
    X, Y, Z, T = dims
    g = f.reshape((T, Z, Y, X) + f.shape[1:])
    return np.roll(g, -n, axis=3 - mu).reshape(f.shape)


def net_transports(dims, fat, field, t_antiperiodic=True):
    """The 9 transported copies [T_h field] of one (V, 3) colour field."""
    c = _coords(dims)
    T = dims[3]
    fat = np.asarray(fat).reshape(-1, 4, 3, 3)
    out = [np.array(field, dtype=np.complex128)]
    for mu in range(4):
        e = np.ones(len(c[0]))
        for nu in range(mu):
            e = e * np.where(c[nu] % 2 == 1, -1.0, 1.0)
        bcf = np.where((mu == 3) & t_antiperiodic & (c[3] == T - 1), -1.0, 1.0) if mu == 3 else np.ones_like(e)
        bcb = np.where(t_antiperiodic & (c[3] == 0), -1.0, 1.0) if mu == 3 else np.ones_like(e)
        U = fat[:, mu]
        fwd = np.einsum("sij,sj->si", U, _shift(dims, field, mu, 1)) * (e * bcf)[:, None]
        Ub = _shift(dims, U, mu, -1)  # F_mu(x - mu)
        bwd = -np.einsum("sji,sj->si", np.conj(Ub), _shift(dims, field, mu, -1)) * (e * bcb)[:, None]
        out += [fwd, bwd]
    return out


def net_layer(dims, fat, w, ins, t_antiperiodic=True):
    """One layer: w (Cout, Cin, 9), ins (Cin, V, 3) -> (Cout, V, 3)."""
    w = np.asarray(w)
    tr = [net_transports(dims, fat, f, t_antiperiodic) for f in ins]
    out = np.zeros((w.shape[0],) + np.asarray(ins).shape[1:], dtype=np.complex128)
    for b in range(w.shape[0]):
        for a in range(w.shape[1]):
            for h in range(9):
                out[b] += w[b, a, h] * tr[a][h]
    return out


def net_wgrad(dims, fat, ins, gouts, t_antiperiodic=True):
    """G[b, a, h] = sum_x gout_b(x) . conj(T_h in_a(x)) (gradient of a real loss
    with respect to conj(w), given gout = its gradient with respect to conj(out))."""
    tr = [net_transports(dims, fat, f, t_antiperiodic) for f in ins]
    G = np.zeros((len(gouts), len(ins), 9), dtype=np.complex128)
    for b in range(len(gouts)):
        for a in range(len(ins)):
            for h in range(9):
                G[b, a, h] = np.vdot(tr[a][h], gouts[b])
    return G


def net_forward(dims, fat, weights, x, t_antiperiodic=True):
    for w in weights:
        x = net_layer(dims, fat, w, x, t_antiperiodic)
    return x
