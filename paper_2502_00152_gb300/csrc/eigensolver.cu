// eigensolver.cu -- thick-restart Lanczos (Section 2 of the paper: the low
// eigenvectors of the squared massless operator, computed once per gauge field
// and reused by every solve) and the eigenpair store (set, get, save, load,
// deflate; Section 3: eigenvalues recomputed from the stored vectors).
//
// Operator: A0 = -D_eo D_oe on even sites (FP32).  Optionally the Lanczos
// process runs on a Chebyshev polynomial T_d(x), x = (a_max + a_min - 2 A0) /
// (a_max - a_min), which maps [a_min, a_max] into [-1, 1] and makes the modes
// below a_min the largest ones.  The basis is FP32; full reorthogonalisation
// (classical Gram-Schmidt, twice) runs on the GPU; the Rayleigh-Ritz step on the
// small real symmetric matrix is FP64 on the host; the final eigenvalues are
// FP64 Rayleigh quotients with the FP64 operator.  Thick restart after Wu &
// Simon (SIAM J. Matrix Anal. Appl. 22 (2000) 602): keep n_keep Ritz vectors,
// append the last Lanczos vector, and continue with the arrowhead matrix.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.cuh"

namespace hisq {

double *eig_eps_dev(hisq_ctx *ctx);
hisq_status read_slots(hisq_ctx *ctx, int slot0, int n, double *out);
hisq_status deflate_add(hisq_ctx *ctx, int n, const double *r, double *x);

#define TRY(x)                                  \
    do {                                        \
        hisq_status s_ = (x);                   \
        if (s_ != HISQ_OK) return s_;           \
    } while (0)

// ------------------------------------------------ host symmetric eigensolver
// Eigen-decomposition of a real symmetric n x n matrix a (row major):
// Householder reduction to tridiagonal form with the transformations
// accumulated in z, then implicit QL iterations with shifts on the tridiagonal
// matrix (Golub & Van Loan, Matrix Computations, Secs. 8.3.1 and 8.3.3; the
// QL iteration is the published tred2/tql2 procedure of Bowdler, Martin,
// Reinsch and Wilkinson, Numer. Math. 11 (1968) 293, as distributed in EISPACK).
// On exit w holds the eigenvalues ascending and column j of z (row major) the
// eigenvector of w[j].
static void sym_eig(int n, std::vector<double> a, std::vector<double> &w, std::vector<double> &z)
{
    z.assign(size_t(n) * n, 0.0);
    for (int i = 0; i < n; i++) z[size_t(i) * n + i] = 1.0;
    std::vector<double> v(n), p(n), q(n);
    auto A = [&](int i, int j) -> double & { return a[size_t(i) * n + j]; };
    for (int k = 0; k + 2 < n; k++) {
        double alpha = 0;
        for (int i = k + 1; i < n; i++) alpha += A(i, k) * A(i, k);
        alpha = std::sqrt(alpha);
        if (alpha == 0) continue;
        if (A(k + 1, k) > 0) alpha = -alpha;
        double vn = 0;
        for (int i = k + 1; i < n; i++) {
            v[i] = A(i, k);
            if (i == k + 1) v[i] -= alpha;
            vn += v[i] * v[i];
        }
        if (vn == 0) continue;
        const double beta = 2.0 / vn;
        // p = beta * A v over the trailing block, K = beta/2 v.p, q = p - K v
        for (int i = k + 1; i < n; i++) {
            double s = 0;
            for (int j = k + 1; j < n; j++) s += A(i, j) * v[j];
            p[i] = beta * s;
        }
        double K = 0;
        for (int i = k + 1; i < n; i++) K += v[i] * p[i];
        K *= 0.5 * beta;
        for (int i = k + 1; i < n; i++) q[i] = p[i] - K * v[i];
        for (int i = k + 1; i < n; i++)
            for (int j = k + 1; j < n; j++) A(i, j) -= v[i] * q[j] + q[i] * v[j];
        A(k + 1, k) = A(k, k + 1) = alpha;
        for (int i = k + 2; i < n; i++) A(i, k) = A(k, i) = 0;
        // z <- z H
        for (int r = 0; r < n; r++) {
            double s = 0;
            for (int j = k + 1; j < n; j++) s += z[size_t(r) * n + j] * v[j];
            s *= beta;
            for (int j = k + 1; j < n; j++) z[size_t(r) * n + j] -= s * v[j];
        }
    }
    std::vector<double> d(n), e(n, 0.0);
    for (int i = 0; i < n; i++) d[i] = A(i, i);
    for (int i = 0; i + 1 < n; i++) e[i] = A(i + 1, i);
    // implicit QL on (d, e); e[i] couples d[i] and d[i+1]
    for (int l = 0; l < n; l++) {
        for (int iter = 0; iter < 60; iter++) {
            int m = l;
            for (; m + 1 < n; m++) {
                const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
                if (std::fabs(e[m]) <= 1e-15 * dd) break;
            }
            if (m == l) break;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + (g >= 0 ? std::fabs(r) : -std::fabs(r)));
            double s = 1.0, c = 1.0, pp = 0.0;
            int i;
            bool early = false;
            for (i = m - 1; i >= l; i--) {
                double f = s * e[i], b = c * e[i];
                r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0) {
                    d[i + 1] -= pp;
                    e[m] = 0;
                    early = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - pp;
                r = (d[i] - g) * s + 2.0 * c * b;
                pp = s * r;
                d[i + 1] = g + pp;
                g = c * r - b;
                for (int k2 = 0; k2 < n; k2++) {
                    double &zi = z[size_t(k2) * n + i], &zi1 = z[size_t(k2) * n + i + 1];
                    const double t = zi1;
                    zi1 = s * zi + c * t;
                    zi = c * zi - s * t;
                }
            }
            if (early) continue;
            d[l] -= pp;
            e[l] = g;
            e[m] = 0;
        }
    }
    // sort ascending
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return d[x] < d[y]; });
    w.resize(n);
    std::vector<double> zs(size_t(n) * n);
    for (int j = 0; j < n; j++) {
        w[j] = d[idx[j]];
        for (int r = 0; r < n; r++) zs[size_t(r) * n + j] = z[size_t(r) * n + idx[j]];
    }
    z.swap(zs);
}

// ------------------------------------------------------------ operators
struct EigWork {
    int Vh;
    void *tmp_odd;    // FP32 odd
    void *c0, *c1;    // Chebyshev recurrence
    double *coef;     // device FP64 complex coefficients
};

enum { ESL_A = 8, ESL_B = 9, ESL_C = 10 };

// w = A0 v = -D_eo D_oe v (FP32)
static hisq_status op_A0(hisq_ctx *ctx, EigWork &W, const void *v, void *w)
{
    TRY(launch_dslash(ctx, 1, 32, 32, v, W.tmp_odd, 0, nullptr, 0, nullptr, 1.0, -1));
    return launch_dslash(ctx, 0, 32, 32, W.tmp_odd, w, 0, nullptr, 0, nullptr, -1.0, -1);
}

// w = T_d(x) v, x = (sigma - 2 A0) / delta
static hisq_status op_cheby(hisq_ctx *ctx, EigWork &W, int deg, double amin, double amax, const void *v, void *w)
{
    const double sigma = amax + amin, delta = amax - amin;
    if (deg == 1) {
        // w = (sigma v - 2 A0 v) / delta = (sigma/delta) v + (2/delta) D_eo D_oe v
        TRY(launch_dslash(ctx, 1, 32, 32, v, W.tmp_odd, 0, nullptr, 0, nullptr, 1.0, -1));
        return launch_dslash(ctx, 0, 32, 32, W.tmp_odd, w, sigma / delta, v, 0, nullptr, 2.0 / delta, -1);
    }
    // T_{k-1} = prev, T_k = cur; T_{k+1} = (2 sigma/delta) T_k + (4/delta) D_eo D_oe T_k - T_{k-1}
    void *pool[3] = {W.c0, W.c1, w};
    const void *prev = v;
    void *cur = W.c0;
    TRY(launch_dslash(ctx, 1, 32, 32, v, W.tmp_odd, 0, nullptr, 0, nullptr, 1.0, -1));
    TRY(launch_dslash(ctx, 0, 32, 32, W.tmp_odd, cur, sigma / delta, v, 0, nullptr, 2.0 / delta, -1));
    for (int k = 1; k < deg; k++) {
        void *next = nullptr;
        for (void *b : pool)
            if (b != prev && b != cur) {
                next = b;
                break;
            }
        TRY(launch_dslash(ctx, 1, 32, 32, cur, W.tmp_odd, 0, nullptr, 0, nullptr, 1.0, -1));
        TRY(launch_dslash(ctx, 0, 32, 32, W.tmp_odd, next, 2.0 * sigma / delta, cur, -1.0, prev, 4.0 / delta, -1));
        prev = cur;
        cur = next;
    }
    if (cur != w) HISQ_CUDA(cudaMemcpyAsync(w, cur, spinor_bytes(32, ctx->g.Vh), cudaMemcpyDeviceToDevice, ctx->stream));
    return HISQ_OK;
}

// FP64 Rayleigh quotient eps = |D_oe v|^2 / |v|^2 and residual |A0 v - eps v| / |v|
// of an even FP64 field v (tmp: FP64 odd, out: FP64 even scratch)
static hisq_status rayleigh_fp64(hisq_ctx *ctx, const double *v, double *tmp, double *out, double *eps, double *res)
{
    TRY(launch_norm2(ctx, 64, v, ESL_A));
    TRY(launch_dslash(ctx, 1, 64, 64, v, tmp, 0, nullptr, 0, nullptr, 1.0, ESL_B));
    double ab[2];
    TRY(read_slots(ctx, ESL_A, 2, ab));
    const double e = ab[0] > 0 ? ab[1] / ab[0] : 0;
    // out = -D_eo tmp - e v
    TRY(launch_dslash(ctx, 0, 64, 64, tmp, out, -e, v, 0, nullptr, -1.0, ESL_C));
    double r2 = 0;
    TRY(read_slots(ctx, ESL_C, 1, &r2));
    *eps = e;
    *res = ab[0] > 0 ? std::sqrt(r2 / ab[0]) : 0;
    return HISQ_OK;
}

static void free_eig(hisq_ctx *ctx)
{
    if (ctx->eig.vecs) dev_free(ctx, ctx->eig.vecs, size_t(ctx->eig.n) * spinor_bytes(ctx->eig.prec, ctx->g.Vh));
    if (ctx->eig.eps_dev) dev_free(ctx, ctx->eig.eps_dev, sizeof(double) * (ctx->eig.n > 0 ? ctx->eig.n : 1));
    ctx->eig.vecs = nullptr;
    ctx->eig.eps_dev = nullptr;
    ctx->eig.n = 0;
    ctx->eig.eps.clear();
}

// Take n FP32 vectors (stride spinor_bytes(32)), recompute FP64 Rayleigh
// quotients, sort ascending, store in precision prec.
static hisq_status store_eigvecs(hisq_ctx *ctx, int n, const void *vf32, int prec, const double *eps_given,
                                 std::vector<double> *residuals)
{
    const int Vh = ctx->g.Vh;
    const size_t sf = spinor_bytes(32, Vh), sp = spinor_bytes(prec, Vh);
    double *vd = (double *)get_buf(ctx, BUF_TEST_A, spinor_bytes(64, Vh));
    double *td = (double *)get_buf(ctx, BUF_TMPHI, spinor_bytes(64, Vh));
    double *od = (double *)get_buf(ctx, BUF_RHI, spinor_bytes(64, Vh));
    if (!vd || !td || !od) return HISQ_ERR_OOM;
    std::vector<double> eps(n), res(n, 0.0);
    for (int i = 0; i < n; i++) {
        const void *vi = (const char *)vf32 + sf * i;
        if (eps_given) {
            eps[i] = eps_given[i];
        } else {
            TRY(launch_convert(ctx, vi, 32, vd, 64));
            TRY(rayleigh_fp64(ctx, vd, td, od, &eps[i], &res[i]));
        }
    }
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return eps[a] < eps[b]; });
    free_eig(ctx);
    void *store = dev_alloc(ctx, sp * (n > 0 ? n : 1));
    if (!store) return HISQ_ERR_OOM;
    double *eps_dev = (double *)dev_alloc(ctx, sizeof(double) * (n > 0 ? n : 1));
    if (!eps_dev) {
        dev_free(ctx, store, sp * (n > 0 ? n : 1));
        return HISQ_ERR_OOM;
    }
    for (int j = 0; j < n; j++) TRY(launch_convert(ctx, (const char *)vf32 + sf * idx[j], 32, (char *)store + sp * j, prec));
    std::vector<double> sorted(n);
    for (int j = 0; j < n; j++) sorted[j] = eps[idx[j]];
    if (n > 0) HISQ_CUDA(cudaMemcpyAsync(eps_dev, sorted.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->eig.vecs = store;
    ctx->eig.eps_dev = eps_dev;
    ctx->eig.n = n;
    ctx->eig.prec = prec;
    ctx->eig.version++;
    ctx->eig.eps = sorted;
    if (residuals) residuals->resize(n);
    for (int j = 0; j < n; j++)
        if (residuals) (*residuals)[j] = res[idx[j]];
    return HISQ_OK;
}

hisq_status block_trlm(hisq_ctx *ctx, const hisq_eig_params *P, int b, int n_ev, int n_kr, int n_keep, int deg,
                       double amin, double amax, void *B, int *conv_out);

// Pairs that pass the final check: the convergence test of the iteration looks
// at the residual of the (filtered) Krylov operator, which in FP32 can accept a
// spurious Ritz pair when the filter's dynamic range is large; every stored
// pair is therefore also checked with the FP64 operator, |A v - theta v| / |v|
// <= 1e-3 a_max (far above the accuracy of a genuine pair, far below the O(1)
// residual of a spurious one).  Returns the number of pairs that pass.
static int verified_pairs(const std::vector<double> &res, double amax)
{
    int good = 0;
    for (double r : res)
        if (r <= 1e-3 * amax) good++;
    if (good < int(res.size()) && log_level() > 0)
        fprintf(stderr, "[hisq] eigensolve: %d of %zu Ritz pairs fail the FP64 residual check\n",
                int(res.size()) - good, res.size());
    return good;
}

// ------------------------------------------------------------ TRLM
static hisq_status trlm(hisq_ctx *ctx, const hisq_eig_params *P, int *n_conv, double *eps_out)
{
    const int Vh = ctx->g.Vh;
    const int n_ev = P->n_ev, n_kr = P->n_kr;
    const int n_keep = P->n_keep > 0 ? P->n_keep : (n_ev + n_kr) / 2;
    const int deg = P->cheby_degree;
    const size_t sf = spinor_bytes(32, Vh);
    const int dim = 3 * Vh;
    if (n_ev < 1 || n_kr <= n_ev + 2 || n_keep < n_ev || n_keep >= n_kr || n_kr > dim || n_kr > 6144)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "need 1 <= n_ev <= n_keep < n_kr <= min(3 Vh, 6144), n_kr > n_ev + 2");
    if (P->storage_precision != 32 && P->storage_precision != 16 && P->storage_precision != HISQ_PREC_BF16 &&
        P->storage_precision != HISQ_PREC_HALF_EV)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "storage_precision must be 32, 16, 15 (BF16) or 14 (FP16 x 2^e)");
    if (!(P->tol > 0)) return set_err(ctx, HISQ_ERR_INVALID_ARG, "tol must be positive");

    // basis (n_kr + 1 vectors, Ritz vectors rotated into its head in place,
    // through a chunk buffer of about 256 MB), work
    const int nrot = std::max(n_keep, n_ev);
    const size_t Lf = size_t(6) * Vh;
    size_t chunk = (size_t(256) << 20) / (sizeof(float) * size_t(nrot));
    chunk = std::max<size_t>(128, std::min(Lf, chunk) / 128 * 128);
    const int bs = P->block_size > 1 ? P->block_size : 1;
    char *B = (char *)dev_alloc(ctx, sf * (n_kr + bs));
    char *R = (char *)dev_alloc(ctx, sizeof(float) * chunk * nrot);
    char *wk = (char *)dev_alloc(ctx, sf * 4);
    double *coef = (double *)dev_alloc(ctx, sizeof(double) * 2 * (n_kr + 1));
    double *Yd = (double *)dev_alloc(ctx, sizeof(double) * size_t(n_kr) * std::max(n_keep, n_ev));
    struct Free {
        hisq_ctx *c;
        void *p[5];
        size_t s[5];
        ~Free()
        {
            cudaStreamSynchronize(c->stream);
            for (int i = 0; i < 5; i++) dev_free(c, p[i], s[i]);
        }
    } guard{ctx, {B, R, wk, coef, Yd}, {sf * (n_kr + bs), sizeof(float) * chunk * nrot, sf * 4, sizeof(double) * 2 * (n_kr + 1), sizeof(double) * size_t(n_kr) * nrot}};
    if (!B || !R || !wk || !coef || !Yd) return HISQ_ERR_OOM;
    void *tmp_odd = get_buf(ctx, BUF_TMP, spinor_bytes(32, Vh));
    if (!tmp_odd) return HISQ_ERR_OOM;
    EigWork W{Vh, tmp_odd, wk + sf * 1, wk + sf * 2, coef};
    void *w = wk; // Lanczos work vector
    auto vec = [&](int i) -> void * { return B + sf * i; };

    // spectrum window
    double amax = P->a_max, amin = P->a_min;
    if (!(amax > 0)) {
        // power iteration on A0 (also the scale of the final residual check)
        TRY(launch_random_f(ctx, P->seed ^ 0x5bd1e995ull, vec(0)));
        double lam = 0;
        for (int it = 0; it < 60; it++) {
            TRY(launch_norm2(ctx, 32, vec(0), ESL_A));
            double nn;
            TRY(read_slots(ctx, ESL_A, 1, &nn));
            TRY(launch_scale_f(ctx, 1.0 / std::sqrt(nn), vec(0), vec(0)));
            TRY(op_A0(ctx, W, vec(0), w));
            TRY(launch_cdot(ctx, 32, vec(0), w, ESL_B));
            double ab[2];
            TRY(read_slots(ctx, ESL_B, 2, ab));
            lam = ab[0];
            HISQ_CUDA(cudaMemcpyAsync(vec(0), w, sf, cudaMemcpyDeviceToDevice, ctx->stream));
        }
        amax = 1.1 * lam + 0.1;
    }
    std::vector<double> alpha(n_kr, 0.0), beta(n_kr, 0.0), theta_keep, s_keep;
    std::vector<double> coefh(2 * (n_kr + 1));
    auto start = [&](uint64_t seed) -> hisq_status {
        TRY(launch_random_f(ctx, seed, vec(0)));
        TRY(launch_norm2(ctx, 32, vec(0), ESL_A));
        double nn;
        TRY(read_slots(ctx, ESL_A, 1, &nn));
        return launch_scale_f(ctx, 1.0 / std::sqrt(nn), vec(0), vec(0));
    };
    // Lanczos steps j0 .. j1-1 with full reorthogonalisation (classical
    // Gram-Schmidt against v_0..v_j, twice): alpha_j, beta_j, v_{j+1}
    auto lanczos = [&](int j0, int j1, bool filtered) -> hisq_status {
        for (int j = j0; j < j1; j++) {
            TRY(filtered ? op_cheby(ctx, W, deg, amin, amax, vec(j), w) : op_A0(ctx, W, vec(j), w));
            for (int pass = 0; pass < 2; pass++) {
                TRY(launch_defl_project(ctx, j + 1, 32, B, 32, w, coef));
                if (pass == 0)
                    HISQ_CUDA(cudaMemcpyAsync(coefh.data(), coef, sizeof(double) * 2 * (j + 1), cudaMemcpyDeviceToHost,
                                              ctx->stream));
                TRY(launch_defl_expand(ctx, j + 1, 32, B, coef, -1.0, 32, w));
            }
            TRY(launch_norm2(ctx, 32, w, ESL_A));
            double bb;
            TRY(read_slots(ctx, ESL_A, 1, &bb));
            alpha[j] = coefh[2 * j];
            beta[j] = std::sqrt(bb);
            if (!std::isfinite(beta[j])) return set_err(ctx, HISQ_ERR_NUMERICAL, "non-finite Lanczos coefficient");
            if (beta[j] < 1e-30) beta[j] = 1e-30;
            TRY(launch_scale_f(ctx, 1.0 / beta[j], w, vec(j + 1)));
        }
        return HISQ_OK;
    };
    if (deg > 0 && !(amin > 0)) {
        // Window edge from a stochastic Lanczos quadrature estimate of the
        // eigenvalue count (Lin, Saad & Yang, SIAM Review 58 (2016) 34): m plain
        // Lanczos steps from a random vector give nodes theta_j with weights
        // tau_j^2 (first components of the Ritz vectors), and the number of
        // eigenvalues below x is about dim * sum_{theta_j <= x} tau_j^2.
        const double want = (amin < 0 ? -amin : 2.0) * n_ev;
        const int m = std::min(n_kr, std::min(dim - 1, 256));
        TRY(start(P->seed ^ 0x9e3779b97f4a7c15ull));
        TRY(lanczos(0, m, false));
        std::vector<double> T(size_t(m) * m, 0.0), th, Z;
        for (int j = 0; j < m; j++) {
            T[size_t(j) * m + j] = alpha[j];
            if (j + 1 < m) T[size_t(j) * m + j + 1] = T[size_t(j + 1) * m + j] = beta[j];
        }
        sym_eig(m, T, th, Z);
        double cum = 0;
        amin = th[m - 1];
        for (int j = 0; j < m; j++) {
            cum += Z[j] * Z[j]; // row 0, column j
            if (double(dim) * cum >= want) {
                amin = th[j];
                break;
            }
        }
        if (!(amin < amax)) amin = 0.5 * amax;
    }
    if (deg > 0 && !(amin > 0 && amin < amax)) return set_err(ctx, HISQ_ERR_INVALID_ARG, "need 0 < a_min < a_max");
    if (log_level() > 0) fprintf(stderr, "[hisq] trlm: degree %d, window [%.6g, %.6g]\n", deg, amin, amax);
    ctx->last_window[0] = amin;
    ctx->last_window[1] = amax;
    const bool want_largest = deg > 0;

    if (bs > 1) {
        // block thick-restart Lanczos (block_eig.cu); Ritz vectors end in B[0 .. n_ev)
        int conv = 0;
        TRY(block_trlm(ctx, P, bs, n_ev, n_kr, n_keep, deg, amin, amax, B, &conv));
        std::vector<double> res;
        TRY(store_eigvecs(ctx, n_ev, B, P->storage_precision, nullptr, &res));
        if (n_conv) *n_conv = std::min(conv, verified_pairs(res, amax));
        if (eps_out)
            for (int i = 0; i < n_ev; i++) eps_out[i] = ctx->eig.eps[i];
        return HISQ_OK;
    }

    // start vector
    TRY(start(P->seed));
    int k = 0; // kept vectors
    int conv = 0;
    std::vector<double> ritz, Y;
    for (int restart = 0; restart <= P->max_restarts; restart++) {
        TRY(lanczos(k, n_kr, deg > 0));
        // Rayleigh-Ritz on the n_kr x n_kr arrowhead + tridiagonal matrix
        std::vector<double> T(size_t(n_kr) * n_kr, 0.0);
        for (int i = 0; i < k; i++) {
            T[size_t(i) * n_kr + i] = theta_keep[i];
            T[size_t(i) * n_kr + k] = T[size_t(k) * n_kr + i] = s_keep[i];
        }
        for (int j = k; j < n_kr; j++) {
            T[size_t(j) * n_kr + j] = alpha[j];
            if (j + 1 < n_kr) T[size_t(j) * n_kr + j + 1] = T[size_t(j + 1) * n_kr + j] = beta[j];
        }
        std::vector<double> th, Z;
        sym_eig(n_kr, T, th, Z);
        // wanted order
        std::vector<int> order(n_kr);
        std::iota(order.begin(), order.end(), 0);
        if (want_largest) std::reverse(order.begin(), order.end());
        double scale = 0;
        for (double t : th) scale = std::max(scale, std::fabs(t));
        const double bl = beta[n_kr - 1];
        conv = 0;
        for (int i = 0; i < n_ev; i++) {
            const double resid = std::fabs(bl * Z[size_t(n_kr - 1) * n_kr + order[i]]);
            if (resid <= P->tol * scale) conv++;
            else break;
        }
        const bool done = conv >= n_ev || restart == P->max_restarts;
        if (log_level() > 0)
            fprintf(stderr, "[hisq] trlm restart %d: %d/%d converged, window [%.4g, %.4g], ritz %.6g .. %.6g\n",
                    restart, conv, n_ev, amin, amax, th[order[0]], th[order[n_ev - 1]]);
        const int nout = done ? n_ev : n_keep;
        Y.assign(size_t(n_kr) * nout, 0.0);
        for (int r = 0; r < n_kr; r++)
            for (int c = 0; c < nout; c++) Y[size_t(r) * nout + c] = Z[size_t(r) * n_kr + order[c]];
        HISQ_CUDA(cudaMemcpyAsync(Yd, Y.data(), sizeof(double) * Y.size(), cudaMemcpyHostToDevice, ctx->stream));
        TRY(launch_rotate_inplace(ctx, n_kr, nout, B, Yd, (float *)R, int(chunk)));
        if (done) break;
        // thick restart: v_0..v_{k-1} = Ritz vectors (rotated in place), v_k <- v_{n_kr}
        HISQ_CUDA(cudaMemcpyAsync(vec(n_keep), vec(n_kr), sf, cudaMemcpyDeviceToDevice, ctx->stream));
        k = n_keep;
        theta_keep.resize(k);
        s_keep.resize(k);
        for (int i = 0; i < k; i++) {
            theta_keep[i] = th[order[i]];
            s_keep[i] = bl * Z[size_t(n_kr - 1) * n_kr + order[i]];
        }
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    // the head of B holds the n_ev wanted Ritz vectors (FP32): FP64 Rayleigh quotients, sort, store
    std::vector<double> res;
    TRY(store_eigvecs(ctx, n_ev, B, P->storage_precision, nullptr, &res));
    if (n_conv) *n_conv = std::min(conv, verified_pairs(res, amax));
    if (eps_out)
        for (int i = 0; i < n_ev; i++) eps_out[i] = ctx->eig.eps[i];
    return HISQ_OK;
}

static uint64_t fnv1a(const unsigned char *p, size_t n, uint64_t h)
{
    for (size_t i = 0; i < n; i++) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct EigFileHeader {
    char magic[8];
    int32_t dims[4];
    int32_t n, prec;
    int64_t bytes_per_vec;
    uint64_t checksum;
};

} // namespace hisq

using namespace hisq;

extern "C" {

hisq_status hisq_eigensolve(hisq_ctx *ctx, const hisq_eig_params *params, int *n_conv, double *eps_out)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!params) return set_err(ctx, HISQ_ERR_INVALID_ARG, "null params");
    if (!ctx->links_loaded) return set_err(ctx, HISQ_ERR_STATE, "links not loaded");
    HISQ_CUDA(cudaSetDevice(ctx->device));
    return trlm(ctx, params, n_conv, eps_out);
}

hisq_status hisq_get_eigvals(hisq_ctx *ctx, int *n_ev, double *eps_out)
{
    if (!ctx || !n_ev) return HISQ_ERR_INVALID_ARG;
    *n_ev = ctx->eig.n;
    if (eps_out)
        for (int i = 0; i < ctx->eig.n; i++) eps_out[i] = ctx->eig.eps[i];
    return HISQ_OK;
}

hisq_status hisq_get_eigvec(hisq_ctx *ctx, int i, double *out)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!out || i < 0 || i >= ctx->eig.n) return set_err(ctx, HISQ_ERR_INVALID_ARG, "eigenvector index out of range");
    HISQ_CUDA(cudaSetDevice(ctx->device));
    const int Vh = ctx->g.Vh;
    const size_t full = size_t(ctx->g.V) * 48;
    double *f = (double *)get_buf(ctx, BUF_ETA_FULL, full);
    if (!f) return HISQ_ERR_OOM;
    HISQ_CUDA(cudaMemsetAsync(f, 0, full, ctx->stream));
    TRY(launch_scatter_parity(ctx, (const char *)ctx->eig.vecs + spinor_bytes(ctx->eig.prec, Vh) * i, ctx->eig.prec, 0, f));
    HISQ_CUDA(cudaMemcpyAsync(out, f, full, cudaMemcpyDeviceToHost, ctx->stream));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return HISQ_OK;
}

hisq_status hisq_set_eigvecs(hisq_ctx *ctx, int n, const double *vecs, const double *eps, int storage_precision)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && !vecs)) return set_err(ctx, HISQ_ERR_INVALID_ARG, "bad eigenvector arguments");
    if (storage_precision != 32 && storage_precision != 16 && storage_precision != HISQ_PREC_BF16 &&
        storage_precision != HISQ_PREC_HALF_EV)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "storage_precision must be 32, 16, 15 (BF16) or 14 (FP16 x 2^e)");
    if (!eps && !ctx->links_loaded) return set_err(ctx, HISQ_ERR_STATE, "links needed to recompute eigenvalues");
    HISQ_CUDA(cudaSetDevice(ctx->device));
    const int Vh = ctx->g.Vh;
    const size_t full = size_t(ctx->g.V) * 48, sf = spinor_bytes(32, Vh);
    double *f = (double *)get_buf(ctx, BUF_ETA_FULL, full);
    char *tmp = (char *)dev_alloc(ctx, sf * (n > 0 ? n : 1));
    if (!f || !tmp) return HISQ_ERR_OOM;
    hisq_status st = HISQ_OK;
    for (int i = 0; i < n && st == HISQ_OK; i++) {
        cudaError_t e = cudaMemcpyAsync(f, vecs + size_t(i) * ctx->g.V * 6, full, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) st = cuda_err(ctx, e, "eigenvector upload");
        if (st == HISQ_OK) st = launch_gather_parity(ctx, f, 0, 32, tmp + sf * i);
    }
    if (st == HISQ_OK) st = store_eigvecs(ctx, n, tmp, storage_precision, eps, nullptr);
    cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, tmp, sf * (n > 0 ? n : 1));
    return st;
}

hisq_status hisq_deflate(hisq_ctx *ctx, int n, const double *b, double *x)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!b || !x) return set_err(ctx, HISQ_ERR_INVALID_ARG, "null field");
    if (ctx->eig.n <= 0) return set_err(ctx, HISQ_ERR_STATE, "no eigenpairs stored");
    if (!(ctx->mass > 0)) return set_err(ctx, HISQ_ERR_STATE, "mass not set");
    if (n <= 0 || n > ctx->eig.n) n = ctx->eig.n;
    HISQ_CUDA(cudaSetDevice(ctx->device));
    const int Vh = ctx->g.Vh;
    const size_t full = size_t(ctx->g.V) * 48;
    double *f = (double *)get_buf(ctx, BUF_ETA_FULL, full);
    double *be = (double *)get_buf(ctx, BUF_ETA_E, spinor_bytes(64, Vh));
    double *xe = (double *)get_buf(ctx, BUF_XHI, spinor_bytes(64, Vh));
    if (!f || !be || !xe) return HISQ_ERR_OOM;
    HISQ_CUDA(cudaMemcpyAsync(f, b, full, cudaMemcpyHostToDevice, ctx->stream));
    TRY(launch_gather_parity(ctx, f, 0, 64, be));
    HISQ_CUDA(cudaMemsetAsync(xe, 0, spinor_bytes(64, Vh), ctx->stream));
    TRY(deflate_add(ctx, n, be, xe));
    HISQ_CUDA(cudaMemsetAsync(f, 0, full, ctx->stream));
    TRY(launch_scatter_parity(ctx, xe, 64, 0, f));
    HISQ_CUDA(cudaMemcpyAsync(x, f, full, cudaMemcpyDeviceToHost, ctx->stream));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return HISQ_OK;
}

hisq_status hisq_save_eigvecs(hisq_ctx *ctx, const char *path)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!path) return set_err(ctx, HISQ_ERR_INVALID_ARG, "null path");
    if (ctx->eig.n <= 0) return set_err(ctx, HISQ_ERR_STATE, "no eigenpairs stored");
    HISQ_CUDA(cudaSetDevice(ctx->device));
    const size_t bpv = spinor_bytes(ctx->eig.prec, ctx->g.Vh);
    std::vector<unsigned char> host(bpv * ctx->eig.n);
    HISQ_CUDA(cudaMemcpy(host.data(), ctx->eig.vecs, host.size(), cudaMemcpyDeviceToHost));
    EigFileHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "HISQEIG1", 8);
    h.dims[0] = ctx->g.X;
    h.dims[1] = ctx->g.Y;
    h.dims[2] = ctx->g.Z;
    h.dims[3] = ctx->g.T;
    h.n = ctx->eig.n;
    h.prec = ctx->eig.prec;
    h.bytes_per_vec = int64_t(bpv);
    h.checksum = fnv1a(host.data(), host.size(), 1469598103934665603ull);
    FILE *fp = fopen(path, "wb");
    if (!fp) return set_err(ctx, HISQ_ERR_INVALID_ARG, "cannot open %s for writing", path);
    bool ok = fwrite(&h, sizeof h, 1, fp) == 1 && fwrite(ctx->eig.eps.data(), sizeof(double), h.n, fp) == size_t(h.n) &&
              fwrite(host.data(), 1, host.size(), fp) == host.size();
    ok = (fclose(fp) == 0) && ok;
    return ok ? HISQ_OK : set_err(ctx, HISQ_ERR_INVALID_ARG, "write to %s failed", path);
}

hisq_status hisq_load_eigvecs(hisq_ctx *ctx, const char *path)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!path) return set_err(ctx, HISQ_ERR_INVALID_ARG, "null path");
    if (!ctx->links_loaded) return set_err(ctx, HISQ_ERR_STATE, "links needed to recompute eigenvalues");
    HISQ_CUDA(cudaSetDevice(ctx->device));
    FILE *fp = fopen(path, "rb");
    if (!fp) return set_err(ctx, HISQ_ERR_INVALID_ARG, "cannot open %s", path);
    EigFileHeader h;
    bool ok = fread(&h, sizeof h, 1, fp) == 1 && memcmp(h.magic, "HISQEIG1", 8) == 0;
    const int Vh = ctx->g.Vh;
    ok = ok && h.dims[0] == ctx->g.X && h.dims[1] == ctx->g.Y && h.dims[2] == ctx->g.Z && h.dims[3] == ctx->g.T &&
         (h.prec == 32 || h.prec == 16 || h.prec == HISQ_PREC_BF16 || h.prec == HISQ_PREC_HALF_EV) && h.n > 0 && h.bytes_per_vec == int64_t(spinor_bytes(h.prec, Vh));
    if (!ok) {
        fclose(fp);
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "%s: bad header or lattice mismatch", path);
    }
    std::vector<double> eps(h.n);
    std::vector<unsigned char> host(size_t(h.bytes_per_vec) * h.n);
    ok = fread(eps.data(), sizeof(double), h.n, fp) == size_t(h.n) && fread(host.data(), 1, host.size(), fp) == host.size();
    fclose(fp);
    if (!ok) return set_err(ctx, HISQ_ERR_INVALID_ARG, "%s: truncated file", path);
    if (fnv1a(host.data(), host.size(), 1469598103934665603ull) != h.checksum)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "%s: checksum mismatch", path);
    // convert to FP32 staging, recompute eigenvalues (FP64 Rayleigh quotients), store
    const size_t sf = spinor_bytes(32, Vh), sp = size_t(h.bytes_per_vec);
    char *raw = (char *)dev_alloc(ctx, host.size());
    char *f32 = (char *)dev_alloc(ctx, sf * h.n);
    if (!raw || !f32) {
        dev_free(ctx, raw, host.size());
        dev_free(ctx, f32, sf * h.n);
        return HISQ_ERR_OOM;
    }
    hisq_status st = HISQ_OK;
    cudaError_t e = cudaMemcpyAsync(raw, host.data(), host.size(), cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) st = cuda_err(ctx, e, "eigenvector upload");
    for (int i = 0; i < h.n && st == HISQ_OK; i++) st = launch_convert(ctx, raw + sp * i, h.prec, f32 + sf * i, 32);
    if (st == HISQ_OK) st = store_eigvecs(ctx, h.n, f32, h.prec, nullptr, nullptr);
    cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, raw, host.size());
    dev_free(ctx, f32, sf * h.n);
    return st;
}

} // extern "C"
