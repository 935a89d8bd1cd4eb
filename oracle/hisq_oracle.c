/*
 * hisq_oracle.c -- plain FP64 CPU oracle of the even-odd HISQ propagator solve.
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code with
 * the CUDA library: it is written from the paper's statement of the problem and
 * kept deliberately plain (full-lattice fields, coordinate arithmetic for every
 * neighbour, explicit parity masks, no blocking or fusion) so it can be checked
 * against the paper by eye.
 *
 * Paper: "Improving HISQ propagator solves using deflation", Section 2.
 *   - M = D + 2m with D the anti-Hermitian HISQ Dirac matrix; the factor 2 is
 *     the MILC convention (Section 2, first paragraph).
 *   - CG is run on the normal equation M^dag M psi = M^dag eta (Eq. 1), even-odd
 *     preconditioned: y = M^dag eta, solve (M^dag M)_ee psi_e = y_e, then
 *     reconstruct the odd sites (Section 2, paragraph on MILC/QUDA).
 *   - lambda_min = eps_min + (2 a m)^2 (Eq. 3): the massive normal operator is
 *     the massless one shifted by 4m^2.
 *
 * Readings taken where the paper is silent (each also listed in the design notes):
 *   - D carries no factor 1/2 (so that the free-field lambda_max is
 *     16 (7/6)^2 = 21.8, the paper's "about 23"):
 *       (D psi)(x) = sum_mu eta_mu(x) [ F_mu(x) psi(x+mu) - F_mu(x-mu)^dag psi(x-mu)
 *                                     + L_mu(x) psi(x+3mu) - L_mu(x-3mu)^dag psi(x-3mu) ]
 *     with the HISQ coefficients c1, c3 already folded into F and L.
 *   - Staggered phases eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y),
 *     eta_t = (-1)^(x+y+z); periodic space, and (flag) antiperiodic time: every
 *     hop that crosses from t = T-1 to t = 0 carries a factor -1.
 *   - Odd reconstruction psi_o = (eta_o - D_oe psi_e) / (2m), from the odd rows
 *     of M psi = eta (the paper's printed formula is dimensionally garbled).
 *   - Stopping rule: the recomputed residual |y_e - A psi_e| <= target, where the
 *     caller passes target = tol * min(|y_e|, 2m |eta|); this bounds both
 *     |r|/|b| of Section 3 and the full-system |eta - M psi| / |eta|.
 *
 * Layouts (shared with the C-ABI's host layouts):
 *   site index s = x + X*(y + Y*(z + Z*t)); parity (x+y+z+t) mod 2 (even = 0)
 *   links  [s][mu][row][col] complex (re, im interleaved doubles), mu = x,y,z,t
 *   fields [s][colour] complex over the full lattice.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ---------------------------------------------------------------- geometry */

static long site_of(const int L[4], const int c[4])
{
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

static void coords_of(const int L[4], long s, int c[4])
{
    for (int mu = 0; mu < 4; mu++) {
        c[mu] = (int)(s % L[mu]);
        s /= L[mu];
    }
}

static int parity_of(const int c[4])
{
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

static long volume_of(const int L[4])
{
    return (long)L[0] * L[1] * L[2] * L[3];
}

/* c + d * mu_hat with periodic wrap */
static void shift(const int L[4], const int c[4], int mu, int d, int out[4])
{
    for (int nu = 0; nu < 4; nu++) out[nu] = c[nu];
    out[mu] = ((c[mu] + d) % L[mu] + L[mu]) % L[mu];
}

/* Staggered phase eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}). */
static double staggered_phase(int mu, const int c[4])
{
    int e = 0;
    for (int nu = 0; nu < mu; nu++) e += c[nu];
    return (e & 1) ? -1.0 : 1.0;
}

/* Sign of a forward hop of n steps along mu that starts at c: -1 when it wraps
 * across the time boundary of an antiperiodic lattice. */
static double boundary_sign(int t_antiperiodic, const int L[4], int mu, const int c[4], int n)
{
    if (mu == 3 && t_antiperiodic && c[3] + n >= L[3]) return -1.0;
    return 1.0;
}

/* ------------------------------------------------------- small linear algebra */

static const cplx *link_at(const double *U, long s, int mu)
{
    return (const cplx *)U + (s * 4 + mu) * 9;
}

/* acc += a * W v */
static void add_mat_vec(cplx *acc, double a, const cplx *W, const cplx *v)
{
    for (int i = 0; i < 3; i++) {
        cplx sum = 0;
        for (int j = 0; j < 3; j++) sum += W[3 * i + j] * v[j];
        acc[i] += a * sum;
    }
}

/* acc += a * W^dag v */
static void add_adj_mat_vec(cplx *acc, double a, const cplx *W, const cplx *v)
{
    for (int i = 0; i < 3; i++) {
        cplx sum = 0;
        for (int j = 0; j < 3; j++) sum += conj(W[3 * j + i]) * v[j];
        acc[i] += a * sum;
    }
}

/* ------------------------------------------------------------- the operator */

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* out = D in over the full lattice (Section 2; formula in the header). */
void oracle_dslash(const int L[4], int t_antiperiodic, const double *fat, const double *lng,
                   const double *in, double *out)
{
    const long V = volume_of(L);
    const cplx *psi = (const cplx *)in;
    cplx *res = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        int c[4], n[4];
        cplx acc[3] = {0, 0, 0};
        coords_of(L, s, c);
        for (int mu = 0; mu < 4; mu++) {
            const double eta = staggered_phase(mu, c);
            long sn;
            /* one-hop forward: F_mu(x) psi(x + mu) */
            shift(L, c, mu, +1, n);
            sn = site_of(L, n);
            add_mat_vec(acc, eta * boundary_sign(t_antiperiodic, L, mu, c, 1),
                        link_at(fat, s, mu), psi + 3 * sn);
            /* one-hop backward: - F_mu(x - mu)^dag psi(x - mu) */
            shift(L, c, mu, -1, n);
            sn = site_of(L, n);
            add_adj_mat_vec(acc, -eta * boundary_sign(t_antiperiodic, L, mu, n, 1),
                            link_at(fat, sn, mu), psi + 3 * sn);
            /* three-hop forward: L_mu(x) psi(x + 3 mu) */
            shift(L, c, mu, +3, n);
            sn = site_of(L, n);
            add_mat_vec(acc, eta * boundary_sign(t_antiperiodic, L, mu, c, 3),
                        link_at(lng, s, mu), psi + 3 * sn);
            /* three-hop backward: - L_mu(x - 3 mu)^dag psi(x - 3 mu) */
            shift(L, c, mu, -3, n);
            sn = site_of(L, n);
            add_adj_mat_vec(acc, -eta * boundary_sign(t_antiperiodic, L, mu, n, 3),
                            link_at(lng, sn, mu), psi + 3 * sn);
        }
        for (int i = 0; i < 3; i++) res[3 * s + i] = acc[i];
    }
}

/* out = M in = D in + 2m in (Section 2). */
void oracle_apply_M(const int L[4], int t_antiperiodic, const double *fat, const double *lng,
                    double m, const double *in, double *out)
{
    const long n = 3 * volume_of(L);
    oracle_dslash(L, t_antiperiodic, fat, lng, in, out);
    const cplx *x = (const cplx *)in;
    cplx *y = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) y[i] += 2.0 * m * x[i];
}

/* Keep the sites of parity `keep`, zero the others. */
static void parity_mask(const int L[4], int keep, const cplx *in, cplx *out)
{
    const long V = volume_of(L);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        int c[4];
        coords_of(L, s, c);
        const int on = parity_of(c) == keep;
        for (int i = 0; i < 3; i++) out[3 * s + i] = on ? in[3 * s + i] : 0;
    }
}

/* out = (M^dag M)_ee in = 4m^2 in_e - D_eo D_oe in_e  (Eq. 1, even block).
 * The odd sites of `in` are ignored and those of `out` are zero. */
void oracle_apply_Aee(const int L[4], int t_antiperiodic, const double *fat, const double *lng,
                      double m, const double *in, double *out)
{
    const long n = 3 * volume_of(L);
    cplx *e = malloc(n * sizeof(cplx)), *t1 = malloc(n * sizeof(cplx)),
         *t2 = malloc(n * sizeof(cplx));
    parity_mask(L, 0, (const cplx *)in, e);                            /* in_e        */
    oracle_dslash(L, t_antiperiodic, fat, lng, (double *)e, (double *)t1);
    parity_mask(L, 1, t1, t1);                                         /* D_oe in_e   */
    oracle_dslash(L, t_antiperiodic, fat, lng, (double *)t1, (double *)t2);
    parity_mask(L, 0, t2, t2);                                         /* D_eo D_oe . */
    cplx *y = (cplx *)out;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) y[i] = 4.0 * m * m * e[i] - t2[i];
    free(e);
    free(t1);
    free(t2);
}

/* y_e = (M^dag eta)_e = 2m eta_e - D_eo eta_o  (Section 2, even-odd step). */
void oracle_prepare_source(const int L[4], int t_antiperiodic, const double *fat,
                           const double *lng, double m, const double *eta, double *y)
{
    const long n = 3 * volume_of(L);
    cplx *eo = malloc(n * sizeof(cplx)), *t = malloc(n * sizeof(cplx)),
         *ee = malloc(n * sizeof(cplx));
    parity_mask(L, 1, (const cplx *)eta, eo);
    parity_mask(L, 0, (const cplx *)eta, ee);
    oracle_dslash(L, t_antiperiodic, fat, lng, (double *)eo, (double *)t);
    parity_mask(L, 0, t, t);
    cplx *out = (cplx *)y;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) out[i] = 2.0 * m * ee[i] - t[i];
    free(eo);
    free(t);
    free(ee);
}

/* psi = (psi_e, (eta_o - D_oe psi_e) / (2m)): odd rows of M psi = eta. */
void oracle_reconstruct(const int L[4], int t_antiperiodic, const double *fat,
                        const double *lng, double m, const double *psi_e, const double *eta,
                        double *psi)
{
    const long V = volume_of(L);
    cplx *e = malloc(3 * V * sizeof(cplx)), *t = malloc(3 * V * sizeof(cplx));
    parity_mask(L, 0, (const cplx *)psi_e, e);
    oracle_dslash(L, t_antiperiodic, fat, lng, (double *)e, (double *)t);
    const cplx *h = (const cplx *)eta;
    cplx *out = (cplx *)psi;
#pragma omp parallel for schedule(static)
    for (long s = 0; s < V; s++) {
        int c[4];
        coords_of(L, s, c);
        for (int i = 0; i < 3; i++) {
            const long k = 3 * s + i;
            out[k] = parity_of(c) == 0 ? e[k] : (h[k] - t[k]) / (2.0 * m);
        }
    }
    free(e);
    free(t);
}

/* ------------------------------------------------------------------- CG */

static double norm2(long n, const cplx *a)
{
    double s = 0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (long i = 0; i < n; i++) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

static double re_dot(long n, const cplx *a, const cplx *b)
{
    double s = 0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (long i = 0; i < n; i++) s += creal(conj(a[i]) * b[i]);
    return s;
}

double oracle_norm2(long n, const double *a)
{
    return norm2(n, (const cplx *)a);
}

/*
 * Conjugate gradient on A = (M^dag M)_ee (Eq. 1), Hestenes-Stiefel form, in FP64.
 * x holds the initial guess on entry (0, or the deflated guess of Eq. 4) and the
 * solution on exit.  The iteration stops when the recomputed residual
 * |b - A x| <= rtarget.  Returns 0 on convergence, 1 when maxiter is reached.
 */
int oracle_cg(const int L[4], int t_antiperiodic, const double *fat, const double *lng,
              double m, const double *b_in, double *x_io, double rtarget, int maxiter,
              int *iters_out, double *true_res_out)
{
    const long n = 3 * volume_of(L);
    const cplx *b = (const cplx *)b_in;
    cplx *x = (cplx *)x_io;
    cplx *r = malloc(n * sizeof(cplx)), *p = malloc(n * sizeof(cplx)),
         *Ap = malloc(n * sizeof(cplx));
    int it = 0, status = 1;

    parity_mask(L, 0, x, x);
    oracle_apply_Aee(L, t_antiperiodic, fat, lng, m, (double *)x, (double *)Ap);
    for (long i = 0; i < n; i++) r[i] = b[i] - Ap[i];
    parity_mask(L, 0, r, r);
    double rr = norm2(n, r);
    memcpy(p, r, n * sizeof(cplx));
    if (sqrt(rr) <= rtarget) status = 0;

    while (status != 0 && it < maxiter) {
        oracle_apply_Aee(L, t_antiperiodic, fat, lng, m, (double *)p, (double *)Ap);
        const double alpha = rr / re_dot(n, p, Ap);
        for (long i = 0; i < n; i++) {
            x[i] += alpha * p[i];
            r[i] -= alpha * Ap[i];
        }
        double rr_new = norm2(n, r);
        it++;
        if (sqrt(rr_new) <= rtarget) {
            /* confirm with the recomputed residual */
            oracle_apply_Aee(L, t_antiperiodic, fat, lng, m, (double *)x, (double *)Ap);
            for (long i = 0; i < n; i++) r[i] = b[i] - Ap[i];
            parity_mask(L, 0, r, r);
            rr_new = norm2(n, r);
            if (sqrt(rr_new) <= rtarget) {
                status = 0;
                rr = rr_new;
                break;
            }
            memcpy(p, r, n * sizeof(cplx)); /* restart from the true residual */
            rr = rr_new;
            continue;
        }
        const double beta = rr_new / rr;
        for (long i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
        rr = rr_new;
    }
    /* final recomputed residual */
    oracle_apply_Aee(L, t_antiperiodic, fat, lng, m, (double *)x, (double *)Ap);
    for (long i = 0; i < n; i++) r[i] = b[i] - Ap[i];
    parity_mask(L, 0, r, r);
    if (true_res_out) *true_res_out = sqrt(norm2(n, r));
    if (iters_out) *iters_out = it;
    free(r);
    free(p);
    free(Ap);
    return status;
}

/*
 * Full propagator solve M psi = eta by the even-odd route of Section 2:
 *   y_e = 2m eta_e - D_eo eta_o; CG on A_ee psi_e = y_e from x0_e (NULL = 0);
 *   psi_o = (eta_o - D_oe psi_e) / (2m).
 * The CG target is tol * min(|y_e|, 2m |eta|).  stats[0] = iterations,
 * stats[1] = even-system residual |y_e - A psi_e| / |y_e|,
 * stats[2] = full-system residual |eta - M psi| / |eta|.
 */
int oracle_solve(const int L[4], int t_antiperiodic, const double *fat, const double *lng,
                 double m, const double *eta, const double *x0_e, double tol, int maxiter,
                 double *psi, double *stats)
{
    const long n = 3 * volume_of(L);
    cplx *y = malloc(n * sizeof(cplx)), *x = calloc(n, sizeof(cplx)),
         *r = malloc(n * sizeof(cplx));
    oracle_prepare_source(L, t_antiperiodic, fat, lng, m, eta, (double *)y);
    if (x0_e) memcpy(x, x0_e, n * sizeof(cplx));
    const double ynorm = sqrt(norm2(n, y));
    const double etanorm = sqrt(norm2(n, (const cplx *)eta));
    double target = tol * fmin(ynorm, 2.0 * m * etanorm);
    int iters = 0;
    double res = 0;
    int status = oracle_cg(L, t_antiperiodic, fat, lng, m, (double *)y, (double *)x, target,
                           maxiter, &iters, &res);
    oracle_reconstruct(L, t_antiperiodic, fat, lng, m, (double *)x, eta, psi);
    oracle_apply_M(L, t_antiperiodic, fat, lng, m, psi, (double *)r);
    const cplx *h = (const cplx *)eta;
    for (long i = 0; i < n; i++) r[i] = h[i] - r[i];
    if (stats) {
        stats[0] = iters;
        stats[1] = ynorm > 0 ? res / ynorm : 0;
        stats[2] = etanorm > 0 ? sqrt(norm2(n, r)) / etanorm : 0;
    }
    free(y);
    free(x);
    free(r);
    return status;
}
