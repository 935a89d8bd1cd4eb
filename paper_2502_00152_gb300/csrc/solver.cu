// solver.cu -- the propagator solve of Sections 2 and 3 of the paper:
//   y_e = (M^dag eta)_e = 2m eta_e - D_eo eta_o
//   x_e = V Lambda^-1 V^dag y_e                       (deflated guess, Eq. 4)
//   CG on (M^dag M)_ee x_e = y_e in sloppy precision with FP64 reliable updates
//     (or double-float ones, certified in FP64 before convergence is reported)
//     (|r| < delta_rd |r_last|, delta_rd = 0.1) and re-deflation
//     (|r| < delta_tr |r_defl|, delta_tr = 1e-3)
//   psi_o = (eta_o - D_oe psi_e) / (2m)
// The host drives the iterations with a one-iteration lag: it queues iteration
// k and only then reads the residual of iteration k-1 from mapped memory, so the
// GPU never idles waiting for the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace hisq {

double *eig_eps_dev(hisq_ctx *ctx);
hisq_status read_slots(hisq_ctx *ctx, int slot0, int n, double *out);

#define TRY(x)                                  \
    do {                                        \
        hisq_status s_ = (x);                   \
        if (s_ != HISQ_OK) return s_;           \
    } while (0)

// force a reliable update when the sloppy residual has not triggered one for
// this many iterations (it can stall when the sloppy operator is too coarse)
constexpr long long kMaxItersBetweenUpdates = 1000;

enum Slot { SL_YNORM = 0, SL_ETAE = 1, SL_ETAO = 2, SL_RHI = 3, SL_RE = 4, SL_RO = 5, SL_PP = 6 };

// r = b - A x  (FP64 operator, A = 4m^2 - D_eo D_oe), |r|^2 -> slot
static hisq_status residual_hi(hisq_ctx *ctx, const double *b, const double *x, double *r, double *tmp_odd, int slot)
{
    const double m4 = 4.0 * ctx->mass * ctx->mass;
    TRY(launch_dslash(ctx, 1, 64, 64, x, tmp_odd, 0, nullptr, 0, nullptr, 1.0, -1));
    return launch_dslash(ctx, 0, 64, 64, tmp_odd, r, -m4, x, 1.0, b, 1.0, slot);
}

// the reliable-update residual r = b - A x in FP64 or, with df, in
// double-float arithmetic on the FP32 units (df64.cu)
hisq_status residual_rel(hisq_ctx *ctx, bool df, const double *b, const double *x, double *r, double *tmp_odd,
                         int slot)
{
    return df ? launch_residual_df(ctx, b, x, r, slot) : residual_hi(ctx, b, x, r, tmp_odd, slot);
}

// Odd reconstruction from t = D_oe psi_e already computed in FP64 (left by the
// last FP64 residual b - A x taken on the final x): psi_o = (eta_o - t) / (2m)
hisq_status odd_from_t(hisq_ctx *ctx, double m, const double *eta_o, const double *t, double *psi_o)
{
    HISQ_CUDA(cudaMemcpyAsync(psi_o, t, spinor_bytes(64, ctx->g.Vh), cudaMemcpyDeviceToDevice, ctx->stream));
    return launch_scale_axpby_d(ctx, 1.0 / (2.0 * m), eta_o, -1.0 / (2.0 * m), psi_o);
}

// odd part of the full residual, r_o = eta_o - 2m psi_o - D_oe psi_e, from the
// same t, written over t; |r_o|^2 -> slot
hisq_status odd_residual_from_t(hisq_ctx *ctx, double m, const double *eta_o, const double *psi_o, double *t, int slot)
{
    TRY(launch_scale_axpby_d(ctx, 1.0, eta_o, -1.0, t));
    TRY(launch_axpy_d(ctx, -2.0 * m, psi_o, 64, t));
    return launch_norm2(ctx, 64, t, slot);
}

// x += V Lambda^-1 V^dag r over the first n stored eigenpairs (Eq. 4)
hisq_status deflate_add(hisq_ctx *ctx, int n, const double *r, double *x)
{
    double *eps = eig_eps_dev(ctx);
    double *c = (double *)get_buf(ctx, BUF_DEFL_C, sizeof(double) * 2 * (n > 0 ? n : 1));
    if (!eps || !c) return set_err(ctx, HISQ_ERR_OOM, "deflation buffers");
    TRY(launch_defl_project(ctx, n, ctx->eig.prec, ctx->eig.vecs, 64, r, c));
    TRY(launch_defl_scale(ctx, n, c, eps, 4.0 * ctx->mass * ctx->mass));
    return launch_defl_expand(ctx, n, ctx->eig.prec, ctx->eig.vecs, c, 1.0, 64, x);
}

hisq_status launch_defl_expand2(hisq_ctx *ctx, int n, int vprec, const void *V, const double *c_dev,
                                const double *eps_dev, double shift, double *x, double *r);

// Deflation step on the pair (x, r = b - A x): c = V^dag r, x += V Lambda^-1 c,
// r -= V c (Eq. 4 applied to the current residual).  The new residual follows
// from A v_i = lambda_i v_i of the stored pairs instead of an FP64 operator
// application; the next reliable update recomputes it exactly.  |r|^2 -> slot.
static hisq_status deflate_pair(hisq_ctx *ctx, int n, bool df, const double *b, double *r, double *x, double *t_odd,
                                int slot)
{
    // beyond the fused kernel, or with FP16 eigenvectors (whose rounding, divided
    // by small lambda_i, breaks A V Lambda^-1 c = V c): x update, then the
    // reliable-update residual
    if (n > 4096 || ctx->eig.prec != 32) {
        TRY(deflate_add(ctx, n, r, x));
        return residual_rel(ctx, df, b, x, r, t_odd, slot);
    }
    double *eps = eig_eps_dev(ctx);
    double *c = (double *)get_buf(ctx, BUF_DEFL_C, sizeof(double) * 2 * (n > 0 ? n : 1));
    if (!eps || !c) return set_err(ctx, HISQ_ERR_OOM, "deflation buffers");
    TRY(launch_defl_project(ctx, n, ctx->eig.prec, ctx->eig.vecs, 64, r, c));
    TRY(launch_defl_expand2(ctx, n, ctx->eig.prec, ctx->eig.vecs, c, eps, 4.0 * ctx->mass * ctx->mass, x, r));
    return launch_norm2(ctx, 64, r, slot);
}

struct HostScalars {
    double rr, pp, m4;
    long long iter;
};

static hisq_status set_scalars(hisq_ctx *ctx, const HostScalars &h)
{
    DevScalars s;
    memset(&s, 0, sizeof s);
    s.rr = h.rr;
    s.pp = h.pp;
    s.m4 = h.m4;
    s.iter = h.iter;
    HISQ_CUDA(cudaMemcpyAsync(ctx->scal, &s, offsetof(DevScalars, slot), cudaMemcpyHostToDevice, ctx->stream));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return HISQ_OK;
}

// CG with reliable updates and re-deflation on one right-hand side.
// b, x: FP64 even fields; x holds the initial guess on entry.
// With double-float reliable updates the FP64 confirmation of a converged
// residual is the even part of the full residual: t = D_oe x,
// psi_o = (eta_o - t) / 2m, r_e = eta_e - 2m x - D_eo psi_o, and y - A x = 2m r_e
// (exact reconstruction), so it also leaves psi_o and |r_e|^2 (*re2_final >= 0)
// for the caller.
static hisq_status cg_reliable(hisq_ctx *ctx, const hisq_solve_params *P, const double *b, double *x, double target,
                               int n_defl, double rn0, hisq_solve_stats *st, double *rfinal, double *defl_seconds,
                               bool *t_final, const double *eta_e, const double *eta_o, double *psi_o,
                               double *re2_final)
{
    const double m = ctx->mass;
    const int Vh = ctx->g.Vh;
    const int prec = P->precision_sloppy;
    const int lprec = prec == 64 ? 64 : P->link_precision_sloppy;
    const int xprec = prec == 64 ? 64 : 32;
    double *r_hi = (double *)get_buf(ctx, BUF_RHI, spinor_bytes(64, Vh));
    double *t_hi = (double *)get_buf(ctx, BUF_TMPHI, spinor_bytes(64, Vh));
    void *x_sl = get_buf(ctx, BUF_XSL, spinor_bytes(xprec, Vh));
    void *r_sl = get_buf(ctx, BUF_RSL, spinor_bytes(prec, Vh));
    void *p = get_buf(ctx, BUF_P, spinor_bytes(prec, Vh));
    void *tmp = get_buf(ctx, BUF_TMP, spinor_bytes(prec, Vh));
    if (!r_hi || !t_hi || !x_sl || !r_sl || !p || !tmp) return HISQ_ERR_OOM;

    double rt = rn0; // true residual norm, r_hi holds b - A x
    // double-float reliable updates; a residual that meets the target is
    // recomputed in FP64 first, and if FP64 does not confirm it the rest of the
    // solve stays on FP64 residuals
    bool use_df = P->precision_reliable == HISQ_PREC_DF64;
    // t_hi = D_oe x for the current x (left by an FP64 residual)
    bool t_ok = false;
    // psi_o and |r_e|^2 of the full residual for the current x (left by a confirmation)
    bool fin_ok = false;
    double re2_fin = -1;
    *t_final = false;
    *re2_final = -1;
    auto certify = [&]() -> hisq_status {
        if (!use_df || rt > target) return HISQ_OK;
        TRY(launch_dslash(ctx, 1, 64, 64, x, t_hi, 0, nullptr, 0, nullptr, 1.0, -1));
        TRY(odd_from_t(ctx, m, eta_o, t_hi, psi_o));
        TRY(launch_dslash(ctx, 0, 64, 64, psi_o, r_hi, -2.0 * m, x, 1.0, eta_e, -1.0, SL_RHI));
        double re2 = 0;
        TRY(read_slots(ctx, SL_RHI, 1, &re2));
        rt = 2.0 * m * std::sqrt(re2);
        t_ok = fin_ok = true;
        re2_fin = re2;
        if (!(rt <= target)) {
            // not confirmed: r_hi = 2m r_e = b - A x, and FP64 residuals from here
            HISQ_CUDA(cudaMemcpyAsync(t_hi, r_hi, spinor_bytes(64, Vh), cudaMemcpyDeviceToDevice, ctx->stream));
            TRY(launch_scale_axpby_d(ctx, 0.0, t_hi, 2.0 * m, r_hi));
            t_ok = fin_ok = false;
            use_df = false;
            if (log_level() > 0) fprintf(stderr, "[hisq] FP64 residual %.4e does not confirm; FP64 from here\n", rt);
        }
        return HISQ_OK;
    };

    TRY(certify());
    *rfinal = rt;
    if (rt <= target) {
        st->converged = 1;
        *t_final = t_ok;
        *re2_final = fin_ok ? re2_fin : -1;
        return HISQ_OK;
    }
    const double m4 = 4.0 * ctx->mass * ctx->mass;
    TRY(launch_convert(ctx, r_hi, 64, r_sl, prec));
    TRY(launch_convert(ctx, r_hi, 64, p, prec));
    TRY(launch_zero(ctx, x_sl, xprec));
    TRY(set_scalars(ctx, HostScalars{rt * rt, rt * rt, m4, 0}));

    cudaEvent_t ev[2], d0, d1;
    HISQ_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    HISQ_CUDA(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    HISQ_CUDA(cudaEventCreate(&d0));
    HISQ_CUDA(cudaEventCreate(&d1));
    struct Cleanup {
        cudaEvent_t *e;
        ~Cleanup()
        {
            for (int i = 0; i < 4; i++) cudaEventDestroy(e[i]);
        }
    };
    cudaEvent_t all[4] = {ev[0], ev[1], d0, d1};
    Cleanup cleanup{all};
    // optional kernel timing: ring of 4 iterations x 3 events
    const bool prof = ctx->profile;
    cudaEvent_t pe[4][3] = {};
    struct ProfFree {
        cudaEvent_t (*e)[3];
        ~ProfFree()
        {
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 3; j++)
                    if (e[i][j]) cudaEventDestroy(e[i][j]);
        }
    } prof_free{pe};
    if (prof)
        for (int i = 0; i < 4; i++)
            for (int j = 0; j < 3; j++) HISQ_CUDA(cudaEventCreate(&pe[i][j]));
    long long retired = 0;
    auto retire = [&](long long n_done) {
        if (!prof) return;
        for (; retired < n_done; retired++) {
            float a = 0, b = 0;
            cudaEvent_t *e = pe[retired & 3];
            if (cudaEventElapsedTime(&a, e[0], e[1]) == cudaSuccess && cudaEventElapsedTime(&b, e[1], e[2]) == cudaSuccess) {
                st->seconds_dslash_oe += a * 1e-3;
                st->seconds_dslash_eo += b * 1e-3;
                st->profiled_iterations++;
            }
        }
    };

    IterGraphs graphs;
    double r_last = rt, r_defl = rt;
    double r_best = rt, rn_last_seen = rt;
    int no_progress = 0; // reliable updates in a row without halving the best true residual
    long long last_update_it = 0;
    long long k = 0, checked = 0;
    const long long maxit = P->max_iter > 0 ? P->max_iter : 1;
    hisq_status result = HISQ_ERR_NOT_CONVERGED;
    for (;;) {
        bool force = false;
        if (k < maxit) {
            const int slot = int(k & 3);
            auto iteration = [&](bool cap) -> hisq_status {
                if (prof) HISQ_CUDA(record_event(ctx, pe[slot][0], cap));
                TRY(launch_cg_dslash_tt(ctx, prec, lprec, p, tmp));
                if (prof) HISQ_CUDA(record_event(ctx, pe[slot][1], cap));
                TRY(launch_cg_dslash_update(ctx, prec, lprec, xprec, tmp, p, x_sl, r_sl));
                if (prof) HISQ_CUDA(record_event(ctx, pe[slot][2], cap));
                TRY(launch_cg_p_update(ctx, prec, r_sl, p));
                HISQ_CUDA(record_event(ctx, ev[slot & 1], cap));
                return HISQ_OK;
            };
            // the first iterations run directly (lazy kernel set-up happens outside capture)
            if (k < 4) {
                TRY(iteration(false));
            } else {
                TRY(graph_run(ctx, graphs, slot, 0, iteration));
            }
            k++;
        } else {
            force = true;
        }
        bool update = force;
        const long long j = k - 2; // the iteration before the one just queued
        if (!force && j >= checked) {
            HISQ_CUDA(cudaEventSynchronize(ev[j & 1]));
            const double rr = ctx->monitor_h[j % ctx->monitor_len];
            if (!std::isfinite(rr)) {
                cudaStreamSynchronize(ctx->stream);
                st->iterations = int(k);
                return set_err(ctx, HISQ_ERR_NUMERICAL, "non-finite residual at iteration %lld", j);
            }
            const double rn = std::sqrt(rr);
            rn_last_seen = rn;
            // a sloppy residual that grows far above the last true one means the
            // sloppy recurrence has lost contact: replace it now
            if (rn < target || rn < P->delta_rd * r_last || rn > 1e3 * r_last) update = true;
            // a sloppy residual that stops falling also needs the true one
            if (j - last_update_it >= kMaxItersBetweenUpdates) update = true;
            checked = j + 1;
            retire(j + 1);
        }
        if (!update) continue;
        // ---- reliable update: x_hi += x_sl; r_hi = b - A x_hi in FP64 (or double-float)
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
        retire(k);
        TRY(launch_axpy_d(ctx, 1.0, x_sl, xprec, x));
        TRY(residual_rel(ctx, use_df, b, x, r_hi, t_hi, SL_RHI));
        t_ok = !use_df;
        fin_ok = false;
        double r2 = 0;
        TRY(read_slots(ctx, SL_RHI, 1, &r2));
        if (!std::isfinite(r2)) return set_err(ctx, HISQ_ERR_NUMERICAL, "non-finite true residual");
        if (log_level() > 1)
            fprintf(stderr, "[hisq] cg it %lld: iterated |r| %.4e\n", k, rn_last_seen);
        rt = std::sqrt(r2);
        TRY(certify());
        st->reliable_updates++;
        checked = k;
        last_update_it = k;
        if (log_level() > 0)
            fprintf(stderr, "[hisq] cg it %lld: reliable update, true |r| %.4e (target %.4e)\n", k, rt, target);
        if (rt <= target) {
            result = HISQ_OK;
            break;
        }
        if (force) break;
        // stagnation: the sloppy operator is too far from the FP64 one for this
        // spectrum (its error exceeds the smallest eigenvalue); give up cleanly
        if (rt < 0.5 * r_best) {
            r_best = rt;
            no_progress = 0;
        } else if (++no_progress >= 8) {
            set_err(ctx, HISQ_ERR_NOT_CONVERGED, "stagnation: %d reliable updates without progress (true |r| %.3e)",
                    no_progress, rt);
            break;
        }
        // restart the search direction when the true residual is far from the
        // iterated one (the kept direction would no longer be conjugate)
        bool restart = rt > 10.0 * rn_last_seen;
        if (n_defl > 0 && P->delta_tr > 0 && rt < P->delta_tr * r_defl) {
            HISQ_CUDA(cudaEventRecord(d0, ctx->stream));
            TRY(deflate_pair(ctx, n_defl, use_df, b, r_hi, x, t_hi, SL_RHI));
            t_ok = fin_ok = false;
            HISQ_CUDA(cudaEventRecord(d1, ctx->stream));
            TRY(read_slots(ctx, SL_RHI, 1, &r2));
            float ms = 0;
            cudaEventElapsedTime(&ms, d0, d1);
            *defl_seconds += ms * 1e-3;
            rt = std::sqrt(r2);
            r_defl = rt;
            st->redeflations++;
            restart = true;
            TRY(certify());
            if (rt <= target) {
                result = HISQ_OK;
                break;
            }
        }
        TRY(launch_convert(ctx, r_hi, 64, r_sl, prec));
        TRY(launch_zero(ctx, x_sl, xprec));
        double pp = -1;
        if (restart) {
            TRY(launch_convert(ctx, r_hi, 64, p, prec));
            pp = rt * rt;
        } else {
            TRY(launch_norm2(ctx, prec, p, SL_PP));
            TRY(read_slots(ctx, SL_PP, 1, &pp));
        }
        TRY(set_scalars(ctx, HostScalars{rt * rt, pp, m4, k}));
        r_last = rt;
    }
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    retire(k);
    st->iterations = int(k);
    st->converged = result == HISQ_OK;
    *rfinal = rt;
    *t_final = t_ok;
    *re2_final = fin_ok ? re2_fin : -1;
    return result;
}

// Solve M psi = eta for one right-hand side; eta, psi: FP64 full-lattice device fields.
hisq_status solve_one(hisq_ctx *ctx, const hisq_solve_params *P, const double *eta, double *psi, hisq_solve_stats *st)
{
    const int Vh = ctx->g.Vh;
    const double m = ctx->mass;
    memset(st, 0, sizeof *st);
    st->full_residual = -1;
    auto t0 = std::chrono::steady_clock::now();
    double *eta_e = (double *)get_buf(ctx, BUF_ETA_E, spinor_bytes(64, Vh));
    double *eta_o = (double *)get_buf(ctx, BUF_ETA_O, spinor_bytes(64, Vh));
    double *y = (double *)get_buf(ctx, BUF_Y, spinor_bytes(64, Vh));
    double *x = (double *)get_buf(ctx, BUF_XHI, spinor_bytes(64, Vh));
    double *r_hi = (double *)get_buf(ctx, BUF_RHI, spinor_bytes(64, Vh));
    double *t_hi = (double *)get_buf(ctx, BUF_TMPHI, spinor_bytes(64, Vh));
    double *psi_o = (double *)get_buf(ctx, BUF_PSI_O, spinor_bytes(64, Vh));
    if (!eta_e || !eta_o || !y || !x || !r_hi || !t_hi || !psi_o) return HISQ_ERR_OOM;

    // (a2) source preparation
    TRY(launch_gather_parity(ctx, eta, 0, 64, eta_e));
    TRY(launch_gather_parity(ctx, eta, 1, 64, eta_o));
    TRY(launch_norm2(ctx, 64, eta_e, SL_ETAE));
    TRY(launch_norm2(ctx, 64, eta_o, SL_ETAO));
    TRY(launch_dslash(ctx, 0, 64, 64, eta_o, y, 2.0 * m, eta_e, 0, nullptr, -1.0, SL_YNORM));
    double nrm[3];
    TRY(read_slots(ctx, SL_YNORM, 3, nrm));
    const double ynorm = std::sqrt(nrm[0]), etanorm = std::sqrt(nrm[1] + nrm[2]);
    if (!std::isfinite(ynorm) || !std::isfinite(etanorm)) return set_err(ctx, HISQ_ERR_NUMERICAL, "non-finite source");
    HISQ_CUDA(cudaMemsetAsync(x, 0, spinor_bytes(64, Vh), ctx->stream));
    if (etanorm == 0) {
        HISQ_CUDA(cudaMemsetAsync(psi, 0, size_t(ctx->g.V) * 48, ctx->stream));
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
        st->converged = 1;
        st->full_residual = 0;
        return HISQ_OK;
    }
    const double target = P->tol * std::fmin(ynorm, 2.0 * m * etanorm);

    // (a8) deflated initial guess
    int n_defl = 0;
    if (P->deflate) {
        if (ctx->eig.n <= 0) return set_err(ctx, HISQ_ERR_STATE, "deflation requested but no eigenpairs stored");
        n_defl = P->n_defl > 0 ? std::min(P->n_defl, ctx->eig.n) : ctx->eig.n;
    }
    double defl_s = 0;
    // x = 0 (or the caller's guess), r = y - A x; with deflation
    // x += V Lambda^-1 V^dag r, r -= V V^dag r
    double r2 = nrm[0];
    if (P->guess) {
        TRY(launch_gather_parity(ctx, psi, 0, 64, x));
        TRY(residual_hi(ctx, y, x, r_hi, t_hi, SL_RHI));
        TRY(read_slots(ctx, SL_RHI, 1, &r2));
    } else {
        HISQ_CUDA(cudaMemcpyAsync(r_hi, y, spinor_bytes(64, Vh), cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (n_defl > 0) {
        auto d0 = std::chrono::steady_clock::now();
        TRY(deflate_pair(ctx, n_defl, P->precision_reliable == HISQ_PREC_DF64, y, r_hi, x, t_hi, SL_RHI));
        TRY(read_slots(ctx, SL_RHI, 1, &r2));
        defl_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - d0).count();
    }

    // (a6) CG with reliable updates
    double rfin = 0;
    bool t_final = false;
    double re2_final = -1;
    hisq_status cst = cg_reliable(ctx, P, y, x, target, n_defl, std::sqrt(r2), st, &rfin, &defl_s, &t_final, eta_e,
                                  eta_o, psi_o, &re2_final);
    if (cst != HISQ_OK && cst != HISQ_ERR_NOT_CONVERGED) return cst;
    st->even_residual = ynorm > 0 ? rfin / ynorm : 0;

    // (a9) odd reconstruction psi_o = (eta_o - D_oe psi_e) / (2m); D_oe psi_e
    // is reused when the last FP64 residual computed it on the final x, and
    // an FP64 confirmation has already formed psi_o and r_e
    const bool fin = re2_final >= 0;
    if (fin) {
        // psi_o is in place
    } else if (t_final) {
        TRY(odd_from_t(ctx, m, eta_o, t_hi, psi_o));
    } else {
        TRY(launch_dslash(ctx, 1, 64, 64, x, psi_o, 1.0 / (2.0 * m), eta_o, 0, nullptr, -1.0 / (2.0 * m), -1));
    }
    if (P->compute_full_residual) {
        // r_e = eta_e - 2m psi_e - D_eo psi_o ; r_o = eta_o - 2m psi_o - D_oe psi_e
        double re2 = re2_final, ro2 = 0;
        if (!fin) {
            TRY(launch_dslash(ctx, 0, 64, 64, psi_o, r_hi, -2.0 * m, x, 1.0, eta_e, -1.0, SL_RE));
            TRY(read_slots(ctx, SL_RE, 1, &re2));
        }
        if (t_final) {
            TRY(odd_residual_from_t(ctx, m, eta_o, psi_o, t_hi, SL_RO));
        } else {
            TRY(launch_dslash(ctx, 1, 64, 64, x, t_hi, -2.0 * m, psi_o, 1.0, eta_o, -1.0, SL_RO));
        }
        TRY(read_slots(ctx, SL_RO, 1, &ro2));
        st->full_residual = std::sqrt(re2 + ro2) / etanorm;
    }
    TRY(launch_scatter_parity(ctx, x, 64, 0, psi));
    TRY(launch_scatter_parity(ctx, psi_o, 64, 1, psi));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    st->seconds_deflate = defl_s;
    st->seconds_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return cst;
}

static hisq_status check_solve_args(hisq_ctx *ctx, const hisq_solve_params *P, int nrhs)
{
    if (!P || nrhs < 0) return set_err(ctx, HISQ_ERR_INVALID_ARG, "bad solve arguments");
    if (!ctx->links_loaded) return set_err(ctx, HISQ_ERR_STATE, "links not loaded");
    if (!(ctx->mass > 0)) return set_err(ctx, HISQ_ERR_STATE, "mass not set");
    if (P->precision_sloppy != 64 && P->precision_sloppy != 32 && P->precision_sloppy != 16)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "precision_sloppy must be 64, 32 or 16");
    if (P->precision_sloppy != 64 && P->link_precision_sloppy != 32 && P->link_precision_sloppy != 16)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "link_precision_sloppy must be 32 or 16");
    if (!(P->tol > 0) || !(P->delta_rd > 0 && P->delta_rd < 1) || P->delta_tr < 0 || P->delta_tr >= 1)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "bad tolerance / delta parameters");
    if (P->precision_reliable != 64 && P->precision_reliable != HISQ_PREC_DF64)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "precision_reliable must be 64 or HISQ_PREC_DF64 (48)");
    return HISQ_OK;
}

hisq_status solve_batched(hisq_ctx *ctx, const hisq_solve_params *P, const double *eta, double *psi, int k,
                          hisq_solve_stats *stats);

static bool use_batched(const hisq_solve_params *P, int nrhs)
{
    return P->batch && nrhs > 1 && (P->precision_sloppy == 32 || P->precision_sloppy == 16) &&
           P->link_precision_sloppy == 32;
}

} // namespace hisq

using namespace hisq;

extern "C" {

hisq_status hisq_solve(hisq_ctx *ctx, const double *eta, double *psi, int nrhs, const hisq_solve_params *params,
                       hisq_solve_stats *stats)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!eta || !psi) return set_err(ctx, HISQ_ERR_INVALID_ARG, "null field");
    TRY(check_solve_args(ctx, params, nrhs));
    ctx->err.clear();
    HISQ_CUDA(cudaSetDevice(ctx->device));
    const size_t bytes = size_t(ctx->g.V) * 48;
    hisq_status worst = HISQ_OK;
    if (use_batched(params, nrhs)) {
        for (int k0 = 0; k0 < nrhs; k0 += kMaxBatch) {
            const int kb = std::min(kMaxBatch, nrhs - k0);
            double *de = (double *)get_buf(ctx, BUF_ETA_FULL, bytes * kb);
            double *dp = (double *)get_buf(ctx, BUF_PSI_FULL, bytes * kb);
            if (!de || !dp) return HISQ_ERR_OOM;
            auto t0 = std::chrono::steady_clock::now();
            HISQ_CUDA(cudaMemcpyAsync(de, eta + size_t(k0) * ctx->g.V * 6, bytes * kb, cudaMemcpyHostToDevice, ctx->stream));
            if (params->guess)
                HISQ_CUDA(cudaMemcpyAsync(dp, psi + size_t(k0) * ctx->g.V * 6, bytes * kb, cudaMemcpyHostToDevice,
                                          ctx->stream));
            hisq_status s = solve_batched(ctx, params, de, dp, kb, stats ? stats + k0 : nullptr);
            if (s != HISQ_OK && s != HISQ_ERR_NOT_CONVERGED) return s;
            HISQ_CUDA(cudaMemcpyAsync(psi + size_t(k0) * ctx->g.V * 6, dp, bytes * kb, cudaMemcpyDeviceToHost, ctx->stream));
            HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
            const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (stats)
                for (int j = 0; j < kb; j++) stats[k0 + j].seconds_total = secs / kb;
            if (s != HISQ_OK) worst = s;
        }
        if (worst != HISQ_OK) {
            const std::string why = ctx->err;
            set_err(ctx, worst, "at least one right-hand side did not converge (%s)", why.c_str());
        }
        return worst;
    }
    double *de = (double *)get_buf(ctx, BUF_ETA_FULL, bytes);
    double *dp = (double *)get_buf(ctx, BUF_PSI_FULL, bytes);
    if (!de || !dp) return HISQ_ERR_OOM;
    for (int k = 0; k < nrhs; k++) {
        hisq_solve_stats st;
        auto t0 = std::chrono::steady_clock::now();
        HISQ_CUDA(cudaMemcpyAsync(de, eta + size_t(k) * ctx->g.V * 6, bytes, cudaMemcpyHostToDevice, ctx->stream));
        if (params->guess)
            HISQ_CUDA(cudaMemcpyAsync(dp, psi + size_t(k) * ctx->g.V * 6, bytes, cudaMemcpyHostToDevice, ctx->stream));
        hisq_status s = solve_one(ctx, params, de, dp, &st);
        if (s != HISQ_OK && s != HISQ_ERR_NOT_CONVERGED) return s;
        HISQ_CUDA(cudaMemcpyAsync(psi + size_t(k) * ctx->g.V * 6, dp, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
        st.seconds_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (stats) stats[k] = st;
        if (s != HISQ_OK) worst = s;
    }
    if (worst != HISQ_OK) {
        const std::string why = ctx->err;
        set_err(ctx, worst, "at least one right-hand side did not converge (%s)", why.c_str());
    }
    return worst;
}

hisq_status hisq_set_profiling(hisq_ctx *ctx, int on)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (on && !ctx->profile) { // the FP64 operator sums restart
        fp64_prof_drain(ctx, true, true);
        ctx->fp64_seconds = 0;
        ctx->fp64_launches = 0;
    }
    ctx->profile = on != 0;
    return HISQ_OK;
}

hisq_status hisq_profiled_fp64(hisq_ctx *ctx, double *seconds, unsigned long long *launches)
{
    if (!ctx || !seconds || !launches) return HISQ_ERR_INVALID_ARG;
    fp64_prof_drain(ctx, true);
    *seconds = ctx->fp64_seconds;
    *launches = ctx->fp64_launches;
    return HISQ_OK;
}

hisq_status hisq_solve_device(hisq_ctx *ctx, const double *eta_dev, double *psi_dev, int nrhs,
                              const hisq_solve_params *params, hisq_solve_stats *stats)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!eta_dev || !psi_dev) return set_err(ctx, HISQ_ERR_INVALID_ARG, "null field");
    TRY(check_solve_args(ctx, params, nrhs));
    ctx->err.clear();
    HISQ_CUDA(cudaSetDevice(ctx->device));
    hisq_status worst = HISQ_OK;
    if (use_batched(params, nrhs)) {
        for (int k0 = 0; k0 < nrhs; k0 += kMaxBatch) {
            const int kb = std::min(kMaxBatch, nrhs - k0);
            hisq_status s = solve_batched(ctx, params, eta_dev + size_t(k0) * ctx->g.V * 6,
                                          psi_dev + size_t(k0) * ctx->g.V * 6, kb, stats ? stats + k0 : nullptr);
            if (s != HISQ_OK && s != HISQ_ERR_NOT_CONVERGED) return s;
            if (s != HISQ_OK) worst = s;
        }
        if (worst != HISQ_OK) {
            const std::string why = ctx->err;
            set_err(ctx, worst, "at least one right-hand side did not converge (%s)", why.c_str());
        }
        return worst;
    }
    for (int k = 0; k < nrhs; k++) {
        hisq_solve_stats st;
        hisq_status s = solve_one(ctx, params, eta_dev + size_t(k) * ctx->g.V * 6, psi_dev + size_t(k) * ctx->g.V * 6, &st);
        if (s != HISQ_OK && s != HISQ_ERR_NOT_CONVERGED) return s;
        if (stats) stats[k] = st;
        if (s != HISQ_OK) worst = s;
    }
    if (worst != HISQ_OK) {
        const std::string why = ctx->err;
        set_err(ctx, worst, "at least one right-hand side did not converge (%s)", why.c_str());
    }
    return worst;
}

} // extern "C"
