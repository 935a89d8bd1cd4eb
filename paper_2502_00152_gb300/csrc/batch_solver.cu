// batch_solver.cu -- several right-hand sides solved together (the paper's
// outlook, Section 4: batched solves raise the arithmetic intensity).
//
// Each right-hand side keeps its own CG recurrence, reliable updates (Section 3,
// delta_rd) and re-deflations (delta_tr); the sloppy operator is applied to all
// active right-hand sides in one batched launch, which reads every link once
// per iteration instead of once per right-hand side.  A right-hand side leaves
// the active set (its slot is removed from the launch list) as soon as its FP64
// true residual meets the tolerance.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include <algorithm>

#include "internal.cuh"

namespace hisq {

double *eig_eps_dev(hisq_ctx *ctx);
hisq_status read_slots(hisq_ctx *ctx, int slot0, int n, double *out);
hisq_status deflate_add(hisq_ctx *ctx, int n, const double *r, double *x);
hisq_status launch_defl_expand2(hisq_ctx *ctx, int n, int vprec, const void *V, const double *c_dev,
                                const double *eps_dev, double shift, double *x, double *r);
hisq_status tc_deflate_batch(hisq_ctx *ctx, int n, int k, double *R, double *X, const double *rnorm, const int *field,
                             bool update_r);

// the tensor-core batched deflation applies to FP32-, BF16- or FP16-stored
// eigenvectors, up to 512 of them and 32 right-hand sides per call; with
// 16-bit storage it also serves a single right-hand side (the GEMMs stream the
// vectors near the HBM rate, and r is updated with the FP32 operator instead of
// recomputing b - A x in FP64)
static bool tc_eligible(const hisq_ctx *ctx, int n, int k)
{
    const bool prec_ok = ctx->eig.prec == 32 || ctx->eig.prec == HISQ_PREC_BF16 || ctx->eig.prec == HISQ_PREC_HALF_EV;
    return prec_ok && n >= 1 && n <= 512 && (k >= 2 || (k == 1 && ctx->eig.prec != 32));
}

// r -= V c is the residual change of x += V Lambda^-1 c only while A v_i =
// lambda_i v_i holds to well below the solve's tolerance.  A rounded vector
// v = v_exact + dv has |A v - lambda v| ~ |A dv| <= lambda_max |dv|: about 5e-2
// for BF16 (|dv| ~ 2e-3, lambda_max ~ 23), far above the low eigenvalues.  For
// 16-bit storage the deflation increment dx is therefore formed on its own and
// the residual updated by r -= A dx with the FP32 operator: dx lies in the low
// modes, so the FP32 error of A dx, ~ 6e-8 |A| |dx| <= 6e-8 (lambda_max /
// lambda_min) |r|, is of the size the FP32-vector update carries anyway, and
// the next FP64 reliable update replaces r with b - A x.
static bool dual_residual(const hisq_ctx *ctx) { return ctx->eig.prec == 32; }

#define TRY(x)                                  \
    do {                                        \
        hisq_status s_ = (x);                   \
        if (s_ != HISQ_OK) return s_;           \
    } while (0)

enum { BS_Y = 0, BS_ETAE = 1, BS_ETAO = 2, BS_R = 3, BS_RE = 4, BS_RO = 5, BS_PP = 6 };

static hisq_status residual_hi_b(hisq_ctx *ctx, const double *b, const double *x, double *r, double *tmp_odd, int slot)
{
    const double m4 = 4.0 * ctx->mass * ctx->mass;
    TRY(launch_dslash(ctx, 1, 64, 64, x, tmp_odd, 0, nullptr, 0, nullptr, 1.0, -1));
    return launch_dslash(ctx, 0, 64, 64, tmp_odd, r, -m4, x, 1.0, b, 1.0, slot);
}

hisq_status residual_rel(hisq_ctx *ctx, bool df, const double *b, const double *x, double *r, double *tmp_odd,
                         int slot);
hisq_status odd_from_t(hisq_ctx *ctx, double m, const double *eta_o, const double *t, double *psi_o);
hisq_status launch_residual_df_batch(hisq_ctx *ctx, const std::vector<int> &ids, const char *Y, const char *X, char *Rr,
                                     size_t s64, double *rr);
hisq_status odd_residual_from_t(hisq_ctx *ctx, double m, const double *eta_o, const double *psi_o, double *t, int slot);

static hisq_status deflate_pair_b(hisq_ctx *ctx, int n, bool df, const double *b, double *r, double *x, double *t_odd,
                                  int slot)
{
    if (n > 4096 || ctx->eig.prec != 32) { // see deflate_pair in solver.cu
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

// copy selected fields of the batch scalars of right-hand side j to the device
static hisq_status set_rhs_scalars(hisq_ctx *ctx, int j, double rr, double pp)
{
    HISQ_CUDA(cudaMemcpyAsync(&ctx->bscal->rr[j], &rr, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    HISQ_CUDA(cudaMemcpyAsync(&ctx->bscal->pp[j], &pp, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    return HISQ_OK;
}

static hisq_status set_active(hisq_ctx *ctx, const std::vector<int> &act)
{
    int buf[kMaxBatch + 1];
    buf[0] = int(act.size());
    for (size_t q = 0; q < act.size(); q++) buf[1 + q] = act[q];
    HISQ_CUDA(cudaMemcpyAsync(&ctx->bscal->kact, buf, sizeof(int) * (1 + act.size()), cudaMemcpyHostToDevice,
                              ctx->stream));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return HISQ_OK;
}

// Solve M psi_j = eta_j for k <= kMaxBatch right-hand sides together; eta, psi:
// k FP64 full-lattice device fields (stride V*48 bytes).
hisq_status solve_batched(hisq_ctx *ctx, const hisq_solve_params *P, const double *eta, double *psi, int k,
                          hisq_solve_stats *stats)
{
    static_assert(offsetof(BatchScalars, idx) == offsetof(BatchScalars, kact) + sizeof(int), "kact, idx adjacent");
    const int Vh = ctx->g.Vh;
    const size_t full = size_t(ctx->g.V) * 6;
    const double m = ctx->mass, m4 = 4.0 * m * m;
    const int prec = P->precision_sloppy, lprec = P->link_precision_sloppy, xprec = 32;
    if (k < 1 || k > kMaxBatch) return set_err(ctx, HISQ_ERR_INVALID_ARG, "batch of 1..%d right-hand sides", kMaxBatch);
    if (prec != 32 && prec != 16) return set_err(ctx, HISQ_ERR_INVALID_ARG, "batched solve: sloppy precision 32 or 16");
    if (lprec != 32) return set_err(ctx, HISQ_ERR_INVALID_ARG, "batched solve: FP32 sloppy links");
    const size_t s64 = spinor_bytes(64, Vh), ssl = spinor_bytes(prec, Vh), sx = spinor_bytes(xprec, Vh);
    char *Y = (char *)get_buf(ctx, BUF_B_Y, s64 * k);
    char *XH = (char *)get_buf(ctx, BUF_B_XHI, s64 * k);
    char *RH = (char *)get_buf(ctx, BUF_B_RHI, s64 * k);
    char *XS = (char *)get_buf(ctx, BUF_B_XSL, sx * k);
    char *RS = (char *)get_buf(ctx, BUF_B_RSL, ssl * k);
    char *PP = (char *)get_buf(ctx, BUF_B_P, ssl * k);
    char *TT = (char *)get_buf(ctx, BUF_B_TMP, ssl * k);
    double *eta_e = (double *)get_buf(ctx, BUF_ETA_E, s64);
    double *eta_o = (double *)get_buf(ctx, BUF_ETA_O, s64);
    double *t_hi = (double *)get_buf(ctx, BUF_TMPHI, s64);
    double *psi_o = (double *)get_buf(ctx, BUF_PSI_O, s64);
    if (!Y || !XH || !RH || !XS || !RS || !PP || !TT || !eta_e || !eta_o || !t_hi || !psi_o) return HISQ_ERR_OOM;
    char *DX = nullptr, *F32 = nullptr;
    const size_t s32 = spinor_bytes(32, Vh);
    if (P->deflate && ctx->eig.n > 0 && !dual_residual(ctx)) {
        DX = (char *)get_buf(ctx, BUF_B_DX, s64 * k);
        F32 = (char *)get_buf(ctx, BUF_B_F32, s32 * 3);
        if (!DX || !F32) return HISQ_ERR_OOM;
    }
    auto y = [&](int j) { return (double *)(Y + s64 * j); };
    auto xh = [&](int j) { return (double *)(XH + s64 * j); };
    auto rh = [&](int j) { return (double *)(RH + s64 * j); };
    auto xs = [&](int j) { return (void *)(XS + sx * j); };
    auto rs = [&](int j) { return (void *)(RS + ssl * j); };
    auto pj = [&](int j) { return (void *)(PP + ssl * j); };
    // tensor-core deflation of the right-hand sides `fields` (at most 32):
    // x_j += V Lambda^-1 V^dag r_j and the matching r_j, |r_j| into rt[j]
    auto tc_group = [&](const std::vector<int> &fields, int n_defl, std::vector<double> &rt) -> hisq_status {
        std::vector<double> nr(fields.size());
        for (size_t q = 0; q < fields.size(); q++) nr[q] = rt[fields[q]];
        const int kb = int(fields.size());
        if (dual_residual(ctx)) {
            TRY(tc_deflate_batch(ctx, n_defl, kb, rh(0), xh(0), nr.data(), fields.data(), true));
        } else {
            auto dx = [&](int j) { return (double *)(DX + s64 * j); };
            void *df = F32, *tf = F32 + s32, *af = F32 + 2 * s32;
            for (int j : fields) HISQ_CUDA(cudaMemsetAsync(dx(j), 0, s64, ctx->stream));
            TRY(tc_deflate_batch(ctx, n_defl, kb, rh(0), dx(0), nr.data(), fields.data(), false));
            for (int j : fields) {
                TRY(launch_convert(ctx, dx(j), 64, df, 32));
                TRY(launch_dslash(ctx, 1, 32, 32, df, tf, 0, nullptr, 0, nullptr, 1.0, -1));  // D_oe dx
                TRY(launch_dslash(ctx, 0, 32, 32, tf, af, m4, df, 0, nullptr, -1.0, -1));     // A dx
                TRY(launch_axpy_d(ctx, -1.0, af, 32, rh(j)));
                TRY(launch_axpy_d(ctx, 1.0, dx(j), 64, xh(j)));
            }
        }
        for (int j : fields) {
            double r2;
            TRY(launch_norm2(ctx, 64, rh(j), BS_R));
            TRY(read_slots(ctx, BS_R, 1, &r2));
            rt[j] = std::sqrt(r2);
        }
        return HISQ_OK;
    };

    int n_defl = 0;
    if (P->deflate) {
        if (ctx->eig.n <= 0) return set_err(ctx, HISQ_ERR_STATE, "deflation requested but no eigenpairs stored");
        n_defl = P->n_defl > 0 ? std::min(P->n_defl, ctx->eig.n) : ctx->eig.n;
    }
    auto t0 = std::chrono::steady_clock::now();
    std::vector<double> target(k), etanorm(k), ynorm(k), rt(k), r_last(k), r_defl(k), r_best(k), rn_seen(k);
    std::vector<int> noprog(k, 0), done(k, 0), its(k, 0), last_upd(k, 0);
    std::vector<hisq_solve_stats> st(k);
    for (int j = 0; j < k; j++) {
        memset(&st[j], 0, sizeof st[j]);
        st[j].full_residual = -1;
    }
    double defl_s = 0;
    // double-float reliable updates per right-hand side; a residual that meets
    // the target is recomputed in FP64 first, and a right-hand side whose FP64
    // residual does not confirm it stays on FP64 residuals from then on
    std::vector<char> use_df(k, P->precision_reliable == HISQ_PREC_DF64);
    // tok[j]: t_hi holds D_oe x_j for the current x_j (left by an FP64
    // residual); tval[j]: rh(j), no longer needed once j has finished, keeps
    // that D_oe x_j for the odd reconstruction
    std::vector<char> tok(k, 0), tval(k, 0);
    // |r_e|^2 of the full residual left by the FP64 confirmation of j (-1: none)
    std::vector<double> re2f(k, -1.0);
    auto keep_t = [&](int j) -> hisq_status {
        if (!tok[j]) return HISQ_OK;
        HISQ_CUDA(cudaMemcpyAsync(rh(j), t_hi, s64, cudaMemcpyDeviceToDevice, ctx->stream));
        tval[j] = 1;
        return HISQ_OK;
    };
    // the FP64 confirmation is the even part of the full residual (see
    // cg_reliable in solver.cu): t = D_oe x_j, psi_o = (eta_o - t) / 2m,
    // r_e = eta_e - 2m x_j - D_eo psi_o, y_j - A x_j = 2m r_e
    auto certify = [&](int j) -> hisq_status {
        if (!use_df[j] || rt[j] > target[j]) return HISQ_OK;
        const double *e = eta + full * j;
        TRY(launch_gather_parity(ctx, e, 0, 64, eta_e));
        TRY(launch_gather_parity(ctx, e, 1, 64, eta_o));
        TRY(launch_dslash(ctx, 1, 64, 64, xh(j), t_hi, 0, nullptr, 0, nullptr, 1.0, -1));
        TRY(odd_from_t(ctx, m, eta_o, t_hi, psi_o));
        TRY(launch_dslash(ctx, 0, 64, 64, psi_o, rh(j), -2.0 * m, xh(j), 1.0, eta_e, -1.0, BS_R));
        double re2;
        TRY(read_slots(ctx, BS_R, 1, &re2));
        rt[j] = 2.0 * m * std::sqrt(re2);
        tok[j] = 1;
        re2f[j] = re2;
        if (!(rt[j] <= target[j])) {
            // not confirmed: rh(j) = 2m r_e = y_j - A x_j, FP64 residuals from here
            HISQ_CUDA(cudaMemcpyAsync(t_hi, rh(j), s64, cudaMemcpyDeviceToDevice, ctx->stream));
            TRY(launch_scale_axpby_d(ctx, 0.0, t_hi, 2.0 * m, rh(j)));
            tok[j] = 0;
            re2f[j] = -1;
            use_df[j] = 0;
        }
        return HISQ_OK;
    };

    // (a2) sources, (a8) deflated guesses
    for (int j = 0; j < k; j++) {
        const double *e = eta + full * j;
        TRY(launch_gather_parity(ctx, e, 0, 64, eta_e));
        TRY(launch_gather_parity(ctx, e, 1, 64, eta_o));
        TRY(launch_norm2(ctx, 64, eta_e, BS_ETAE));
        TRY(launch_norm2(ctx, 64, eta_o, BS_ETAO));
        TRY(launch_dslash(ctx, 0, 64, 64, eta_o, y(j), 2.0 * m, eta_e, 0, nullptr, -1.0, BS_Y));
        double nrm[3];
        TRY(read_slots(ctx, BS_Y, 3, nrm));
        ynorm[j] = std::sqrt(nrm[0]);
        etanorm[j] = std::sqrt(nrm[1] + nrm[2]);
        if (!std::isfinite(ynorm[j]) || !std::isfinite(etanorm[j]))
            return set_err(ctx, HISQ_ERR_NUMERICAL, "non-finite source %d", j);
        target[j] = P->tol * std::fmin(ynorm[j], 2.0 * m * etanorm[j]);
        HISQ_CUDA(cudaMemsetAsync(xh(j), 0, s64, ctx->stream));
        if (P->guess) { // start from the caller's guess (even sites of psi_j)
            TRY(launch_gather_parity(ctx, psi + full * j, 0, 64, xh(j)));
            TRY(residual_hi_b(ctx, y(j), xh(j), rh(j), t_hi, BS_R));
            double r2;
            TRY(read_slots(ctx, BS_R, 1, &r2));
            rt[j] = std::sqrt(r2);
        } else {
            HISQ_CUDA(cudaMemcpyAsync(rh(j), y(j), s64, cudaMemcpyDeviceToDevice, ctx->stream));
            rt[j] = ynorm[j];
        }
    }
    // deflated guesses of all right-hand sides: one tensor-core projection and
    // one expansion for the whole batch, else one pair of passes per RHS
    if (n_defl > 0) {
        auto d0 = std::chrono::steady_clock::now();
        if (tc_eligible(ctx, n_defl, k)) {
            for (int j0 = 0; j0 < k; j0 += 32) {
                std::vector<int> fields;
                for (int j = j0; j < std::min(k, j0 + 32); j++) fields.push_back(j);
                TRY(tc_group(fields, n_defl, rt));
            }
        } else {
            for (int j = 0; j < k; j++) {
                double r2;
                TRY(deflate_pair_b(ctx, n_defl, use_df[j], y(j), rh(j), xh(j), t_hi, BS_R));
                TRY(read_slots(ctx, BS_R, 1, &r2));
                rt[j] = std::sqrt(r2);
            }
        }
        defl_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - d0).count();
    }
    for (int j = 0; j < k; j++) {
        if (etanorm[j] > 0) TRY(certify(j));
        r_last[j] = r_defl[j] = r_best[j] = rn_seen[j] = rt[j];
        if (etanorm[j] == 0 || rt[j] <= target[j]) {
            if (etanorm[j] > 0) TRY(keep_t(j));
            done[j] = 1;
            st[j].converged = 1;
            continue;
        }
        TRY(launch_convert(ctx, rh(j), 64, rs(j), prec));
        TRY(launch_convert(ctx, rh(j), 64, pj(j), prec));
        TRY(launch_zero(ctx, xs(j), xprec));
        TRY(set_rhs_scalars(ctx, j, rt[j] * rt[j], rt[j] * rt[j]));
    }
    std::vector<int> act;
    for (int j = 0; j < k; j++)
        if (!done[j]) act.push_back(j);
    {
        double hm4 = m4;
        long long it0 = 0;
        HISQ_CUDA(cudaMemcpyAsync(&ctx->bscal->m4, &hm4, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        HISQ_CUDA(cudaMemcpyAsync(&ctx->bscal->iter, &it0, sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
    }
    TRY(set_active(ctx, act));

    cudaEvent_t ev[2];
    HISQ_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    HISQ_CUDA(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    struct EvFree {
        cudaEvent_t *e;
        ~EvFree()
        {
            cudaEventDestroy(e[0]);
            cudaEventDestroy(e[1]);
        }
    } evfree{ev};
    const long long maxit = P->max_iter > 0 ? P->max_iter : 1;
    long long it = 0, checked = 0;
    std::vector<std::vector<int>> act_at(4); // active list of the iteration in each slot (it mod 4)
    IterGraphs graphs;
    int direct_ka = -1;
    // optional kernel timing of the two batched Dslash launches: ring of 4
    // iterations x 3 events; a launch's time is shared by its active right-hand sides
    const bool prof = ctx->profile;
    cudaEvent_t pe[4][3] = {};
    struct ProfFree {
        cudaEvent_t (*e)[3];
        ~ProfFree()
        {
            for (int i = 0; i < 4; i++)
                for (int q = 0; q < 3; q++)
                    if (e[i][q]) cudaEventDestroy(e[i][q]);
        }
    } prof_free{pe};
    if (prof)
        for (int i = 0; i < 4; i++)
            for (int q = 0; q < 3; q++) HISQ_CUDA(cudaEventCreate(&pe[i][q]));
    long long retired = 0;
    auto retire = [&](long long n_done) {
        if (!prof) return;
        for (; retired < n_done; retired++) {
            float a = 0, b = 0;
            cudaEvent_t *e = pe[retired & 3];
            const std::vector<int> &on = act_at[retired & 3];
            if (on.empty() || cudaEventElapsedTime(&a, e[0], e[1]) != cudaSuccess ||
                cudaEventElapsedTime(&b, e[1], e[2]) != cudaSuccess)
                continue;
            for (int j : on) {
                st[j].seconds_dslash_oe += a * 1e-3 / on.size();
                st[j].seconds_dslash_eo += b * 1e-3 / on.size();
                st[j].profiled_iterations++;
            }
        }
    };
    // the persistent form of the iterations between host interventions
    const bool persist = P->persistent && lprec == 32 && (prec == 16 || prec == 32) &&
                         (ctx->long_recon == 12 || ctx->long_recon == 18);
    std::vector<double> lo2(kMaxBatch, 0.0), hi2(kMaxBatch, 0.0), rrh(kMaxBatch, 0.0);
    // one persistent launch up to the next iteration in which a right-hand side
    // meets a condition the host acts on (the same conditions as below)
    auto persistent_round = [&](std::vector<int> &upd) -> hisq_status {
        long long mx = maxit - it;
        for (int j : act) mx = std::min<long long>(mx, 1000 - (its[j] - last_upd[j]));
        mx = std::max<long long>(1, std::min<long long>(mx, 1 << 30));
        std::fill(lo2.begin(), lo2.end(), 0.0);
        std::fill(hi2.begin(), hi2.end(), 0.0);
        for (int j : act) {
            const double lo = std::max(target[j], P->delta_rd * r_last[j]);
            lo2[j] = lo * lo;
            hi2[j] = 1e6 * r_last[j] * r_last[j];
        }
        int n = 0, itr[kMaxBatch] = {};
        double ph[2] = {0, 0};
        TRY(launch_bcg_persistent(ctx, prec, lprec, PP, TT, RS, XS, int(act.size()), int(mx), lo2.data(), hi2.data(),
                                  &n, itr, prof ? ph : nullptr));
        HISQ_CUDA(cudaMemcpyAsync(rrh.data(), ctx->bscal->rr, sizeof(double) * kMaxBatch, cudaMemcpyDeviceToHost,
                                  ctx->stream));
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
        long long rhs_its = 0;
        for (int j : act) {
            its[j] += itr[j];
            rhs_its += itr[j];
        }
        it += n;
        if (prof && rhs_its > 0)
            for (int j : act) { // launch time shared in proportion to each one's iterations
                st[j].seconds_dslash_oe += ph[0] * itr[j] / double(rhs_its);
                st[j].seconds_dslash_eo += ph[1] * itr[j] / double(rhs_its);
                st[j].profiled_iterations += itr[j];
            }
        for (int j : act) {
            const double rr = rrh[j];
            if (!std::isfinite(rr)) return set_err(ctx, HISQ_ERR_NUMERICAL, "non-finite residual of right-hand side %d", j);
            const double rn = std::sqrt(rr);
            rn_seen[j] = rn;
            if (rn < target[j] || rn < P->delta_rd * r_last[j] || rn > 1e3 * r_last[j] || its[j] - last_upd[j] >= 1000)
                upd.push_back(j);
        }
        retired = it; // no per-launch events in this form
        checked = it;
        return HISQ_OK;
    };
    while (!act.empty()) {
        const bool force = it >= maxit;
        std::vector<int> upd;
        if (persist && !force) {
            TRY(persistent_round(upd));
        } else {
            if (!force) {
                const int ka = int(act.size());
                const int slot = int(it & 3);
                auto iteration = [&](bool cap) -> hisq_status {
                    if (prof) HISQ_CUDA(record_event(ctx, pe[slot][0], cap));
                    TRY(launch_mrhs_dslash_tt(ctx, prec, lprec, PP, TT, ka));
                    if (prof) HISQ_CUDA(record_event(ctx, pe[slot][1], cap));
                    TRY(launch_mrhs_dslash_update(ctx, prec, lprec, TT, PP, XS, RS, ka));
                    if (prof) HISQ_CUDA(record_event(ctx, pe[slot][2], cap));
                    TRY(launch_mrhs_p_update(ctx, prec, RS, PP, ka));
                    HISQ_CUDA(record_event(ctx, ev[slot & 1], cap));
                    return HISQ_OK;
                };
                // the first iteration of each active-set size runs directly (lazy
                // kernel set-up happens outside capture), later ones replay a graph
                if (ka != direct_ka) {
                    TRY(iteration(false));
                    direct_ka = ka;
                } else {
                    TRY(graph_run(ctx, graphs, slot, ka, iteration));
                }
                act_at[it & 3] = act;
                for (int j : act) its[j]++;
                it++;
            }
            const long long jj = it - 2;
            if (force) {
                upd = act;
            } else if (jj >= checked) {
                HISQ_CUDA(cudaEventSynchronize(ev[jj & 1]));
                if (*(volatile int *)ctx->wait_status_h != 0) {
                    const int code = *ctx->wait_status_h;
                    cudaStreamSynchronize(ctx->stream);
                    *ctx->wait_status_h = 0;
                    return set_err(ctx, HISQ_ERR_TIMEOUT, "batched operator: a pipeline wait ran out (code %d)", code);
                }
                retire(jj + 1);
                for (int j : act_at[jj & 3]) {
                    const double rr = ctx->bmonitor_h[size_t(jj % ctx->bmonitor_len) * kMaxBatch + j];
                    if (!std::isfinite(rr)) {
                        cudaStreamSynchronize(ctx->stream);
                        return set_err(ctx, HISQ_ERR_NUMERICAL, "non-finite residual of right-hand side %d", j);
                    }
                    const double rn = std::sqrt(rr);
                    rn_seen[j] = rn;
                    if (rn < target[j] || rn < P->delta_rd * r_last[j] || rn > 1e3 * r_last[j] ||
                        its[j] - last_upd[j] >= 1000)
                        upd.push_back(j);
                }
                checked = jj + 1;
            }
        }
        if (upd.empty()) continue;
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
        retire(it);
        checked = it;
        bool changed = false;
        std::vector<int> redefl;
        // sloppy state of right-hand side j after a reliable update or a re-deflation
        auto finalize = [&](int j, bool restart) -> hisq_status {
            TRY(launch_convert(ctx, rh(j), 64, rs(j), prec));
            TRY(launch_zero(ctx, xs(j), xprec));
            double pp = rt[j] * rt[j];
            if (restart) {
                TRY(launch_convert(ctx, rh(j), 64, pj(j), prec));
            } else {
                TRY(launch_norm2(ctx, prec, pj(j), BS_PP));
                TRY(read_slots(ctx, BS_PP, 1, &pp));
            }
            TRY(set_rhs_scalars(ctx, j, rt[j] * rt[j], pp));
            r_last[j] = rt[j];
            return HISQ_OK;
        };
        // the double-float residuals of this round together (one pass over the links)
        std::vector<int> gdf;
        std::vector<double> r2df(k, 0.0);
        for (int j : upd)
            if (use_df[j]) gdf.push_back(j);
        if (gdf.size() > 1) {
            std::vector<double> rr(gdf.size());
            for (int j : gdf) TRY(launch_axpy_d(ctx, 1.0, xs(j), xprec, xh(j)));
            TRY(launch_residual_df_batch(ctx, gdf, Y, XH, RH, s64, rr.data()));
            for (size_t q = 0; q < gdf.size(); q++) r2df[gdf[q]] = rr[q];
        } else {
            gdf.clear();
        }
        for (int j : upd) {
            // reliable update of right-hand side j (FP64 or double-float true residual)
            double r2;
            if (std::find(gdf.begin(), gdf.end(), j) != gdf.end()) {
                r2 = r2df[j];
            } else {
                TRY(launch_axpy_d(ctx, 1.0, xs(j), xprec, xh(j)));
                TRY(residual_rel(ctx, use_df[j], y(j), xh(j), rh(j), t_hi, BS_R));
                TRY(read_slots(ctx, BS_R, 1, &r2));
            }
            tok[j] = !use_df[j];
            if (!std::isfinite(r2)) return set_err(ctx, HISQ_ERR_NUMERICAL, "non-finite true residual");
            rt[j] = std::sqrt(r2);
            TRY(certify(j));
            st[j].reliable_updates++;
            last_upd[j] = its[j];
            bool finish = false;
            if (rt[j] <= target[j]) {
                st[j].converged = 1;
                finish = true;
            } else if (force || its[j] >= maxit) {
                finish = true;
            } else if (rt[j] < 0.5 * r_best[j]) {
                r_best[j] = rt[j];
                noprog[j] = 0;
            } else if (++noprog[j] >= 8) {
                set_err(ctx, HISQ_ERR_NOT_CONVERGED, "stagnation of right-hand side %d", j);
                finish = true;
            }
            if (finish) {
                TRY(keep_t(j));
                done[j] = 1;
                changed = true;
                continue;
            }
            const bool restart = rt[j] > 10.0 * rn_seen[j];
            if (n_defl > 0 && P->delta_tr > 0 && rt[j] < P->delta_tr * r_defl[j]) {
                redefl.push_back(j);
                continue;
            }
            TRY(finalize(j, restart));
        }
        // re-deflations of this round, together on the tensor cores when possible
        if (!redefl.empty()) {
            auto d0 = std::chrono::steady_clock::now();
            if (tc_eligible(ctx, n_defl, int(redefl.size()))) {
                for (size_t q0 = 0; q0 < redefl.size(); q0 += 32) {
                    const size_t q1 = std::min(redefl.size(), q0 + 32);
                    TRY(tc_group(std::vector<int>(redefl.begin() + q0, redefl.begin() + q1), n_defl, rt));
                }
            } else {
                for (int j : redefl) {
                    double r2;
                    TRY(deflate_pair_b(ctx, n_defl, use_df[j], y(j), rh(j), xh(j), t_hi, BS_R));
                    TRY(read_slots(ctx, BS_R, 1, &r2));
                    rt[j] = std::sqrt(r2);
                }
            }
            defl_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - d0).count();
            for (int j : redefl) {
                r_defl[j] = rt[j];
                st[j].redeflations++;
                tok[j] = 0;
                TRY(certify(j));
                if (rt[j] <= target[j]) {
                    TRY(keep_t(j));
                    st[j].converged = 1;
                    done[j] = 1;
                    changed = true;
                    continue;
                }
                TRY(finalize(j, true));
            }
        }
        if (changed) {
            act.clear();
            for (int j = 0; j < k; j++)
                if (!done[j]) act.push_back(j);
        }
        TRY(set_active(ctx, act));
    }
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    retire(it);

    // (a9) reconstruction and FP64 full residuals
    hisq_status worst = HISQ_OK;
    for (int j = 0; j < k; j++) {
        const double *e = eta + full * j;
        double *out = psi + full * j;
        TRY(launch_gather_parity(ctx, e, 0, 64, eta_e));
        TRY(launch_gather_parity(ctx, e, 1, 64, eta_o));
        if (tval[j]) {
            TRY(odd_from_t(ctx, m, eta_o, rh(j), psi_o));
        } else {
            TRY(launch_dslash(ctx, 1, 64, 64, xh(j), psi_o, 1.0 / (2.0 * m), eta_o, 0, nullptr, -1.0 / (2.0 * m), -1));
        }
        if (P->compute_full_residual && etanorm[j] > 0) {
            double rr[2] = {re2f[j], 0.0};
            if (tval[j]) {
                // an FP64 confirmation of this x_j has already formed |r_e|^2
                if (re2f[j] < 0)
                    TRY(launch_dslash(ctx, 0, 64, 64, psi_o, t_hi, -2.0 * m, xh(j), 1.0, eta_e, -1.0, BS_RE));
                TRY(odd_residual_from_t(ctx, m, eta_o, psi_o, rh(j), BS_RO));
            } else {
                re2f[j] = -1;
                TRY(launch_dslash(ctx, 0, 64, 64, psi_o, rh(j), -2.0 * m, xh(j), 1.0, eta_e, -1.0, BS_RE));
                TRY(launch_dslash(ctx, 1, 64, 64, xh(j), t_hi, -2.0 * m, psi_o, 1.0, eta_o, -1.0, BS_RO));
            }
            if (re2f[j] < 0) {
                TRY(read_slots(ctx, BS_RE, 2, rr));
            } else {
                TRY(read_slots(ctx, BS_RO, 1, &rr[1]));
            }
            st[j].full_residual = std::sqrt(rr[0] + rr[1]) / etanorm[j];
        } else if (etanorm[j] == 0) {
            st[j].full_residual = 0;
        }
        TRY(launch_scatter_parity(ctx, xh(j), 64, 0, out));
        TRY(launch_scatter_parity(ctx, psi_o, 64, 1, out));
        st[j].iterations = its[j];
        st[j].even_residual = ynorm[j] > 0 ? rt[j] / ynorm[j] : 0;
        if (!st[j].converged) worst = HISQ_ERR_NOT_CONVERGED;
    }
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int j = 0; j < k; j++) {
        st[j].seconds_total = secs / k;
        st[j].seconds_deflate = defl_s / k;
        if (stats) stats[j] = st[j];
    }
    return worst;
}

} // namespace hisq
