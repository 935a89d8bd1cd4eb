// block_eig.cu -- block thick-restart Lanczos for the low modes of
// A0 = -D_eo D_oe (the block variant the paper names as an outlook, Section 4).
//
// b basis vectors are generated per step, so the (Chebyshev-filtered) operator
// is applied to b fields at once with the batched Dslash, which reads each link
// once for all b.  The projected matrix H = V^dag A V is formed explicitly from
// the block Gram-Schmidt coefficients (classical, twice), which also carries the
// thick-restart coupling without special cases:
//   expand block j:  W = Op V_j;  C = V^dag W (twice);  H[:, j] = C;  W = Q R
//   (Cholesky QR, twice);  V_{j+1} = Q;  H[j+1, j] = R
//   restart:  H = Z Theta Z^dag (FP64, on the device);  V_keep = V Z_keep;
//   V_{k} = residual block;  H = diag(theta_keep) + coupling R Z_last.
// Dense block operations are plain FP32 complex GEMMs (cuBLAS); the small
// Hermitian eigenproblem is cuSOLVER's Zheevd.  Fields use the FP32 colour-vector
// storage, which is 3 Vh complex numbers per field in a fixed order, so a set of
// fields is a column-major complex matrix with leading dimension 3 Vh.
#include <cublas_v2.h>
#include <cuComplex.h>
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

#include "internal.cuh"

namespace hisq {

hisq_status read_slots(hisq_ctx *ctx, int slot0, int n, double *out);

#define TRY_B(x)                                \
    do {                                        \
        hisq_status s_ = (x);                   \
        if (s_ != HISQ_OK) return s_;           \
    } while (0)
#define BLAS(call)                                                                              \
    do {                                                                                        \
        cublasStatus_t e_ = (call);                                                             \
        if (e_ != CUBLAS_STATUS_SUCCESS) return set_err(ctx, HISQ_ERR_CUDA, "cuBLAS %d: %s", int(e_), #call); \
    } while (0)
#define SOLVER(call)                                                                              \
    do {                                                                                          \
        cusolverStatus_t e_ = (call);                                                             \
        if (e_ != CUSOLVER_STATUS_SUCCESS) return set_err(ctx, HISQ_ERR_CUDA, "cuSOLVER %d: %s", int(e_), #call); \
    } while (0)

typedef std::complex<double> cd;

namespace {

struct Handles {
    cublasHandle_t blas = nullptr;
    cusolverDnHandle_t solver = nullptr;
    ~Handles()
    {
        if (blas) cublasDestroy(blas);
        if (solver) cusolverDnDestroy(solver);
    }
};

// Cholesky of a Hermitian positive b x b matrix G (column-major): G = R^dag R,
// R upper triangular; returns false when G is not numerically positive
bool cholesky_upper(int b, const std::vector<cd> &G, std::vector<cd> &R)
{
    R.assign(size_t(b) * b, cd(0));
    for (int j = 0; j < b; j++) {
        cd s = G[size_t(j) * b + j];
        for (int k = 0; k < j; k++) s -= std::conj(R[size_t(j) * b + k]) * R[size_t(j) * b + k];
        const double d = s.real();
        if (!(d > 0) || !std::isfinite(d)) return false;
        const double rjj = std::sqrt(d);
        R[size_t(j) * b + j] = rjj;
        for (int i = j + 1; i < b; i++) {
            cd t = G[size_t(i) * b + j]; // G(j, i)
            for (int k = 0; k < j; k++) t -= std::conj(R[size_t(j) * b + k]) * R[size_t(i) * b + k];
            R[size_t(i) * b + j] = t / rjj; // R(j, i)
        }
    }
    return true;
}

// inverse of an upper triangular b x b matrix (column-major)
std::vector<cd> inv_upper(int b, const std::vector<cd> &R)
{
    std::vector<cd> X(size_t(b) * b, cd(0));
    for (int j = 0; j < b; j++) {
        X[size_t(j) * b + j] = 1.0 / R[size_t(j) * b + j];
        for (int i = j - 1; i >= 0; i--) {
            cd s = 0;
            for (int k = i + 1; k <= j; k++) s += R[size_t(k) * b + i] * X[size_t(j) * b + k];
            X[size_t(j) * b + i] = -s / R[size_t(i) * b + i];
        }
    }
    return X;
}

} // namespace

// Block thick-restart Lanczos.  B holds n_kr + b FP32 fields; on success the
// n_ev wanted Ritz vectors are in B[0 .. n_ev).  Op: the Chebyshev filter of
// degree deg on [amin, amax] (wanted: largest) or A0 itself (wanted: smallest).
hisq_status block_trlm(hisq_ctx *ctx, const hisq_eig_params *P, int b, int n_ev, int n_kr, int n_keep, int deg,
                       double amin, double amax, void *B, int *conv_out)
{
    const int Vh = ctx->g.Vh;
    const size_t sf = spinor_bytes(32, Vh);
    const int L = 3 * Vh;                  // complex rows of a field
    const bool filtered = deg > 0;
    if (b < 2 || b > kMaxBatch) return set_err(ctx, HISQ_ERR_INVALID_ARG, "block size 2..%d", kMaxBatch);
    // a restart keeps n_keep >= n_ev vectors and adds at least two blocks (one
    // block per restart was measured 3x slower: 28.0 s against 8.8 s for 256 pairs)
    b = std::min(b, (n_kr - std::max(n_keep, n_ev)) / 2);
    if (b < 2 || n_kr < 2 * b) return set_err(ctx, HISQ_ERR_INVALID_ARG, "block Lanczos needs n_kr >= n_keep + 4");
    // n_kr and n_keep on the block grid: n_kr multiple of b, n_kr - n_keep a multiple of b
    n_kr = std::max(b * 2, (n_kr / b) * b);
    n_keep = n_kr - b * std::max(1, (n_kr - n_keep) / b);
    if (n_keep < n_ev) n_keep = std::min(n_kr - b, ((n_ev + b - 1) / b) * b);
    if (n_keep < n_ev || n_keep >= n_kr) return set_err(ctx, HISQ_ERR_INVALID_ARG, "block Lanczos: n_kr too small for n_ev");

    Handles h;
    BLAS(cublasCreate(&h.blas));
    BLAS(cublasSetStream(h.blas, ctx->stream));
    SOLVER(cusolverDnCreate(&h.solver));
    SOLVER(cusolverDnSetStream(h.solver, ctx->stream));

    // work: three blocks for the Chebyshev recurrence (W is one of them), one
    // odd block, projection coefficients, small matrices, rotation chunk
    const size_t rot_rows = std::max<size_t>(4096, (size_t(192) << 20) / (sizeof(cuComplex) * size_t(n_kr)));
    std::vector<std::pair<void *, size_t>> mem;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = dev_alloc(ctx, bytes);
        if (p) mem.emplace_back(p, bytes);
        return p;
    };
    struct Free {
        hisq_ctx *c;
        std::vector<std::pair<void *, size_t>> *m;
        ~Free()
        {
            cudaStreamSynchronize(c->stream);
            for (auto &e : *m) dev_free(c, e.first, e.second);
        }
    } guard{ctx, &mem};
    char *blk = (char *)alloc(sf * b * 3);
    char *odd = (char *)alloc(sf * b);
    cuComplex *Cd = (cuComplex *)alloc(sizeof(cuComplex) * size_t(n_kr + b) * b * 2);
    cuComplex *Sd = (cuComplex *)alloc(sizeof(cuComplex) * size_t(b) * b);
    cuComplex *Zd = (cuComplex *)alloc(sizeof(cuComplex) * size_t(n_kr) * n_kr);
    cuComplex *Td = (cuComplex *)alloc(sizeof(cuComplex) * rot_rows * n_kr);
    cuDoubleComplex *Hd = (cuDoubleComplex *)alloc(sizeof(cuDoubleComplex) * size_t(n_kr) * n_kr);
    double *Wd = (double *)alloc(sizeof(double) * n_kr);
    int *infod = (int *)alloc(sizeof(int));
    if (!blk || !odd || !Cd || !Sd || !Zd || !Td || !Hd || !Wd || !infod) return HISQ_ERR_OOM;
    int lwork = 0;
    SOLVER(cusolverDnZheevd_bufferSize(h.solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n_kr, Hd, n_kr, Wd,
                                       &lwork));
    cuDoubleComplex *work = (cuDoubleComplex *)alloc(sizeof(cuDoubleComplex) * std::max(lwork, 1));
    if (!work) return HISQ_ERR_OOM;

    auto fld = [&](int i) -> cuComplex * { return (cuComplex *)((char *)B + sf * i); };
    auto blkp = [&](int q) -> void * { return blk + sf * b * q; };
    const cuComplex one = make_cuComplex(1.f, 0.f), zero = make_cuComplex(0.f, 0.f), mone = make_cuComplex(-1.f, 0.f);

    TRY_B(mrhs_set_identity(ctx, b));
    // W = Op(V[j .. j+b)) into one of the three blocks; returns which
    auto op_block = [&](const void *in) -> void * {
        if (!filtered) {
            if (launch_mrhs_dslash_lin(ctx, 1, in, odd, 0, nullptr, 0, nullptr, 1.0, b) != HISQ_OK) return nullptr;
            if (launch_mrhs_dslash_lin(ctx, 0, odd, blkp(0), 0, nullptr, 0, nullptr, -1.0, b) != HISQ_OK) return nullptr;
            return blkp(0);
        }
        const double sigma = amax + amin, delta = amax - amin;
        // T1 = (sigma v + 2 D_eo D_oe v) / delta
        const void *prev = in;
        void *cur = blkp(0);
        if (launch_mrhs_dslash_lin(ctx, 1, in, odd, 0, nullptr, 0, nullptr, 1.0, b) != HISQ_OK) return nullptr;
        if (launch_mrhs_dslash_lin(ctx, 0, odd, cur, sigma / delta, in, 0, nullptr, 2.0 / delta, b) != HISQ_OK)
            return nullptr;
        for (int k = 1; k < deg; k++) {
            void *next = nullptr;
            for (int q = 0; q < 3; q++)
                if (blkp(q) != prev && blkp(q) != cur) {
                    next = blkp(q);
                    break;
                }
            if (launch_mrhs_dslash_lin(ctx, 1, cur, odd, 0, nullptr, 0, nullptr, 1.0, b) != HISQ_OK) return nullptr;
            if (launch_mrhs_dslash_lin(ctx, 0, odd, next, 2.0 * sigma / delta, cur, -1.0, prev, 4.0 / delta, b) !=
                HISQ_OK)
                return nullptr;
            prev = cur;
            cur = next;
        }
        return cur;
    };

    // W (b fields) -> orthogonal to V[0 .. m); coefficients V^dag W summed over
    // both passes into Cacc (host, m x b, column-major)
    auto project_out = [&](cuComplex *W, int m, std::vector<cd> &Cacc) -> hisq_status {
        Cacc.assign(size_t(m) * b, cd(0));
        std::vector<cuComplex> Ch(size_t(m) * b);
        for (int pass = 0; pass < 2; pass++) {
            BLAS(cublasCgemm(h.blas, CUBLAS_OP_C, CUBLAS_OP_N, m, b, L, &one, fld(0), L, W, L, &zero, Cd, m));
            BLAS(cublasCgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, L, b, m, &mone, fld(0), L, Cd, m, &one, W, L));
            HISQ_CUDA(cudaMemcpyAsync(Ch.data(), Cd, sizeof(cuComplex) * Ch.size(), cudaMemcpyDeviceToHost,
                                      ctx->stream));
            HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
            for (size_t i = 0; i < Ch.size(); i++) Cacc[i] += cd(Ch[i].x, Ch[i].y);
        }
        return HISQ_OK;
    };

    // W = Q R (Cholesky QR, twice) with Q written to `out` (b fields); R (b x b,
    // column-major) returned; a rank-deficient W is replaced by random fields
    // made orthogonal to V[0 .. m) (then R = 0)
    auto block_qr = [&](cuComplex *W, cuComplex *out, int m, std::vector<cd> &Rtot, uint64_t seed) -> hisq_status {
        std::vector<cd> Racc(size_t(b) * b, cd(0));
        for (int i = 0; i < b; i++) Racc[size_t(i) * b + i] = 1;
        cuComplex *src = W;
        bool deficient = false;
        for (int pass = 0; pass < 2; pass++) {
            BLAS(cublasCgemm(h.blas, CUBLAS_OP_C, CUBLAS_OP_N, b, b, L, &one, src, L, src, L, &zero, Sd, b));
            std::vector<cuComplex> Gh(size_t(b) * b);
            HISQ_CUDA(cudaMemcpyAsync(Gh.data(), Sd, sizeof(cuComplex) * Gh.size(), cudaMemcpyDeviceToHost, ctx->stream));
            HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
            std::vector<cd> G(Gh.size()), R;
            double tr = 0;
            for (size_t i = 0; i < Gh.size(); i++) G[i] = cd(Gh[i].x, Gh[i].y);
            for (int i = 0; i < b; i++) tr += G[size_t(i) * b + i].real();
            if (!(tr > 0) || !cholesky_upper(b, G, R)) {
                deficient = true;
                break;
            }
            // a direction whose norm fell below 1e-4 of the block's is noise
            double rmin = 1e300, rmax = 0;
            for (int i = 0; i < b; i++) {
                rmin = std::min(rmin, std::abs(R[size_t(i) * b + i]));
                rmax = std::max(rmax, std::abs(R[size_t(i) * b + i]));
            }
            if (pass == 0 && rmin < 1e-4 * rmax) {
                deficient = true;
                break;
            }
            const std::vector<cd> Ri = inv_upper(b, R);
            std::vector<cuComplex> Rih(Ri.size());
            for (size_t i = 0; i < Ri.size(); i++) Rih[i] = make_cuComplex(float(Ri[i].real()), float(Ri[i].imag()));
            HISQ_CUDA(cudaMemcpyAsync(Sd, Rih.data(), sizeof(cuComplex) * Rih.size(), cudaMemcpyHostToDevice,
                                      ctx->stream));
            cuComplex *dst = pass == 0 ? out : W;
            BLAS(cublasCgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, L, b, b, &one, src, L, Sd, b, &zero, dst, L));
            // Racc = R * Racc (the second factor applies after the first)
            std::vector<cd> N(size_t(b) * b, cd(0));
            for (int j = 0; j < b; j++)
                for (int i = 0; i < b; i++) {
                    cd s = 0;
                    for (int k = i; k < b; k++) s += R[size_t(k) * b + i] * Racc[size_t(j) * b + k];
                    N[size_t(j) * b + i] = s;
                }
            Racc.swap(N);
            src = dst;
        }
        if (deficient) {
            for (int i = 0; i < b; i++)
                TRY_B(launch_random_f(ctx, seed + 7919ull * uint64_t(i + 1), (char *)W + sf * i));
            std::vector<cd> dummy;
            TRY_B(project_out(W, m, dummy));
            std::vector<cd> Rn;
            // orthonormalise the random block (it is well conditioned)
            for (int pass = 0; pass < 2; pass++) {
                cuComplex *s2 = pass == 0 ? W : out;
                cuComplex *d2 = pass == 0 ? out : W;
                BLAS(cublasCgemm(h.blas, CUBLAS_OP_C, CUBLAS_OP_N, b, b, L, &one, s2, L, s2, L, &zero, Sd, b));
                std::vector<cuComplex> Gh(size_t(b) * b);
                HISQ_CUDA(cudaMemcpyAsync(Gh.data(), Sd, sizeof(cuComplex) * Gh.size(), cudaMemcpyDeviceToHost,
                                          ctx->stream));
                HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
                std::vector<cd> G(Gh.size());
                for (size_t i = 0; i < Gh.size(); i++) G[i] = cd(Gh[i].x, Gh[i].y);
                if (!cholesky_upper(b, G, Rn)) return set_err(ctx, HISQ_ERR_NUMERICAL, "block Lanczos: restart block");
                const std::vector<cd> Ri = inv_upper(b, Rn);
                std::vector<cuComplex> Rih(Ri.size());
                for (size_t i = 0; i < Ri.size(); i++) Rih[i] = make_cuComplex(float(Ri[i].real()), float(Ri[i].imag()));
                HISQ_CUDA(cudaMemcpyAsync(Sd, Rih.data(), sizeof(cuComplex) * Rih.size(), cudaMemcpyHostToDevice,
                                          ctx->stream));
                BLAS(cublasCgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, L, b, b, &one, s2, L, Sd, b, &zero, d2, L));
            }
            HISQ_CUDA(cudaMemcpyAsync(out, W, sf * b, cudaMemcpyDeviceToDevice, ctx->stream));
            Racc.assign(size_t(b) * b, cd(0));
        } else {
            // the second pass wrote W: copy the final Q to `out`
            HISQ_CUDA(cudaMemcpyAsync(out, W, sf * b, cudaMemcpyDeviceToDevice, ctx->stream));
        }
        Rtot.swap(Racc);
        return HISQ_OK;
    };

    // start block: random fields, orthonormal
    {
        for (int i = 0; i < b; i++) TRY_B(launch_random_f(ctx, P->seed + 104729ull * uint64_t(i + 1), fld(i)));
        HISQ_CUDA(cudaMemcpyAsync(blkp(1), fld(0), sf * b, cudaMemcpyDeviceToDevice, ctx->stream));
        std::vector<cd> Rs;
        TRY_B(block_qr((cuComplex *)blkp(1), fld(0), 0, Rs, P->seed ^ 0xabcdefull));
        TRY_B(mrhs_set_identity(ctx, b));
    }
    std::vector<cd> H(size_t(n_kr) * n_kr, cd(0)), Rlast;
    int k = 0, conv = 0;
    // phase times (logging only: the stream is synchronised at each boundary)
    const bool timing = log_level() > 0;
    double t_filter = 0, t_gs = 0, t_rr = 0, t_rot = 0;
    auto t_last = std::chrono::steady_clock::now();
    auto tick = [&](double &acc) {
        if (!timing) return;
        cudaStreamSynchronize(ctx->stream);
        const auto now = std::chrono::steady_clock::now();
        acc += std::chrono::duration<double>(now - t_last).count();
        t_last = now;
    };
    for (int restart = 0; restart <= P->max_restarts; restart++) {
        for (int j = k; j < n_kr; j += b) {
            tick(t_rr);
            void *Wv = op_block(fld(j));
            if (!Wv) return HISQ_ERR_CUDA;
            tick(t_filter);
            const int m = j + b;
            std::vector<cd> C;
            TRY_B(project_out((cuComplex *)Wv, m, C));
            for (int c = 0; c < b; c++)
                for (int r = 0; r < m; r++) H[size_t(j + c) * n_kr + r] = C[size_t(c) * m + r];
            std::vector<cd> R;
            TRY_B(block_qr((cuComplex *)Wv, fld(m), m, R, P->seed + 31ull * uint64_t(restart * n_kr + j)));
            TRY_B(mrhs_set_identity(ctx, b));
            if (m < n_kr) {
                for (int c = 0; c < b; c++)
                    for (int r = 0; r < b; r++) H[size_t(j + c) * n_kr + (m + r)] = R[size_t(c) * b + r];
            } else {
                Rlast = R;
            }
        }
        tick(t_gs);
        // Rayleigh-Ritz: H Hermitian (mean of H and H^dag), eigenpairs on the device in FP64
        std::vector<cuDoubleComplex> Hh(H.size());
        for (int c = 0; c < n_kr; c++)
            for (int r = 0; r < n_kr; r++) {
                const cd v = 0.5 * (H[size_t(c) * n_kr + r] + std::conj(H[size_t(r) * n_kr + c]));
                Hh[size_t(c) * n_kr + r] = make_cuDoubleComplex(v.real(), v.imag());
            }
        HISQ_CUDA(cudaMemcpyAsync(Hd, Hh.data(), sizeof(cuDoubleComplex) * Hh.size(), cudaMemcpyHostToDevice, ctx->stream));
        SOLVER(cusolverDnZheevd(h.solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, n_kr, Hd, n_kr, Wd, work,
                                lwork, infod));
        std::vector<double> th(n_kr);
        int info = 0;
        HISQ_CUDA(cudaMemcpyAsync(th.data(), Wd, sizeof(double) * n_kr, cudaMemcpyDeviceToHost, ctx->stream));
        HISQ_CUDA(cudaMemcpyAsync(Hh.data(), Hd, sizeof(cuDoubleComplex) * Hh.size(), cudaMemcpyDeviceToHost, ctx->stream));
        HISQ_CUDA(cudaMemcpyAsync(&info, infod, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
        if (info != 0) return set_err(ctx, HISQ_ERR_NUMERICAL, "block Lanczos: projected eigenproblem failed (%d)", info);
        std::vector<int> order(n_kr);
        std::iota(order.begin(), order.end(), 0);
        if (filtered) std::reverse(order.begin(), order.end());
        double scale = 0;
        for (double t : th) scale = std::max(scale, std::fabs(t));
        // residual of Ritz pair i: |R_last Z[n_kr-b .. n_kr, i]|
        auto resid = [&](int i) {
            double s = 0;
            for (int r = 0; r < b; r++) {
                cd acc = 0;
                for (int c = 0; c < b; c++) {
                    const cuDoubleComplex z = Hh[size_t(i) * n_kr + (n_kr - b + c)];
                    acc += Rlast[size_t(c) * b + r] * cd(z.x, z.y);
                }
                s += std::norm(acc);
            }
            return std::sqrt(s);
        };
        conv = 0;
        for (int i = 0; i < n_ev; i++) {
            if (resid(order[i]) <= P->tol * scale) conv++;
            else break;
        }
        const bool done = conv >= n_ev || restart == P->max_restarts;
        if (log_level() > 0)
            fprintf(stderr, "[hisq] block trlm (b = %d) restart %d: %d/%d converged, ritz %.6g .. %.6g\n", b, restart,
                    conv, n_ev, th[order[0]], th[order[n_ev - 1]]);
        const int nout = done ? n_ev : n_keep;
        // V[:, 0 .. nout) = V[:, 0 .. n_kr) Z[:, order[0 .. nout)] in place by row chunks
        std::vector<cuComplex> Zh(size_t(n_kr) * nout);
        for (int c = 0; c < nout; c++)
            for (int r = 0; r < n_kr; r++) {
                const cuDoubleComplex z = Hh[size_t(order[c]) * n_kr + r];
                Zh[size_t(c) * n_kr + r] = make_cuComplex(float(z.x), float(z.y));
            }
        HISQ_CUDA(cudaMemcpyAsync(Zd, Zh.data(), sizeof(cuComplex) * Zh.size(), cudaMemcpyHostToDevice, ctx->stream));
        tick(t_rr);
        for (size_t r0 = 0; r0 < size_t(L); r0 += rot_rows) {
            const int len = int(std::min(rot_rows, size_t(L) - r0));
            BLAS(cublasCgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, len, nout, n_kr, &one, fld(0) + r0, L, Zd, n_kr, &zero, Td,
                             len));
            HISQ_CUDA(cudaMemcpy2DAsync(fld(0) + r0, sizeof(cuComplex) * L, Td, sizeof(cuComplex) * len,
                                        sizeof(cuComplex) * len, nout, cudaMemcpyDeviceToDevice, ctx->stream));
        }
        tick(t_rot);
        if (timing)
            fprintf(stderr, "[hisq] block trlm times so far: filter %.2f s, Gram-Schmidt %.2f s, Rayleigh-Ritz %.2f s, "
                            "rotation %.2f s\n", t_filter, t_gs, t_rr, t_rot);
        if (done) break;
        // thick restart: kept Ritz vectors, then the residual block V[n_kr .. n_kr+b)
        HISQ_CUDA(cudaMemcpyAsync(fld(n_keep), fld(n_kr), sf * b, cudaMemcpyDeviceToDevice, ctx->stream));
        std::fill(H.begin(), H.end(), cd(0));
        for (int i = 0; i < n_keep; i++) {
            H[size_t(i) * n_kr + i] = th[order[i]];
            for (int r = 0; r < b; r++) {
                cd acc = 0;
                for (int c = 0; c < b; c++) {
                    const cuDoubleComplex z = Hh[size_t(order[i]) * n_kr + (n_kr - b + c)];
                    acc += Rlast[size_t(c) * b + r] * cd(z.x, z.y);
                }
                H[size_t(i) * n_kr + (n_keep + r)] = acc;             // row n_keep + r, column i
                H[size_t(n_keep + r) * n_kr + i] = std::conj(acc);    // row i, column n_keep + r
            }
        }
        k = n_keep;
    }
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    *conv_out = conv;
    return HISQ_OK;
}

} // namespace hisq
