// api.cu -- the C ABI (include/hisq.h): context lifetime, errors, device
// memory, link ingest, the operator test entry points and the eigenpair store.
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>

#include "internal.cuh"

using namespace hisq;

namespace hisq {
void tc_forget(hisq_ctx *ctx);
hisq_status noalloc_scratch_address(hisq_ctx *ctx, unsigned char **out);

int log_level()
{
    static int lvl = -1;
    if (lvl < 0) {
        const char *e = getenv("HISQ_LOG");
        lvl = e ? atoi(e) : 0;
    }
    return lvl;
}

bool tuning_enabled()
{
    static int on = -1;
    if (on < 0) {
        const char *e = getenv("HISQ_TUNE");
        on = (e && atoi(e) == 0) ? 0 : 1;
    }
    return on;
}

bool graphs_enabled(const hisq_ctx *ctx)
{
    static int on = -1;
    if (on < 0) {
        const char *e = getenv("HISQ_GRAPHS");
        on = (e && atoi(e) == 0) ? 0 : 1;
    }
    const cudaStream_t s = ctx->stream;
    return on && s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
}

hisq_status set_err(hisq_ctx *c, hisq_status s, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

hisq_status cuda_err(hisq_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) return set_err(c, HISQ_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return set_err(c, HISQ_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void *dev_alloc(hisq_ctx *c, size_t bytes)
{
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (c->alloc_fail_after == 0) {
        set_err(c, HISQ_ERR_OOM, "allocation of %zu bytes refused (injected failure)", bytes);
        return nullptr;
    }
    if (c->alloc_fail_after > 0) c->alloc_fail_after--;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_err(c, HISQ_ERR_OOM, "cudaMalloc of %zu bytes failed", bytes);
        return nullptr;
    }
    c->bytes += bytes;
    return p;
}

void dev_free(hisq_ctx *c, void *p, size_t bytes)
{
    if (p) {
        cudaFree(p);
        c->bytes -= bytes;
    }
}

void *get_buf(hisq_ctx *c, int id, size_t bytes)
{
    if (c->buf_cap[id] >= bytes && c->bufs[id]) return c->bufs[id];
    if (c->bufs[id]) {
        cudaStreamSynchronize(c->stream);
        dev_free(c, c->bufs[id], c->buf_cap[id]);
        c->bufs[id] = nullptr;
        c->buf_cap[id] = 0;
    }
    void *p = dev_alloc(c, bytes);
    if (!p) return nullptr;
    c->bufs[id] = p;
    c->buf_cap[id] = bytes;
    return p;
}

// device copy of the stored eigenvalues eps (FP64, ascending), written when
// the eigenpairs are stored
double *eig_eps_dev(hisq_ctx *ctx)
{
    if (!ctx->eig.eps_dev) set_err(ctx, HISQ_ERR_STATE, "no eigenpairs stored");
    return ctx->eig.eps_dev;
}

// scalar slot readback (synchronises the stream)
hisq_status read_slots(hisq_ctx *ctx, int slot0, int n, double *out)
{
    HISQ_CUDA(cudaMemcpyAsync(out, &ctx->scal->slot[slot0], sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return HISQ_OK;
}

} // namespace hisq

// ---------------------------------------------------------------------- ABI
extern "C" {

const char *hisq_status_string(hisq_status s)
{
    switch (s) {
    case HISQ_OK: return "ok";
    case HISQ_ERR_INVALID_ARG: return "invalid argument";
    case HISQ_ERR_CUDA: return "CUDA error";
    case HISQ_ERR_OOM: return "out of memory";
    case HISQ_ERR_NOT_CONVERGED: return "not converged";
    case HISQ_ERR_NUMERICAL: return "numerical error (NaN/Inf)";
    case HISQ_ERR_TIMEOUT: return "timeout";
    case HISQ_ERR_STATE: return "invalid call order";
    }
    return "unknown status";
}

const char *hisq_last_error(const hisq_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t hisq_device_bytes(const hisq_ctx *ctx) { return ctx ? ctx->bytes : 0; }

unsigned long long hisq_kernel_launches(const hisq_ctx *ctx) { return ctx ? ctx->launches : 0; }

void hisq_default_solve_params(hisq_solve_params *p)
{
    if (!p) return;
    p->tol = 1e-10;
    p->max_iter = 100000;
    p->precision_sloppy = 32;
    p->link_precision_sloppy = 32;
    p->delta_rd = 0.1;
    p->deflate = 0;
    p->n_defl = 0;
    p->delta_tr = 1e-3;
    p->compute_full_residual = 1;
    p->batch = 1;
    p->guess = 0;
    p->precision_reliable = 64;
    p->persistent = 0;
}

void hisq_default_eig_params(hisq_eig_params *p)
{
    if (!p) return;
    p->n_ev = 16;
    p->n_kr = 64;
    p->n_keep = 0;
    p->tol = 1e-6;
    p->max_restarts = 200;
    p->cheby_degree = 0;
    p->a_min = 0;
    p->a_max = 0;
    p->storage_precision = 32;
    p->seed = 1234;
    p->block_size = 1;
}

hisq_status hisq_create(const int dims[4], int t_antiperiodic, int device, void *cuda_stream, hisq_ctx **out)
{
    if (!out || !dims) return HISQ_ERR_INVALID_ARG;
    *out = nullptr;
    long V = 1;
    for (int i = 0; i < 4; i++) {
        if (dims[i] < 4 || dims[i] % 2 || dims[i] >= (1 << 15)) return HISQ_ERR_INVALID_ARG;
        V *= dims[i];
    }
    if (V / 2 > (1L << 30)) return HISQ_ERR_INVALID_ARG;
    hisq_ctx *ctx = new hisq_ctx();
    ctx->device = device;
    Geom &g = ctx->g;
    g.X = dims[0];
    g.Y = dims[1];
    g.Z = dims[2];
    g.T = dims[3];
    g.X2 = g.X / 2;
    g.V = int(V);
    g.Vh = int(V / 2);
    g.t_antiperiodic = t_antiperiodic ? 1 : 0;
    g.stride[0] = 1;
    g.stride[1] = g.X;
    g.stride[2] = g.X * g.Y;
    g.stride[3] = g.X * g.Y * g.Z;
    g.dX2 = make_fastdiv(g.X2);
    g.dY = make_fastdiv(g.Y);
    g.dZ = make_fastdiv(g.Z);
    auto fail = [&](hisq_status s) {
        hisq_destroy(ctx);
        return s;
    };
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return HISQ_ERR_CUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return fail(HISQ_ERR_CUDA);
    ctx->num_sms = prop.multiProcessorCount;
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(HISQ_ERR_CUDA);
        ctx->own_stream = true;
    }
    ctx->g.oob = (int *)dev_alloc(ctx, sizeof(int));
    if (!ctx->g.oob || cudaMemset(ctx->g.oob, 0, sizeof(int)) != cudaSuccess) return fail(HISQ_ERR_OOM);
    ctx->max_red_blocks = ctx->num_sms * 16;
    ctx->partials = (double *)dev_alloc(ctx, sizeof(double) * ctx->max_red_blocks * kMaxRedVals);
    ctx->ticket = (unsigned int *)dev_alloc(ctx, 256);
    ctx->scal = (DevScalars *)dev_alloc(ctx, sizeof(DevScalars));
    if (!ctx->partials || !ctx->ticket || !ctx->scal) return fail(HISQ_ERR_OOM);
    if (cudaMemset(ctx->ticket, 0, 256) != cudaSuccess || cudaMemset(ctx->scal, 0, sizeof(DevScalars)) != cudaSuccess)
        return fail(HISQ_ERR_CUDA);
    if (cudaHostAlloc((void **)&ctx->monitor_h, sizeof(double) * ctx->monitor_len, cudaHostAllocMapped) != cudaSuccess)
        return fail(HISQ_ERR_OOM);
    if (cudaHostGetDevicePointer((void **)&ctx->monitor_d, ctx->monitor_h, 0) != cudaSuccess) return fail(HISQ_ERR_CUDA);
    ctx->bscal = (BatchScalars *)dev_alloc(ctx, sizeof(BatchScalars));
    ctx->bpartials = (double *)dev_alloc(ctx, sizeof(double) * ctx->max_red_blocks * kMaxBatch);
    if (!ctx->bscal || !ctx->bpartials) return fail(HISQ_ERR_OOM);
    if (cudaMemset(ctx->bscal, 0, sizeof(BatchScalars)) != cudaSuccess) return fail(HISQ_ERR_CUDA);
    if (cudaHostAlloc((void **)&ctx->bmonitor_h, sizeof(double) * ctx->bmonitor_len * kMaxBatch,
                      cudaHostAllocMapped) != cudaSuccess)
        return fail(HISQ_ERR_OOM);
    if (cudaHostGetDevicePointer((void **)&ctx->bmonitor_d, ctx->bmonitor_h, 0) != cudaSuccess) return fail(HISQ_ERR_CUDA);
    if (cudaHostAlloc((void **)&ctx->wait_status_h, sizeof(int), cudaHostAllocMapped) != cudaSuccess)
        return fail(HISQ_ERR_OOM);
    *ctx->wait_status_h = 0;
    if (cudaHostGetDevicePointer((void **)&ctx->wait_status_d, ctx->wait_status_h, 0) != cudaSuccess)
        return fail(HISQ_ERR_CUDA);
    // the fixed scratch of hisq_deflate_noalloc is reserved on this device now,
    // so that the no-allocation entry point itself never causes a reservation
    if (noalloc_scratch_address(ctx, nullptr) != HISQ_OK) return fail(HISQ_ERR_CUDA);
    *out = ctx;
    return HISQ_OK;
}

void hisq_destroy(hisq_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    tc_forget(ctx);
    for (int p = 0; p < 2; p++) {
        cudaFree(ctx->links_d[p]);
        cudaFree(ctx->links_f[p]);
        cudaFree(ctx->links_f12[p]);
        cudaFree(ctx->links_h[p]);
        cudaFree(ctx->links_h12[p]);
        cudaFree(ctx->links_df[p]);
    }
    for (int i = 0; i < BUF_COUNT; i++) cudaFree(ctx->bufs[i]);
    cudaFree(ctx->eig.vecs);
    cudaFree(ctx->eig.eps_dev);
    cudaFree(ctx->partials);
    cudaFree(ctx->g.oob);
    cudaFree(ctx->ticket);
    cudaFree(ctx->scal);
    if (ctx->monitor_h) cudaFreeHost(ctx->monitor_h);
    cudaFree(ctx->bscal);
    cudaFree(ctx->bpartials);
    if (ctx->bmonitor_h) cudaFreeHost(ctx->bmonitor_h);
    if (ctx->wait_status_h) cudaFreeHost(ctx->wait_status_h);
    for (auto &e : ctx->fp64_pending) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    for (cudaEvent_t e : ctx->fp64_pool) cudaEventDestroy(e);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

hisq_status hisq_load_links(hisq_ctx *ctx, const double *fat, const double *lng, int long_recon, double long_scale)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!fat || !lng) return set_err(ctx, HISQ_ERR_INVALID_ARG, "null link array");
    if (long_recon != 18 && long_recon != 12 && long_recon != 8)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "long_recon must be 18, 12 or 8");
    if (long_recon != 18 && (!(std::fabs(long_scale) > 0) || !std::isfinite(long_scale)))
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "long_scale must be finite and non-zero");
    HISQ_CUDA(cudaSetDevice(ctx->device));
    const int Vh = ctx->g.Vh;
    const size_t nlink = size_t(ctx->g.V) * 4 * 18 * sizeof(double);
    // (re)allocate gathered arrays
    for (int p = 0; p < 2; p++) {
        dev_free(ctx, ctx->links_d[p], size_t(Vh) * 16 * 9 * 16);
        ctx->links_d[p] = nullptr;
        dev_free(ctx, ctx->links_f[p], size_t(Vh) * (ctx->long_recon == 18 ? 8 : 4) * 9 * 16);
        ctx->links_f[p] = nullptr;
        dev_free(ctx, ctx->links_f12[p], size_t(Vh) * long_f32_bytes_per_site(ctx->long_recon));
        ctx->links_f12[p] = nullptr;
        dev_free(ctx, ctx->links_h[p], size_t(Vh) * (ctx->long_recon == 18 ? 8 : 4) * 9 * 8);
        ctx->links_h[p] = nullptr;
        dev_free(ctx, ctx->links_h12[p], size_t(Vh) * 4 * 6 * 8);
        ctx->links_h12[p] = nullptr;
        dev_free(ctx, ctx->links_df[p], size_t(Vh) * 16 * 9 * 16);
        ctx->links_df[p] = nullptr;
    }
    ctx->links_loaded = false;
    for (int p = 0; p < 2; p++) {
        ctx->links_d[p] = (double2 *)dev_alloc(ctx, size_t(Vh) * 16 * 9 * 16);
        ctx->links_f[p] = (float4 *)dev_alloc(ctx, size_t(Vh) * (long_recon == 18 ? 8 : 4) * 9 * 16);
        if (long_recon != 18) ctx->links_f12[p] = (float4 *)dev_alloc(ctx, size_t(Vh) * long_f32_bytes_per_site(long_recon));
        if (!ctx->links_d[p] || !ctx->links_f[p] || (long_recon != 18 && !ctx->links_f12[p])) return HISQ_ERR_OOM;
        // FP16 links are built from the FP32 ones on first use (ensure_half_links)
    }
    ctx->long_recon = long_recon;
    ctx->long_scale = long_recon != 18 ? long_scale : 1.0;
    double *stage = nullptr;
    HISQ_CUDA(cudaMalloc(&stage, 2 * nlink));
    cudaError_t e1 = cudaMemcpyAsync(stage, fat, nlink, cudaMemcpyHostToDevice, ctx->stream);
    cudaError_t e2 = cudaMemcpyAsync((char *)stage + nlink, lng, nlink, cudaMemcpyHostToDevice, ctx->stream);
    hisq_status st = HISQ_OK;
    double dev = 0;
    if (e1 != cudaSuccess || e2 != cudaSuccess) st = cuda_err(ctx, e1 != cudaSuccess ? e1 : e2, "link upload");
    if (st == HISQ_OK) st = ingest_links(ctx, stage, (const double *)((char *)stage + nlink), long_recon, long_scale, &dev);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(stage);
    if (st != HISQ_OK) return st;
    if (long_recon != 18 && !(dev <= 1e-6))
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "long links / long_scale are not SU(3) (deviation %.3g)", dev);
    ctx->links_loaded = true;
    return HISQ_OK;
}

hisq_status hisq_set_mass(hisq_ctx *ctx, double m)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!(m > 0) || !std::isfinite(m)) return set_err(ctx, HISQ_ERR_INVALID_ARG, "mass must be positive and finite");
    ctx->mass = m;
    return HISQ_OK;
}

static hisq_status upload_full(hisq_ctx *ctx, const double *host, int id, double **dev)
{
    const size_t bytes = size_t(ctx->g.V) * 6 * sizeof(double);
    *dev = (double *)get_buf(ctx, id, bytes);
    if (!*dev) return HISQ_ERR_OOM;
    HISQ_CUDA(cudaMemcpyAsync(*dev, host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return HISQ_OK;
}

static hisq_status download_full(hisq_ctx *ctx, const double *dev, double *host)
{
    const size_t bytes = size_t(ctx->g.V) * 6 * sizeof(double);
    HISQ_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return HISQ_OK;
}

#define TRY(x)                                  \
    do {                                        \
        hisq_status s_ = (x);                   \
        if (s_ != HISQ_OK) return s_;           \
    } while (0)

static bool bad_precisions(int prec, int link_prec)
{
    if (prec == HISQ_PREC_DF64 || link_prec == HISQ_PREC_DF64) return prec != link_prec;
    if (prec != 64 && prec != 32 && prec != 16) return true;
    if (link_prec != 64 && link_prec != 32 && link_prec != 16) return true;
    return (prec == 64) != (link_prec == 64);
}

hisq_status hisq_apply_dslash(hisq_ctx *ctx, int out_parity, int precision, int link_precision, const double *in,
                              double *out)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!in || !out || (out_parity != 0 && out_parity != 1)) return set_err(ctx, HISQ_ERR_INVALID_ARG, "bad argument");
    if (bad_precisions(precision, link_precision))
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "precisions must be 64/64, 48/48 or 32|16 with 32|16 links");
    if (!ctx->links_loaded) return set_err(ctx, HISQ_ERR_STATE, "links not loaded");
    HISQ_CUDA(cudaSetDevice(ctx->device));
    const int Vh = ctx->g.Vh;
    double *full = nullptr;
    TRY(upload_full(ctx, in, BUF_TEST_A, &full));
    void *a = get_buf(ctx, BUF_TEST_B, spinor_bytes(precision, Vh));
    void *b = get_buf(ctx, BUF_TEST_C, spinor_bytes(precision, Vh));
    if (!a || !b) return HISQ_ERR_OOM;
    if (precision == HISQ_PREC_DF64) {
        void *d = get_buf(ctx, BUF_DF_X, spinor_bytes(HISQ_PREC_DF64, Vh));
        if (!d) return HISQ_ERR_OOM;
        TRY(launch_gather_parity(ctx, full, 1 - out_parity, 64, a));
        TRY(launch_to_df64(ctx, (const double *)a, d));
        TRY(launch_dslash_df_xpay(ctx, out_parity, d, (double *)b, 0, nullptr, 0, nullptr, 1.0, -1));
        HISQ_CUDA(cudaMemsetAsync(full, 0, size_t(ctx->g.V) * 48, ctx->stream));
        TRY(launch_scatter_parity(ctx, b, 64, out_parity, full));
        return download_full(ctx, full, out);
    }
    TRY(launch_gather_parity(ctx, full, 1 - out_parity, precision, a));
    TRY(launch_dslash(ctx, out_parity, precision, link_precision, a, b, 0, nullptr, 0, nullptr, 1.0, -1));
    HISQ_CUDA(cudaMemsetAsync(full, 0, size_t(ctx->g.V) * 48, ctx->stream));
    TRY(launch_scatter_parity(ctx, b, precision, out_parity, full));
    return download_full(ctx, full, out);
}

hisq_status hisq_bounds_violations(hisq_ctx *ctx, int *flag)
{
    if (!ctx || !flag) return HISQ_ERR_INVALID_ARG;
    HISQ_CUDA(cudaSetDevice(ctx->device));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    HISQ_CUDA(cudaMemcpy(flag, ctx->g.oob, sizeof(int), cudaMemcpyDeviceToHost));
    HISQ_CUDA(cudaMemset(ctx->g.oob, 0, sizeof(int)));
#ifdef HISQ_BOUNDS_CHECK
    return HISQ_OK;
#else
    return set_err(ctx, HISQ_ERR_STATE, "library built without HISQ_BOUNDS_CHECK: indices are not checked");
#endif
}

hisq_status hisq_inject_alloc_failure(hisq_ctx *ctx, int after)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    ctx->alloc_fail_after = after < 0 ? -1 : after;
    return HISQ_OK;
}

hisq_status hisq_set_batched_kernel(hisq_ctx *ctx, int kind, int rhs_per_thread, int budget)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (kind < 0 || kind > 3) return set_err(ctx, HISQ_ERR_INVALID_ARG, "kind must be 0, 1, 2 or 3");
    if (kind != 0 && (rhs_per_thread < 2 || rhs_per_thread > 4 || (kind == 3 && rhs_per_thread == 3)))
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "rhs_per_thread must be 2, 3 or 4 (2 or 4 for kind 3)");
    if (((kind == 1 || kind == 3) && (budget < 0 || budget > 1)) || (kind == 2 && (budget < 2 || budget > 4)))
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "budget out of range for this kind");
    ctx->mrhs_force_kind = kind;
    ctx->mrhs_force_R = kind ? rhs_per_thread : 0;
    ctx->mrhs_force_budget = kind ? budget : 0;
    return HISQ_OK;
}

hisq_status hisq_apply_dslash_batch(hisq_ctx *ctx, int out_parity, int precision, int nrhs, const double *in,
                                    double *out)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!in || !out || (out_parity != 0 && out_parity != 1) || nrhs < 1 || nrhs > kMaxBatch)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "bad argument");
    if (precision != 32 && precision != 16) return set_err(ctx, HISQ_ERR_INVALID_ARG, "precision must be 32 or 16");
    if (!ctx->links_loaded) return set_err(ctx, HISQ_ERR_STATE, "links not loaded");
    HISQ_CUDA(cudaSetDevice(ctx->device));
    const int Vh = ctx->g.Vh;
    const size_t sb = spinor_bytes(precision, Vh), full_bytes = size_t(ctx->g.V) * 48;
    double *full = (double *)get_buf(ctx, BUF_TEST_A, full_bytes);
    char *a = (char *)get_buf(ctx, BUF_B_P, sb * nrhs);
    char *b = (char *)get_buf(ctx, BUF_B_TMP, sb * nrhs);
    if (!full || !a || !b) return HISQ_ERR_OOM;
    for (int j = 0; j < nrhs; j++) {
        HISQ_CUDA(cudaMemcpyAsync(full, in + size_t(j) * ctx->g.V * 6, full_bytes, cudaMemcpyHostToDevice, ctx->stream));
        TRY(launch_gather_parity(ctx, full, 1 - out_parity, precision, a + sb * j));
    }
    TRY(mrhs_set_identity(ctx, nrhs));
    TRY(launch_mrhs_dslash_store(ctx, out_parity, precision, a, b, nrhs));
    for (int j = 0; j < nrhs; j++) {
        HISQ_CUDA(cudaMemsetAsync(full, 0, full_bytes, ctx->stream));
        TRY(launch_scatter_parity(ctx, b + sb * j, precision, out_parity, full));
        HISQ_CUDA(cudaMemcpyAsync(out + size_t(j) * ctx->g.V * 6, full, full_bytes, cudaMemcpyDeviceToHost, ctx->stream));
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    if (*(volatile int *)ctx->wait_status_h != 0) {
        const int code = *ctx->wait_status_h;
        *ctx->wait_status_h = 0;
        return set_err(ctx, HISQ_ERR_TIMEOUT, "batched operator: a pipeline wait ran out (code %d)", code);
    }
    return HISQ_OK;
}

hisq_status hisq_inject_wait_timeout(hisq_ctx *ctx, int on)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    ctx->inject_wait_timeout = on != 0;
    return HISQ_OK;
}

hisq_status hisq_apply_normal_op(hisq_ctx *ctx, int precision, int link_precision, const double *in, double *out)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!in || !out) return set_err(ctx, HISQ_ERR_INVALID_ARG, "bad argument");
    if (bad_precisions(precision, link_precision))
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "precisions must be 64/64, 48/48 or 32|16 with 32|16 links");
    if (!ctx->links_loaded) return set_err(ctx, HISQ_ERR_STATE, "links not loaded");
    if (!(ctx->mass > 0)) return set_err(ctx, HISQ_ERR_STATE, "mass not set");
    HISQ_CUDA(cudaSetDevice(ctx->device));
    const int Vh = ctx->g.Vh;
    double *full = nullptr;
    TRY(upload_full(ctx, in, BUF_TEST_A, &full));
    void *a = get_buf(ctx, BUF_TEST_B, spinor_bytes(precision, Vh));
    void *b = get_buf(ctx, BUF_TEST_C, spinor_bytes(precision, Vh));
    void *t = get_buf(ctx, BUF_TMP, spinor_bytes(precision, Vh));
    if (!a || !b || !t) return HISQ_ERR_OOM;
    const int lp = link_precision;
    const double m4 = 4.0 * ctx->mass * ctx->mass;
    if (precision == HISQ_PREC_DF64) {
        void *d = get_buf(ctx, BUF_DF_X, spinor_bytes(HISQ_PREC_DF64, Vh));
        void *dt = get_buf(ctx, BUF_DF_T, spinor_bytes(HISQ_PREC_DF64, Vh));
        if (!d || !dt) return HISQ_ERR_OOM;
        TRY(launch_gather_parity(ctx, full, 0, 64, a));
        TRY(launch_to_df64(ctx, (const double *)a, d));
        TRY(launch_dslash_df(ctx, 1, d, dt));                                                        // D_oe a
        TRY(launch_dslash_df_xpay(ctx, 0, dt, (double *)b, m4, (const double *)a, 0, nullptr, -1.0, -1)); // 4m^2 a - D_eo t
        HISQ_CUDA(cudaMemsetAsync(full, 0, size_t(ctx->g.V) * 48, ctx->stream));
        TRY(launch_scatter_parity(ctx, b, 64, 0, full));
        return download_full(ctx, full, out);
    }
    TRY(launch_gather_parity(ctx, full, 0, precision, a));
    TRY(launch_dslash(ctx, 1, precision, lp, a, t, 0, nullptr, 0, nullptr, 1.0, -1));       // t = D_oe a
    TRY(launch_dslash(ctx, 0, precision, lp, t, b, m4, a, 0, nullptr, -1.0, -1));           // b = 4m^2 a - D_eo t
    HISQ_CUDA(cudaMemsetAsync(full, 0, size_t(ctx->g.V) * 48, ctx->stream));
    TRY(launch_scatter_parity(ctx, b, precision, 0, full));
    return download_full(ctx, full, out);
}

} // extern "C"
