// noalloc.cu -- the deflated guess of hisq_deflate for callers that may not
// allocate device memory.  All scratch lives in one file-scope device array of
// fixed size; the caller passes its input and output in device memory.
#include <mutex>

#include "internal.cuh"

namespace hisq {
int defl_project_chunks(int Vh);
hisq_status launch_defl_project_ext(hisq_ctx *ctx, int n, int vprec, const void *V, const double *b, double *c_dev,
                                    void *part_buf);
} // namespace hisq

using namespace hisq;

namespace {

// Scratch of hisq_deflate_noalloc: 16 MiB on every device where a context has
// been created, held until the process exits.  Holds the projection partial
// sums (n x chunks complex) and the n coefficients.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

} // namespace

namespace hisq {

// Device address of the scratch array on the current device (ctx->device),
// looked up once per device.  The lookup loads the module that holds the array,
// which is when the device reserves its 16 MiB; hisq_create calls this, so the
// reservation happens at context creation and never inside
// hisq_deflate_noalloc.
hisq_status noalloc_scratch_address(hisq_ctx *ctx, unsigned char **out)
{
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "device index %d out of range", ctx->device);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[ctx->device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_err(ctx, e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_scratch_addr[ctx->device] = p;
    }
    if (out) *out = static_cast<unsigned char *>(g_scratch_addr[ctx->device]);
    return HISQ_OK;
}

} // namespace hisq

extern "C" hisq_status hisq_deflate_noalloc(hisq_ctx *ctx, int n, const double *b_dev, double *x_dev)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!b_dev || !x_dev) return set_err(ctx, HISQ_ERR_INVALID_ARG, "null device field");
    if (ctx->eig.n <= 0 || !ctx->eig.eps_dev) return set_err(ctx, HISQ_ERR_STATE, "no eigenpairs stored");
    if (!(ctx->mass > 0)) return set_err(ctx, HISQ_ERR_STATE, "mass not set");
    if (n <= 0 || n > ctx->eig.n) n = ctx->eig.n;
    const int Vh = ctx->g.Vh;
    const size_t part_bytes = align256(size_t(n) * defl_project_chunks(Vh) * sizeof(double2));
    const size_t c_bytes = align256(size_t(n) * sizeof(double2));
    if (part_bytes + c_bytes > kNoAllocScratchBytes)
        return set_err(ctx, HISQ_ERR_INVALID_ARG,
                       "hisq_deflate_noalloc: %d eigenpairs on %d sites need %zu bytes of scratch, more than the "
                       "fixed %zu; use hisq_deflate or fewer eigenpairs",
                       n, Vh, part_bytes + c_bytes, kNoAllocScratchBytes);
    HISQ_CUDA(cudaSetDevice(ctx->device));
    unsigned char *scratch = nullptr;
    hisq_status st = noalloc_scratch_address(ctx, &scratch);
    if (st != HISQ_OK) return st;
    double *part = reinterpret_cast<double *>(scratch);
    double *c = reinterpret_cast<double *>(scratch + part_bytes);
    // every scratch byte used below is written by this call's kernels before it
    // is read; the eigenvalues come from the device copy kept with the pairs
    st = launch_defl_project_ext(ctx, n, ctx->eig.prec, ctx->eig.vecs, b_dev, c, part);
    if (st != HISQ_OK) return st;
    st = launch_defl_scale(ctx, n, c, ctx->eig.eps_dev, 4.0 * ctx->mass * ctx->mass);
    if (st != HISQ_OK) return st;
    HISQ_CUDA(cudaMemsetAsync(x_dev, 0, spinor_bytes(64, Vh), ctx->stream));
    return launch_defl_expand(ctx, n, ctx->eig.prec, ctx->eig.vecs, c, 1.0, 64, x_dev);
}
