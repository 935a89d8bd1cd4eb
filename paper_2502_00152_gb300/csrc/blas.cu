// blas.cu -- one-parity vector kernels: layout conversion, norms and inner
// products with deterministic grid reductions, the CG direction update, the
// deflation projection and expansion of Eq. 4 (x = sum_i v_i lambda_i^-1 v_i^dag b),
// and the Ritz basis rotation of the thick-restart Lanczos eigensolver.
#include <algorithm>

#include "internal.cuh"

namespace hisq {

template <typename K>
static int occ(K kernel, int threads, size_t smem = 0)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) n = 1;
    return n;
}

#define LAUNCH_CHECK(what)                                                  \
    do {                                                                    \
        cudaError_t e_ = cudaGetLastError();                                \
        if (e_ != cudaSuccess) return cuda_err(ctx, e_, what);              \
    } while (0)

// run f(spinor accessor) for a runtime precision
template <class F>
static hisq_status with_spinor(hisq_ctx *ctx, int prec, const void *p, F &&f)
{
    const int Vh = ctx->g.Vh;
    void *q = const_cast<void *>(p);
    switch (prec) {
    case 64: return f(make_spinorD(q, Vh));
    case 32: return f(make_spinorF(q, Vh));
    case 16: return f(make_spinorH(q, Vh));
    case HISQ_PREC_BF16: return f(make_spinorB(q, Vh));
    case HISQ_PREC_HALF_EV: return f(make_spinorE(q, Vh));
    }
    return set_err(ctx, HISQ_ERR_INVALID_ARG, "precision must be 64, 32, 16, 15 (BF16) or 14 (FP16 eigenvectors)");
}

// ------------------------------------------------------------- layout
template <class S>
__global__ void k_gather_parity(Geom g, const double2 *__restrict__ full, int par, S out)
{
    for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < g.Vh; cb += gridDim.x * blockDim.x) {
        int c[4];
        cb_coords(g, par, cb, c);
        const size_t s = full_site(g, c);
        CVec<double> v;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            double2 a = full[3 * s + i];
            v.re[i] = a.x;
            v.im[i] = a.y;
        }
        out.store(cb, cvt<typename S::real>(v));
    }
}

template <class S>
__global__ void k_scatter_parity(Geom g, S in, int par, double2 *__restrict__ full)
{
    for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < g.Vh; cb += gridDim.x * blockDim.x) {
        int c[4];
        cb_coords(g, par, cb, c);
        const size_t s = full_site(g, c);
        CVec<double> v = cvt<double>(in.load(cb));
#pragma unroll
        for (int i = 0; i < 3; i++) full[3 * s + i] = make_double2(v.re[i], v.im[i]);
    }
}

hisq_status launch_gather_parity(hisq_ctx *ctx, const double *full, int parity, int prec, void *out)
{
    return with_spinor(ctx, prec, out, [&](auto S) -> hisq_status {
        auto k = k_gather_parity<decltype(S)>;
        int grid = grid_for(ctx, ctx->g.Vh, 256, occ(k, 256));
        k<<<grid, 256, 0, ctx->stream>>>(ctx->g, (const double2 *)full, parity, S);
        LAUNCH_CHECK("gather_parity");
        return HISQ_OK;
    });
}

hisq_status launch_scatter_parity(hisq_ctx *ctx, const void *in, int prec, int parity, double *full)
{
    return with_spinor(ctx, prec, in, [&](auto S) -> hisq_status {
        auto k = k_scatter_parity<decltype(S)>;
        int grid = grid_for(ctx, ctx->g.Vh, 256, occ(k, 256));
        k<<<grid, 256, 0, ctx->stream>>>(ctx->g, S, parity, (double2 *)full);
        LAUNCH_CHECK("scatter_parity");
        return HISQ_OK;
    });
}

template <class SI, class SO>
__global__ void k_convert(int Vh, SI in, SO out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x)
        out.store(i, cvt<typename SO::real>(in.load(i)));
}

hisq_status launch_convert(hisq_ctx *ctx, const void *in, int prec_in, void *out, int prec_out)
{
    if (prec_in == prec_out) {
        cudaError_t e = cudaMemcpyAsync(out, in, spinor_bytes(prec_in, ctx->g.Vh), cudaMemcpyDeviceToDevice,
                                        ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "convert copy");
        return HISQ_OK;
    }
    return with_spinor(ctx, prec_in, in, [&](auto SI) -> hisq_status {
        return with_spinor(ctx, prec_out, out, [&](auto SO) -> hisq_status {
            auto k = k_convert<decltype(SI), decltype(SO)>;
            int grid = grid_for(ctx, ctx->g.Vh, 256, occ(k, 256));
            k<<<grid, 256, 0, ctx->stream>>>(ctx->g.Vh, SI, SO);
            LAUNCH_CHECK("convert");
            return HISQ_OK;
        });
    });
}

template <class S>
__global__ void k_zero(int Vh, S x)
{
    CVec<typename S::real> z;
    z.zero();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) x.store(i, z);
}

hisq_status launch_zero(hisq_ctx *ctx, void *x, int prec)
{
    cudaError_t e = cudaMemsetAsync(x, 0, spinor_bytes(prec, ctx->g.Vh), ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "zero");
    return HISQ_OK;
}

// ------------------------------------------------------------- reductions
template <class S>
__global__ void __launch_bounds__(256) k_norm2(int Vh, S x, RedArgs ra)
{
    double v[1] = {0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x)
        v[0] += double(x.load(i).norm2());
    grid_reduce<1>(v, ra);
}

hisq_status launch_norm2(hisq_ctx *ctx, int prec, const void *x, int slot)
{
    return with_spinor(ctx, prec, x, [&](auto S) -> hisq_status {
        auto k = k_norm2<decltype(S)>;
        int grid = grid_for(ctx, ctx->g.Vh, 256, occ(k, 256));
        k<<<grid, 256, 0, ctx->stream>>>(ctx->g.Vh, S, red_args(ctx, FIN_STORE, slot));
        LAUNCH_CHECK("norm2");
        return HISQ_OK;
    });
}

template <class S>
__global__ void __launch_bounds__(256) k_cdot(int Vh, S x, S y, RedArgs ra)
{
    double v[2] = {0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
        auto a = x.load(i);
        auto b = y.load(i);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            v[0] += double(a.re[c]) * b.re[c] + double(a.im[c]) * b.im[c];
            v[1] += double(a.re[c]) * b.im[c] - double(a.im[c]) * b.re[c];
        }
    }
    grid_reduce<2>(v, ra);
}

hisq_status launch_cdot(hisq_ctx *ctx, int prec, const void *x, const void *y, int slot)
{
    return with_spinor(ctx, prec, x, [&](auto S) -> hisq_status {
        typedef decltype(S) ST;
        const ST Y = make_like<ST>(const_cast<void *>(y), ctx->g.Vh);
        auto k = k_cdot<ST>;
        int grid = grid_for(ctx, ctx->g.Vh, 256, occ(k, 256));
        k<<<grid, 256, 0, ctx->stream>>>(ctx->g.Vh, S, Y, red_args(ctx, FIN_STORE, slot));
        LAUNCH_CHECK("cdot");
        return HISQ_OK;
    });
}

// y (FP64) += a x
template <class S>
__global__ void k_axpy_d(int Vh, double a, S x, SpinorD y)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
        CVec<double> xv = cvt<double>(x.load(i));
        CVec<double> yv = y.load(i);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            yv.re[c] = fma(a, xv.re[c], yv.re[c]);
            yv.im[c] = fma(a, xv.im[c], yv.im[c]);
        }
        y.store(i, yv);
    }
}

hisq_status launch_axpy_d(hisq_ctx *ctx, double a, const void *x, int xprec, double *y)
{
    return with_spinor(ctx, xprec, x, [&](auto S) -> hisq_status {
        auto k = k_axpy_d<decltype(S)>;
        int grid = grid_for(ctx, ctx->g.Vh, 256, occ(k, 256));
        k<<<grid, 256, 0, ctx->stream>>>(ctx->g.Vh, a, S, make_spinorD(y, ctx->g.Vh));
        LAUNCH_CHECK("axpy_d");
        return HISQ_OK;
    });
}

__global__ void k_axpby_d(int n, double a, const double *__restrict__ x, double b, double *__restrict__ y)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = a * x[i] + b * y[i];
}

hisq_status launch_scale_axpby_d(hisq_ctx *ctx, double a, const double *x, double b, double *y)
{
    const int n = ctx->g.Vh * 6;
    int grid = grid_for(ctx, n, 256, occ(k_axpby_d, 256));
    k_axpby_d<<<grid, 256, 0, ctx->stream>>>(n, a, x, b, y);
    LAUNCH_CHECK("axpby_d");
    return HISQ_OK;
}

// p = r + beta p; |p|^2 (third kernel of a CG iteration)
template <class S>
__global__ void __launch_bounds__(256) k_p_update(int Vh, S r, S p, const DevScalars *scal, RedArgs ra)
{
    typedef typename S::real R;
    const R beta = R(scal->beta);
    double v[1] = {0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Vh; i += gridDim.x * blockDim.x) {
        auto rv = r.load(i);
        auto pv = p.load(i);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            pv.re[c] = fma(beta, pv.re[c], rv.re[c]);
            pv.im[c] = fma(beta, pv.im[c], rv.im[c]);
        }
        p.store(i, pv);
        v[0] += double(pv.norm2());
    }
    grid_reduce<1>(v, ra);
}

hisq_status launch_cg_p_update(hisq_ctx *ctx, int prec, const void *r, void *p)
{
    return with_spinor(ctx, prec, p, [&](auto S) -> hisq_status {
        typedef decltype(S) ST;
        const ST R = make_like<ST>(const_cast<void *>(r), ctx->g.Vh);
        auto k = k_p_update<ST>;
        int grid = grid_for(ctx, ctx->g.Vh, 256, occ(k, 256));
        k<<<grid, 256, 0, ctx->stream>>>(ctx->g.Vh, R, S, ctx->scal, red_args(ctx, FIN_CG_P));
        LAUNCH_CHECK("p_update");
        return HISQ_OK;
    });
}

// ------------------------------------------------------------- deflation
template <class S>
__device__ __forceinline__ S spinor_at(const char *base, size_t stride, int i, int Vh);
template <>
__device__ __forceinline__ SpinorF spinor_at<SpinorF>(const char *base, size_t stride, int i, int Vh)
{
    char *p = const_cast<char *>(base) + stride * i;
    return SpinorF{(float4 *)p, (float2 *)(p + size_t(Vh) * 16), Vh};
}
template <>
__device__ __forceinline__ SpinorH spinor_at<SpinorH>(const char *base, size_t stride, int i, int Vh)
{
    char *p = const_cast<char *>(base) + stride * i;
    return SpinorH{(uint4 *)p, Vh};
}
template <>
__device__ __forceinline__ SpinorB spinor_at<SpinorB>(const char *base, size_t stride, int i, int Vh)
{
    char *p = const_cast<char *>(base) + stride * i;
    return SpinorB{(__nv_bfloat162 *)p, Vh};
}
template <>
__device__ __forceinline__ SpinorE spinor_at<SpinorE>(const char *base, size_t stride, int i, int Vh)
{
    return make_spinorE(const_cast<char *>(base) + stride * i, Vh);
}

constexpr int kDeflVG = 8;        // vectors per block in the projection
constexpr int kDeflSites = 4096;  // sites per block in the projection

// partial[i][chunk] = sum over the chunk's sites of v_i^dag b
// (16 vectors per block with unconditional loads was measured 1.8x slower:
// at 128 registers it halves the resident blocks; 8 vectors fit 80 registers)
template <class SV, class SB>
__global__ void __launch_bounds__(256, 3)
    k_defl_project(int Vh, int n, const char *__restrict__ V0, size_t vstride, SB b, double2 *part, int nchunks)
{
    const int g0 = blockIdx.x * kDeflVG;
    const int chunk = blockIdx.y;
    const int cb0 = chunk * kDeflSites;
    const int cb1 = min(Vh, cb0 + kDeflSites);
    float ar[kDeflVG], ai[kDeflVG];
#pragma unroll
    for (int j = 0; j < kDeflVG; j++) ar[j] = ai[j] = 0.f;
    for (int cb = cb0 + threadIdx.x; cb < cb1; cb += blockDim.x) {
        CVec<float> bv = cvt<float>(b.load(cb));
        // every vector's load is unconditional (a vector past n reads vector
        // n - 1 and is not accumulated), so all of them are in flight at once
        CVec<float> v[kDeflVG];
#pragma unroll
        for (int j = 0; j < kDeflVG; j++) v[j] = spinor_at<SV>(V0, vstride, min(g0 + j, n - 1), Vh).load(cb);
#pragma unroll
        for (int j = 0; j < kDeflVG; j++) {
            if (g0 + j < n) {
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    ar[j] = fmaf(v[j].re[c], bv.re[c], fmaf(v[j].im[c], bv.im[c], ar[j]));
                    ai[j] = fmaf(v[j].re[c], bv.im[c], fmaf(-v[j].im[c], bv.re[c], ai[j]));
                }
            }
        }
    }
    // block reduction (fixed order)
    __shared__ double sh[2 * kDeflVG][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kDeflVG; j++) {
        double xr = ar[j], xi = ai[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            xr += __shfl_down_sync(0xffffffffu, xr, o);
            xi += __shfl_down_sync(0xffffffffu, xi, o);
        }
        if (lane == 0) {
            sh[2 * j][warp] = xr;
            sh[2 * j + 1][warp] = xi;
        }
    }
    __syncthreads();
    if (threadIdx.x < kDeflVG && g0 + threadIdx.x < n) {
        const int j = threadIdx.x;
        double xr = 0, xi = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            xr += sh[2 * j][w];
            xi += sh[2 * j + 1][w];
        }
        part[size_t(g0 + j) * nchunks + chunk] = make_double2(xr, xi);
    }
}

// c_i = sum_chunks partial[i][chunk] (fixed order); optional d_i = c_i / lam_i
__global__ void k_defl_finish(int n, int nchunks, const double2 *part, double2 *c, const double *lam, double shift)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double xr = 0, xi = 0;
        const double2 *q = part + size_t(i) * nchunks;
        for (int k = 0; k < nchunks; k++) {
            xr += q[k].x;
            xi += q[k].y;
        }
        if (lam) {
            const double l = lam[i] + shift;
            xr /= l;
            xi /= l;
        }
        c[i] = make_double2(xr, xi);
    }
}

static hisq_status ensure_defl_scratch(hisq_ctx *ctx, size_t bytes, double2 **out);

hisq_status launch_defl_project(hisq_ctx *ctx, int n, int vprec, const void *V, int bprec, const void *b,
                                double *c_dev)
{
    const int Vh = ctx->g.Vh;
    const int nchunks = (Vh + kDeflSites - 1) / kDeflSites;
    double2 *part = nullptr;
    hisq_status st = ensure_defl_scratch(ctx, size_t(n) * nchunks * sizeof(double2), &part);
    if (st != HISQ_OK) return st;
    dim3 grid((n + kDeflVG - 1) / kDeflVG, nchunks);
    const size_t stride = spinor_bytes(vprec, Vh);
    if (vprec != 32 && vprec != 16 && vprec != HISQ_PREC_BF16 && vprec != HISQ_PREC_HALF_EV)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "eigenvector precision must be 32, 16, 15 (BF16) or 14 (FP16)");
    if (bprec != 64 && bprec != 32) return set_err(ctx, HISQ_ERR_INVALID_ARG, "projected vector must be FP64 or FP32");
    void *bb = const_cast<void *>(b);
    if (vprec == 32 && bprec == 64)
        k_defl_project<SpinorF, SpinorD><<<grid, 256, 0, ctx->stream>>>(Vh, n, (const char *)V, stride, make_spinorD(bb, Vh), part, nchunks);
    else if (vprec == 32)
        k_defl_project<SpinorF, SpinorF><<<grid, 256, 0, ctx->stream>>>(Vh, n, (const char *)V, stride, make_spinorF(bb, Vh), part, nchunks);
    else if (vprec == HISQ_PREC_BF16 && bprec == 64)
        k_defl_project<SpinorB, SpinorD><<<grid, 256, 0, ctx->stream>>>(Vh, n, (const char *)V, stride, make_spinorD(bb, Vh), part, nchunks);
    else if (vprec == HISQ_PREC_BF16)
        k_defl_project<SpinorB, SpinorF><<<grid, 256, 0, ctx->stream>>>(Vh, n, (const char *)V, stride, make_spinorF(bb, Vh), part, nchunks);
    else if (vprec == HISQ_PREC_HALF_EV && bprec == 64)
        k_defl_project<SpinorE, SpinorD><<<grid, 256, 0, ctx->stream>>>(Vh, n, (const char *)V, stride, make_spinorD(bb, Vh), part, nchunks);
    else if (vprec == HISQ_PREC_HALF_EV)
        k_defl_project<SpinorE, SpinorF><<<grid, 256, 0, ctx->stream>>>(Vh, n, (const char *)V, stride, make_spinorF(bb, Vh), part, nchunks);
    else if (bprec == 64)
        k_defl_project<SpinorH, SpinorD><<<grid, 256, 0, ctx->stream>>>(Vh, n, (const char *)V, stride, make_spinorD(bb, Vh), part, nchunks);
    else
        k_defl_project<SpinorH, SpinorF><<<grid, 256, 0, ctx->stream>>>(Vh, n, (const char *)V, stride, make_spinorF(bb, Vh), part, nchunks);
    LAUNCH_CHECK("defl_project");
    ctx->launches += 2;
    k_defl_finish<<<(n + 127) / 128, 128, 0, ctx->stream>>>(n, nchunks, part, (double2 *)c_dev, nullptr, 0.0);
    LAUNCH_CHECK("defl_finish");
    return HISQ_OK;
}

// x += coef * sum_i d_i v_i  (d in FP64 on the device, FP32 accumulation per site)
template <class SV, class SX>
__global__ void __launch_bounds__(256)
    k_defl_expand(int Vh, int n, const char *__restrict__ V0, size_t vstride, const double2 *d, double coef, SX x)
{
    extern __shared__ float2 sd[];
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        sd[i] = make_float2(float(coef * d[i].x), float(coef * d[i].y));
    __syncthreads();
    for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < Vh; cb += gridDim.x * blockDim.x) {
        CVec<float> acc;
        acc.zero();
#pragma unroll 4
        for (int i = 0; i < n; i++) {
            CVec<float> v = spinor_at<SV>(V0, vstride, i, Vh).load(cb);
            const float2 w = sd[i];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                acc.re[c] = fmaf(w.x, v.re[c], fmaf(-w.y, v.im[c], acc.re[c]));
                acc.im[c] = fmaf(w.x, v.im[c], fmaf(w.y, v.re[c], acc.im[c]));
            }
        }
        auto xv = x.load(cb);
        typedef typename SX::real XR;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            xv.re[c] += XR(acc.re[c]);
            xv.im[c] += XR(acc.im[c]);
        }
        x.store(cb, xv);
    }
}

template <class SV, class SX>
static hisq_status expand_go(hisq_ctx *ctx, int n, const void *V, size_t stride, const double *d, double coef, SX xs,
                             size_t smem)
{
    auto k = k_defl_expand<SV, SX>;
    int grid = grid_for(ctx, ctx->g.Vh, 256, occ(k, 256, smem));
    k<<<grid, 256, smem, ctx->stream>>>(ctx->g.Vh, n, (const char *)V, stride, (const double2 *)d, coef, xs);
    LAUNCH_CHECK("defl_expand");
    return HISQ_OK;
}

hisq_status launch_defl_expand(hisq_ctx *ctx, int n, int vprec, const void *V, const double *d_dev, double coef,
                               int xprec, void *x)
{
    const int Vh = ctx->g.Vh;
    if (n > 6144) return set_err(ctx, HISQ_ERR_INVALID_ARG, "at most 6144 deflation vectors");
    const size_t smem = size_t(n) * sizeof(float2);
    const size_t stride = spinor_bytes(vprec, Vh);
    if (vprec == 32 && xprec == 64) return expand_go<SpinorF>(ctx, n, V, stride, d_dev, coef, make_spinorD(x, Vh), smem);
    if (vprec == 32 && xprec == 32) return expand_go<SpinorF>(ctx, n, V, stride, d_dev, coef, make_spinorF(x, Vh), smem);
    if (vprec == 16 && xprec == 64) return expand_go<SpinorH>(ctx, n, V, stride, d_dev, coef, make_spinorD(x, Vh), smem);
    if (vprec == 16 && xprec == 32) return expand_go<SpinorH>(ctx, n, V, stride, d_dev, coef, make_spinorF(x, Vh), smem);
    if (vprec == HISQ_PREC_BF16 && xprec == 64)
        return expand_go<SpinorB>(ctx, n, V, stride, d_dev, coef, make_spinorD(x, Vh), smem);
    if (vprec == HISQ_PREC_BF16 && xprec == 32)
        return expand_go<SpinorB>(ctx, n, V, stride, d_dev, coef, make_spinorF(x, Vh), smem);
    if (vprec == HISQ_PREC_HALF_EV && xprec == 64)
        return expand_go<SpinorE>(ctx, n, V, stride, d_dev, coef, make_spinorD(x, Vh), smem);
    if (vprec == HISQ_PREC_HALF_EV && xprec == 32)
        return expand_go<SpinorE>(ctx, n, V, stride, d_dev, coef, make_spinorF(x, Vh), smem);
    return set_err(ctx, HISQ_ERR_INVALID_ARG, "bad deflation precisions");
}

// out = s * in (FP32 fields)
__global__ void k_scale_f(int n, float s, const float *__restrict__ in, float *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = s * in[i];
}

hisq_status launch_scale_f(hisq_ctx *ctx, double s, const void *in, void *out)
{
    const int n = ctx->g.Vh * 6;
    int grid = grid_for(ctx, n, 256, occ(k_scale_f, 256));
    k_scale_f<<<grid, 256, 0, ctx->stream>>>(n, float(s), (const float *)in, (float *)out);
    LAUNCH_CHECK("scale_f");
    return HISQ_OK;
}

// counter-based uniform (-1, 1) fill of an FP32 field (splitmix64 of seed and index)
__global__ void k_random_f(int n, unsigned long long seed, float *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned long long z = seed * 0x9E3779B97F4A7C15ull + (unsigned long long)(i + 1) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        out[i] = float(double(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    }
}

hisq_status launch_random_f(hisq_ctx *ctx, unsigned long long seed, void *out)
{
    const int n = ctx->g.Vh * 6;
    int grid = grid_for(ctx, n, 256, occ(k_random_f, 256));
    k_random_f<<<grid, 256, 0, ctx->stream>>>(n, seed, (float *)out);
    LAUNCH_CHECK("random_f");
    return HISQ_OK;
}

// d_i = c_i / (eps_i + shift) on the device
__global__ void k_defl_scale(int n, double2 *c, const double *eps, double shift)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double l = eps[i] + shift;
        c[i] = make_double2(c[i].x / l, c[i].y / l);
    }
}

hisq_status launch_defl_scale(hisq_ctx *ctx, int n, double *c_dev, const double *eps_dev, double shift)
{
    ctx->launches++;
    k_defl_scale<<<(n + 127) / 128, 128, 0, ctx->stream>>>(n, (double2 *)c_dev, eps_dev, shift);
    LAUNCH_CHECK("defl_scale");
    return HISQ_OK;
}

// ------------------------------------------------------------- basis rotation
// Out (Lf x k_out) = In (Lf x k_in) * Y (k_in x k_out), vectors are columns of
// Lf floats (rows of FP32 colour-vector storage; ld / ld_out floats between
// columns), Y real (FP64 row major).
constexpr int RBM = 128, RBN = 64, RBK = 16;

__global__ void __launch_bounds__(256)
    k_rotate(int Lf, int k_in, int k_out, const float *__restrict__ In, size_t ld, const double *__restrict__ Y,
             float *__restrict__ Out, size_t ld_out)
{
    __shared__ __align__(16) float As[RBK][RBM];
    __shared__ __align__(16) float Bs[RBK][RBN];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.x * RBM, n0 = blockIdx.y * RBN;
    const int tx = tid & 15, ty = tid >> 4; // 16 x 16 threads
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.f;

    for (int k0 = 0; k0 < k_in; k0 += RBK) {
        { // A tile: 16 vectors x 128 floats, 8 floats per thread
            const int kk = tid >> 4, mm = (tid & 15) * 8;
            float4 a0 = make_float4(0, 0, 0, 0), a1 = a0;
            if (k0 + kk < k_in) {
                const float *src = In + size_t(k0 + kk) * ld + m0 + mm;
                if (m0 + mm + 3 < Lf) a0 = *reinterpret_cast<const float4 *>(src);
                if (m0 + mm + 7 < Lf) a1 = *reinterpret_cast<const float4 *>(src + 4);
            }
            *reinterpret_cast<float4 *>(&As[kk][mm]) = a0;
            *reinterpret_cast<float4 *>(&As[kk][mm + 4]) = a1;
        }
        { // B tile: 16 x 64, 4 per thread
            const int kk = tid >> 4, nn = (tid & 15) * 4;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int r = k0 + kk, c = n0 + nn + j;
                Bs[kk][nn + j] = (r < k_in && c < k_out) ? float(Y[size_t(r) * k_out + c]) : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < RBK; kk++) {
            float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][tx * 8]);
            float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][tx * 8 + 4]);
            float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][ty * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int c = n0 + ty * 4 + j;
        if (c >= k_out) continue;
        float *dst = Out + size_t(c) * ld_out + m0 + tx * 8;
        if (m0 + tx * 8 + 3 < Lf) *reinterpret_cast<float4 *>(dst) = make_float4(acc[0][j], acc[1][j], acc[2][j], acc[3][j]);
        if (m0 + tx * 8 + 7 < Lf) *reinterpret_cast<float4 *>(dst + 4) = make_float4(acc[4][j], acc[5][j], acc[6][j], acc[7][j]);
    }
}

// V[:, 0..k_out) = V[:, 0..k_in) Y in place (k_out <= k_in): rows of V are taken
// in chunks of `chunk` floats (a multiple of RBM), each chunk rotated into
// `tmp` (k_out x chunk floats) and copied back, so no second basis is needed.
hisq_status launch_rotate_inplace(hisq_ctx *ctx, int k_in, int k_out, void *V, const double *Y_dev, float *tmp,
                                  int chunk)
{
    const int Lf = 6 * ctx->g.Vh;
    const size_t ld = size_t(ctx->g.Vh) * 6;
    if (k_out > k_in || chunk < RBM || chunk % RBM) return set_err(ctx, HISQ_ERR_INVALID_ARG, "in-place rotation shape");
    for (int m0 = 0; m0 < Lf; m0 += chunk) {
        const int len = std::min(chunk, Lf - m0);
        dim3 grid((len + RBM - 1) / RBM, (k_out + RBN - 1) / RBN);
        ctx->launches++;
        k_rotate<<<grid, 256, 0, ctx->stream>>>(len, k_in, k_out, (const float *)V + m0, ld, Y_dev, tmp, size_t(chunk));
        LAUNCH_CHECK("rotate chunk");
        cudaError_t e = cudaMemcpy2DAsync((float *)V + m0, ld * sizeof(float), tmp, size_t(chunk) * sizeof(float),
                                          size_t(len) * sizeof(float), size_t(k_out), cudaMemcpyDeviceToDevice,
                                          ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "rotate copy-back");
    }
    return HISQ_OK;
}

// ------------------------------------------------------------- scratch
static hisq_status ensure_defl_scratch(hisq_ctx *ctx, size_t bytes, double2 **out)
{
    void *p = get_buf(ctx, BUF_DEFL_PART, bytes);
    if (!p) return HISQ_ERR_OOM;
    *out = (double2 *)p;
    return HISQ_OK;
}

} // namespace hisq

namespace hisq {

// number of site chunks of the deflation projection (partials per vector)
int defl_project_chunks(int Vh) { return (Vh + kDeflSites - 1) / kDeflSites; }

// The projection c_i = v_i^dag b with the partial sums in a buffer the caller
// provides (at least n * defl_project_chunks(Vh) double2); b is FP64.
hisq_status launch_defl_project_ext(hisq_ctx *ctx, int n, int vprec, const void *V, const double *b, double *c_dev,
                                    void *part_buf)
{
    const int Vh = ctx->g.Vh;
    const int nchunks = defl_project_chunks(Vh);
    double2 *part = (double2 *)part_buf;
    dim3 grid((n + kDeflVG - 1) / kDeflVG, nchunks);
    const size_t stride = spinor_bytes(vprec, Vh);
    SpinorD bs = make_spinorD(const_cast<double *>(b), Vh);
    if (vprec == 32)
        k_defl_project<SpinorF, SpinorD><<<grid, 256, 0, ctx->stream>>>(Vh, n, (const char *)V, stride, bs, part, nchunks);
    else if (vprec == 16)
        k_defl_project<SpinorH, SpinorD><<<grid, 256, 0, ctx->stream>>>(Vh, n, (const char *)V, stride, bs, part, nchunks);
    else if (vprec == HISQ_PREC_BF16)
        k_defl_project<SpinorB, SpinorD><<<grid, 256, 0, ctx->stream>>>(Vh, n, (const char *)V, stride, bs, part, nchunks);
    else if (vprec == HISQ_PREC_HALF_EV)
        k_defl_project<SpinorE, SpinorD><<<grid, 256, 0, ctx->stream>>>(Vh, n, (const char *)V, stride, bs, part, nchunks);
    else
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "eigenvector precision must be 32, 16, 15 (BF16) or 14 (FP16)");
    LAUNCH_CHECK("defl_project_ext");
    ctx->launches += 2;
    k_defl_finish<<<(n + 127) / 128, 128, 0, ctx->stream>>>(n, nchunks, part, (double2 *)c_dev, nullptr, 0.0);
    LAUNCH_CHECK("defl_finish_ext");
    return HISQ_OK;
}

} // namespace hisq

namespace hisq {

// One pass over the eigenvectors for a deflation step on an FP64 pair (x, r):
//   x += sum_i c_i / (eps_i + shift) v_i,   r -= sum_i c_i v_i
// With A v_i = lambda_i v_i (lambda_i = eps_i + shift) the second update is the
// residual change of the first, so r stays b - A x without applying A.
template <class SV>
__global__ void __launch_bounds__(256) k_defl_expand2(int Vh, int n, const char *__restrict__ V0, size_t vstride,
                                                      const double2 *c, const double *eps, double shift, SpinorD x,
                                                      SpinorD r)
{
    extern __shared__ float smem[];
    float2 *sc = reinterpret_cast<float2 *>(smem);
    float *sinv = smem + 2 * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sc[i] = make_float2(float(c[i].x), float(c[i].y));
        sinv[i] = float(1.0 / (eps[i] + shift));
    }
    __syncthreads();
    for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < Vh; cb += gridDim.x * blockDim.x) {
        CVec<float> ax, ar;
        ax.zero();
        ar.zero();
#pragma unroll 4
        for (int i = 0; i < n; i++) {
            CVec<float> v = spinor_at<SV>(V0, vstride, i, Vh).load(cb);
            const float2 w = sc[i];
            const float s = sinv[i];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float pr = fmaf(w.x, v.re[k], -w.y * v.im[k]);
                const float pi = fmaf(w.x, v.im[k], w.y * v.re[k]);
                ar.re[k] += pr;
                ar.im[k] += pi;
                ax.re[k] = fmaf(s, pr, ax.re[k]);
                ax.im[k] = fmaf(s, pi, ax.im[k]);
            }
        }
        CVec<double> xv = x.load(cb), rv = r.load(cb);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            xv.re[k] += double(ax.re[k]);
            xv.im[k] += double(ax.im[k]);
            rv.re[k] -= double(ar.re[k]);
            rv.im[k] -= double(ar.im[k]);
        }
        x.store(cb, xv);
        r.store(cb, rv);
    }
}

hisq_status launch_defl_expand2(hisq_ctx *ctx, int n, int vprec, const void *V, const double *c_dev,
                                const double *eps_dev, double shift, double *x, double *r)
{
    const int Vh = ctx->g.Vh;
    if (n > 4096) return set_err(ctx, HISQ_ERR_INVALID_ARG, "dual expansion supports at most 4096 vectors");
    const size_t smem = size_t(n) * 12;
    const size_t stride = spinor_bytes(vprec, Vh);
    SpinorD xs = make_spinorD(x, Vh), rs = make_spinorD(r, Vh);
    if (vprec == 32) {
        auto k = k_defl_expand2<SpinorF>;
        int grid = grid_for(ctx, Vh, 256, occ(k, 256, smem));
        k<<<grid, 256, smem, ctx->stream>>>(Vh, n, (const char *)V, stride, (const double2 *)c_dev, eps_dev, shift, xs, rs);
    } else if (vprec == 16) {
        auto k = k_defl_expand2<SpinorH>;
        int grid = grid_for(ctx, Vh, 256, occ(k, 256, smem));
        k<<<grid, 256, smem, ctx->stream>>>(Vh, n, (const char *)V, stride, (const double2 *)c_dev, eps_dev, shift, xs, rs);
    } else if (vprec == HISQ_PREC_BF16) {
        auto k = k_defl_expand2<SpinorB>;
        int grid = grid_for(ctx, Vh, 256, occ(k, 256, smem));
        k<<<grid, 256, smem, ctx->stream>>>(Vh, n, (const char *)V, stride, (const double2 *)c_dev, eps_dev, shift, xs, rs);
    } else if (vprec == HISQ_PREC_HALF_EV) {
        auto k = k_defl_expand2<SpinorE>;
        int grid = grid_for(ctx, Vh, 256, occ(k, 256, smem));
        k<<<grid, 256, smem, ctx->stream>>>(Vh, n, (const char *)V, stride, (const double2 *)c_dev, eps_dev, shift, xs, rs);
    } else {
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "eigenvector precision must be 32, 16, 15 or 14");
    }
    LAUNCH_CHECK("defl_expand2");
    return HISQ_OK;
}

} // namespace hisq
