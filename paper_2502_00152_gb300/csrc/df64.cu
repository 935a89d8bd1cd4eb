// df64.cu -- the reliable-update residual r = b - A x (A = 4m^2 - D_eo D_oe,
// Section 3) in double-float arithmetic on the FP32 units.
//
// GB300 issues FP64 at 1/64 of its FP32 rate, so the FP64 Dslash of the
// reliable updates is bound by the FP64 pipe (about 1.1 TFLOP/s), not by HBM.
// Here every real number is the unevaluated sum hi + lo of two FP32 numbers
// (Dekker's double-length arithmetic, 1971): a product of two such numbers is
// made exact in its leading part with one FMA (two-product) and every addition
// keeps its rounding error through Knuth's two-sum, so each of the 96 terms of
// an output component enters with a relative error of about 2^-47 (FP64:
// 2^-53) and the kernel runs on the FP32 pipes at the HBM rate of its 2.3 KB of
// link data per site.  The solver certifies the final residual in FP64 before
// it reports convergence.
//
// Storage (one parity, Vh sites):
//   links: float4 [p][mu][kind][fwd,bwd][k=0..8][Vh], float4 = (re_hi, re_lo,
//          im_hi, im_lo) of element k of the gathered FP64 hop matrix (the
//          same matrices as the FP64 copy, phases and signs folded in)
//   colour vectors: float4 [3][Vh] = (re_hi, re_lo, im_hi, im_lo)   48 B / site
#include <algorithm>

#include "internal.cuh"

namespace hisq {

// ---------------------------------------------------------- arithmetic
// the (hi, lo) split of an FP64 number: hi = fl32(d), lo = fl32(d - hi)
__device__ __forceinline__ float2 split_df(double d)
{
    const float hi = __double2float_rn(d);
    return make_float2(hi, __double2float_rn(d - double(hi)));
}

// S + E += (ah + al) * (bh + bl): S is a running FP32 sum, E collects the
// rounding error of every product and of every addition into S.
__device__ __forceinline__ void df_mac(float &S, float &E, float ah, float al, float bh, float bl)
{
    const float p = __fmul_rn(ah, bh);
    float q = __fmaf_rn(ah, bh, -p); // ah * bh = p + q exactly
    q = __fmaf_rn(ah, bl, q);
    q = __fmaf_rn(al, bh, q);        // al * bl (relative size 2^-48) is dropped
    const float t = __fadd_rn(S, p); // two-sum: S + p = t + err exactly
    const float z = __fsub_rn(t, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(t, z)), __fsub_rn(p, z));
    S = t;
    E = __fadd_rn(E, __fadd_rn(err, q));
}

// (S, E) -> normalised (hi, lo) with hi = fl32(S + E) (two-sum)
__device__ __forceinline__ float2 df_norm(float S, float E)
{
    const float h = __fadd_rn(S, E);
    const float z = __fsub_rn(h, S);
    return make_float2(h, __fadd_rn(__fsub_rn(S, __fsub_rn(h, z)), __fsub_rn(E, z)));
}

// accumulator of one colour vector: (S, E) of re and im of three colours
struct AccDF {
    float S[6], E[6];
};

// acc += W v for one complex matrix element W_ij and colour component v_j
__device__ __forceinline__ void cmac_df(AccDF &a, int i, float4 w, float4 v)
{
    df_mac(a.S[2 * i], a.E[2 * i], w.x, w.y, v.x, v.y);       //  Re W Re v
    df_mac(a.S[2 * i], a.E[2 * i], -w.z, -w.w, v.z, v.w);     // -Im W Im v
    df_mac(a.S[2 * i + 1], a.E[2 * i + 1], w.x, w.y, v.z, v.w); // Re W Im v
    df_mac(a.S[2 * i + 1], a.E[2 * i + 1], w.z, w.w, v.x, v.y); // Im W Re v
}

// ------------------------------------------------------------- epilogues
// out (double-float colour vector) = D in
struct EpiDFStore {
    float4 *out;
    int Vh;
    __device__ __forceinline__ void operator()(int cb, const AccDF &a, double &) const
    {
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float2 re = df_norm(a.S[2 * c], a.E[2 * c]);
            const float2 im = df_norm(a.S[2 * c + 1], a.E[2 * c + 1]);
            out[size_t(c) * Vh + cb] = make_float4(re.x, re.y, im.x, im.y);
        }
    }
};

// out (FP64) = a x + b y + c D in, optional |out|^2
struct EpiDFXpay {
    double2 *out;
    const double2 *x, *y;
    double a, b, c;
    int Vh;
    int want_norm;
    __device__ __forceinline__ void operator()(int cb, const AccDF &acc, double &red) const
    {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const size_t i = size_t(k) * Vh + cb;
            double re = c * (double(acc.S[2 * k]) + double(acc.E[2 * k]));
            double im = c * (double(acc.S[2 * k + 1]) + double(acc.E[2 * k + 1]));
            if (x) {
                const double2 v = x[i];
                re = fma(a, v.x, re);
                im = fma(a, v.y, im);
            }
            if (y) {
                const double2 v = y[i];
                re = fma(b, v.x, re);
                im = fma(b, v.y, im);
            }
            out[i] = make_double2(re, im);
            if (want_norm) red += re * re + im * im;
        }
    }
};

// ------------------------------------------------------------- the kernel
// One thread per output site; the 16 hop matrices are streamed (read once per
// launch), the 16 neighbour colour vectors come from L2.
// One resident block of 256 threads is all the bound asks for: the compiler
// then keeps a whole hop matrix of loads in flight per thread (106 registers,
// 16 warps per SM), which measured faster than 64 registers at 32 warps per SM
// and than an L2 prefetch of the next direction's links.
template <class Epi>
__global__ void __launch_bounds__(256, 1)
    k_dslash_df(Geom g, int par, const float4 *__restrict__ L, const float4 *__restrict__ in, Epi epi, RedArgs ra,
                int do_red)
{
    const int Vh = g.Vh;
    double red = 0;
    for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < Vh; cb += gridDim.x * blockDim.x) {
        int c[4];
        cb_coords(g, par, cb, c);
        const int s = full_site(g, c);
        AccDF acc;
#pragma unroll
        for (int k = 0; k < 6; k++) acc.S[k] = acc.E[k] = 0.f;
#pragma unroll 1
        for (int mu = 0; mu < 4; mu++) {
#pragma unroll
            for (int h = 0; h < 4; h++) { // fat fwd, fat bwd, long fwd, long bwd
                const int kind = h >> 1, bwd = h & 1;
                const int nb = nb_cb(g, c, s, mu, (kind ? 3 : 1) * (bwd ? -1 : 1));
                float4 v[3];
#pragma unroll
                for (int j = 0; j < 3; j++) v[j] = in[size_t(j) * Vh + nb];
                const float4 *w = L + size_t(((mu * 2 + kind) * 2 + bwd) * 9) * Vh + cb;
#pragma unroll
                for (int i = 0; i < 3; i++)
#pragma unroll
                    for (int j = 0; j < 3; j++) cmac_df(acc, i, __ldcs(w + size_t(3 * i + j) * Vh), v[j]);
            }
        }
        epi(cb, acc, red);
    }
    if (do_red) {
        double v[1] = {red};
        grid_reduce<1>(v, ra);
    }
}

__global__ void k_split_df(size_t n, const double2 *__restrict__ in, float4 *__restrict__ out)
{
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        const double2 d = in[i];
        const float2 re = split_df(d.x), im = split_df(d.y);
        out[i] = make_float4(re.x, re.y, im.x, im.y);
    }
}

// ------------------------------------------------------------- launch glue
static hisq_status launch_split(hisq_ctx *ctx, size_t n, const double2 *in, float4 *out)
{
    ctx->launches++;
    k_split_df<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(n, in, out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HISQ_OK : cuda_err(ctx, e, "double-float split");
}

// the double-float links exist once a double-float operator is first applied
hisq_status ensure_df_links(hisq_ctx *ctx)
{
    if (ctx->links_df[0]) return HISQ_OK;
    if (!ctx->links_loaded) return set_err(ctx, HISQ_ERR_STATE, "links not loaded");
    const size_t n = size_t(ctx->g.Vh) * 16 * 9;
    float4 *d[2] = {(float4 *)dev_alloc(ctx, n * sizeof(float4)), nullptr};
    if (d[0]) d[1] = (float4 *)dev_alloc(ctx, n * sizeof(float4));
    hisq_status s = (d[0] && d[1]) ? HISQ_OK : HISQ_ERR_OOM;
    for (int p = 0; p < 2 && s == HISQ_OK; p++) s = launch_split(ctx, n, ctx->links_d[p], d[p]);
    if (s != HISQ_OK) { // neither parity is kept, so the next call starts over (message set by the failing call)
        for (int p = 0; p < 2; p++) dev_free(ctx, d[p], d[p] ? n * sizeof(float4) : 0);
        return s;
    }
    ctx->links_df[0] = d[0];
    ctx->links_df[1] = d[1];
    return HISQ_OK;
}

hisq_status launch_to_df64(hisq_ctx *ctx, const double *in, void *out)
{
    return launch_split(ctx, size_t(ctx->g.Vh) * 3, (const double2 *)in, (float4 *)out);
}

template <class Epi>
static hisq_status run_df(hisq_ctx *ctx, int par, const void *in, const Epi &epi, RedArgs ra, int do_red)
{
    if (!ctx->links_loaded) return set_err(ctx, HISQ_ERR_STATE, "links not loaded");
    const hisq_status s = ensure_df_links(ctx);
    if (s != HISQ_OK) return s;
    auto kern = k_dslash_df<Epi>;
    static int bps = -1;
    if (bps < 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 256, 0) != cudaSuccess || bps < 1))
        bps = 1;
    const int grid = grid_for(ctx, ctx->g.Vh, 256, bps);
    kern<<<grid, 256, 0, ctx->stream>>>(ctx->g, par, ctx->links_df[par], (const float4 *)in, epi, ra, do_red);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HISQ_OK : cuda_err(ctx, e, "double-float dslash launch");
}

hisq_status launch_dslash_df(hisq_ctx *ctx, int out_parity, const void *in, void *out)
{
    return run_df(ctx, out_parity, in, EpiDFStore{(float4 *)out, ctx->g.Vh}, red_args(ctx, FIN_STORE), 0);
}

hisq_status launch_dslash_df_xpay(hisq_ctx *ctx, int out_parity, const void *in, double *out, double a,
                                  const double *x, double b, const double *y, double c, int norm_slot)
{
    EpiDFXpay epi{(double2 *)out, (const double2 *)x, (const double2 *)y, a, b, c, ctx->g.Vh, norm_slot >= 0};
    return run_df(ctx, out_parity, in, epi, red_args(ctx, FIN_STORE, norm_slot < 0 ? 0 : norm_slot), norm_slot >= 0);
}

// r = b - A x = b - 4m^2 x + D_eo D_oe x, |r|^2 -> slot (x, b, r: FP64 even fields)
hisq_status launch_residual_df(hisq_ctx *ctx, const double *b, const double *x, double *r, int slot)
{
    const int Vh = ctx->g.Vh;
    void *xd = get_buf(ctx, BUF_DF_X, spinor_bytes(HISQ_PREC_DF64, Vh));
    void *td = get_buf(ctx, BUF_DF_T, spinor_bytes(HISQ_PREC_DF64, Vh));
    if (!xd || !td) return HISQ_ERR_OOM;
    const double m4 = 4.0 * ctx->mass * ctx->mass;
    hisq_status s = launch_to_df64(ctx, x, xd);
    if (s == HISQ_OK) s = launch_dslash_df(ctx, 1, xd, td);
    if (s == HISQ_OK) s = launch_dslash_df_xpay(ctx, 0, td, r, -m4, x, 1.0, b, 1.0, slot);
    return s;
}


// ------------------------------------------------- several right-hand sides
// The reliable updates of a batched solve that fall in the same round are
// computed together.  A block holds one group of 32 consecutive sites and up to
// 8 warps, warp w taking field blockIdx.y * 8 + w: the warps of a block load the
// same link lines at about the same time, so after the first they come from L1
// and the links (2304 B per site) leave DRAM about once per 8 fields, while
// every warp keeps the register budget of the one-field kernel (two blocks of
// 8 warps per SM).  The arithmetic per field is that of k_dslash_df.
struct DFGroup {
    int k;               // fields in the group (<= kMaxBatch)
    int id[kMaxBatch];   // group slot -> right-hand-side index
};

struct DFBatchOut {
    float4 *t;           // store: k double-float fields at a stride of 3 Vh float4
    double2 *r;          // residual: r_id = b_id - m4 x_id + D t_slot at a stride of 3 Vh double2
    const double2 *x, *b;
    double m4;
};

constexpr int kDFWarps = 8;

template <bool STORE>
__global__ void __launch_bounds__(256, 2)
    k_dslash_df_batch(Geom g, int par, const float4 *__restrict__ L, const float4 *__restrict__ in, DFBatchOut o,
                      DFGroup grp, double *partials, unsigned int *ticket, double *norms)
{
    const int Vh = g.Vh;
    const size_t fs = size_t(3) * Vh;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int q = blockIdx.y * (blockDim.x >> 5) + w; // field of this warp
    const bool on = q < grp.k;                         // warp-uniform
    double red = 0;
    if (on) {
        const float4 *src = in + size_t(q) * fs;
        for (int sg = blockIdx.x; sg * 32 < Vh; sg += gridDim.x) {
            const int cb = sg * 32 + lane;
            if (cb >= Vh) continue;
            int cc[4];
            cb_coords(g, par, cb, cc);
            const int s = full_site(g, cc);
            AccDF acc;
#pragma unroll
            for (int u = 0; u < 6; u++) acc.S[u] = acc.E[u] = 0.f;
#pragma unroll 1
            for (int mu = 0; mu < 4; mu++) {
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    const int kind = h >> 1, bwd = h & 1;
                    const int nb = nb_cb(g, cc, s, mu, (kind ? 3 : 1) * (bwd ? -1 : 1));
                    float4 v[3];
#pragma unroll
                    for (int j = 0; j < 3; j++) v[j] = src[size_t(j) * Vh + nb];
                    const float4 *wl = L + size_t(((mu * 2 + kind) * 2 + bwd) * 9) * Vh + cb;
#pragma unroll
                    for (int i = 0; i < 3; i++)
#pragma unroll
                        for (int j = 0; j < 3; j++) cmac_df(acc, i, __ldg(wl + size_t(3 * i + j) * Vh), v[j]);
                }
            }
            if constexpr (STORE) {
#pragma unroll
                for (int u = 0; u < 3; u++) {
                    const float2 re = df_norm(acc.S[2 * u], acc.E[2 * u]);
                    const float2 im = df_norm(acc.S[2 * u + 1], acc.E[2 * u + 1]);
                    o.t[size_t(q) * fs + size_t(u) * Vh + cb] = make_float4(re.x, re.y, im.x, im.y);
                }
            } else {
                const size_t base = size_t(grp.id[q]) * fs + cb;
#pragma unroll
                for (int u = 0; u < 3; u++) {
                    const size_t i = base + size_t(u) * Vh;
                    const double2 xv = o.x[i], bv = o.b[i];
                    const double re = fma(-o.m4, xv.x, bv.x) + (double(acc.S[2 * u]) + double(acc.E[2 * u]));
                    const double im = fma(-o.m4, xv.y, bv.y) + (double(acc.S[2 * u + 1]) + double(acc.E[2 * u + 1]));
                    o.r[i] = make_double2(re, im);
                    red += re * re + im * im;
                }
            }
        }
    }
    if constexpr (!STORE) {
        // per-field sums: lanes by a fixed shuffle tree, blocks in block order
        __shared__ bool am_last;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) red += __shfl_down_sync(0xffffffffu, red, off);
        if (lane == 0 && on) partials[size_t(blockIdx.x) * kMaxBatch + q] = red;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) am_last = (atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1);
        __syncthreads();
        if (!am_last) return;
        __threadfence();
        for (int f = threadIdx.x; f < grp.k; f += blockDim.x) {
            double t = 0;
            for (int b = 0; b < (int)gridDim.x; b++) t += ((volatile double *)partials)[size_t(b) * kMaxBatch + f];
            norms[grp.id[f]] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            *ticket = 0u;
            __threadfence();
        }
    }
}

static hisq_status run_df_batch(hisq_ctx *ctx, const DFGroup &grp, const float4 *xd, float4 *td, const DFBatchOut &o)
{
    const int Vh = ctx->g.Vh;
    const int wpb = std::min(grp.k, kDFWarps);
    const int ny = (grp.k + wpb - 1) / wpb;
    auto go = [&](auto kern, int par, const float4 *in) -> hisq_status {
        static int bps = -1;
        if (bps < 0 && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 256, 0) != cudaSuccess || bps < 1))
            bps = 1;
        // all ny field chunks resident together (blocks of fewer warps fit
        // proportionally more per SM), so that the chunks sweep the sites in
        // step and re-read each link line from L2 rather than DRAM
        ctx->launches++;
        const long resident = long(ctx->num_sms) * bps * (kDFWarps / wpb);
        long gx = std::min(long((Vh + 31) / 32), std::max(1L, resident / ny));
        gx = std::min(gx, long(ctx->max_red_blocks));
        dim3 grid(unsigned(gx), unsigned(ny), 1u);
        kern<<<grid, 32 * wpb, 0, ctx->stream>>>(ctx->g, par, ctx->links_df[par], in, o, grp, ctx->bpartials,
                                                 ctx->ticket + 48, ctx->bscal->out);
        const cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? HISQ_OK : cuda_err(ctx, e, "batched double-float dslash launch");
    };
    hisq_status st = go(k_dslash_df_batch<true>, 1, xd);
    if (st == HISQ_OK) st = go(k_dslash_df_batch<false>, 0, td);
    return st;
}

// r_j = y_j - (4m^2 - D_eo D_oe) x_j for the right-hand sides `ids` of a batched
// solve (FP64 fields at a stride of s64 bytes from Y, X, Rr); |r_j|^2 -> rr[q]
hisq_status launch_residual_df_batch(hisq_ctx *ctx, const std::vector<int> &ids, const char *Y, const char *X, char *Rr,
                                     size_t s64, double *rr)
{
    const int Vh = ctx->g.Vh;
    const size_t sdf = spinor_bytes(HISQ_PREC_DF64, Vh);
    hisq_status st = ensure_df_links(ctx);
    if (st != HISQ_OK) return st;
    double out[kMaxBatch];
    for (size_t q0 = 0; q0 < ids.size(); q0 += kMaxBatch) {
        const int k = int(std::min(ids.size() - q0, size_t(kMaxBatch)));
        char *xd = (char *)get_buf(ctx, BUF_DF_X, sdf * k);
        char *td = (char *)get_buf(ctx, BUF_DF_T, sdf * k);
        if (!xd || !td) return HISQ_ERR_OOM;
        DFGroup grp;
        grp.k = k;
        for (int q = 0; q < k; q++) {
            grp.id[q] = ids[q0 + q];
            st = launch_to_df64(ctx, (const double *)(X + s64 * grp.id[q]), xd + sdf * q);
            if (st != HISQ_OK) return st;
        }
        DFBatchOut o{(float4 *)td, (double2 *)Rr, (const double2 *)X, (const double2 *)Y,
                     4.0 * ctx->mass * ctx->mass};
        st = run_df_batch(ctx, grp, (const float4 *)xd, (float4 *)td, o);
        if (st != HISQ_OK) return st;
        HISQ_CUDA(cudaMemcpyAsync(out, ctx->bscal->out, sizeof out, cudaMemcpyDeviceToHost, ctx->stream));
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
        for (int q = 0; q < k; q++) rr[q0 + q] = out[grp.id[q]];
    }
    return HISQ_OK;
}

} // namespace hisq
