// mrhs.cu -- multi right-hand-side kernels (the paper's outlook, Section 4:
// several right-hand sides at once raise the arithmetic intensity).
//
// A batch is k ordinary one-parity colour fields at a fixed byte stride; a list
// of active slots (idx[q] = right-hand side of slot q) masks converged ones.
// Work item t = site * groups + group: the `groups` lanes of one site are
// adjacent in a warp, so their link loads hit the same addresses and each link
// is read from memory once for all right-hand sides.  Each thread accumulates
// kMrhsChunk right-hand sides.  Per-RHS reductions are deterministic: lanes of
// equal group are combined by shuffles, warps in a fixed order, blocks by the
// last block in block order.
#include "internal.cuh"

namespace hisq {

constexpr int kMrhsChunk = 4;

template <class S>
struct BatchF {
    char *base;
    size_t stride;
    int Vh;
    __device__ __forceinline__ S at(int j) const;
};
template <>
__device__ __forceinline__ SpinorD BatchF<SpinorD>::at(int j) const
{
    return SpinorD{(double2 *)(base + stride * j), Vh};
}
template <>
__device__ __forceinline__ SpinorF BatchF<SpinorF>::at(int j) const
{
    char *p = base + stride * j;
    return SpinorF{(float4 *)p, (float2 *)(p + size_t(Vh) * 16), Vh};
}
template <>
__device__ __forceinline__ SpinorH BatchF<SpinorH>::at(int j) const
{
    return SpinorH{(uint4 *)(base + stride * j), Vh};
}

template <class S>
static BatchF<S> batchf(void *base, int Vh, int prec)
{
    return BatchF<S>{(char *)base, spinor_bytes(prec, Vh), Vh};
}

// per-slot reduction of kMrhsChunk values per thread into partials[block][slot]
// and, in the last block, the batch finish operation
__device__ __forceinline__ void batch_reduce(const double (&v)[kMrhsChunk], int groups, int kact, const BatchRed &br)
{
    __shared__ double sh[8][kMaxBatch];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    double x[kMrhsChunk];
#pragma unroll
    for (int u = 0; u < kMrhsChunk; u++) {
        x[u] = v[u];
        for (int o = 16; o >= groups; o >>= 1) x[u] += __shfl_down_sync(0xffffffffu, x[u], o);
    }
    if (lane < groups) {
#pragma unroll
        for (int u = 0; u < kMrhsChunk; u++) {
            const int q = lane * kMrhsChunk + u;
            if (q < kMaxBatch) sh[warp][q] = x[u];
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kact; q += blockDim.x) {
        double s = 0;
        for (int w = 0; w < nwarps; w++) s += sh[w][q];
        br.partials[size_t(blockIdx.x) * kMaxBatch + q] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(br.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    for (int q = threadIdx.x; q < kact; q += blockDim.x) {
        double s = 0;
        for (int b = 0; b < (int)gridDim.x; b++) s += ((volatile double *)br.partials)[size_t(b) * kMaxBatch + q];
        BatchScalars *B = br.scal;
        const int j = B->idx[q];
        switch (br.op) {
        case BFIN_STORE: B->out[j] = s; break;
        case BFIN_ALPHA:
            B->tt[j] = s;
            B->alpha[j] = B->rr[j] / (B->m4 * B->pp[j] + s);
            break;
        case BFIN_BETA:
            B->rr_new[j] = s;
            B->beta[j] = s / B->rr[j];
            if (br.monitor) br.monitor[size_t(B->iter % br.monitor_len) * kMaxBatch + j] = s;
            break;
        case BFIN_P:
            B->pp[j] = s;
            B->rr[j] = B->rr_new[j];
            break;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (br.op == BFIN_P) br.scal->iter += 1;
        *br.ticket = 0u;
        __threadfence();
    }
}

// ------------------------------------------------------------- epilogues
// tmp_j = acc, |tmp_j|^2
template <class S>
struct BEpiStore {
    BatchF<S> out;
    template <typename R>
    __device__ __forceinline__ void operator()(int cb, int j, const CVec<R> &acc, double &red) const
    {
        out.at(j).store(cb, acc);
        red += double(acc.norm2());
    }
};

// Ap = 4m^2 p - acc; x += alpha_j p; r -= alpha_j Ap; |r|^2
template <class S, class SX>
struct BEpiCG {
    BatchF<S> p, r;
    BatchF<SX> x;
    const BatchScalars *scal;
    template <typename R>
    __device__ __forceinline__ void operator()(int cb, int j, const CVec<R> &acc, double &red) const
    {
        const R alpha = R(scal->alpha[j]);
        const R m4 = R(scal->m4);
        const S pj = p.at(j), rj = r.at(j);
        const SX xj = x.at(j);
        CVec<R> pv = pj.load(cb);
        CVec<R> rv = rj.load(cb);
        auto xv = xj.load(cb);
        typedef typename SX::real XR;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            R apr = fma(m4, pv.re[i], -acc.re[i]);
            R api = fma(m4, pv.im[i], -acc.im[i]);
            rv.re[i] = fma(-alpha, apr, rv.re[i]);
            rv.im[i] = fma(-alpha, api, rv.im[i]);
            xv.re[i] = fma(XR(alpha), XR(pv.re[i]), xv.re[i]);
            xv.im[i] = fma(XR(alpha), XR(pv.im[i]), xv.im[i]);
        }
        xj.store(cb, xv);
        rj.store(cb, rv);
        red += double(rv.norm2());
    }
};

// ------------------------------------------------------------- the kernel
template <class S, class Lk, class L12T, bool R12, class Epi>
__global__ void __launch_bounds__(256)
    k_dslash_mrhs(Geom g, int par, Lk L, L12T L12, float c3, BatchF<S> in, const BatchScalars *scal, int groups,
                  Epi epi, BatchRed br)
{
    typedef typename Lk::real R;
    const int kact = scal->kact;
    double red[kMrhsChunk];
#pragma unroll
    for (int u = 0; u < kMrhsChunk; u++) red[u] = 0;
    const long total = long(g.Vh) * groups;
    for (long t = long(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += long(gridDim.x) * blockDim.x) {
        const int cb = int(t / groups), gi = int(t % groups);
        int c[4];
        cb_coords(g, par, cb, c);
        const int s = full_site(g, c);
        int jj[kMrhsChunk];
#pragma unroll
        for (int u = 0; u < kMrhsChunk; u++) {
            const int q = gi * kMrhsChunk + u;
            jj[u] = q < kact ? scal->idx[q] : -1;
        }
        CVec<R> acc[kMrhsChunk];
#pragma unroll
        for (int u = 0; u < kMrhsChunk; u++) acc[u].zero();
#pragma unroll 1
        for (int mu = 0; mu < 4; mu++) {
            const int f1 = nb_cb(g, c, s, mu, +1), b1 = nb_cb(g, c, s, mu, -1);
            const int f3 = nb_cb(g, c, s, mu, +3), b3 = nb_cb(g, c, s, mu, -3);
            CMat<R> f, b;
            L.load(mu, 0, cb, f, b);
#pragma unroll
            for (int u = 0; u < kMrhsChunk; u++) {
                if (jj[u] < 0) continue;
                const S v = in.at(jj[u]);
                mv_acc(acc[u], f, cvt<R>(v.load(f1)));
                mv_acc(acc[u], b, cvt<R>(v.load(b1)));
            }
            if constexpr (R12) {
                CMat<float> f3m, b3m;
                L12.load(mu, cb, f3m, b3m);
                const float eta = stag_phase(mu, c);
                float sf = eta * c3, sb = -eta * c3;
                if (mu == 3 && g.t_antiperiodic) {
                    if (c[3] + 3 >= g.T) sf = -sf;
                    if (c[3] < 3) sb = -sb;
                }
#pragma unroll
                for (int u = 0; u < kMrhsChunk; u++) {
                    if (jj[u] < 0) continue;
                    const S v = in.at(jj[u]);
                    mv_acc_scaled(acc[u], sf, f3m, cvt<float>(v.load(f3)));
                    mv_acc_scaled(acc[u], sb, b3m, cvt<float>(v.load(b3)));
                }
            } else {
                L.load(mu, 1, cb, f, b);
#pragma unroll
                for (int u = 0; u < kMrhsChunk; u++) {
                    if (jj[u] < 0) continue;
                    const S v = in.at(jj[u]);
                    mv_acc(acc[u], f, cvt<R>(v.load(f3)));
                    mv_acc(acc[u], b, cvt<R>(v.load(b3)));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kMrhsChunk; u++)
            if (jj[u] >= 0) epi(cb, jj[u], acc[u], red[u]);
    }
    batch_reduce(red, groups, kact, br);
}

// p_j = r_j + beta_j p_j, |p_j|^2
template <class S>
__global__ void __launch_bounds__(256)
    k_p_update_mrhs(int Vh, BatchF<S> r, BatchF<S> p, const BatchScalars *scal, int groups, BatchRed br)
{
    typedef typename S::real R;
    const int kact = scal->kact;
    double red[kMrhsChunk];
#pragma unroll
    for (int u = 0; u < kMrhsChunk; u++) red[u] = 0;
    const long total = long(Vh) * groups;
    for (long t = long(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += long(gridDim.x) * blockDim.x) {
        const int cb = int(t / groups), gi = int(t % groups);
#pragma unroll
        for (int u = 0; u < kMrhsChunk; u++) {
            const int q = gi * kMrhsChunk + u;
            if (q >= kact) continue;
            const int j = scal->idx[q];
            const R beta = R(scal->beta[j]);
            const S rj = r.at(j), pj = p.at(j);
            auto rv = rj.load(cb);
            auto pv = pj.load(cb);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                pv.re[c] = fma(beta, pv.re[c], rv.re[c]);
                pv.im[c] = fma(beta, pv.im[c], rv.im[c]);
            }
            pj.store(cb, pv);
            red[u] += double(pv.norm2());
        }
    }
    batch_reduce(red, groups, kact, br);
}

// ------------------------------------------------------------- launch glue
static int groups_for(int kact)
{
    int g = (kact + kMrhsChunk - 1) / kMrhsChunk;
    int p = 1;
    while (p < g) p <<= 1;
    return p; // power of two <= kMaxBatch / kMrhsChunk
}

struct LinksFvB {
    const float4 *base;
    int Vh;
    int nk;
    typedef float real;
    __device__ __forceinline__ void load(int mu, int kind, int i, CMat<float> &f, CMat<float> &b) const
    {
        const float4 *q = base + size_t((mu * nk + kind) * 9) * Vh + i;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            float4 a = __ldg(q + size_t(k) * Vh); // shared by the lanes of one site
            f.re[k] = a.x;
            f.im[k] = a.y;
            b.re[k] = a.z;
            b.im[k] = a.w;
        }
    }
};

template <class S, class Epi>
static hisq_status run_mrhs(hisq_ctx *ctx, int par, int link_prec, const BatchF<S> &in, int kact, const Epi &epi,
                            BatchRed br)
{
    const int Vh = ctx->g.Vh;
    const int groups = groups_for(kact);
    if (link_prec != 32) return set_err(ctx, HISQ_ERR_INVALID_ARG, "batched operator: FP32 links only");
    LinksFvB L{ctx->links_f[par], Vh, ctx->long_recon == 12 ? 1 : 2};
    auto launch = [&](auto kern, auto L12) -> hisq_status {
        static int bps = -1;
        if (bps < 0) {
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 256, 0) != cudaSuccess || n < 1) n = 1;
            bps = n;
        }
        const int grid = grid_for(ctx, long(Vh) * groups, 256, bps);
        kern<<<grid, 256, 0, ctx->stream>>>(ctx->g, par, L, L12, float(ctx->long_scale), in, ctx->bscal, groups, epi, br);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(ctx, e, "batched dslash launch");
        return HISQ_OK;
    };
    if (ctx->long_recon == 12)
        return launch(k_dslash_mrhs<S, LinksFvB, LinksF12, true, Epi>, LinksF12{ctx->links_f12[par], Vh});
    return launch(k_dslash_mrhs<S, LinksFvB, LinksF12, false, Epi>, LinksF12{nullptr, Vh});
}

BatchRed batch_red(hisq_ctx *ctx, int op)
{
    BatchRed b;
    b.partials = ctx->bpartials;
    b.ticket = ctx->ticket + 32; // a ticket of its own
    b.scal = ctx->bscal;
    b.monitor = ctx->bmonitor_d;
    b.monitor_len = ctx->bmonitor_len;
    b.op = op;
    return b;
}

// (1) tmp_j = D_oe p_j, tt_j -> alpha_j
hisq_status launch_mrhs_dslash_tt(hisq_ctx *ctx, int prec, int link_prec, void *p, void *tmp, int kact)
{
    const int Vh = ctx->g.Vh;
    BatchRed br = batch_red(ctx, BFIN_ALPHA);
    switch (prec) {
    case 32: return run_mrhs(ctx, 1, link_prec, batchf<SpinorF>(p, Vh, 32), kact, BEpiStore<SpinorF>{batchf<SpinorF>(tmp, Vh, 32)}, br);
    case 16: return run_mrhs(ctx, 1, link_prec, batchf<SpinorH>(p, Vh, 16), kact, BEpiStore<SpinorH>{batchf<SpinorH>(tmp, Vh, 16)}, br);
    }
    return set_err(ctx, HISQ_ERR_INVALID_ARG, "batched sloppy precision must be 32 or 16");
}

// (2) even output: CG update of every active right-hand side, rr_new_j -> beta_j
hisq_status launch_mrhs_dslash_update(hisq_ctx *ctx, int prec, int link_prec, void *tmp, void *p, void *x, void *r,
                                      int kact)
{
    const int Vh = ctx->g.Vh;
    BatchRed br = batch_red(ctx, BFIN_BETA);
    switch (prec) {
    case 32: {
        BEpiCG<SpinorF, SpinorF> epi{batchf<SpinorF>(p, Vh, 32), batchf<SpinorF>(r, Vh, 32), batchf<SpinorF>(x, Vh, 32), ctx->bscal};
        return run_mrhs(ctx, 0, link_prec, batchf<SpinorF>(tmp, Vh, 32), kact, epi, br);
    }
    case 16: {
        BEpiCG<SpinorH, SpinorF> epi{batchf<SpinorH>(p, Vh, 16), batchf<SpinorH>(r, Vh, 16), batchf<SpinorF>(x, Vh, 32), ctx->bscal};
        return run_mrhs(ctx, 0, link_prec, batchf<SpinorH>(tmp, Vh, 16), kact, epi, br);
    }
    }
    return set_err(ctx, HISQ_ERR_INVALID_ARG, "batched sloppy precision must be 32 or 16");
}

// (3) p_j = r_j + beta_j p_j, pp_j
hisq_status launch_mrhs_p_update(hisq_ctx *ctx, int prec, void *r, void *p, int kact)
{
    const int Vh = ctx->g.Vh;
    const int groups = groups_for(kact);
    BatchRed br = batch_red(ctx, BFIN_P);
    auto go = [&](auto kern, auto R, auto P) -> hisq_status {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, 256, 0) != cudaSuccess || n < 1) n = 1;
        const int grid = grid_for(ctx, long(Vh) * groups, 256, n);
        kern<<<grid, 256, 0, ctx->stream>>>(Vh, R, P, ctx->bscal, groups, br);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(ctx, e, "batched p update");
        return HISQ_OK;
    };
    switch (prec) {
    case 32: return go(k_p_update_mrhs<SpinorF>, batchf<SpinorF>(r, Vh, 32), batchf<SpinorF>(p, Vh, 32));
    case 16: return go(k_p_update_mrhs<SpinorH>, batchf<SpinorH>(r, Vh, 16), batchf<SpinorH>(p, Vh, 16));
    }
    return set_err(ctx, HISQ_ERR_INVALID_ARG, "batched sloppy precision must be 32 or 16");
}

} // namespace hisq
