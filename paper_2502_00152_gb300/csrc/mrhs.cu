// mrhs.cu -- multi right-hand-side kernels (the paper's outlook, Section 4:
// several right-hand sides at once raise the arithmetic intensity).
//
// A batch is k ordinary one-parity colour fields at a fixed byte stride; a list
// of active slots (idx[q] = right-hand side of slot q) masks converged ones.
// Each thread computes one site for R right-hand sides, so every link it loads
// serves R matrix-vector products from registers; the lanes of a warp take 32
// consecutive sites of the same fields, so neighbour gathers are coalesced.
// Per-RHS reductions are deterministic: lanes by a fixed shuffle tree, warps in
// a fixed order, blocks by the last block in block order.
#include <algorithm>
#include <cstddef>
#include <functional>

#include "internal.cuh"

namespace hisq {


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

// Thread tiling of the batched kernels: a block holds nsg site groups of 32
// consecutive sites; within a site group, warp c handles right-hand-side slots
// c*R .. c*R+R-1 (nch = ceil(kact / R) warps per site group).  The lanes of a
// warp therefore read one colour field at 32 consecutive sites (coalesced), and
// the nch warps of a site group read the same links at about the same time, so
// the links come from DRAM once per launch.
struct MrhsTile {
    int nch, nsg;
    __device__ __forceinline__ int chunk() const { return (threadIdx.x >> 5) % nch; }
    __device__ __forceinline__ int group() const { return (threadIdx.x >> 5) / nch; }
};

// per-slot sums of R values per thread into partials[block][slot] (lanes by a
// fixed shuffle tree, site groups in order) and, in the last block, the sums
// over blocks in block order followed by the batch finish operation
template <int R>
__device__ __forceinline__ void batch_reduce(double (&v)[R], const MrhsTile &tl, int kact, const BatchRed &br)
{
    __shared__ double sh[8][kMaxBatch]; // [site group][slot]
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int u = 0; u < R; u++)
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v[u] += __shfl_down_sync(0xffffffffu, v[u], o);
    if (lane == 0) {
#pragma unroll
        for (int u = 0; u < R; u++) {
            const int q = tl.chunk() * R + u;
            if (q < kMaxBatch) sh[tl.group()][q] = v[u];
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kact; q += blockDim.x) {
        double s = 0;
        for (int w = 0; w < tl.nsg; w++) s += sh[w][q];
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

// out_j = a x_j + b y_j + c acc (x, y nullable), FP32 fields; no reduction
struct BEpiLin {
    BatchF<SpinorF> out, x, y;
    float a, b, c;
    bool hx, hy;
    template <typename R>
    __device__ __forceinline__ void operator()(int cb, int j, const CVec<R> &acc, double &) const
    {
        CVec<float> o;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            o.re[i] = c * float(acc.re[i]);
            o.im[i] = c * float(acc.im[i]);
        }
        if (hx) {
            const CVec<float> v = x.at(j).load(cb);
#pragma unroll
            for (int i = 0; i < 3; i++) {
                o.re[i] = fmaf(a, v.re[i], o.re[i]);
                o.im[i] = fmaf(a, v.im[i], o.im[i]);
            }
        }
        if (hy) {
            const CVec<float> v = y.at(j).load(cb);
#pragma unroll
            for (int i = 0; i < 3; i++) {
                o.re[i] = fmaf(b, v.re[i], o.re[i]);
                o.im[i] = fmaf(b, v.im[i], o.im[i]);
            }
        }
        out.at(j).store(cb, o);
    }
};

// ------------------------------------------------------------- the kernel
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void prefetch_long(const LinksF12 &L, int mu, int i)
{
    if (!L.base) return;
    const float4 *q = L.base + size_t(mu * 6) * L.Vh + i;
#pragma unroll
    for (int k = 0; k < 6; k++) prefetch_l2(q + size_t(k) * L.Vh);
}
__device__ __forceinline__ void prefetch_long(const LinksF8 &L, int mu, int i)
{
    const float4 *q = L.base + size_t(mu * 4) * L.Vh + i;
#pragma unroll
    for (int k = 0; k < 4; k++) prefetch_l2(q + size_t(k) * L.Vh);
}

template <int R, class S, class Lk, class L12T, bool R12, class Epi>
__global__ void __launch_bounds__(512, 1)
    k_dslash_mrhs(Geom g, int par, Lk L, L12T L12, float c3, BatchF<S> in, const BatchScalars *scal, MrhsTile tl,
                  Epi epi, BatchRed br)
{
    typedef typename Lk::real Rl;
    const int kact = scal->kact;
    // slots past kact (a partial last chunk) gather an active field again and
    // skip only the epilogue, so every gather is unconditional and the
    // compiler can issue them all ahead of the arithmetic
    int jj[R];
    bool on[R];
#pragma unroll
    for (int u = 0; u < R; u++) {
        const int q = tl.chunk() * R + u;
        on[u] = q < kact; // uniform over the warp
        jj[u] = scal->idx[on[u] ? q : kact - 1];
    }
    double red[R];
#pragma unroll
    for (int u = 0; u < R; u++) red[u] = 0;
    const int step = gridDim.x * tl.nsg * 32;
    for (int cb = (blockIdx.x * tl.nsg + tl.group()) * 32 + (threadIdx.x & 31); cb < g.Vh; cb += step) {
        int c[4];
        cb_coords(g, par, cb, c);
        const int s = full_site(g, c);
        CVec<Rl> acc[R];
#pragma unroll
        for (int u = 0; u < R; u++) acc[u].zero();
#pragma unroll 1
        for (int mu = 0; mu < 4; mu++) {
            const int f1 = nb_cb(g, c, s, mu, +1), b1 = nb_cb(g, c, s, mu, -1);
            const int f3 = nb_cb(g, c, s, mu, +3), b3 = nb_cb(g, c, s, mu, -3);
            // the next direction's links (read from DRAM once per launch) are
            // requested into L2 while this direction is computed
            if (mu < 3) {
                L.prefetch(mu + 1, cb);
                prefetch_long(L12, mu + 1, cb);
            }
            CMat<Rl> f, b;
            L.load(mu, 0, cb, f, b);
#pragma unroll
            for (int u = 0; u < R; u++) {
                const S v = in.at(jj[u]);
                mv_acc(acc[u], f, cvt<Rl>(v.load(f1)));
                mv_acc(acc[u], b, cvt<Rl>(v.load(b1)));
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
                for (int u = 0; u < R; u++) {
                    const S v = in.at(jj[u]);
                    mv_acc_scaled(acc[u], sf, f3m, cvt<float>(v.load(f3)));
                    mv_acc_scaled(acc[u], sb, b3m, cvt<float>(v.load(b3)));
                }
            } else {
                L.load(mu, 1, cb, f, b);
#pragma unroll
                for (int u = 0; u < R; u++) {
                    const S v = in.at(jj[u]);
                    mv_acc(acc[u], f, cvt<Rl>(v.load(f3)));
                    mv_acc(acc[u], b, cvt<Rl>(v.load(b3)));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < R; u++)
            if (on[u]) epi(cb, jj[u], acc[u], red[u]);
    }
    batch_reduce<R>(red, tl, kact, br);
}

// p_j = r_j + beta_j p_j, |p_j|^2
template <int R, class S>
__global__ void __launch_bounds__(512, 1)
    k_p_update_mrhs(int Vh, BatchF<S> r, BatchF<S> p, const BatchScalars *scal, MrhsTile tl, BatchRed br)
{
    typedef typename S::real Rl;
    const int kact = scal->kact;
    int jj[R];
#pragma unroll
    for (int u = 0; u < R; u++) {
        const int q = tl.chunk() * R + u;
        jj[u] = q < kact ? scal->idx[q] : -1;
    }
    double red[R];
#pragma unroll
    for (int u = 0; u < R; u++) red[u] = 0;
    const int step = gridDim.x * tl.nsg * 32;
    for (int cb = (blockIdx.x * tl.nsg + tl.group()) * 32 + (threadIdx.x & 31); cb < Vh; cb += step) {
#pragma unroll
        for (int u = 0; u < R; u++) {
            if (jj[u] < 0) continue;
            const int j = jj[u];
            const Rl beta = Rl(scal->beta[j]);
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
    batch_reduce<R>(red, tl, kact, br);
}

// ------------------------------------------------------------- launch glue
// Launch shapes of the batched kernels, tried by the autotuner on the first
// D_oe launch of each (batch size, precision, link format): R right-hand
// sides per thread (2, 3 or 4: more spills the link matrices, accumulators and
// gathers out of 128 registers) and 1 or 2 site groups per block (up to 512
// threads).  Candidate 0, R = 4 with blocks of about 8 warps, is the default.
struct MrhsShape {
    int R;
    MrhsTile tile;
};

static int mrhs_candidates(int kact, MrhsShape *out)
{
    int n = 0;
    for (int R : {4, 3, 2}) {
        const int nch = (kact + R - 1) / R;
        if (nch > 16) continue;
        const int nsg0 = std::max(1, 8 / nch);
        for (int nsg : {nsg0, 2 * nsg0}) {
            if (32 * nch * nsg > 512 || nsg > 8) continue; // batch_reduce holds 8 site groups
            out[n].R = R;
            out[n].tile.nch = nch;
            out[n].tile.nsg = nsg;
            n++;
        }
    }
    return n;
}

static unsigned long long mrhs_key(const hisq_ctx *ctx, int kact, int prec)
{
    return (1ull << 40) | (unsigned long long)kact | ((unsigned long long)prec << 8) |
           ((unsigned long long)ctx->long_recon << 16);
}

// blocks per SM of `kern` at `threads` threads, cached per kernel and shape
template <class K>
static int mrhs_blocks_per_sm(K kern, int threads)
{
    static int cache[17] = {0};
    const int slot = threads / 32 > 16 ? 16 : threads / 32;
    if (cache[slot] == 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, 0) != cudaSuccess || n < 1) {
            cudaGetLastError();
            n = 1;
        }
        cache[slot] = n;
    }
    return cache[slot];
}

struct LinksFvB {
    const float4 *base;
    int Vh;
    int nk;
    typedef float real;
    __device__ __forceinline__ void prefetch(int mu, int i) const
    {
        const float4 *q = base + size_t((mu * nk) * 9) * Vh + i;
#pragma unroll
        for (int k = 0; k < 9; k++) prefetch_l2(q + size_t(k) * Vh);
    }
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

template <int R, class S, class Epi>
static hisq_status run_mrhs_r(hisq_ctx *ctx, int par, const BatchF<S> &in, const MrhsTile &tl, const Epi &epi,
                              BatchRed br)
{
    const int Vh = ctx->g.Vh;
    const int threads = 32 * tl.nch * tl.nsg;
    LinksFvB L{ctx->links_f[par], Vh, ctx->long_recon == 18 ? 2 : 1};
    auto launch = [&](auto kern, auto L12) -> hisq_status {
        const int grid = grid_for(ctx, long(Vh), 32 * tl.nsg, mrhs_blocks_per_sm(kern, threads));
        kern<<<grid, threads, 0, ctx->stream>>>(ctx->g, par, L, L12, float(ctx->long_scale), in, ctx->bscal, tl, epi,
                                               br);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(ctx, e, "batched dslash launch");
        return HISQ_OK;
    };
    if (ctx->long_recon == 12)
        return launch(k_dslash_mrhs<R, S, LinksFvB, LinksF12, true, Epi>, LinksF12{ctx->links_f12[par], Vh});
    if (ctx->long_recon == 8)
        return launch(k_dslash_mrhs<R, S, LinksFvB, LinksF8, true, Epi>, LinksF8{ctx->links_f12[par], Vh});
    return launch(k_dslash_mrhs<R, S, LinksFvB, LinksF12, false, Epi>, LinksF12{nullptr, Vh});
}

template <class S, class Epi>
static hisq_status run_shape(hisq_ctx *ctx, int par, const BatchF<S> &in, const MrhsShape &sh, const Epi &epi,
                             BatchRed br)
{
    switch (sh.R) {
    case 2: return run_mrhs_r<2>(ctx, par, in, sh.tile, epi, br);
    case 3: return run_mrhs_r<3>(ctx, par, in, sh.tile, epi, br);
    default: return run_mrhs_r<4>(ctx, par, in, sh.tile, epi, br);
    }
}

// the shape for this batch: tuned on an idempotent launch (may_tune), else
// the one tuned before, else the default
static hisq_status mrhs_shape(hisq_ctx *ctx, int kact, int prec, MrhsShape *sh, bool may_tune,
                              const std::function<hisq_status(const MrhsShape &)> &launch)
{
    MrhsShape cand[16];
    const int n = mrhs_candidates(kact, cand);
    int idx = 0;
    const unsigned long long key = mrhs_key(ctx, kact, prec);
    if (may_tune) {
        hisq_status st = autotune(ctx, key, n, 0, [&](int i) { return launch(cand[i]); }, &idx);
        if (st != HISQ_OK) return st;
    } else {
        auto it = ctx->tuned.find(key);
        if (it != ctx->tuned.end()) idx = it->second;
    }
    *sh = cand[idx < n ? idx : 0];
    return HISQ_OK;
}

template <class S, class Epi>
static hisq_status run_mrhs(hisq_ctx *ctx, int par, int link_prec, int prec, const BatchF<S> &in, int kact,
                            const Epi &epi, BatchRed br, bool may_tune)
{
    if (link_prec != 32) return set_err(ctx, HISQ_ERR_INVALID_ARG, "batched operator: FP32 links only");
    if (kact < 1 || kact > kMaxBatch) return set_err(ctx, HISQ_ERR_INVALID_ARG, "batched operator: 1..64 right-hand sides");
    MrhsShape sh;
    hisq_status st = mrhs_shape(ctx, kact, prec, &sh, may_tune,
                                [&](const MrhsShape &c) { return run_shape(ctx, par, in, c, epi, br); });
    if (st != HISQ_OK) return st;
    return run_shape(ctx, par, in, sh, epi, br);
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
    case 32:
        return run_mrhs(ctx, 1, link_prec, 32, batchf<SpinorF>(p, Vh, 32), kact,
                        BEpiStore<SpinorF>{batchf<SpinorF>(tmp, Vh, 32)}, br, true);
    case 16:
        return run_mrhs(ctx, 1, link_prec, 16, batchf<SpinorH>(p, Vh, 16), kact,
                        BEpiStore<SpinorH>{batchf<SpinorH>(tmp, Vh, 16)}, br, true);
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
        return run_mrhs(ctx, 0, link_prec, 32, batchf<SpinorF>(tmp, Vh, 32), kact, epi, br, false);
    }
    case 16: {
        BEpiCG<SpinorH, SpinorF> epi{batchf<SpinorH>(p, Vh, 16), batchf<SpinorH>(r, Vh, 16), batchf<SpinorF>(x, Vh, 32), ctx->bscal};
        return run_mrhs(ctx, 0, link_prec, 16, batchf<SpinorH>(tmp, Vh, 16), kact, epi, br, false);
    }
    }
    return set_err(ctx, HISQ_ERR_INVALID_ARG, "batched sloppy precision must be 32 or 16");
}

// active slots 0..k-1 = right-hand sides 0..k-1 (a block of ordinary fields)
hisq_status mrhs_set_identity(hisq_ctx *ctx, int k)
{
    if (k < 1 || k > kMaxBatch) return set_err(ctx, HISQ_ERR_INVALID_ARG, "batched operator: 1..64 fields");
    int buf[kMaxBatch + 1];
    buf[0] = k;
    for (int q = 0; q < k; q++) buf[1 + q] = q;
    static_assert(offsetof(BatchScalars, idx) == offsetof(BatchScalars, kact) + sizeof(int), "kact, idx adjacent");
    HISQ_CUDA(cudaMemcpyAsync(&ctx->bscal->kact, buf, sizeof(int) * (1 + k), cudaMemcpyHostToDevice, ctx->stream));
    return HISQ_OK;
}

// out_j = a x_j + b y_j + c D(in_j) on output parity par for the k FP32 fields
// of a block (slots 0..k-1 active, mrhs_set_identity); x, y nullable
hisq_status launch_mrhs_dslash_lin(hisq_ctx *ctx, int par, const void *in, void *out, double a, const void *x,
                                   double b, const void *y, double c, int k)
{
    const int Vh = ctx->g.Vh;
    BEpiLin epi{batchf<SpinorF>(out, Vh, 32), batchf<SpinorF>(const_cast<void *>(x), Vh, 32),
                batchf<SpinorF>(const_cast<void *>(y), Vh, 32), float(a), float(b), float(c), x != nullptr,
                y != nullptr};
    return run_mrhs(ctx, par, 32, 32, batchf<SpinorF>(const_cast<void *>(in), Vh, 32), k, epi,
                    batch_red(ctx, BFIN_STORE), false);
}

// (3) p_j = r_j + beta_j p_j, pp_j (the shape of the batch's Dslash)
template <int R, class S>
static hisq_status run_p_update(hisq_ctx *ctx, void *r, void *p, const MrhsTile &tl, int prec)
{
    const int Vh = ctx->g.Vh;
    const int threads = 32 * tl.nch * tl.nsg;
    auto kern = k_p_update_mrhs<R, S>;
    const int grid = grid_for(ctx, long(Vh), 32 * tl.nsg, mrhs_blocks_per_sm(kern, threads));
    kern<<<grid, threads, 0, ctx->stream>>>(Vh, batchf<S>(r, Vh, prec), batchf<S>(p, Vh, prec), ctx->bscal, tl,
                                            batch_red(ctx, BFIN_P));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(ctx, e, "batched p update");
    return HISQ_OK;
}

hisq_status launch_mrhs_p_update(hisq_ctx *ctx, int prec, void *r, void *p, int kact)
{
    if (kact < 1 || kact > kMaxBatch) return set_err(ctx, HISQ_ERR_INVALID_ARG, "batched p update: 1..64 right-hand sides");
    if (prec != 32 && prec != 16) return set_err(ctx, HISQ_ERR_INVALID_ARG, "batched sloppy precision must be 32 or 16");
    MrhsShape sh;
    hisq_status st = mrhs_shape(ctx, kact, prec, &sh, false, nullptr);
    if (st != HISQ_OK) return st;
    auto go = [&](auto tagS) -> hisq_status {
        typedef decltype(tagS) S;
        switch (sh.R) {
        case 2: return run_p_update<2, S>(ctx, r, p, sh.tile, prec);
        case 3: return run_p_update<3, S>(ctx, r, p, sh.tile, prec);
        default: return run_p_update<4, S>(ctx, r, p, sh.tile, prec);
        }
    };
    return prec == 32 ? go(SpinorF{}) : go(SpinorH{});
}

} // namespace hisq
