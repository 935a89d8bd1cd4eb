// dslash.cu -- the HISQ Dirac operator on one parity (Section 2 of the paper:
// M = D + 2m, D with one-hop fat links and three-hop Naik long links) and the
// fused kernels of one CG iteration on (M^dag M)_ee = 4m^2 - D_eo D_oe (Eq. 1).
//
// One thread computes one output site: 16 link matrices are streamed from the
// gathered per-parity link arrays (read once per half-apply, evict-first), the
// 16 neighbour colour vectors are gathered from the opposite parity (they stay
// in L2: a parity field is at most a few hundred MB and the sweep order keeps
// the +-3 time-slice window resident).
#include "internal.cuh"

namespace hisq {

// ------------------------------------------------------------- epilogues
// out = a*x + b*y + c*acc; optional |out|^2
template <class S>
struct EpiXpay {
    S out, x, y;
    typename S::real a, b, c;
    int has_x, has_y, want_norm;
    template <typename R>
    __device__ __forceinline__ void operator()(int cb, const CVec<R> &acc, double &red) const
    {
        CVec<R> o;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            o.re[i] = c * acc.re[i];
            o.im[i] = c * acc.im[i];
        }
        if (has_x) {
            CVec<R> v = x.load(cb);
#pragma unroll
            for (int i = 0; i < 3; i++) {
                o.re[i] = fma(a, v.re[i], o.re[i]);
                o.im[i] = fma(a, v.im[i], o.im[i]);
            }
        }
        if (has_y) {
            CVec<R> v = y.load(cb);
#pragma unroll
            for (int i = 0; i < 3; i++) {
                o.re[i] = fma(b, v.re[i], o.re[i]);
                o.im[i] = fma(b, v.im[i], o.im[i]);
            }
        }
        out.store(cb, o);
        if (want_norm) red += double(o.norm2());
    }
};

// second half of a CG iteration: Ap = 4m^2 p - D_eo tmp; x += alpha p;
// r -= alpha Ap; |r|^2.  Ap is never stored.
template <class S, class SX>
struct EpiCG {
    S p, r;
    SX x;
    const DevScalars *scal;
    template <typename R>
    __device__ __forceinline__ void operator()(int cb, const CVec<R> &acc, double &red) const
    {
        const R alpha = R(scal->alpha);
        const R m4 = R(scal->m4);
        CVec<R> pv = p.load(cb);
        CVec<R> rv = r.load(cb);
        auto xv = x.load(cb);
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
        x.store(cb, xv);
        r.store(cb, rv);
        red += double(rv.norm2());
    }
};

// ------------------------------------------------------------- link formats
// FP32, kinds per mu = 2 (fat + long, 18 reals) or 1 (fat only; long in recon 12)
struct LinksFv {
    const float4 *base;
    int Vh;
    int nk;
    typedef float real;
    __device__ __forceinline__ void load(int mu, int kind, int i, CMat<float> &f, CMat<float> &b) const
    {
        const float4 *q = base + size_t((mu * nk + kind) * 9) * Vh + i;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            float4 a = __ldcs(q + size_t(k) * Vh);
            f.re[k] = a.x;
            f.im[k] = a.y;
            b.re[k] = a.z;
            b.im[k] = a.w;
        }
    }
};

__device__ __forceinline__ float2 h2f(unsigned u)
{
    __half2 h = *reinterpret_cast<__half2 *>(&u);
    return __half22float2(h);
}

// FP16: uint2 = (fwd_k, bwd_k) as two half2, [mu][kind][k<9][Vh]
struct LinksHv {
    const uint2 *base;
    int Vh;
    int nk;
    typedef float real;
    __device__ __forceinline__ void load(int mu, int kind, int i, CMat<float> &f, CMat<float> &b) const
    {
        const uint2 *q = base + size_t((mu * nk + kind) * 9) * Vh + i;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            uint2 a = __ldcs(q + size_t(k) * Vh);
            float2 x = h2f(a.x), y = h2f(a.y);
            f.re[k] = x.x;
            f.im[k] = x.y;
            b.re[k] = y.x;
            b.im[k] = y.y;
        }
    }
};

// FP16 12-real long links: uint2 (fwd_k, bwd_k), rows 0,1 of the SU(3) factor
struct LinksH12 {
    const uint2 *base;
    int Vh;
    __device__ __forceinline__ void load(int mu, int i, CMat<float> &f, CMat<float> &b) const
    {
        const uint2 *q = base + size_t(mu * 6) * Vh + i;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            uint2 a = __ldcs(q + size_t(k) * Vh);
            float2 x = h2f(a.x), y = h2f(a.y);
            f.re[k] = x.x;
            f.im[k] = x.y;
            b.re[k] = y.x;
            b.im[k] = y.y;
        }
        su3_third_row(f);
        su3_third_row(b);
    }
};

// ------------------------------------------------------------- the kernel
template <class SIn, class Lk, class L12T, bool R12, class Epi>
__global__ void __launch_bounds__(256)
    k_dslash(Geom g, int par, Lk L, L12T L12, float c3, SIn in, Epi epi, RedArgs ra, int do_red)
{
    typedef typename Lk::real R;
    double red = 0;
    for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < g.Vh; cb += gridDim.x * blockDim.x) {
        int c[4];
        cb_coords(g, par, cb, c);
        const int s = full_site(g, c);
        CVec<R> acc;
        acc.zero();
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            CMat<R> f, b;
            L.load(mu, 0, cb, f, b);
            {
                CVec<R> vf = cvt<R>(in.load(nb_cb(g, c, s, mu, +1)));
                CVec<R> vb = cvt<R>(in.load(nb_cb(g, c, s, mu, -1)));
                mv_acc(acc, f, vf);
                mv_acc(acc, b, vb);
            }
            if constexpr (R12) {
                CMat<float> f3, b3;
                L12.load(mu, cb, f3, b3);
                const float eta = stag_phase(mu, c);
                float sf = eta * c3, sb = -eta * c3;
                if (mu == 3 && g.t_antiperiodic) {
                    if (c[3] + 3 >= g.T) sf = -sf;
                    if (c[3] < 3) sb = -sb;
                }
                CVec<float> vf = cvt<float>(in.load(nb_cb(g, c, s, mu, +3)));
                CVec<float> vb = cvt<float>(in.load(nb_cb(g, c, s, mu, -3)));
                mv_acc_scaled(acc, sf, f3, vf);
                mv_acc_scaled(acc, sb, b3, vb);
            } else {
                L.load(mu, 1, cb, f, b);
                CVec<R> vf = cvt<R>(in.load(nb_cb(g, c, s, mu, +3)));
                CVec<R> vb = cvt<R>(in.load(nb_cb(g, c, s, mu, -3)));
                mv_acc(acc, f, vf);
                mv_acc(acc, b, vb);
            }
        }
        epi(cb, acc, red);
    }
    if (do_red) {
        double v[1] = {red};
        grid_reduce<1>(v, ra);
    }
}

// ------------------------------------------------------------- launch glue
template <typename K>
static int blocks_per_sm(K kernel)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, 256, 0) != cudaSuccess || n < 1) n = 1;
    return n;
}

template <class SIn, class Lk, class L12T, bool R12, class Epi>
static hisq_status run_dslash(hisq_ctx *ctx, int par, const Lk &L, const L12T &L12, const SIn &in, const Epi &epi,
                              RedArgs ra, int do_red)
{
    auto kern = k_dslash<SIn, Lk, L12T, R12, Epi>;
    static int bps = -1;
    if (bps < 0) bps = blocks_per_sm(kern);
    const int grid = grid_for(ctx, ctx->g.Vh, 256, bps);
    kern<<<grid, 256, 0, ctx->stream>>>(ctx->g, par, L, L12, float(ctx->long_scale), in, epi, ra, do_red);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(ctx, e, "dslash launch");
    return HISQ_OK;
}

// Run the Dslash with output parity `par` on links of precision link_prec
// (64, 32 or 16) in the context's long-link format.
template <class S, class Epi>
static hisq_status run_any(hisq_ctx *ctx, int par, int link_prec, const S &in, const Epi &epi, RedArgs ra, int dored)
{
    typedef typename S::real R;
    const int Vh = ctx->g.Vh;
    const bool r12 = ctx->long_recon == 12, r8 = ctx->long_recon == 8;
    const int nk = (r12 || r8) ? 1 : 2;
    if (link_prec == 64) {
        if constexpr (sizeof(R) == 8)
            return run_dslash<S, LinksD, LinksF12, false>(ctx, par, LinksD{ctx->links_d[par], Vh}, LinksF12{nullptr, Vh},
                                                          in, epi, ra, dored);
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "FP64 links need FP64 vectors");
    }
    if constexpr (sizeof(R) == 4) {
        if (link_prec == 32) {
            LinksFv L{ctx->links_f[par], Vh, nk};
            if (r12) return run_dslash<S, LinksFv, LinksF12, true>(ctx, par, L, LinksF12{ctx->links_f12[par], Vh}, in, epi, ra, dored);
            if (r8) return run_dslash<S, LinksFv, LinksF8, true>(ctx, par, L, LinksF8{ctx->links_f12[par], Vh}, in, epi, ra, dored);
            return run_dslash<S, LinksFv, LinksF12, false>(ctx, par, L, LinksF12{nullptr, Vh}, in, epi, ra, dored);
        }
        if (link_prec == 16) {
            if (!ctx->links_h[par]) {
                const hisq_status hs = ensure_half_links(ctx);
                if (hs != HISQ_OK) return hs;
            }
            LinksHv L{ctx->links_h[par], Vh, nk};
            if (r12) return run_dslash<S, LinksHv, LinksH12, true>(ctx, par, L, LinksH12{ctx->links_h12[par], Vh}, in, epi, ra, dored);
            return run_dslash<S, LinksHv, LinksH12, false>(ctx, par, L, LinksH12{nullptr, Vh}, in, epi, ra, dored);
        }
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "link precision must be 64, 32 or 16");
    }
    return set_err(ctx, HISQ_ERR_INVALID_ARG, "FP32/FP16 links need FP32 or FP16 vectors");
}

void fp64_prof_drain(hisq_ctx *ctx, bool all, bool discard)
{
    size_t n = 0;
    for (; n < ctx->fp64_pending.size(); n++) {
        const auto &e = ctx->fp64_pending[n];
        if (all || discard) {
            cudaEventSynchronize(e.second);
        } else if (cudaEventQuery(e.second) != cudaSuccess) {
            cudaGetLastError(); // not ready yet: later pairs are not either
            break;
        }
        float ms = 0;
        if (!discard && cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) {
            ctx->fp64_seconds += 1e-3 * ms;
            ctx->fp64_launches++;
        }
        cudaGetLastError();
        ctx->fp64_pool.push_back(e.first);
        ctx->fp64_pool.push_back(e.second);
    }
    ctx->fp64_pending.erase(ctx->fp64_pending.begin(), ctx->fp64_pending.begin() + n);
}

static hisq_status dslash_xpay(hisq_ctx *ctx, int out_parity, int prec, int link_prec, const void *in, void *out,
                               double a, const void *x, double b, const void *y, double c, int norm_slot);

// With profiling on, an FP64 launch outside stream capture is bracketed by a
// pair of events (from a pool); the pairs are summed once they have completed,
// so the host never waits for a launch it has just issued.
hisq_status launch_dslash(hisq_ctx *ctx, int out_parity, int prec, int link_prec, const void *in, void *out, double a,
                          const void *x, double b, const void *y, double c, int norm_slot)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (prec != 64 || !ctx->profile || cudaStreamIsCapturing(ctx->stream, &cap) != cudaSuccess ||
        cap != cudaStreamCaptureStatusNone)
        return dslash_xpay(ctx, out_parity, prec, link_prec, in, out, a, x, b, y, c, norm_slot);
    cudaEvent_t e[2];
    for (int i = 0; i < 2; i++) {
        if (!ctx->fp64_pool.empty()) {
            e[i] = ctx->fp64_pool.back();
            ctx->fp64_pool.pop_back();
        } else {
            HISQ_CUDA(cudaEventCreate(&e[i]));
        }
    }
    HISQ_CUDA(cudaEventRecord(e[0], ctx->stream));
    const hisq_status st = dslash_xpay(ctx, out_parity, prec, link_prec, in, out, a, x, b, y, c, norm_slot);
    HISQ_CUDA(cudaEventRecord(e[1], ctx->stream));
    ctx->fp64_pending.emplace_back(e[0], e[1]);
    fp64_prof_drain(ctx, ctx->fp64_pending.size() > 4096);
    return st;
}

static hisq_status dslash_xpay(hisq_ctx *ctx, int out_parity, int prec, int link_prec, const void *in, void *out,
                               double a, const void *x, double b, const void *y, double c, int norm_slot)
{
    const int Vh = ctx->g.Vh;
    if (!ctx->links_loaded) return set_err(ctx, HISQ_ERR_STATE, "links not loaded");
    if ((prec == 64) != (link_prec == 64)) return set_err(ctx, HISQ_ERR_INVALID_ARG, "FP64 vectors go with FP64 links");
    void *xx = const_cast<void *>(x ? x : out), *yy = const_cast<void *>(y ? y : out);
    RedArgs ra = red_args(ctx, FIN_STORE, norm_slot < 0 ? 0 : norm_slot);
    const int dored = norm_slot >= 0;
    auto go = [&](auto in_, auto out_, auto x_, auto y_) -> hisq_status {
        typedef decltype(in_) S;
        typedef typename S::real R;
        EpiXpay<S> epi{out_, x_, y_, R(a), R(b), R(c), x != nullptr, y != nullptr, dored};
        return run_any(ctx, out_parity, link_prec, in_, epi, ra, dored);
    };
    void *ii = const_cast<void *>(in);
    switch (prec) {
    case 64: return go(make_spinorD(ii, Vh), make_spinorD(out, Vh), make_spinorD(xx, Vh), make_spinorD(yy, Vh));
    case 32: return go(make_spinorF(ii, Vh), make_spinorF(out, Vh), make_spinorF(xx, Vh), make_spinorF(yy, Vh));
    case 16: return go(make_spinorH(ii, Vh), make_spinorH(out, Vh), make_spinorH(xx, Vh), make_spinorH(yy, Vh));
    }
    return set_err(ctx, HISQ_ERR_INVALID_ARG, "precision must be 64, 32 or 16");
}

// ---------------------------------------------------------- CG iteration
// (1) tmp = D_oe p (odd output) with tt = |tmp|^2 -> alpha = rr / (4m^2 pp + tt)
//     using <p, A p> = 4m^2 |p|^2 + |D_oe p|^2 (D_eo = -D_oe^dag).
hisq_status launch_cg_dslash_tt(hisq_ctx *ctx, int prec, int link_prec, const void *p, void *tmp)
{
    const int Vh = ctx->g.Vh;
    RedArgs ra = red_args(ctx, FIN_CG_ALPHA);
    void *pp = const_cast<void *>(p);
    auto go = [&](auto in_, auto out_) -> hisq_status {
        typedef decltype(in_) S;
        typedef typename S::real R;
        EpiXpay<S> epi{out_, out_, out_, R(0), R(0), R(1), 0, 0, 1};
        return run_any(ctx, 1, link_prec, in_, epi, ra, 1);
    };
    switch (prec) {
    case 64: return go(make_spinorD(pp, Vh), make_spinorD(tmp, Vh));
    case 32: return go(make_spinorF(pp, Vh), make_spinorF(tmp, Vh));
    case 16: return go(make_spinorH(pp, Vh), make_spinorH(tmp, Vh));
    }
    return set_err(ctx, HISQ_ERR_INVALID_ARG, "bad sloppy precision");
}

// (2) even output: Ap = 4m^2 p - D_eo tmp; x += alpha p; r -= alpha Ap; rr_new = |r|^2,
//     beta = rr_new / rr.
hisq_status launch_cg_dslash_update(hisq_ctx *ctx, int prec, int link_prec, int xprec, const void *tmp,
                                    const void *p, void *x, void *r)
{
    const int Vh = ctx->g.Vh;
    RedArgs ra = red_args(ctx, FIN_CG_BETA);
    void *tt = const_cast<void *>(tmp), *pp = const_cast<void *>(p);
    switch (prec) {
    case 64: {
        EpiCG<SpinorD, SpinorD> epi{make_spinorD(pp, Vh), make_spinorD(r, Vh), make_spinorD(x, Vh), ctx->scal};
        return run_any(ctx, 0, link_prec, make_spinorD(tt, Vh), epi, ra, 1);
    }
    case 32: {
        if (xprec != 32) return set_err(ctx, HISQ_ERR_INVALID_ARG, "x precision");
        EpiCG<SpinorF, SpinorF> epi{make_spinorF(pp, Vh), make_spinorF(r, Vh), make_spinorF(x, Vh), ctx->scal};
        return run_any(ctx, 0, link_prec, make_spinorF(tt, Vh), epi, ra, 1);
    }
    case 16: {
        if (xprec != 32) return set_err(ctx, HISQ_ERR_INVALID_ARG, "x precision");
        EpiCG<SpinorH, SpinorF> epi{make_spinorH(pp, Vh), make_spinorH(r, Vh), make_spinorF(x, Vh), ctx->scal};
        return run_any(ctx, 0, link_prec, make_spinorH(tt, Vh), epi, ra, 1);
    }
    }
    return set_err(ctx, HISQ_ERR_INVALID_ARG, "bad sloppy precision");
}

} // namespace hisq
