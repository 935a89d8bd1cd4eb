// net.cu -- a gauge-covariant parallel-transport network that predicts an
// initial guess for CG (the learned part of the method, built on the paper's
// solver: CG still runs from the guess to the same true residual).
//
// One layer maps Cin complex colour-vector channels to Cout channels on the
// full lattice:
//   out_b(x) = sum_a sum_h w[b][a][h] (T_h in_a)(x)
//   T_0 = identity, T_{mu,fwd} in(x) = W_fwd(x) in(x+mu), T_{mu,bwd} in(x) = W_bwd(x) in(x-mu)
// with W the one-hop fat-link hop matrices of the Dirac operator (staggered
// phases, boundary signs and the backward minus sign included), so a layer with
// w = (0, 1, 1, ..., 1) is exactly the fat-link part of D and the map commutes
// with gauge transformations (scalar weights, covariant transports).
// Because T_{mu,fwd}^dag = -T_{mu,bwd}, the adjoint of a layer is the same layer
// with weights w'[a][b][0] = conj(w[b][a][0]), w'[a][b][mu,d] = -conj(w[b][a][mu,1-d]).
//
// Channel tensors: (C, V, 3) complex64, full lattice, s = x + X(y + Y(z + Z t)).
// Weights: (Cout, Cin, 9) complex64; optionally rounded to BF16 when staged.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace hisq {

constexpr int kNetHops = 9;
constexpr int kNetSites = 16; // sites per block
constexpr int kNetMaxC = 16;

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// transports of site (parity p, cb) for input channel a and hop h -> 3 complex
__device__ __forceinline__ void net_transport(const Geom &g, const float4 *links_p, int nk, const float2 *in, int V,
                                              int a, int h, int p, int cb, const int c[4], int s, float2 (&t)[3])
{
    const float2 *ch = in + size_t(a) * V * 3;
    if (h == 0) {
#pragma unroll
        for (int i = 0; i < 3; i++) t[i] = ch[size_t(s) * 3 + i];
        return;
    }
    const int mu = (h - 1) >> 1, d = (h - 1) & 1;
    int cn[4] = {c[0], c[1], c[2], c[3]};
    const int L = dim_of(g, mu);
    cn[mu] = d == 0 ? (c[mu] + 1 == L ? 0 : c[mu] + 1) : (c[mu] == 0 ? L - 1 : c[mu] - 1);
    const int sn = checked_index(g, full_site(g, cn), g.V);
    float2 v[3];
#pragma unroll
    for (int i = 0; i < 3; i++) v[i] = ch[size_t(sn) * 3 + i];
    const float4 *q = links_p + size_t((mu * nk + 0) * 9) * g.Vh + cb;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float4 w = __ldg(q + size_t(3 * i + j) * g.Vh);
            const float2 m = d == 0 ? make_float2(w.x, w.y) : make_float2(w.z, w.w);
            const float2 pr = cmulf(m, v[j]);
            acc.x += pr.x;
            acc.y += pr.y;
        }
        t[i] = acc;
    }
}

// stage the (possibly adjoint) weights of one layer into shared memory
__device__ __forceinline__ void net_stage_weights(float2 *sw, const float2 *w, int cin, int cout, int adjoint, int bf16)
{
    // staged layout: [b][a][h] for the layer as applied (cout_eff x cin_eff)
    const int co = adjoint ? cin : cout, ci = adjoint ? cout : cin;
    for (int t = threadIdx.x; t < co * ci * kNetHops; t += blockDim.x) {
        const int b = t / (ci * kNetHops), a = (t / kNetHops) % ci, h = t % kNetHops;
        float2 v;
        if (!adjoint) {
            v = w[(size_t(b) * cin + a) * kNetHops + h];
        } else {
            // applied weight w'[b][a][h] from the stored w[a][b][h'] (b < cin, a < cout)
            const int hs = h == 0 ? 0 : (1 + (((h - 1) >> 1) << 1) + (1 - ((h - 1) & 1)));
            const float2 u = w[(size_t(a) * cin + b) * kNetHops + hs];
            v = h == 0 ? make_float2(u.x, -u.y) : make_float2(-u.x, u.y);
        }
        if (bf16) {
            v.x = __bfloat162float(__float2bfloat16_rn(v.x));
            v.y = __bfloat162float(__float2bfloat16_rn(v.y));
        }
        sw[t] = v;
    }
}

// out = layer(in) (adjoint = 0) or layer^dag(in) (adjoint = 1)
__global__ void __launch_bounds__(256)
    k_net_layer(Geom g, const float4 *links0, const float4 *links1, int nk, const float2 *__restrict__ w, int cin,
                int cout, int adjoint, int bf16, const float2 *__restrict__ in, float2 *__restrict__ out)
{
    extern __shared__ float2 sm[];
    const int co = adjoint ? cin : cout, ci = adjoint ? cout : cin;
    float2 *sw = sm;                                   // co * ci * 9
    float2 *st = sm + co * ci * kNetHops;              // kNetSites * ci * 9 * 3
    net_stage_weights(sw, w, cin, cout, adjoint, bf16);
    const int V = g.V;
    const int nblk = (V + kNetSites - 1) / kNetSites;
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        __syncthreads();
        // phase 1: transports of every (site, input channel, hop)
        for (int t = threadIdx.x; t < kNetSites * ci * kNetHops; t += blockDim.x) {
            const int ls = t / (ci * kNetHops), a = (t / kNetHops) % ci, h = t % kNetHops;
            const int s = blk * kNetSites + ls;
            float2 tr[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            if (s < V) {
                int c[4];
                int r = s;
                c[0] = r % g.X;
                r /= g.X;
                c[1] = r % g.Y;
                r /= g.Y;
                c[2] = r % g.Z;
                c[3] = r / g.Z;
                const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
                net_transport(g, p ? links1 : links0, nk, in, V, a, h, p, s >> 1, c, s, tr);
            }
#pragma unroll
            for (int i = 0; i < 3; i++) st[size_t(t) * 3 + i] = tr[i];
        }
        __syncthreads();
        // phase 2: channel mixing, one (site, output channel) per thread
        for (int t = threadIdx.x; t < kNetSites * co; t += blockDim.x) {
            const int ls = t / co, b = t % co;
            const int s = blk * kNetSites + ls;
            if (s >= V) continue;
            float2 acc[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            const float2 *tb = st + size_t(ls) * ci * kNetHops * 3;
            const float2 *wb = sw + size_t(b) * ci * kNetHops;
            for (int q = 0; q < ci * kNetHops; q++) {
                const float2 wv = wb[q];
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    const float2 pr = cmulf(wv, tb[q * 3 + i]);
                    acc[i].x += pr.x;
                    acc[i].y += pr.y;
                }
            }
#pragma unroll
            for (int i = 0; i < 3; i++) out[(size_t(b) * V + s) * 3 + i] = acc[i];
        }
    }
}

// per-block partial weight gradients: G[b][a][h] = sum_x gout_b(x) . conj(T_h in_a(x))
__global__ void __launch_bounds__(256)
    k_net_wgrad(Geom g, const float4 *links0, const float4 *links1, int nk, int cin, int cout,
                const float2 *__restrict__ in, const float2 *__restrict__ gout, double2 *part)
{
    extern __shared__ float2 sm[];
    float2 *st = sm;                                           // kNetSites * cin * 9 * 3
    float2 *sg = sm + size_t(kNetSites) * cin * kNetHops * 3;  // kNetSites * cout * 3
    const int V = g.V;
    const int ntrip = cout * cin * kNetHops;
    constexpr int kPer = (kNetMaxC * kNetMaxC * kNetHops + 255) / 256;
    double accr[kPer], acci[kPer];
#pragma unroll
    for (int u = 0; u < kPer; u++) accr[u] = acci[u] = 0;
    const int nblk = (V + kNetSites - 1) / kNetSites;
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        __syncthreads();
        for (int t = threadIdx.x; t < kNetSites * cin * kNetHops; t += blockDim.x) {
            const int ls = t / (cin * kNetHops), a = (t / kNetHops) % cin, h = t % kNetHops;
            const int s = blk * kNetSites + ls;
            float2 tr[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            if (s < V) {
                int c[4];
                int r = s;
                c[0] = r % g.X;
                r /= g.X;
                c[1] = r % g.Y;
                r /= g.Y;
                c[2] = r % g.Z;
                c[3] = r / g.Z;
                const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
                net_transport(g, p ? links1 : links0, nk, in, V, a, h, p, s >> 1, c, s, tr);
            }
#pragma unroll
            for (int i = 0; i < 3; i++) st[size_t(t) * 3 + i] = tr[i];
        }
        for (int t = threadIdx.x; t < kNetSites * cout * 3; t += blockDim.x) {
            const int ls = t / (cout * 3), b = (t / 3) % cout, i = t % 3;
            const int s = blk * kNetSites + ls;
            sg[t] = s < V ? gout[(size_t(b) * V + s) * 3 + i] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kPer; u++) {
            const int q = threadIdx.x + u * blockDim.x;
            if (q >= ntrip) continue;
            const int b = q / (cin * kNetHops), ah = q % (cin * kNetHops);
            float sr = 0.f, si = 0.f;
            for (int ls = 0; ls < kNetSites; ls++) {
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    const float2 gv = sg[(ls * cout + b) * 3 + i];
                    const float2 tv = st[(size_t(ls) * cin * kNetHops + ah) * 3 + i];
                    // gv * conj(tv)
                    sr += gv.x * tv.x + gv.y * tv.y;
                    si += gv.y * tv.x - gv.x * tv.y;
                }
            }
            accr[u] += sr;
            acci[u] += si;
        }
    }
#pragma unroll
    for (int u = 0; u < kPer; u++) {
        const int q = threadIdx.x + u * blockDim.x;
        if (q < ntrip) part[size_t(blockIdx.x) * ntrip + q] = make_double2(accr[u], acci[u]);
    }
}

__global__ void k_net_wgrad_finish(int nblocks, int ntrip, const double2 *part, float2 *gw)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < ntrip; q += gridDim.x * blockDim.x) {
        double r = 0, i = 0;
        for (int b = 0; b < nblocks; b++) {
            r += part[size_t(b) * ntrip + q].x;
            i += part[size_t(b) * ntrip + q].y;
        }
        gw[q] = make_float2(float(r), float(i));
    }
}

// Adam step on n real parameters (Kingma & Ba, ICLR 2015)
__global__ void k_adam(int n, float *w, const float *gr, float *m1, float *m2, float lr, float b1, float b2, float eps,
                       float bc1, float bc2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gv = gr[i];
        m1[i] = b1 * m1[i] + (1.f - b1) * gv;
        m2[i] = b2 * m2[i] + (1.f - b2) * gv * gv;
        const float mh = m1[i] / bc1, vh = m2[i] / bc2;
        w[i] -= lr * mh / (sqrtf(vh) + eps);
    }
}

} // namespace hisq

using namespace hisq;

extern "C" {

hisq_status hisq_net_layer(hisq_ctx *ctx, int cin, int cout, const float *w_dev, int w_bf16, int adjoint,
                           const float *in_dev, float *out_dev)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!w_dev || !in_dev || !out_dev || cin < 1 || cout < 1 || cin > kNetMaxC || cout > kNetMaxC)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "network layer: 1..16 channels, device pointers");
    if (!ctx->links_loaded) return set_err(ctx, HISQ_ERR_STATE, "links not loaded");
    HISQ_CUDA(cudaSetDevice(ctx->device));
    const int co = adjoint ? cin : cout, ci = adjoint ? cout : cin;
    const size_t smem = sizeof(float2) * (size_t(co) * ci * kNetHops + size_t(kNetSites) * ci * kNetHops * 3);
    static bool attr = false;
    if (!attr) {
        HISQ_CUDA(cudaFuncSetAttribute(k_net_layer, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
        attr = true;
    }
    const int nblk = (ctx->g.V + kNetSites - 1) / kNetSites;
    const int grid = std::min(nblk, ctx->num_sms * 4);
    const int nk = ctx->long_recon == 18 ? 2 : 1;
    ctx->launches++;
    k_net_layer<<<grid, 256, smem, ctx->stream>>>(ctx->g, ctx->links_f[0], ctx->links_f[1], nk, (const float2 *)w_dev,
                                                  cin, cout, adjoint, w_bf16, (const float2 *)in_dev, (float2 *)out_dev);
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

hisq_status hisq_net_wgrad(hisq_ctx *ctx, int cin, int cout, const float *in_dev, const float *gout_dev, float *gw_dev)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!in_dev || !gout_dev || !gw_dev || cin < 1 || cout < 1 || cin > kNetMaxC || cout > kNetMaxC)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "network gradient: 1..16 channels, device pointers");
    if (!ctx->links_loaded) return set_err(ctx, HISQ_ERR_STATE, "links not loaded");
    HISQ_CUDA(cudaSetDevice(ctx->device));
    const size_t smem = sizeof(float2) * (size_t(kNetSites) * cin * kNetHops * 3 + size_t(kNetSites) * cout * 3);
    static bool attr = false;
    if (!attr) {
        HISQ_CUDA(cudaFuncSetAttribute(k_net_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
        attr = true;
    }
    const int nblk = (ctx->g.V + kNetSites - 1) / kNetSites;
    const int grid = std::min(nblk, ctx->num_sms * 2);
    const int ntrip = cin * cout * kNetHops;
    double2 *part = (double2 *)get_buf(ctx, BUF_NET_PART, sizeof(double2) * size_t(grid) * ntrip);
    if (!part) return HISQ_ERR_OOM;
    const int nk = ctx->long_recon == 18 ? 2 : 1;
    ctx->launches += 2;
    k_net_wgrad<<<grid, 256, smem, ctx->stream>>>(ctx->g, ctx->links_f[0], ctx->links_f[1], nk, cin, cout,
                                                  (const float2 *)in_dev, (const float2 *)gout_dev, part);
    HISQ_CUDA(cudaGetLastError());
    k_net_wgrad_finish<<<(ntrip + 255) / 256, 256, 0, ctx->stream>>>(grid, ntrip, part, (float2 *)gw_dev);
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

hisq_status hisq_net_adam(hisq_ctx *ctx, int n, float *w_dev, const float *g_dev, float *m1_dev, float *m2_dev,
                          float lr, float beta1, float beta2, float eps, int step)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (n < 1 || !w_dev || !g_dev || !m1_dev || !m2_dev || step < 1)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "adam: bad arguments");
    HISQ_CUDA(cudaSetDevice(ctx->device));
    const float bc1 = 1.f - std::pow(beta1, float(step)), bc2 = 1.f - std::pow(beta2, float(step));
    ctx->launches++;
    k_adam<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, w_dev, g_dev, m1_dev, m2_dev, lr, beta1, beta2, eps, bc1, bc2);
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

} // extern "C"
