// ingest.cu -- link ingest: from the caller's FP64 fat and long links (host
// layout [s][mu][3][3]) to the library's gathered per-parity device copies.
//
// For output parity p, site x and direction mu the 16 hop matrices of the HISQ
// operator (Section 2: one-hop fat links, three-hop Naik long links) are
//   fwd, n hops:  W = eta_mu(x) * bc(x, n)        * U_mu(x)
//   bwd, n hops:  W = -eta_mu(x) * bc(x - n mu, n) * U_mu(x - n mu)^dag
// with bc = -1 for a hop that wraps the time boundary of an antiperiodic
// lattice.  They are written in FP64, FP32 and FP16 (see internal.cuh for layouts).
// With 12-real long links only rows 0 and 1 of S = U_long / long_scale are kept
// (for fwd and bwd); the Dslash rebuilds row 2 and applies the sign and scale.
#include "internal.cuh"

namespace hisq {

__device__ __forceinline__ void load_link(const double2 *U, int s, int mu, double2 (&m)[9])
{
    const double2 *q = U + (size_t(s) * 4 + mu) * 9;
#pragma unroll
    for (int k = 0; k < 9; k++) m[k] = q[k];
}

__device__ __forceinline__ void adjoint(const double2 (&a)[9], double2 (&b)[9])
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) b[3 * i + j] = make_double2(a[3 * j + i].x, -a[3 * j + i].y);
}

// max |S S^dag - 1| and |det S - 1| for the 12-real check
__device__ double su3_deviation(const double2 (&S)[9])
{
    double dev = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double re = 0, im = 0;
            for (int k = 0; k < 3; k++) {
                const double2 a = S[3 * i + k], b = S[3 * j + k];
                re += a.x * b.x + a.y * b.y;
                im += a.y * b.x - a.x * b.y;
            }
            if (i == j) re -= 1.0;
            dev = fmax(dev, fmax(fabs(re), fabs(im)));
        }
    // det via the cofactor expansion along row 0
    double2 c[3];
    for (int k = 0; k < 3; k++) {
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        const double2 a1 = S[3 + k1], a2 = S[3 + k2], b1 = S[6 + k1], b2 = S[6 + k2];
        c[k] = make_double2((a1.x * b2.x - a1.y * b2.y) - (a2.x * b1.x - a2.y * b1.y),
                            (a1.x * b2.y + a1.y * b2.x) - (a2.x * b1.y + a2.y * b1.x));
    }
    double dr = 0, di = 0;
    for (int k = 0; k < 3; k++) {
        dr += S[k].x * c[k].x - S[k].y * c[k].y;
        di += S[k].x * c[k].y + S[k].y * c[k].x;
    }
    dev = fmax(dev, fmax(fabs(dr - 1.0), fabs(di)));
    return dev;
}

__device__ __forceinline__ void atomic_max_nonneg(float *addr, float v)
{
    atomicMax(reinterpret_cast<int *>(addr), __float_as_int(v));
}

struct IngestOut {
    double2 *d;    // FP64 [mu][kind][fb][k][Vh] for this parity
    float4 *f;     // FP32 [mu][nk][k][Vh]
    float4 *f12;   // FP32 compressed long: recon 12 [mu][6][Vh], recon 8 [mu][4][Vh], or null
    int nk;
};


// one thread per (output site cb, mu) of parity `par`
__global__ void k_ingest(Geom g, int par, const double2 *__restrict__ fat, const double2 *__restrict__ lng,
                         IngestOut o, double inv_scale, int recon, float *max_dev, int *nonfinite)
{
    const int Vh = g.Vh;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 4 * Vh; t += gridDim.x * blockDim.x) {
        const int cb = t % Vh, mu = t / Vh;
        int c[4];
        cb_coords(g, par, cb, c);
        const int s = full_site(g, c);
        const int L = dim_of(g, mu);
        const double eta = stag_phase(mu, c);
        for (int kind = 0; kind < 2; kind++) {
            const int n = kind == 0 ? 1 : 3;
            const double2 *U = kind == 0 ? fat : lng;
            // backward source site x - n mu
            int cb_[4] = {c[0], c[1], c[2], c[3]};
            cb_[mu] = (c[mu] - n + L) % L;
            const int sb = checked_index(g, full_site(g, cb_), g.V);
            double sf = eta, sbk = -eta;
            if (mu == 3 && g.t_antiperiodic) {
                if (c[3] + n >= g.T) sf = -sf;
                if (cb_[3] + n >= g.T) sbk = -sbk;
            }
            double2 Mf[9], Mb0[9], Mb[9];
            load_link(U, s, mu, Mf);
            load_link(U, sb, mu, Mb0);
            adjoint(Mb0, Mb);
            int bad = 0;
#pragma unroll
            for (int k = 0; k < 9; k++)
                bad |= !isfinite(Mf[k].x) | !isfinite(Mf[k].y) | !isfinite(Mb[k].x) | !isfinite(Mb[k].y);
            if (bad) atomicOr(nonfinite, 1);
            // FP64 copy, signs folded
            double2 *qd = o.d + size_t((mu * 2 + kind) * 2) * 9 * Vh + cb;
#pragma unroll
            for (int k = 0; k < 9; k++) {
                qd[size_t(k) * Vh] = make_double2(sf * Mf[k].x, sf * Mf[k].y);
                qd[size_t(9 + k) * Vh] = make_double2(sbk * Mb[k].x, sbk * Mb[k].y);
            }
            if (kind == 1 && recon != 18) {
                // SU(3) factor, rows 0 and 1
                double2 Sf[9], Sb[9];
#pragma unroll
                for (int k = 0; k < 9; k++) {
                    Sf[k] = make_double2(Mf[k].x * inv_scale, Mf[k].y * inv_scale);
                    Sb[k] = make_double2(Mb[k].x * inv_scale, Mb[k].y * inv_scale);
                }
                const double dev = fmax(su3_deviation(Sf), su3_deviation(Sb));
                atomic_max_nonneg(max_dev, isfinite(dev) ? float(dev) : 1e30f);
                if (recon == 12) {
                    float4 *q = o.f12 + size_t(mu * 6) * Vh + cb;
#pragma unroll
                    for (int k = 0; k < 6; k++)
                        __stcs(q + size_t(k) * Vh,
                               make_float4(float(Sf[k].x), float(Sf[k].y), float(Sb[k].x), float(Sb[k].y)));
                } else { // recon 8: (a2, a3), (b1, arg a1, arg c1) of fwd, then of bwd
                    float4 *q = o.f12 + size_t(mu * 4) * Vh + cb;
                    const double2 *S2[2] = {Sf, Sb};
                    for (int fb = 0; fb < 2; fb++) {
                        const double2 *S = S2[fb];
                        __stcs(q + size_t(2 * fb) * Vh, make_float4(float(S[1].x), float(S[1].y), float(S[2].x), float(S[2].y)));
                        __stcs(q + size_t(2 * fb + 1) * Vh, make_float4(float(S[3].x), float(S[3].y), float(atan2(S[0].y, S[0].x)),
                                                                        float(atan2(S[6].y, S[6].x))));
                    }
                }
            } else {
                float4 *q = o.f + size_t((mu * o.nk + kind) * 9) * Vh + cb;
#pragma unroll
                for (int k = 0; k < 9; k++)
                    __stcs(q + size_t(k) * Vh, make_float4(float(sf * Mf[k].x), float(sf * Mf[k].y),
                                                           float(sbk * Mb[k].x), float(sbk * Mb[k].y)));
            }
        }
    }
}

hisq_status ingest_links(hisq_ctx *ctx, const double *fat_dev, const double *lng_dev, int recon, double long_scale,
                         double *max_unitarity_err)
{
    const int Vh = ctx->g.Vh;
    float *d_dev = nullptr;
    int *d_bad = nullptr;
    HISQ_CUDA(cudaMallocAsync((void **)&d_dev, sizeof(float) + sizeof(int), ctx->stream));
    d_bad = reinterpret_cast<int *>(d_dev + 1);
    HISQ_CUDA(cudaMemsetAsync(d_dev, 0, sizeof(float) + sizeof(int), ctx->stream));
    const int nk = recon == 18 ? 2 : 1;
    for (int par = 0; par < 2; par++) {
        IngestOut o{ctx->links_d[par], ctx->links_f[par], recon != 18 ? ctx->links_f12[par] : nullptr, nk};
        int grid = (4 * Vh + 255) / 256;
        if (grid > ctx->num_sms * 16) grid = ctx->num_sms * 16;
        ctx->launches++;
        k_ingest<<<grid, 256, 0, ctx->stream>>>(ctx->g, par, (const double2 *)fat_dev, (const double2 *)lng_dev, o,
                                                1.0 / long_scale, recon, d_dev, d_bad);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(ctx, e, "ingest launch");
    }
    float hdev = 0;
    int hbad = 0;
    HISQ_CUDA(cudaMemcpyAsync(&hdev, d_dev, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    HISQ_CUDA(cudaMemcpyAsync(&hbad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    HISQ_CUDA(cudaFreeAsync(d_dev, ctx->stream));
    if (max_unitarity_err) *max_unitarity_err = hdev;
    if (hbad) return set_err(ctx, HISQ_ERR_NUMERICAL, "non-finite link element");
    return HISQ_OK;
}

} // namespace hisq

namespace hisq {

// FP16 gathered links: each FP32 (fwd, bwd) pair rounded to two half2 values
__global__ void k_links_to_half(size_t n, const float4 *__restrict__ f, uint2 *__restrict__ h)
{
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        const float4 a = f[i];
        const __half2 x = __floats2half2_rn(a.x, a.y), y = __floats2half2_rn(a.z, a.w);
        h[i] = make_uint2(*reinterpret_cast<const unsigned *>(&x), *reinterpret_cast<const unsigned *>(&y));
    }
}

// the FP16 sloppy links exist only once an operator asks for them (they are
// the rounding of the FP32 gathered links, so nothing else is needed)
hisq_status ensure_half_links(hisq_ctx *ctx)
{
    if (ctx->links_h[0]) return HISQ_OK;
    if (ctx->long_recon == 8) return set_err(ctx, HISQ_ERR_INVALID_ARG, "FP16 links need long_recon 18 or 12");
    const size_t Vh = size_t(ctx->g.Vh);
    const bool r12 = ctx->long_recon == 12;
    const size_t nf = Vh * (r12 ? 4 : 8) * 9, n12 = Vh * 4 * 6;
    for (int p = 0; p < 2; p++) {
        ctx->links_h[p] = (uint2 *)dev_alloc(ctx, nf * 8);
        if (r12) ctx->links_h12[p] = (uint2 *)dev_alloc(ctx, n12 * 8);
        if (!ctx->links_h[p] || (r12 && !ctx->links_h12[p])) return HISQ_ERR_OOM;
        ctx->launches++;
        k_links_to_half<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(nf, ctx->links_f[p], ctx->links_h[p]);
        HISQ_CUDA(cudaGetLastError());
        if (r12) {
            ctx->launches++;
            k_links_to_half<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(n12, ctx->links_f12[p], ctx->links_h12[p]);
            HISQ_CUDA(cudaGetLastError());
        }
    }
    return HISQ_OK;
}

} // namespace hisq
