// tc_gemm.cu -- the deflation projection and expansion of a batch of right-hand
// sides as complex GEMMs on the 5th-generation tensor cores (tcgen05, FP16
// operands, FP32 accumulation in tensor memory, TMA-fed shared memory).
// Eq. 4 of the paper for k right-hand sides at once:
//   C = V^dag R   (n x k),   X += V Lambda^-1 C,   R -= V C.
//
// Complex -> real: with V stored as interleaved (re, im) FP16 and
//   R'_{2j} = (Re r_j, Im r_j),  R'_{2j+1} = (Im r_j, -Re r_j)
// the real product V R'^T gives (Re c_ij, Im c_ij) in columns (2j, 2j+1).  The
// expansion uses the site-major copy of V, rows s, K = (i, re/im), against
// D'_{4j..4j+3} built from d = c / lambda and c, so one GEMM updates x and r.
// FP32 eigenvectors: every operand is split into an FP16 high part and an FP16
// residual part and three MMAs (hi*hi + hi*lo + lo*hi) are accumulated, which
// gives about 22 significant bits: enough for the updated residual to stay
// consistent with the updated solution (r -= V c uses A v_i = lambda_i v_i).
// BF16 or FP16 (HISQ_PREC_HALF_EV) eigenvectors: the stored vectors are the A
// operand as they are (their colour-major layout is the GEMM's K order); only
// the other operand is split into high and low parts of the same type, two MMAs
// (a*hi + a*lo) per step, so the products are those of the stored vectors to
// about 16 (BF16) or 22 (FP16) bits of the other side.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "internal.cuh"
#include "tc.cuh"

namespace hisq {

hisq_status read_slots(hisq_ctx *ctx, int slot0, int n, double *out);

#define TRY_HISQ(x)                             \
    do {                                        \
        hisq_status s_ = (x);                   \
        if (s_ != HISQ_OK) return s_;           \
    } while (0)

constexpr int TC_BK = 64;   // K elements per stage (128 B of FP16)
constexpr int TC_ROWB = 128; // bytes per swizzled row

// ------------------------------------------------------------- tensor maps
typedef CUresult (*PFN_encodeTiled_t)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                       const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                       CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled_t encode_fn()
{
    static std::once_flag once;
    static PFN_encodeTiled_t fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encodeTiled_t>(p);
    });
    return fn;
}

// 2D FP16 (or BF16) tensor: inner dimension `inner` elements (contiguous), `rows` rows of
// `row_bytes`; box {64, box_rows}, 128-byte swizzle, zero fill out of bounds.
static bool make_tmap(CUtensorMap *tm, const void *base, uint64_t inner, uint64_t rows, uint64_t row_bytes,
                      uint32_t box_rows, bool bf16 = false)
{
    PFN_encodeTiled_t enc = encode_fn();
    if (!enc) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (row_bytes & 15) || box_rows == 0 || box_rows > 256) return false;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {uint32_t(TC_BK), box_rows};
    cuuint32_t estr[2] = {1, 1};
    return enc(tm, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ------------------------------------------------------------- the GEMM kernel
// D[m][nn] = sum_k A[m][k] B[nn][k] over this CTA's K range for MT row tiles of
// 128 and N columns, operands split into hi/lo FP16 tensors (4 maps).
//   mode 0 (projection): blockIdx.x = K split, rows m0 = blockIdx.y * MT * 128;
//            the FP32 tile is written to part[split][m][nn].
//   mode 1 (expansion):  persistent over row tiles (MT = 1), full K range; the
//            epilogue applies the result to the right-hand-side fields.
struct ExpandEpi {
    uint32_t spin_limit; // polls of a bounded wait before it gives up
    int no_loads;     // failure injection (tests): the producer issues no copy
    double2 *x;       // k FP64 even fields, element s of field j at x + j*xs + s
    double2 *r;       // nullptr: x only (the caller recomputes r = b - A x)
    size_t fstride;   // double2 elements between fields
    const float *scale; // 4 per right-hand side: x re/im, r re/im column factors
    const int *field; // column group j -> field index
    int k;
    int rows;         // L = 3 Vh
};

// Warp roles (192 threads): warp 0 issues the TMA loads, warp 1 issues the MMAs
// and owns the TMEM allocation, warps 2..5 read the accumulator (warp w may
// only access TMEM lanes 32 * (w % 4) .. +31, so these four cover all 128 rows).
constexpr int TC_THREADS = 192;

// operand kinds of A (the eigenvectors): FP16 high + low parts of FP32 vectors,
// stored BF16 vectors, stored FP16 vectors; B is split into high and low parts
// of A's type in every case
enum : int { AK_F16_SPLIT = 0, AK_BF16 = 1, AK_F16 = 2 };

template <int MT, int N, int STAGES, int MODE, int AK>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
              const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, int K, int kchunk,
              int Mrows, float *part, ExpandEpi epi, int *status)
{
    constexpr int A_TILE = 128 * TC_ROWB;               // 16 KB per 128-row tile
    constexpr int B_TILE = N * TC_ROWB;
    constexpr int AP = AK == AK_F16_SPLIT ? 2 : 1;        // A parts: hi (+ lo for split FP32)
    constexpr int STAGE = AP * MT * A_TILE + 2 * B_TILE;  // B: hi + lo
    // the expansion walks several row tiles per CTA: two accumulators, so that the
    // MMAs of tile t+1 run while the epilogue drains tile t
    constexpr int NBUF = MODE == 1 ? 2 : 1;
    constexpr int BUFC = MT * N; // TMEM columns of one accumulator
    constexpr int NCOLS = (NBUF * BUFC <= 32) ? 32 : (NBUF * BUFC <= 64) ? 64 : (NBUF * BUFC <= 128) ? 128
                        : (NBUF * BUFC <= 256) ? 256 : 512;
    constexpr uint32_t IDESC = AK == AK_BF16 ? tc::idesc_bf16_f32(128, N) : tc::idesc_f16_f32(128, N);
    static_assert(N % 16 == 0 && N >= 16 && N <= 256, "N");
    static_assert(NBUF * BUFC <= 512, "TMEM columns");

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE);
    uint64_t *empty = full + STAGES;
    uint64_t *done = empty + STAGES;     // [NBUF] MMAs of a tile finished
    uint64_t *drained = done + NBUF;     // [NBUF] epilogue has read the accumulator
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(drained + NBUF);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < NBUF; b++) {
            tc::mbar_init(&done[b], 1);
            tc::mbar_init(&drained[b], 128);
        }
        tc::fence_mbar_init();
    }
    if (warp == 1) tc::tmem_alloc(tmem_holder, NCOLS);
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t taddr = *tmem_holder;

    // work list: (row tile, K range)
    int ntiles, tile0, tstride, kbeg, kend;
    if (MODE == 0) {
        ntiles = 1;
        tile0 = blockIdx.y;
        tstride = 1;
        kbeg = blockIdx.x * kchunk;
        kend = min(K, kbeg + kchunk);
    } else {
        ntiles = (Mrows + 127) / 128;
        tile0 = blockIdx.x;
        tstride = gridDim.x;
        kbeg = 0;
        kend = K;
    }
    const int nk = (kend - kbeg + TC_BK - 1) / TC_BK;

    const uint32_t lim = epi.spin_limit;
    if (warp == 0 && lane == 0 && !epi.no_loads) {
        // ---------------- TMA producer
        tc::prefetch_tmap(&tmAh);
        if (AK == AK_F16_SPLIT) tc::prefetch_tmap(&tmAl);
        tc::prefetch_tmap(&tmBh);
        tc::prefetch_tmap(&tmBl);
        uint32_t it = 0;
        for (int t = tile0; t < (MODE == 0 ? tile0 + 1 : ntiles); t += tstride) {
            const int m0 = (MODE == 0) ? t * MT * 128 : t * 128;
            for (int kk = 0; kk < nk; kk++, it++) {
                const int s = it % STAGES;
                if (it >= STAGES && !tc::mbar_wait(&empty[s], ((it / STAGES) - 1) & 1, status, tc::TC_TIMEOUT_EMPTY, lim))
                    goto producer_done;
                uint8_t *st = smem + s * STAGE;
                tc::mbar_arrive_expect_tx(&full[s], STAGE);
                const int kx = kbeg + kk * TC_BK;
                for (int mt = 0; mt < MT; mt++) {
                    tc::tma_load_2d(st + mt * A_TILE, &tmAh, &full[s], kx, m0 + mt * 128);
                    if (AK == AK_F16_SPLIT) tc::tma_load_2d(st + (MT + mt) * A_TILE, &tmAl, &full[s], kx, m0 + mt * 128);
                }
                tc::tma_load_2d(st + AP * MT * A_TILE, &tmBh, &full[s], kx, 0);
                tc::tma_load_2d(st + AP * MT * A_TILE + B_TILE, &tmBl, &full[s], kx, 0);
            }
        }
    producer_done:
        // the loads of the last stages must have landed before the CTA exits
        // (already true on the normal path; bounded if the pipeline broke)
        for (uint32_t j = (it > STAGES ? it - STAGES : 0); j < it; j++)
            if (!tc::mbar_try_wait(&full[j % STAGES], (j / STAGES) & 1))
                for (int spin = 0; spin < (1 << 20) && !tc::mbar_try_wait(&full[j % STAGES], (j / STAGES) & 1); spin++) {
                }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        uint32_t it = 0, tcount = 0;
        for (int t = tile0; t < (MODE == 0 ? tile0 + 1 : ntiles); t += tstride, tcount++) {
            // accumulator b is used for the (use)-th time: the epilogue must have
            // drained its previous use
            const uint32_t b = tcount % NBUF, use = tcount / NBUF;
            if (use > 0 && !tc::mbar_wait(&drained[b], (use - 1) & 1, status, tc::TC_TIMEOUT_DONE, lim)) break;
            tc::tc_fence_after();
            for (int kk = 0; kk < nk; kk++, it++) {
                const int s = it % STAGES;
                if (!tc::mbar_wait(&full[s], (it / STAGES) & 1, status, tc::TC_TIMEOUT_FULL, lim)) goto mma_done;
                tc::tc_fence_after();
                const uint32_t st = tc::smem_addr(smem + s * STAGE);
                const uint32_t bh = st + AP * MT * A_TILE, bl = bh + B_TILE;
#pragma unroll
                for (int mt = 0; mt < MT; mt++) {
                    const uint32_t ah = st + mt * A_TILE, al = st + (MT + mt) * A_TILE;
#pragma unroll
                    for (int q = 0; q < TC_BK / 16; q++) {
                        const uint32_t off = q * 32; // 16 16-bit values along K inside the swizzle atom
                        const uint32_t d = taddr + b * BUFC + mt * N;
                        const uint32_t acc0 = (kk > 0 || q > 0) ? 1u : 0u;
                        tc::mma_f16(d, tc::smem_desc_sw128(ah + off), tc::smem_desc_sw128(bh + off), IDESC, acc0);
                        tc::mma_f16(d, tc::smem_desc_sw128(ah + off), tc::smem_desc_sw128(bl + off), IDESC, 1u);
                        if (AK == AK_F16_SPLIT)
                            tc::mma_f16(d, tc::smem_desc_sw128(al + off), tc::smem_desc_sw128(bh + off), IDESC, 1u);
                    }
                }
                tc::mma_commit(&empty[s]);
            }
            tc::mma_commit(&done[b]);
        }
    mma_done:;
    }

    // ---------------- epilogue (warps 2..5)
    if (warp >= 2) {
        const int quarter = warp & 3;
        uint32_t tcount = 0;
        for (int t = tile0; t < (MODE == 0 ? tile0 + 1 : ntiles); t += tstride, tcount++) {
            const uint32_t b = tcount % NBUF, use = tcount / NBUF;
            bool ok = tc::mbar_wait(&done[b], use & 1, status, tc::TC_TIMEOUT_DONE, lim);
            tc::tc_fence_after();
            const uint32_t tbuf = taddr + b * BUFC;
            const int row = quarter * 32 + lane;
            if (MODE == 0) {
                for (int mt = 0; mt < MT; mt++) {
                    const int m = t * MT * 128 + mt * 128 + row;
#pragma unroll
                    for (int c0 = 0; c0 < N; c0 += 16) {
                        float v[16];
                        tc::tmem_ld16(tbuf + (uint32_t(quarter * 32) << 16) + mt * N + c0, v);
                        if (ok && nk > 0 && m < Mrows) {
                            float *dst = part + (size_t(blockIdx.x) * Mrows + m) * N + c0;
#pragma unroll
                            for (int i = 0; i < 16; i++) dst[i] = v[i];
                        }
                    }
                }
            } else {
                // 32 accumulator columns (8 right-hand sides) at a time: the FP64
                // x and r values of all 8 are loaded before the accumulator is
                // read and before any store, so a thread has up to 16 loads in
                // flight instead of one read-modify-write at a time
                const int s = t * 128 + row;
                const bool live = ok && s < epi.rows;
                const uint32_t tl = tbuf + (uint32_t(quarter * 32) << 16);
                for (int c0 = 0; c0 < N; c0 += 32) {
                    double2 xv[8], rv[8];
                    double2 *xp[8], *rp[8];
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const int j = (c0 >> 2) + q; // columns 4j .. 4j+3 belong to right-hand side j
                        xp[q] = nullptr;
                        rp[q] = nullptr;
                        if (live && j < epi.k) {
                            const size_t f = size_t(epi.field[j]);
                            xp[q] = epi.x + epi.fstride * f + s;
                            xv[q] = *xp[q];
                            if (epi.r) {
                                rp[q] = epi.r + epi.fstride * f + s;
                                rv[q] = *rp[q];
                            }
                        }
                    }
                    float v0[16], v1[16];
                    tc::tmem_ld16(tl + c0, v0); // warp-wide: c0 and N are uniform
                    if (c0 + 16 < N) {
                        tc::tmem_ld16(tl + c0 + 16, v1);
                    } else {
#pragma unroll
                        for (int i = 0; i < 16; i++) v1[i] = 0.f;
                    }
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        if (!xp[q]) continue;
                        const float *sc = epi.scale + 4 * ((c0 >> 2) + q);
                        const float *v = q < 4 ? v0 + 4 * q : v1 + 4 * (q - 4);
                        xv[q].x += double(v[0]) * sc[0];
                        xv[q].y += double(v[1]) * sc[1];
                        *xp[q] = xv[q];
                        if (rp[q]) {
                            rv[q].x -= double(v[2]) * sc[2];
                            rv[q].y -= double(v[3]) * sc[3];
                            *rp[q] = rv[q];
                        }
                    }
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&drained[b]);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(taddr, NCOLS);
    }
}

// ------------------------------------------------------------- operand builders
// V (n stored FP32 even fields) -> FP16 hi/lo copies scaled by sigma:
//   vector-major  [i][s][re,im]   (projection A)
//   site-major    [s][i][re,im]   (expansion A, row pitch ld_sm halves)
__global__ void k_build_v(int Vh, int n, const char *__restrict__ V32, size_t vstride, float sigma, __half *vm_hi,
                          __half *vm_lo, __half *sm_hi, __half *sm_lo, size_t ld_sm)
{
    const size_t L = size_t(3) * Vh;
    const size_t total = L * n;
    for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += size_t(gridDim.x) * blockDim.x) {
        const int i = int(t / L);
        const size_t s = t % L; // s = c * Vh + cb
        const int c = int(s / Vh), cb = int(s % Vh);
        const char *p = V32 + vstride * i;
        float re, im;
        if (c < 2) {
            const float4 a = reinterpret_cast<const float4 *>(p)[cb];
            re = c == 0 ? a.x : a.z;
            im = c == 0 ? a.y : a.w;
        } else {
            const float2 b = reinterpret_cast<const float2 *>(p + size_t(Vh) * 16)[cb];
            re = b.x;
            im = b.y;
        }
        re *= sigma;
        im *= sigma;
        const __half hr = __float2half_rn(re), hi_ = __float2half_rn(im);
        const __half lr = __float2half_rn(re - __half2float(hr)), li = __float2half_rn(im - __half2float(hi_));
        const size_t vm = (size_t(i) * L + s) * 2, sm = s * ld_sm + size_t(i) * 2;
        vm_hi[vm] = hr;
        vm_hi[vm + 1] = hi_;
        vm_lo[vm] = lr;
        vm_lo[vm + 1] = li;
        sm_hi[sm] = hr;
        sm_hi[sm + 1] = hi_;
        sm_lo[sm] = lr;
        sm_lo[sm + 1] = li;
    }
}

// R' columns 2j = (Re r_j, Im r_j), 2j+1 = (Im r_j, -Re r_j), times scale[j], hi/lo
__global__ void k_build_r(int L, int k, const double2 *__restrict__ R, size_t fstride, const int *field,
                          const float *scale, __half *rh, __half *rl)
{
    const size_t total = size_t(L) * k;
    for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += size_t(gridDim.x) * blockDim.x) {
        const int j = int(t / L);
        const size_t s = t % L;
        const double2 v = R[fstride * size_t(field[j]) + s];
        const float a = float(v.x * scale[j]), b = float(v.y * scale[j]);
        const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
        const __half la = __float2half_rn(a - __half2float(ha)), lb = __float2half_rn(b - __half2float(hb));
        const size_t c0 = (size_t(2 * j) * L + s) * 2, c1 = (size_t(2 * j + 1) * L + s) * 2;
        rh[c0] = ha;
        rh[c0 + 1] = hb;
        rl[c0] = la;
        rl[c0 + 1] = lb;
        rh[c1] = hb;
        rh[c1 + 1] = __hneg(ha);
        rl[c1] = lb;
        rl[c1 + 1] = __hneg(la);
    }
}

// BF16 eigenvectors: site-major copy sm[s][i] (row pitch ld_sm bf16x2 pairs) of
// the stored vector-major vectors V[i][s], s = colour * Vh + cb; 32 x 32 tiles
// through shared memory so that both sides are coalesced.
__global__ void k_build_v_sm_bf16(int L, int n, const __nv_bfloat162 *__restrict__ V, size_t vstride,
                                  __nv_bfloat162 *__restrict__ sm, size_t ld_sm)
{
    __shared__ __nv_bfloat162 tile[32][33];
    const int s0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r, s = s0 + threadIdx.x;
        if (i < n && s < L) tile[r][threadIdx.x] = V[vstride * i + s];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int s = s0 + r, i = i0 + threadIdx.x;
        if (i < n && s < L) sm[ld_sm * s + i] = tile[threadIdx.x][r];
    }
}

// R' for the BF16 GEMM: columns 2j = (Re r_j, Im r_j), 2j+1 = (Im r_j, -Re r_j),
// times scale[j], split into BF16 high and low parts
__global__ void k_build_r_bf16(int L, int k, const double2 *__restrict__ R, size_t fstride, const int *field,
                               const float *scale, __nv_bfloat16 *rh, __nv_bfloat16 *rl)
{
    const size_t total = size_t(L) * k;
    for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += size_t(gridDim.x) * blockDim.x) {
        const int j = int(t / L);
        const size_t s = t % L;
        const double2 v = R[fstride * size_t(field[j]) + s];
        const float a = float(v.x * scale[j]), b = float(v.y * scale[j]);
        const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
        const __nv_bfloat16 la = __float2bfloat16_rn(a - __bfloat162float(ha));
        const __nv_bfloat16 lb = __float2bfloat16_rn(b - __bfloat162float(hb));
        const size_t c0 = (size_t(2 * j) * L + s) * 2, c1 = (size_t(2 * j + 1) * L + s) * 2;
        rh[c0] = ha;
        rh[c0 + 1] = hb;
        rl[c0] = la;
        rl[c0 + 1] = lb;
        rh[c1] = hb;
        rh[c1 + 1] = __hneg(ha);
        rl[c1] = lb;
        rl[c1 + 1] = __hneg(la);
    }
}

// C[i][col] = sum_split part[split][i][col] (fixed order), i < n, col < ncol;
// each split holds Mrows rows of N columns
__global__ void k_reduce_part(int nsplit, int n, int Mrows, int N, int ncol, const float *__restrict__ part, double *C)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * ncol; t += gridDim.x * blockDim.x) {
        const int i = t / ncol, col = t % ncol;
        double s = 0;
        for (int p = 0; p < nsplit; p++) s += part[(size_t(p) * Mrows + i) * N + col];
        C[t] = s;
    }
}

// ------------------------------------------------------------- host driver
struct TcState {
    unsigned version = ~0u;     // eigenpair version the copies were built from
    int n = 0, Vh = 0;
    int akind = AK_F16_SPLIT;   // AK_BF16 / AK_F16: vm_hi is the stored vectors, no lo parts
    void *vm_hi = nullptr, *vm_lo = nullptr, *sm_hi = nullptr, *sm_lo = nullptr;
    void *owned = nullptr;      // device copies owned by this state
    size_t ld_sm = 0;           // 16-bit values per site-major row
    size_t bytes = 0;
    float sigma = 1;
};

static TcState &tc_state(hisq_ctx *ctx)
{
    // one state per context, kept in a side table keyed by the context pointer
    static std::mutex mu;
    static std::vector<std::pair<hisq_ctx *, TcState>> table;
    std::lock_guard<std::mutex> lock(mu);
    for (auto &e : table)
        if (e.first == ctx) return e.second;
    table.emplace_back(ctx, TcState{});
    return table.back().second;
}

void tc_release(hisq_ctx *ctx)
{
    TcState &S = tc_state(ctx);
    if (S.owned) dev_free(ctx, S.owned, S.bytes);
    S = TcState{};
}

// forget the context's state (called when the context is destroyed)
void tc_forget(hisq_ctx *ctx)
{
    tc_release(ctx);
}

static hisq_status tc_prepare_v(hisq_ctx *ctx, int n)
{
    TcState &S = tc_state(ctx);
    const int Vh = ctx->g.Vh;
    if (S.version == ctx->eig.version && S.n == n && S.Vh == Vh && S.vm_hi) return HISQ_OK;
    if (ctx->eig.prec != 32 && ctx->eig.prec != HISQ_PREC_BF16 && ctx->eig.prec != HISQ_PREC_HALF_EV)
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "tensor-core deflation needs FP32, BF16 or FP16 (14) eigenvectors");
    tc_release(ctx);
    const size_t L = size_t(3) * Vh;
    const size_t ld_sm = ((size_t(2) * n + 63) / 64) * 64; // 16-bit values per site-major row (128 B multiple)
    if (ctx->eig.prec == HISQ_PREC_BF16 || ctx->eig.prec == HISQ_PREC_HALF_EV) {
        // the stored vectors are the projection operand; build the site-major copy
        // (a transpose of 32-bit (re, im) pairs, the same for both 16-bit types)
        const size_t bytes = L * ld_sm * sizeof(__nv_bfloat16);
        void *sm = dev_alloc(ctx, bytes);
        if (!sm) return HISQ_ERR_OOM;
        HISQ_CUDA(cudaMemsetAsync(sm, 0, bytes, ctx->stream));
        S.akind = ctx->eig.prec == HISQ_PREC_BF16 ? AK_BF16 : AK_F16;
        S.vm_hi = ctx->eig.vecs;
        S.sm_hi = sm;
        S.owned = sm;
        S.ld_sm = ld_sm;
        S.bytes = bytes;
        S.n = n;
        S.Vh = Vh;
        S.version = ctx->eig.version;
        // FP16 vectors are stored times 2^e (exact); BF16 ones unscaled
        S.sigma = S.akind == AK_F16 ? pow2f(ev_half_exponent(Vh)) : 1.f;
        ctx->launches++;
        dim3 grid(unsigned((L + 31) / 32), unsigned((n + 31) / 32));
        k_build_v_sm_bf16<<<grid, dim3(32, 8), 0, ctx->stream>>>(int(L), n, (const __nv_bfloat162 *)ctx->eig.vecs, L,
                                                                 (__nv_bfloat162 *)sm, ld_sm / 2);
        HISQ_CUDA(cudaGetLastError());
        return HISQ_OK;
    }
    const size_t vm = L * n * 2, sm = L * ld_sm;
    const size_t bytes = (2 * vm + 2 * sm) * sizeof(__half);
    __half *base = (__half *)dev_alloc(ctx, bytes);
    if (!base) return HISQ_ERR_OOM;
    HISQ_CUDA(cudaMemsetAsync(base, 0, bytes, ctx->stream));
    S.owned = base;
    S.vm_hi = base;
    S.vm_lo = base + vm;
    S.sm_hi = base + 2 * vm;
    S.sm_lo = base + 2 * vm + sm;
    S.ld_sm = ld_sm;
    S.bytes = bytes;
    S.n = n;
    S.Vh = Vh;
    S.version = ctx->eig.version;
    S.sigma = float(std::sqrt(double(L)));
    ctx->launches++;
    k_build_v<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(Vh, n, (const char *)ctx->eig.vecs, spinor_bytes(32, Vh),
                                                          S.sigma, (__half *)S.vm_hi, (__half *)S.vm_lo,
                                                          (__half *)S.sm_hi, (__half *)S.sm_lo, ld_sm);
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

template <int MT, int N, int ST, int MODE, int AK>
static hisq_status launch_gemm(hisq_ctx *ctx, dim3 grid, const CUtensorMap *m, int K, int kchunk, int Mrows, float *part,
                               ExpandEpi epi, int *status)
{
    constexpr int STAGE = (AK == AK_F16_SPLIT ? 2 : 1) * MT * 128 * TC_ROWB + 2 * N * TC_ROWB;
    const size_t smem = size_t(ST) * STAGE + 1024 + 256;
    static_assert(ST * STAGE + 1024 + 256 <= 227 * 1024, "shared memory");
    auto kern = k_tc_gemm<MT, N, ST, MODE, AK>;
    static bool attr = false;
    if (!attr) {
        HISQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
        attr = true;
    }
    ctx->launches++;
    kern<<<grid, TC_THREADS, smem, ctx->stream>>>(m[0], m[1], m[2], m[3], K, kchunk, Mrows, part, epi, status);
    HISQ_CUDA(cudaGetLastError());
    return HISQ_OK;
}

// value a as a 16-bit high part and the 16-bit rounding of the remainder
// (FP16 via the CUDA host conversions; BF16 by round-to-nearest-even on the
// FP32 bit pattern: BF16 is the upper half of an FP32)
static uint16_t bf16_bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) == 0x7F800000u) return uint16_t(u >> 16); // Inf/NaN: not produced here
    u += 0x7FFFu + ((u >> 16) & 1u);
    return uint16_t(u >> 16);
}
static float bf16_value(uint16_t h)
{
    const uint32_t u = uint32_t(h) << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
static void split16(double a, bool bf, uint16_t *hi, uint16_t *lo)
{
    if (bf) {
        *hi = bf16_bits(float(a));
        *lo = bf16_bits(float(a - double(bf16_value(*hi))));
    } else {
        const __half h = __float2half_rn(float(a));
        const __half l = __float2half_rn(float(a - double(__half2float(h))));
        std::memcpy(hi, &h, 2);
        std::memcpy(lo, &l, 2);
    }
}

// Batched deflation of k right-hand sides with the first n stored eigenpairs:
// x_j += sum_i v_i c_ij / lambda_i, r_j -= sum_i v_i c_ij, c = V^dag r.
// R, X: k FP64 even fields (element s of field j at base + j*fstride + s).
// rnorm[j] = |r_j| (host values) for the operand scaling.  `field` (host,
// nullable) maps right-hand side j to field field[j] of R and X.  With
// update_r = false only X is updated (R is then the caller's to recompute).
hisq_status tc_deflate_batch(hisq_ctx *ctx, int n, int k, double *R, double *X, const double *rnorm, const int *field,
                             bool update_r)
{
    if (k < 1 || k > 32) return set_err(ctx, HISQ_ERR_INVALID_ARG, "tensor-core deflation: 1..32 right-hand sides");
    if (n < 1 || n > 512) return set_err(ctx, HISQ_ERR_INVALID_ARG, "tensor-core deflation: 1..512 eigenpairs");
    const int Vh = ctx->g.Vh;
    const int L = 3 * Vh;
    const size_t fstride = size_t(L); // double2 elements per even field
    TRY_HISQ(tc_prepare_v(ctx, n));
    TcState &S = tc_state(ctx);

    // ---- projection operands: R' (2k columns), hi/lo
    const int NP = 64;                        // 2k <= 64 columns, padded by zero fill
    std::vector<float> sc(k);
    for (int j = 0; j < k; j++) sc[j] = rnorm[j] > 0 ? float(std::sqrt(double(L)) / rnorm[j]) : 1.f;
    const int ak = S.akind;
    const bool bf = ak == AK_BF16, single = ak != AK_F16_SPLIT;
    const size_t rbytes = size_t(2) * k * L * 2 * sizeof(__half); // same size for BF16
    char *w = (char *)get_buf(ctx, BUF_TC_WORK, 2 * rbytes + 4096 + sizeof(float) * 8 * 64);
    if (!w) return HISQ_ERR_OOM;
    void *rh = w, *rl = w + rbytes;
    float *dscale = (float *)(w + 2 * rbytes);
    int *dfield = (int *)(w + 2 * rbytes + 1024);
    int *status = (int *)(w + 2 * rbytes + 2048);
    std::vector<int> fl(k);
    for (int j = 0; j < k; j++) fl[j] = field ? field[j] : j;
    HISQ_CUDA(cudaMemcpyAsync(dscale, sc.data(), sizeof(float) * k, cudaMemcpyHostToDevice, ctx->stream));
    HISQ_CUDA(cudaMemcpyAsync(dfield, fl.data(), sizeof(int) * k, cudaMemcpyHostToDevice, ctx->stream));
    HISQ_CUDA(cudaMemsetAsync(status, 0, sizeof(int), ctx->stream));
    ctx->launches++;
    if (bf)
        k_build_r_bf16<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(L, k, (const double2 *)R, fstride, dfield, dscale,
                                                                  (__nv_bfloat16 *)rh, (__nv_bfloat16 *)rl);
    else
        k_build_r<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(L, k, (const double2 *)R, fstride, dfield, dscale,
                                                             (__half *)rh, (__half *)rl);
    HISQ_CUDA(cudaGetLastError());

    CUtensorMap mp[4];
    const uint64_t Kp = uint64_t(2) * L;
    const void *alo = single ? S.vm_hi : S.vm_lo; // stored 16-bit vectors: no low part (the map is not read)
    if (!make_tmap(&mp[0], S.vm_hi, Kp, n, Kp * 2, 128, bf) || !make_tmap(&mp[1], alo, Kp, n, Kp * 2, 128, bf) ||
        !make_tmap(&mp[2], rh, Kp, 2 * k, Kp * 2, NP, bf) || !make_tmap(&mp[3], rl, Kp, 2 * k, Kp * 2, NP, bf))
        return set_err(ctx, HISQ_ERR_CUDA, "tensor map encoding failed");
    // split K over about one CTA per SM; rows per CTA: FP16 hi + lo A tiles of
    // 256 rows, or BF16 A tiles of 512 rows, with B fit two 80 KB stages
    const int mtiles = (n + 127) / 128;
    const int MTP = single ? (mtiles >= 4 ? 4 : (mtiles >= 2 ? 2 : 1)) : 2;
    const int mgroups = (mtiles + MTP - 1) / MTP;
    int nsplit = std::max(1, ctx->num_sms / mgroups);
    int kchunk = int(((Kp + nsplit - 1) / nsplit + TC_BK - 1) / TC_BK) * TC_BK;
    nsplit = int((Kp + kchunk - 1) / kchunk);
    const int Mrows = mgroups * MTP * 128;
    float *part = (float *)get_buf(ctx, BUF_TC_PART, sizeof(float) * size_t(nsplit) * Mrows * NP);
    double *C = (double *)get_buf(ctx, BUF_TC_C, sizeof(double) * size_t(n) * 2 * k);
    if (!part || !C) return HISQ_ERR_OOM;
    // failure injection (tests): one call whose producers issue nothing and
    // whose waits give up after a few thousand polls
    const bool inject = ctx->inject_wait_timeout;
    ctx->inject_wait_timeout = false;
    const uint32_t lim = inject ? 4096u : tc::kSpinLimit;
    ExpandEpi none{};
    none.spin_limit = lim;
    none.no_loads = inject ? 1 : 0;
    const dim3 pgrid(nsplit, mgroups);
    auto project = [&](auto akc) -> hisq_status {
        constexpr int AKC = decltype(akc)::value;
        if (MTP == 4) return launch_gemm<4, NP, 2, 0, AKC>(ctx, pgrid, mp, int(Kp), kchunk, Mrows, part, none, status);
        if (MTP == 2) return launch_gemm<2, NP, 2, 0, AKC>(ctx, pgrid, mp, int(Kp), kchunk, Mrows, part, none, status);
        return launch_gemm<1, NP, 4, 0, AKC>(ctx, pgrid, mp, int(Kp), kchunk, Mrows, part, none, status);
    };
    if (ak == AK_BF16)
        TRY_HISQ(project(std::integral_constant<int, AK_BF16>{}));
    else if (ak == AK_F16)
        TRY_HISQ(project(std::integral_constant<int, AK_F16>{}));
    else
        TRY_HISQ((launch_gemm<2, NP, 2, 0, AK_F16_SPLIT>(ctx, pgrid, mp, int(Kp), kchunk, Mrows, part, none, status)));
    ctx->launches++;
    k_reduce_part<<<(n * 2 * k + 255) / 256, 256, 0, ctx->stream>>>(nsplit, n, Mrows, NP, 2 * k, part, C);
    HISQ_CUDA(cudaGetLastError());

    // ---- expansion operands on the host (n x k small): D' columns 4j..4j+3
    std::vector<double> Ch(size_t(n) * 2 * k);
    int hstatus = 0;
    HISQ_CUDA(cudaMemcpyAsync(Ch.data(), C, sizeof(double) * Ch.size(), cudaMemcpyDeviceToHost, ctx->stream));
    HISQ_CUDA(cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    if (hstatus != 0)
        return set_err(ctx, HISQ_ERR_TIMEOUT, "tensor-core projection: a pipeline wait ran out (code %d: %s)", hstatus,
                       hstatus == tc::TC_TIMEOUT_FULL ? "operands never arrived"
                                                      : (hstatus == tc::TC_TIMEOUT_EMPTY ? "stage never released"
                                                                                          : "accumulator never ready"));
    const double shift = 4.0 * ctx->mass * ctx->mass;
    const int NE = 4 * k;                     // columns of the expansion
    const int NEP = ((NE + 15) / 16) * 16;
    const int ldk = int(S.ld_sm);             // K extent of the expansion (2n padded)
    std::vector<uint16_t> dh(size_t(NEP) * ldk, 0), dl(size_t(NEP) * ldk, 0); // FP16 or BF16 bit patterns
    std::vector<float> esc(4 * k);
    const double sig = S.sigma;
    for (int j = 0; j < k; j++) {
        // c_ij = G_ij / (sigma_v * sc_j); d = c / lambda
        double cmax = 0, dmax = 0;
        std::vector<double> cr(n), ci(n), dr(n), di(n);
        for (int i = 0; i < n; i++) {
            const double g = 1.0 / (sig * sc[j]);
            cr[i] = Ch[size_t(i) * 2 * k + 2 * j] * g;
            ci[i] = Ch[size_t(i) * 2 * k + 2 * j + 1] * g;
            const double lam = ctx->eig.eps[i] + shift;
            dr[i] = cr[i] / lam;
            di[i] = ci[i] / lam;
            cmax = std::max(cmax, std::max(std::fabs(cr[i]), std::fabs(ci[i])));
            dmax = std::max(dmax, std::max(std::fabs(dr[i]), std::fabs(di[i])));
        }
        const double tx = dmax > 0 ? 1.0 / dmax : 1.0, tr = cmax > 0 ? 1.0 / cmax : 1.0;
        // GEMM column value = sigma_v * t * (sum v d) -> factor 1 / (sigma_v t)
        esc[4 * j + 0] = esc[4 * j + 1] = float(1.0 / (sig * tx));
        esc[4 * j + 2] = esc[4 * j + 3] = float(1.0 / (sig * tr));
        auto put = [&](int col, int i, double a_re, double a_im) {
            // K index (i, 0) multiplies Re v_i, (i, 1) multiplies Im v_i
            const double a[2] = {a_re, a_im};
            for (int q = 0; q < 2; q++) {
                uint16_t h, l;
                split16(a[q], bf, &h, &l);
                dh[size_t(col) * ldk + 2 * i + q] = h;
                dl[size_t(col) * ldk + 2 * i + q] = l;
            }
        };
        for (int i = 0; i < n; i++) {
            const double xr = dr[i] * tx, xi = di[i] * tx, rr = cr[i] * tr, ri = ci[i] * tr;
            // Re(v d) = Re v Re d - Im v Im d ; Im(v d) = Re v Im d + Im v Re d
            put(4 * j + 0, i, xr, -xi);
            put(4 * j + 1, i, xi, xr);
            put(4 * j + 2, i, rr, -ri);
            put(4 * j + 3, i, ri, rr);
        }
    }
    const size_t dbytes = size_t(NEP) * ldk * sizeof(uint16_t);
    char *dbuf = (char *)get_buf(ctx, BUF_TC_D, 2 * dbytes + sizeof(float) * 4 * 64);
    if (!dbuf) return HISQ_ERR_OOM;
    void *ddh = dbuf, *ddl = dbuf + dbytes;
    float *desc = (float *)(dbuf + 2 * dbytes);
    HISQ_CUDA(cudaMemcpyAsync(ddh, dh.data(), dbytes, cudaMemcpyHostToDevice, ctx->stream));
    HISQ_CUDA(cudaMemcpyAsync(ddl, dl.data(), dbytes, cudaMemcpyHostToDevice, ctx->stream));
    HISQ_CUDA(cudaMemcpyAsync(desc, esc.data(), sizeof(float) * 4 * k, cudaMemcpyHostToDevice, ctx->stream));
    // the TMA box of D' is as tall as the kernel's N (rows beyond NEP are zero filled)
    const int NT = NEP <= 32 ? 32 : (NEP <= 64 ? 64 : 128);
    CUtensorMap me[4];
    const void *slo = single ? S.sm_hi : S.sm_lo;
    if (!make_tmap(&me[0], S.sm_hi, ldk, L, S.ld_sm * 2, 128, bf) || !make_tmap(&me[1], slo, ldk, L, S.ld_sm * 2, 128, bf) ||
        !make_tmap(&me[2], ddh, ldk, NEP, size_t(ldk) * 2, NT, bf) ||
        !make_tmap(&me[3], ddl, ldk, NEP, size_t(ldk) * 2, NT, bf))
        return set_err(ctx, HISQ_ERR_CUDA, "tensor map encoding failed");
    ExpandEpi epi{lim, inject ? 1 : 0, (double2 *)X, update_r ? (double2 *)R : nullptr, fstride, desc, dfield, k, L};
    const int ntiles = (L + 127) / 128;
    const int grid = std::min(ntiles, ctx->num_sms);
    hisq_status st;
    auto expand = [&](auto akc) -> hisq_status {
        constexpr int AKC = decltype(akc)::value;
        if (NT == 32) return launch_gemm<1, 32, 4, 1, AKC>(ctx, dim3(grid), me, ldk, ldk, L, nullptr, epi, status);
        if (NT == 64) return launch_gemm<1, 64, 4, 1, AKC>(ctx, dim3(grid), me, ldk, ldk, L, nullptr, epi, status);
        return launch_gemm<1, 128, (AKC == AK_F16_SPLIT ? 3 : 4), 1, AKC>(ctx, dim3(grid), me, ldk, ldk, L, nullptr,
                                                                          epi, status);
    };
    if (ak == AK_BF16) st = expand(std::integral_constant<int, AK_BF16>{});
    else if (ak == AK_F16) st = expand(std::integral_constant<int, AK_F16>{});
    else st = expand(std::integral_constant<int, AK_F16_SPLIT>{});
    if (st != HISQ_OK) return st;
    HISQ_CUDA(cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    if (hstatus != 0) return set_err(ctx, HISQ_ERR_TIMEOUT, "tensor-core expansion: pipeline wait timed out (%d)", hstatus);
    return HISQ_OK;
}

} // namespace hisq

using namespace hisq;

// x_j = V Lambda^-1 V^dag b_j and r_j = b_j - V V^dag b_j for nrhs <= 32 host
// fields, through the tensor-core batched deflation (test entry point).
extern "C" hisq_status hisq_deflate_batch(hisq_ctx *ctx, int n, int nrhs, const double *b, double *x, double *r)
{
    if (!ctx) return HISQ_ERR_INVALID_ARG;
    if (!b || !x || !r || nrhs < 1 || nrhs > 32) return set_err(ctx, HISQ_ERR_INVALID_ARG, "bad batched deflation arguments");
    if (ctx->eig.n <= 0) return set_err(ctx, HISQ_ERR_STATE, "no eigenpairs stored");
    if (!(ctx->mass > 0)) return set_err(ctx, HISQ_ERR_STATE, "mass not set");
    if (n <= 0 || n > ctx->eig.n) n = ctx->eig.n;
    HISQ_CUDA(cudaSetDevice(ctx->device));
    const int Vh = ctx->g.Vh;
    const size_t full = size_t(ctx->g.V) * 48, s64 = spinor_bytes(64, Vh);
    double *f = (double *)get_buf(ctx, BUF_ETA_FULL, full);
    char *R = (char *)get_buf(ctx, BUF_B_RHI, s64 * nrhs);
    char *X = (char *)get_buf(ctx, BUF_B_XHI, s64 * nrhs);
    if (!f || !R || !X) return HISQ_ERR_OOM;
    std::vector<double> norms(nrhs);
    for (int j = 0; j < nrhs; j++) {
        HISQ_CUDA(cudaMemcpyAsync(f, b + size_t(j) * ctx->g.V * 6, full, cudaMemcpyHostToDevice, ctx->stream));
        TRY_HISQ(launch_gather_parity(ctx, f, 0, 64, R + s64 * j));
        TRY_HISQ(launch_norm2(ctx, 64, R + s64 * j, 12));
        double n2;
        TRY_HISQ(read_slots(ctx, 12, 1, &n2));
        norms[j] = std::sqrt(n2);
    }
    HISQ_CUDA(cudaMemsetAsync(X, 0, s64 * nrhs, ctx->stream));
    TRY_HISQ(tc_deflate_batch(ctx, n, nrhs, (double *)R, (double *)X, norms.data(), nullptr, true));
    for (int j = 0; j < nrhs; j++) {
        HISQ_CUDA(cudaMemsetAsync(f, 0, full, ctx->stream));
        TRY_HISQ(launch_scatter_parity(ctx, X + s64 * j, 64, 0, f));
        HISQ_CUDA(cudaMemcpyAsync(x + size_t(j) * ctx->g.V * 6, f, full, cudaMemcpyDeviceToHost, ctx->stream));
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
        HISQ_CUDA(cudaMemsetAsync(f, 0, full, ctx->stream));
        TRY_HISQ(launch_scatter_parity(ctx, R + s64 * j, 64, 0, f));
        HISQ_CUDA(cudaMemcpyAsync(r + size_t(j) * ctx->g.V * 6, f, full, cudaMemcpyDeviceToHost, ctx->stream));
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    return HISQ_OK;
}
