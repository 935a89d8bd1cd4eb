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
#include <map>
#include <mutex>
#include <utility>

#include "internal.cuh"
#include "tc.cuh"

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
    const double *alpha; // alpha[j] by right-hand side (global or shared memory)
    const double *m4;    // 4 m^2
    template <typename R>
    __device__ __forceinline__ void operator()(int cb, int j, const CVec<R> &acc, double &red) const
    {
        const R alpha_j = R(alpha[j]);
        const R m4v = R(*m4);
        const S pj = p.at(j), rj = r.at(j);
        const SX xj = x.at(j);
        CVec<R> pv = pj.load(cb);
        CVec<R> rv = rj.load(cb);
        auto xv = xj.load(cb);
        typedef typename SX::real XR;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            R apr = fma(m4v, pv.re[i], -acc.re[i]);
            R api = fma(m4v, pv.im[i], -acc.im[i]);
            rv.re[i] = fma(-alpha_j, apr, rv.re[i]);
            rv.im[i] = fma(-alpha_j, api, rv.im[i]);
            xv.re[i] = fma(XR(alpha_j), XR(pv.re[i]), xv.re[i]);
            xv.im[i] = fma(XR(alpha_j), XR(pv.im[i]), xv.im[i]);
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

// gathered FP32 links of the batched kernels: fat (and, with 18-real long
// links, long) rows per direction, read through the read-only path
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

// The sites of a batched operator launch: D on output parity `par` applied to
// the R fields jj[] of `in` at this thread's sites (one site per lane, site
// groups of 32 over the grid), each result handed to the epilogue with its
// running reduction red[u].  Slots past kact (a partial last chunk) gather an
// active field again and skip only the epilogue, so every gather is
// unconditional and the compiler can issue them all ahead of the arithmetic.
template <int R, class S, class Lk, class L12T, bool R12, class Epi, bool PF>
__device__ __forceinline__ void mrhs_sites(const Geom &g, int par, const Lk &L, const L12T &L12, float c3,
                                           const BatchF<S> &in, const int (&jj)[R], const bool (&on)[R],
                                           const MrhsTile &tl, const Epi &epi, double (&red)[R])
{
    typedef typename Lk::real Rl;
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
            if (PF && mu < 3) {
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
}

// slots of this thread: chunk c holds slots c*R .. c*R+R-1
template <int R>
__device__ __forceinline__ void mrhs_slots(const BatchScalars *scal, const MrhsTile &tl, int kact, int (&jj)[R],
                                           bool (&on)[R])
{
#pragma unroll
    for (int u = 0; u < R; u++) {
        const int q = tl.chunk() * R + u;
        on[u] = q < kact; // uniform over the warp
        jj[u] = scal->idx[on[u] ? q : kact - 1];
    }
}

// PF: request the next direction's links into L2 while this one is computed
// (15 prefetch instructions per thread and direction; the autotuner weighs them
// against the latency they hide)
template <int R, class S, class Lk, class L12T, bool R12, class Epi, bool PF = true>
__global__ void __launch_bounds__(512, 1)
    k_dslash_mrhs(Geom g, int par, Lk L, L12T L12, float c3, BatchF<S> in, const BatchScalars *scal, MrhsTile tl,
                  Epi epi, BatchRed br)
{
    const int kact = scal->kact;
    int jj[R];
    bool on[R];
    mrhs_slots<R>(scal, tl, kact, jj, on);
    double red[R];
#pragma unroll
    for (int u = 0; u < R; u++) red[u] = 0;
    mrhs_sites<R, S, Lk, L12T, R12, Epi, PF>(g, par, L, L12, c3, in, jj, on, tl, epi, red);
    batch_reduce<R>(red, tl, kact, br);
}

// p_j = r_j + beta_j p_j at this thread's sites for its R slots (jj[u] < 0:
// inactive), |p_j|^2 into red[u]; beta by right-hand side (global or shared)
template <int R, class S>
__device__ __forceinline__ void pupd_sites(int Vh, const BatchF<S> &r, const BatchF<S> &p, const double *beta,
                                           const int (&jj)[R], const MrhsTile &tl, double (&red)[R])
{
    typedef typename S::real Rl;
    const int step = gridDim.x * tl.nsg * 32;
    for (int cb = (blockIdx.x * tl.nsg + tl.group()) * 32 + (threadIdx.x & 31); cb < Vh; cb += step) {
#pragma unroll
        for (int u = 0; u < R; u++) {
            if (jj[u] < 0) continue;
            const int j = jj[u];
            const Rl bj = Rl(beta[j]);
            const S rj = r.at(j), pj = p.at(j);
            auto rv = rj.load(cb);
            auto pv = pj.load(cb);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                pv.re[c] = fma(bj, pv.re[c], rv.re[c]);
                pv.im[c] = fma(bj, pv.im[c], rv.im[c]);
            }
            pj.store(cb, pv);
            red[u] += double(pv.norm2());
        }
    }
}

// p_j = r_j + beta_j p_j, |p_j|^2
template <int R, class S>
__global__ void __launch_bounds__(512, 1)
    k_p_update_mrhs(int Vh, BatchF<S> r, BatchF<S> p, const BatchScalars *scal, MrhsTile tl, BatchRed br)
{
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
    pupd_sites<R, S>(Vh, r, p, scal->beta, jj, tl, red);
    batch_reduce<R>(red, tl, kact, br);
}

// ------------------------------------------------- persistent batched CG
// The sloppy CG iterations of a batch between two host interventions (reliable
// updates, re-deflations, convergence) in one cooperative launch, all blocks
// resident.  Each iteration is three grid-wide phases as in the launch-per-phase
// loop: tmp_j = D_oe p_j; the fused D_eo + update of x_j and r_j; p_j = r_j +
// beta_j p_j.  Between phases a grid barrier (bounded: a wait that runs out
// records its code in *status and every block leaves); after it every block
// sums the per-block partials itself, in block order, so all blocks hold the
// same alpha, beta and |p|^2 without another barrier.  The launch stops after
// the iteration in which any right-hand side's |r|^2 leaves [lo2_j, hi2_j]
// (the host's reliable-update, convergence and divergence thresholds) or is
// not finite (the launch then ends two iterations later, see below), or after
// max_iters iterations.
struct PersistArgs {
    double *part;              // [gridDim.x][3][kMaxBatch] per-block partial sums
    unsigned *bar;             // grid barrier: [0] arrivals, [1] generation
    int *status;               // bounded-wait status (0: fine)
    const double *lo2, *hi2;   // thresholds by right-hand side
    int max_iters;
    double *monitor;           // host-mapped [monitor_len][kMaxBatch] |r|^2 history
    int monitor_len;
    unsigned long long *phase_ns; // [2]: time of the D_oe and D_eo phases (nullable)
    int *iters_done;           // iterations of the launch
    int *iters_rhs;            // iterations of each right-hand side (by id)
    unsigned long long wait_ns; // a barrier wait longer than this gives up
};

constexpr int kGridWaitCode = 4;          // status code of a grid barrier that ran out
constexpr unsigned long long kGridWaitNs = 4000000000ull; // 4 s

// (A block that gives up still arrives at the barrier exactly once, so the
// arrival counter returns to zero and the next launch starts clean.)

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded grid barrier: returns false when a wait ran out (here or elsewhere)
__device__ __forceinline__ bool grid_sync(unsigned *bar, int *status, unsigned long long wait_ns)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen0 = *reinterpret_cast<volatile unsigned *>(&bar[1]);
        __threadfence(); // this block's writes before the arrival
        if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            const unsigned long long t0 = globaltimer_ns();
            for (unsigned i = 0;; i++) {
                if (*reinterpret_cast<volatile unsigned *>(&bar[1]) != gen0) break;
                if ((i & 255) == 0) {
                    if (*reinterpret_cast<volatile int *>(status) != 0 || globaltimer_ns() - t0 >= wait_ns) {
                        atomicCAS(status, 0, kGridWaitCode);
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(64);
            }
        }
        __threadfence(); // the other blocks' writes after it (acquire)
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// per-slot sums of this block's R values per thread into out[slot]
template <int R>
__device__ __forceinline__ void block_partials(double (&v)[R], const MrhsTile &tl, int kact, double *out)
{
    __shared__ double sh[8][kMaxBatch];
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
        double t = 0;
        for (int w = 0; w < tl.nsg; w++) t += sh[w][q];
        out[q] = t;
    }
    __syncthreads();
}

template <int R, class S, class SX, class L12T, bool R12>
__global__ void __launch_bounds__(512, 1)
    k_bcg_persistent(Geom g, LinksFvB Lo, LinksFvB Le, L12T L12o, L12T L12e, float c3, BatchF<S> p, BatchF<S> tmp,
                     BatchF<S> r, BatchF<SX> x, BatchScalars *scal, MrhsTile tl, PersistArgs pa)
{
    __shared__ double alpha_s[kMaxBatch], beta_s[kMaxBatch], rr_s[kMaxBatch], rrn_s[kMaxBatch], pp_s[kMaxBatch];
    __shared__ double m4_s;
    __shared__ int idx_s[kMaxBatch], its_s[kMaxBatch], trig_s[kMaxBatch], ntrig_s;
    const int kact = scal->kact;
    for (int q = threadIdx.x; q < kact; q += blockDim.x) {
        const int j = scal->idx[q];
        idx_s[q] = j;
        its_s[j] = trig_s[j] = 0;
        rr_s[j] = scal->rr[j];
        pp_s[j] = scal->pp[j];
    }
    if (threadIdx.x == 0) {
        m4_s = scal->m4;
        ntrig_s = 0;
    }
    __syncthreads();
    int jj[R];
    bool on[R];
    mrhs_slots<R>(scal, tl, kact, jj, on);
    const long long iter0 = scal->iter;
    const bool timer = pa.phase_ns && blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long t_oe = 0, t_eo = 0;
    double *part = pa.part + size_t(blockIdx.x) * 3 * kMaxBatch;
    // sum of phase `ph`'s partials over the blocks, in block order (L2 reads)
    auto grid_total = [&](int ph, int q) {
        double t = 0;
        for (int b = 0; b < int(gridDim.x); b++) t += __ldcg(pa.part + (size_t(b) * 3 + ph) * kMaxBatch + q);
        return t;
    };
    // After the first iteration in which a right-hand side reaches its
    // threshold, every right-hand side runs two more iterations (the host-driven
    // loop notices a threshold two iterations late as well), so that the host
    // takes the right-hand sides that reach theirs at about the same time at once.
    int it = 0, first_trig = -1;
    bool ok = true;
    while (ok && it < pa.max_iters) {
        unsigned long long ta = timer ? globaltimer_ns() : 0;
        int jp[R]; // slots of the p update (-1: inactive)
#pragma unroll
        for (int u = 0; u < R; u++) jp[u] = on[u] ? jj[u] : -1;
        double red[R];
        // (1) tmp_j = D_oe p_j, |tmp_j|^2 -> alpha_j
#pragma unroll
        for (int u = 0; u < R; u++) red[u] = 0;
        mrhs_sites<R, S, LinksFvB, L12T, R12, BEpiStore<S>, true>(g, 1, Lo, L12o, c3, p, jj, on, tl,
                                                                  BEpiStore<S>{tmp}, red);
        block_partials<R>(red, tl, kact, part);
        if (!(ok = grid_sync(pa.bar, pa.status, pa.wait_ns))) break;
        for (int q = threadIdx.x; q < kact; q += blockDim.x) {
            const int j = idx_s[q];
            alpha_s[j] = rr_s[j] / (m4_s * pp_s[j] + grid_total(0, q));
        }
        __syncthreads();
        unsigned long long tb = timer ? globaltimer_ns() : 0;
        // (2) Ap = 4m^2 p - D_eo tmp; x += alpha p; r -= alpha Ap; |r|^2 -> beta_j
#pragma unroll
        for (int u = 0; u < R; u++) red[u] = 0;
        mrhs_sites<R, S, LinksFvB, L12T, R12, BEpiCG<S, SX>, true>(
            g, 0, Le, L12e, c3, tmp, jj, on, tl, BEpiCG<S, SX>{p, r, x, alpha_s, &m4_s}, red);
        block_partials<R>(red, tl, kact, part + kMaxBatch);
        if (!(ok = grid_sync(pa.bar, pa.status, pa.wait_ns))) break;
        for (int q = threadIdx.x; q < kact; q += blockDim.x) {
            const int j = idx_s[q];
            const double rn = grid_total(1, q);
            rrn_s[j] = rn;
            beta_s[j] = rn / rr_s[j];
            trig_s[j] = !(rn >= pa.lo2[j] && rn <= pa.hi2[j]); // also NaN
            if (blockIdx.x == 0 && pa.monitor)
                pa.monitor[size_t((iter0 + it) % pa.monitor_len) * kMaxBatch + j] = rn;
        }
        __syncthreads();
        if (timer) {
            const unsigned long long tc = globaltimer_ns();
            t_oe += tb - ta;
            t_eo += tc - tb;
        }
        // (3) p_j = r_j + beta_j p_j, |p_j|^2
#pragma unroll
        for (int u = 0; u < R; u++) red[u] = 0;
        pupd_sites<R, S>(g.Vh, r, p, beta_s, jp, tl, red);
        block_partials<R>(red, tl, kact, part + 2 * kMaxBatch);
        if (!(ok = grid_sync(pa.bar, pa.status, pa.wait_ns))) break;
        for (int q = threadIdx.x; q < kact; q += blockDim.x) {
            const int j = idx_s[q];
            pp_s[j] = grid_total(2, q);
            rr_s[j] = rrn_s[j];
            its_s[j]++;
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int q = 0; q < kact; q++)
                if (trig_s[idx_s[q]]) ntrig_s++;
        __syncthreads();
        if (ntrig_s > 0 && first_trig < 0) first_trig = it;
        it++;
        if (first_trig >= 0 && it - first_trig > 2) break;
    }
    if (blockIdx.x == 0) {
        for (int q = threadIdx.x; q < kact; q += blockDim.x) {
            const int j = idx_s[q];
            scal->rr[j] = rr_s[j];
            scal->rr_new[j] = rr_s[j];
            scal->pp[j] = pp_s[j];
            scal->alpha[j] = alpha_s[j];
            scal->beta[j] = beta_s[j];
            pa.iters_rhs[j] = its_s[j];
        }
        if (threadIdx.x == 0) {
            scal->iter = iter0 + it;
            *pa.iters_done = it;
            if (pa.phase_ns) {
                pa.phase_ns[0] += t_oe;
                pa.phase_ns[1] += t_eo;
            }
        }
    }
}

// ------------------------------------------------- packed FP32 pairs
// Blackwell executes two FP32 FMAs of a register pair in one instruction
// (fma.rn.f32x2: each half is an IEEE fused multiply-add, the same result as
// two scalar ones).  The packed kernel carries right-hand sides in pairs, so
// the colour algebra of two right-hand sides issues as one instruction stream:
// with the link entries broadcast to both halves, a complex multiply-add of a
// pair is four packed FMAs instead of eight scalar ones.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// a colour vector of two right-hand sides: (re, im) of each colour as pairs,
// and -im for the real part of the complex products
struct CVec2 {
    float2 re[3], im[3], nim[3];
};
struct CAcc2 {
    float2 re[3], im[3];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int c = 0; c < 3; c++) re[c] = im[c] = make_float2(0.f, 0.f);
    }
};

template <class S>
__device__ __forceinline__ CVec2 load_pair(const S &a, const S &b, int i)
{
    const CVec<float> x = a.load(i), y = b.load(i);
    CVec2 v;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        v.re[c] = make_float2(x.re[c], y.re[c]);
        v.im[c] = make_float2(x.im[c], y.im[c]);
        v.nim[c] = make_float2(-x.im[c], -y.im[c]);
    }
    return v;
}
// FP16 storage: the per-site scales of the two right-hand sides are applied
// as packed multiplies
template <>
__device__ __forceinline__ CVec2 load_pair<SpinorH>(const SpinorH &a, const SpinorH &b, int i)
{
    const uint4 ua = a.p[i], ub = b.p[i];
    const float2 s2 = make_float2(__uint_as_float(ua.w), __uint_as_float(ub.w));
    const float2 n2 = make_float2(-s2.x, -s2.y);
    const unsigned ha[3] = {ua.x, ua.y, ua.z}, hb[3] = {ub.x, ub.y, ub.z};
    CVec2 v;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float2 fa = __half22float2(*reinterpret_cast<const __half2 *>(&ha[c]));
        const float2 fb = __half22float2(*reinterpret_cast<const __half2 *>(&hb[c]));
        const float2 re = make_float2(fa.x, fb.x), im = make_float2(fa.y, fb.y);
        v.re[c] = mul2(re, s2);
        v.im[c] = mul2(im, s2);
        v.nim[c] = mul2(im, n2);
    }
    return v;
}

// acc += W v for a pair (W shared by both)
__device__ __forceinline__ void mv_acc2(CAcc2 &acc, const CMat<float> &W, const CVec2 &v)
{
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float2 wr = make_float2(W.re[3 * i + j], W.re[3 * i + j]);
            const float2 wi = make_float2(W.im[3 * i + j], W.im[3 * i + j]);
            acc.re[i] = fma2(wr, v.re[j], acc.re[i]);
            acc.re[i] = fma2(wi, v.nim[j], acc.re[i]);
            acc.im[i] = fma2(wr, v.im[j], acc.im[i]);
            acc.im[i] = fma2(wi, v.re[j], acc.im[i]);
        }
}
// acc += s (W v), s real
__device__ __forceinline__ void mv_acc2_scaled(CAcc2 &acc, float s, const CMat<float> &W, const CVec2 &v)
{
    CAcc2 t;
    t.zero();
    mv_acc2(t, W, v);
    const float2 s2 = make_float2(s, s);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        acc.re[i] = fma2(s2, t.re[i], acc.re[i]);
        acc.im[i] = fma2(s2, t.im[i], acc.im[i]);
    }
}

// The batched operator with P pairs (R = 2P right-hand sides) per thread;
// tiling, masking and reductions as k_dslash_mrhs.
template <int P, class S, class Lk, class L12T, bool R12, class Epi, bool PF>
__global__ void __launch_bounds__(512, 1)
    k_dslash_mrhs_x2(Geom g, int par, Lk L, L12T L12, float c3, BatchF<S> in, const BatchScalars *scal, MrhsTile tl,
                     Epi epi, BatchRed br)
{
    constexpr int R = 2 * P;
    const int kact = scal->kact;
    int jj[R];
    bool on[R];
#pragma unroll
    for (int u = 0; u < R; u++) {
        const int q = tl.chunk() * R + u;
        on[u] = q < kact;
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
        CAcc2 acc[P];
#pragma unroll
        for (int q = 0; q < P; q++) acc[q].zero();
#pragma unroll 1
        for (int mu = 0; mu < 4; mu++) {
            const int f1 = nb_cb(g, c, s, mu, +1), b1 = nb_cb(g, c, s, mu, -1);
            const int f3 = nb_cb(g, c, s, mu, +3), b3 = nb_cb(g, c, s, mu, -3);
            if (PF && mu < 3) {
                L.prefetch(mu + 1, cb);
                prefetch_long(L12, mu + 1, cb);
            }
            CMat<float> f, b;
            L.load(mu, 0, cb, f, b);
#pragma unroll
            for (int q = 0; q < P; q++) {
                const S va = in.at(jj[2 * q]), vb = in.at(jj[2 * q + 1]);
                mv_acc2(acc[q], f, load_pair(va, vb, f1));
                mv_acc2(acc[q], b, load_pair(va, vb, b1));
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
                for (int q = 0; q < P; q++) {
                    const S va = in.at(jj[2 * q]), vb = in.at(jj[2 * q + 1]);
                    mv_acc2_scaled(acc[q], sf, f3m, load_pair(va, vb, f3));
                    mv_acc2_scaled(acc[q], sb, b3m, load_pair(va, vb, b3));
                }
            } else {
                L.load(mu, 1, cb, f, b);
#pragma unroll
                for (int q = 0; q < P; q++) {
                    const S va = in.at(jj[2 * q]), vb = in.at(jj[2 * q + 1]);
                    mv_acc2(acc[q], f, load_pair(va, vb, f3));
                    mv_acc2(acc[q], b, load_pair(va, vb, b3));
                }
            }
        }
#pragma unroll
        for (int q = 0; q < P; q++) {
            CVec<float> x, y;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                x.re[i] = acc[q].re[i].x;
                x.im[i] = acc[q].im[i].x;
                y.re[i] = acc[q].re[i].y;
                y.im[i] = acc[q].im[i].y;
            }
            if (on[2 * q]) epi(cb, jj[2 * q], x, red[2 * q]);
            if (on[2 * q + 1]) epi(cb, jj[2 * q + 1], y, red[2 * q + 1]);
        }
    }
    batch_reduce<R>(red, tl, kact, br);
}

// ------------------------------------------------- the TMA-fed batched kernel
// The same operator with the links of each (site group, direction) copied into
// shared memory by the bulk-copy engine (one elected thread per site group
// issues 15 copies of 512 B: the 9 fat rows and the 6 stored long rows of 32
// consecutive sites) into a ring of `stages` slots guarded by mbarriers.  The
// warps then read each link element from shared memory once per R right-hand
// sides, so no link load is held in registers while the DRAM latency elapses:
// registers go to accumulators and neighbour gathers, and more warps fit.  The
// third row of each long link is rebuilt on the fly from the two stored rows,
// with the staggered phase, boundary sign and c3 applied to the rows first
// (row 2 of s*S is conj(s a x s b) / s).  Every wait is bounded: a wait that
// runs out records its code in *status and the warp gives up on the rest of its
// items (the reduction still runs, so the launch ends).
constexpr int kTmaRows = 15;                 // 9 fat + 6 long rows per (site group, direction)
constexpr int kTmaStageBytes = kTmaRows * 512; // 32 sites x float4 per row

template <int R, class S, class Epi, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_dslash_mrhs_tma(Geom g, int par, const float4 *__restrict__ fat, const float4 *__restrict__ lng, float c3,
                      float inv_c3, BatchF<S> in, const BatchScalars *scal, MrhsTile tl, Epi epi, BatchRed br,
                      int stages, int *status)
{
    extern __shared__ __align__(128) unsigned char dsm[];
    const int grp = tl.group(), chk = tl.chunk(), lane = threadIdx.x & 31;
    unsigned char *ring = dsm + size_t(grp) * stages * kTmaStageBytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(dsm + size_t(tl.nsg) * stages * kTmaStageBytes) + 2 * grp * stages;
    uint64_t *empty = full + stages;
    const bool producer = chk == 0 && lane == 0;
    if (producer) {
        for (int q = 0; q < stages; q++) {
            tc::mbar_init(&full[q], 1);
            tc::mbar_init(&empty[q], tl.nch);
        }
        tc::fence_mbar_init();
    }
    __syncthreads();

    const int kact = scal->kact;
    int jj[R];
    bool on[R];
#pragma unroll
    for (int u = 0; u < R; u++) {
        const int q = chk * R + u;
        on[u] = q < kact;
        jj[u] = scal->idx[on[u] ? q : kact - 1];
    }
    double red[R];
#pragma unroll
    for (int u = 0; u < R; u++) red[u] = 0;

    const int Vh = g.Vh;
    const int ngroups = (Vh + 31) / 32;
    const int first = blockIdx.x * tl.nsg + grp, gstride = gridDim.x * tl.nsg;
    const int nitems = first < ngroups ? ((ngroups - 1 - first) / gstride + 1) * 4 : 0;
    // item j = (site-group iteration j / 4, direction j % 4) into slot j % stages
    auto issue = [&](int j) {
        const int mu = j & 3;
        const int cb0 = (first + (j >> 2) * gstride) * 32;
        const uint32_t rb = uint32_t(min(32, Vh - cb0)) * 16u;
        uint64_t *fb = &full[j % stages];
        unsigned char *st = ring + size_t(j % stages) * kTmaStageBytes;
        tc::mbar_arrive_expect_tx(fb, kTmaRows * rb);
#pragma unroll 1
        for (int k = 0; k < 9; k++) tc::bulk_load_1d(st + k * 512, fat + size_t(mu * 9 + k) * Vh + cb0, rb, fb);
#pragma unroll 1
        for (int k = 0; k < 6; k++) tc::bulk_load_1d(st + (9 + k) * 512, lng + size_t(mu * 6 + k) * Vh + cb0, rb, fb);
    };
    int issued = 0;
    if (producer)
        for (; issued < min(stages - 1, nitems); issued++) issue(issued);

    bool ok = true;
    CVec<float> acc[R];
    int c[4] = {0, 0, 0, 0}, s = 0, cb = 0;
    bool valid = false;
#pragma unroll 1
    for (int it = 0; it < nitems; it++) {
        const int mu = it & 3;
        if (producer) {
            // keep up to `stages` items in flight; a slot is refilled once every
            // warp of the group has released it, and the producer blocks only
            // when the item its own warp needs next has not been issued yet
            while (ok && issued < nitems && issued < it + stages) {
                if (issued >= stages) {
                    const uint32_t par_e = ((issued / stages) - 1) & 1;
                    if (!tc::mbar_try_wait(&empty[issued % stages], par_e)) {
                        if (issued > it) break; // not needed yet: try again at the next item
                        ok = tc::mbar_wait(&empty[issued % stages], par_e, status, tc::TC_TIMEOUT_EMPTY);
                        if (!ok) break;
                    }
                }
                issue(issued++);
            }
        }
        if (!ok) break;
        if (mu == 0) {
            cb = (first + (it >> 2) * gstride) * 32 + lane;
            valid = cb < Vh;
            cb_coords(g, par, valid ? cb : Vh - 1, c);
            s = full_site(g, c);
#pragma unroll
            for (int u = 0; u < R; u++) acc[u].zero();
        }
        // the neighbour gathers do not depend on the links: issue them before
        // waiting for the slot, so their latency overlaps the copies'
        const int f1 = nb_cb(g, c, s, mu, +1), b1 = nb_cb(g, c, s, mu, -1);
        const int f3 = nb_cb(g, c, s, mu, +3), b3 = nb_cb(g, c, s, mu, -3);
        CVec<float> v[4][R];
#pragma unroll
        for (int u = 0; u < R; u++) {
            const S f = in.at(jj[u]);
            v[0][u] = cvt<float>(f.load(f1));
            v[1][u] = cvt<float>(f.load(b1));
            v[2][u] = cvt<float>(f.load(f3));
            v[3][u] = cvt<float>(f.load(b3));
        }
        if (!tc::mbar_wait(&full[it % stages], (it / stages) & 1, status, tc::TC_TIMEOUT_FULL)) {
            ok = false;
            break;
        }
        const float4 *rows = reinterpret_cast<const float4 *>(ring + size_t(it % stages) * kTmaStageBytes) + lane;
        // fat links: forward (x, y of each row element) and backward (z, w)
#pragma unroll
        for (int d = 0; d < 2; d++) {
#pragma unroll
            for (int k = 0; k < 9; k++) {
                const float2 w = d == 0 ? *reinterpret_cast<const float2 *>(rows + 32 * k)
                                        : *(reinterpret_cast<const float2 *>(rows + 32 * k) + 1);
                const int i = k / 3, j = k % 3;
#pragma unroll
                for (int u = 0; u < R; u++) {
                    acc[u].re[i] = fmaf(w.x, v[d][u].re[j], fmaf(-w.y, v[d][u].im[j], acc[u].re[i]));
                    acc[u].im[i] = fmaf(w.x, v[d][u].im[j], fmaf(w.y, v[d][u].re[j], acc[u].im[i]));
                }
            }
        }
        // long links: rows a, b of the SU(3) factor times the hop's sign s,
        // row 2 = conj(s a x s b) / s
        const float eta = stag_phase(mu, c);
        float sgn[2] = {eta, -eta};
        if (mu == 3 && g.t_antiperiodic) {
            if (c[3] + 3 >= g.T) sgn[0] = -sgn[0];
            if (c[3] < 3) sgn[1] = -sgn[1];
        }
#pragma unroll
        for (int d = 0; d < 2; d++) {
            const float sc = sgn[d] * c3, isc = sgn[d] * inv_c3;
            float ar[6], ai[6]; // rows 0 and 1: (a0, a1, a2, b0, b1, b2)
#pragma unroll
            for (int k = 0; k < 6; k++) {
                const float2 w = d == 0 ? *reinterpret_cast<const float2 *>(rows + 32 * (9 + k))
                                        : *(reinterpret_cast<const float2 *>(rows + 32 * (9 + k)) + 1);
                ar[k] = sc * w.x;
                ai[k] = sc * w.y;
                const int i = k / 3, j = k % 3;
#pragma unroll
                for (int u = 0; u < R; u++) {
                    acc[u].re[i] = fmaf(ar[k], v[2 + d][u].re[j], fmaf(-ai[k], v[2 + d][u].im[j], acc[u].re[i]));
                    acc[u].im[i] = fmaf(ar[k], v[2 + d][u].im[j], fmaf(ai[k], v[2 + d][u].re[j], acc[u].im[i]));
                }
            }
#pragma unroll
            for (int j = 0; j < 3; j++) {
                // (a x b)_j = a_{j+1} b_{j+2} - a_{j+2} b_{j+1}; row 2 entry = conj(.) / s
                const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
                const float xr = (ar[j1] * ar[3 + j2] - ai[j1] * ai[3 + j2]) - (ar[j2] * ar[3 + j1] - ai[j2] * ai[3 + j1]);
                const float xi = (ar[j1] * ai[3 + j2] + ai[j1] * ar[3 + j2]) - (ar[j2] * ai[3 + j1] + ai[j2] * ar[3 + j1]);
                const float wr = xr * isc, wi = -xi * isc;
#pragma unroll
                for (int u = 0; u < R; u++) {
                    acc[u].re[2] = fmaf(wr, v[2 + d][u].re[j], fmaf(-wi, v[2 + d][u].im[j], acc[u].re[2]));
                    acc[u].im[2] = fmaf(wr, v[2 + d][u].im[j], fmaf(wi, v[2 + d][u].re[j], acc[u].im[2]));
                }
            }
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&empty[it % stages]);
        if (mu == 3 && valid) {
#pragma unroll
            for (int u = 0; u < R; u++)
                if (on[u]) epi(cb, jj[u], acc[u], red[u]);
        }
    }
    // copies still in flight (only after a wait gave up) land before the CTA exits
    if (producer && !ok) {
        for (int j = max(0, issued - stages); j < issued; j++)
            for (int spin = 0; spin < (1 << 20) && !tc::mbar_try_wait(&full[j % stages], (j / stages) & 1); spin++) {
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
    int rc;  // k_dslash_mrhs: 0 with the L2 link prefetch, 1 without; k_dslash_mrhs_tma: blocks per SM
    int tma; // 1: the TMA-fed kernel (FP32 links with 12-real long links only)
    int x2;  // 1: the packed-pair kernel (R even)
};
constexpr int kTmaStages = 4;

constexpr int kMaxMrhsCandidates = 40;

// Candidates the autotuner times: the register kernel with R = 4, 3, 2 right-hand
// sides per thread, one or two site-group counts per block, with and without
// the link prefetch.  With `all` it also lists the packed-pair kernel and the
// TMA-fed kernel (12-real long links), which run only when a caller selects
// them: both measured slower on GB300 (packed FMAs save issue slots but take
// two FMA-pipe cycles each, and both hold fewer warps per SM at 128 registers).
static int mrhs_candidates(int kact, MrhsShape *out, bool tma_ok, bool all)
{
    int n = 0;
    for (int x2 : {0, 1})
        for (int pf : {0, 1})
            for (int R : {4, 3, 2}) {
                if (x2 && (R % 2 || !all)) continue;
                const int nch = (kact + R - 1) / R;
                if (nch > 16) continue;
                const int nsg0 = std::max(1, 8 / nch);
                for (int nsg : {nsg0, 2 * nsg0}) {
                    if (32 * nch * nsg > 512 || nsg > 8) continue; // batch_reduce holds 8 site groups
                    out[n].R = R;
                    out[n].tile.nch = nch;
                    out[n].tile.nsg = nsg;
                    out[n].rc = pf;
                    out[n].tma = 0;
                    out[n].x2 = x2;
                    n++;
                }
            }
    if (!all || !tma_ok) return n;
    for (int minb : {2, 3, 4})
        for (int R : {4, 3, 2}) {
            const int nch = (kact + R - 1) / R;
            if (32 * nch > 256 || n >= kMaxMrhsCandidates) continue;
            out[n].R = R;
            out[n].tile.nch = nch;
            out[n].tile.nsg = std::min(8, std::max(1, 256 / (32 * nch)));
            out[n].rc = minb;
            out[n].tma = 1;
            out[n].x2 = 0;
            n++;
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


template <int P, class S, class Epi>
static hisq_status run_mrhs_x2(hisq_ctx *ctx, int par, const BatchF<S> &in, const MrhsTile &tl, int pf, const Epi &epi,
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
        if (e != cudaSuccess) return cuda_err(ctx, e, "batched dslash (packed) launch");
        return HISQ_OK;
    };
    if (ctx->long_recon == 12) {
        const LinksF12 l12{ctx->links_f12[par], Vh};
        if (pf == 1) return launch(k_dslash_mrhs_x2<P, S, LinksFvB, LinksF12, true, Epi, false>, l12);
        return launch(k_dslash_mrhs_x2<P, S, LinksFvB, LinksF12, true, Epi, true>, l12);
    }
    if (ctx->long_recon == 8)
        return launch(k_dslash_mrhs_x2<P, S, LinksFvB, LinksF8, true, Epi, true>, LinksF8{ctx->links_f12[par], Vh});
    return launch(k_dslash_mrhs_x2<P, S, LinksFvB, LinksF12, false, Epi, true>, LinksF12{nullptr, Vh});
}

template <int R, class S, class Epi>
static hisq_status run_mrhs_r(hisq_ctx *ctx, int par, const BatchF<S> &in, const MrhsTile &tl, int rc, const Epi &epi,
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
    if (ctx->long_recon == 12) {
        const LinksF12 l12{ctx->links_f12[par], Vh};
        if (rc == 1) return launch(k_dslash_mrhs<R, S, LinksFvB, LinksF12, true, Epi, false>, l12);
        return launch(k_dslash_mrhs<R, S, LinksFvB, LinksF12, true, Epi>, l12);
    }
    if (ctx->long_recon == 8)
        return launch(k_dslash_mrhs<R, S, LinksFvB, LinksF8, true, Epi>, LinksF8{ctx->links_f12[par], Vh});
    return launch(k_dslash_mrhs<R, S, LinksFvB, LinksF12, false, Epi>, LinksF12{nullptr, Vh});
}

// dynamic shared memory of the TMA-fed kernel for a tile: the slot rings and
// two mbarriers per slot, per site group
static size_t tma_smem_bytes(const MrhsTile &tl)
{
    return size_t(tl.nsg) * kTmaStages * (kTmaStageBytes + 2 * sizeof(uint64_t));
}

template <int R, class S, class Epi>
static hisq_status run_mrhs_tma(hisq_ctx *ctx, int par, const BatchF<S> &in, const MrhsTile &tl, int minb,
                                const Epi &epi, BatchRed br)
{
    const int Vh = ctx->g.Vh;
    const int threads = 32 * tl.nch * tl.nsg;
    const size_t smem = tma_smem_bytes(tl);
    auto launch = [&](auto kern) -> hisq_status {
        static std::mutex mu;
        static std::map<std::pair<const void *, size_t>, int> bps_cache; // (kernel, smem) -> blocks per SM
        int bps = 1;
        {
            std::lock_guard<std::mutex> lock(mu);
            const auto key = std::make_pair(reinterpret_cast<const void *>(kern), smem * 1024 + size_t(threads));
            auto itc = bps_cache.find(key);
            if (itc == bps_cache.end()) {
                HISQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
                int n = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem) != cudaSuccess || n < 1) {
                    cudaGetLastError();
                    n = 1;
                }
                itc = bps_cache.emplace(key, n).first;
            }
            bps = itc->second;
        }
        const int grid = grid_for(ctx, long(Vh), 32 * tl.nsg, bps);
        kern<<<grid, threads, smem, ctx->stream>>>(ctx->g, par, ctx->links_f[par], ctx->links_f12[par],
                                                   float(ctx->long_scale), float(1.0 / ctx->long_scale), in,
                                                   ctx->bscal, tl, epi, br, kTmaStages, ctx->wait_status_d);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(ctx, e, "batched dslash (TMA) launch");
        return HISQ_OK;
    };
    if (minb == 3) return launch(k_dslash_mrhs_tma<R, S, Epi, 3>);
    if (minb == 4) return launch(k_dslash_mrhs_tma<R, S, Epi, 4>);
    return launch(k_dslash_mrhs_tma<R, S, Epi, 2>);
}

template <class S, class Epi>
static hisq_status run_shape(hisq_ctx *ctx, int par, const BatchF<S> &in, const MrhsShape &sh, const Epi &epi,
                             BatchRed br)
{
    if (sh.x2) {
        if (sh.R == 4) return run_mrhs_x2<2>(ctx, par, in, sh.tile, sh.rc, epi, br);
        return run_mrhs_x2<1>(ctx, par, in, sh.tile, sh.rc, epi, br);
    }
    if (sh.tma) {
        switch (sh.R) {
        case 2: return run_mrhs_tma<2>(ctx, par, in, sh.tile, sh.rc, epi, br);
        case 3: return run_mrhs_tma<3>(ctx, par, in, sh.tile, sh.rc, epi, br);
        default: return run_mrhs_tma<4>(ctx, par, in, sh.tile, sh.rc, epi, br);
        }
    }
    switch (sh.R) {
    case 2: return run_mrhs_r<2>(ctx, par, in, sh.tile, sh.rc, epi, br);
    case 3: return run_mrhs_r<3>(ctx, par, in, sh.tile, sh.rc, epi, br);
    default: return run_mrhs_r<4>(ctx, par, in, sh.tile, sh.rc, epi, br);
    }
}

// the shape for this batch: tuned on an idempotent launch (may_tune), else
// the one tuned before, else the default
static hisq_status mrhs_shape(hisq_ctx *ctx, int kact, int prec, MrhsShape *sh, bool may_tune,
                              const std::function<hisq_status(const MrhsShape &)> &launch)
{
    MrhsShape cand[kMaxMrhsCandidates];
    const bool forced = ctx->mrhs_force_kind != 0;
    const int n = mrhs_candidates(kact, cand, ctx->long_recon == 12, forced);
    int idx = 0;
    if (forced) {
        // a launch shape chosen by the caller (hisq_set_batched_kernel)
        for (int i = 0; i < n; i++)
            if (cand[i].tma == (ctx->mrhs_force_kind == 2) && cand[i].x2 == (ctx->mrhs_force_kind == 3) &&
                cand[i].R == ctx->mrhs_force_R && cand[i].rc == ctx->mrhs_force_budget) {
                *sh = cand[i];
                return HISQ_OK;
            }
        return set_err(ctx, HISQ_ERR_INVALID_ARG,
                       "batched operator: no launch shape of kind %d with %d right-hand sides per thread and budget %d "
                       "for %d right-hand sides and these links",
                       ctx->mrhs_force_kind, ctx->mrhs_force_R, ctx->mrhs_force_budget, kact);
    }
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
        BEpiCG<SpinorF, SpinorF> epi{batchf<SpinorF>(p, Vh, 32), batchf<SpinorF>(r, Vh, 32), batchf<SpinorF>(x, Vh, 32),
                                     ctx->bscal->alpha, &ctx->bscal->m4};
        return run_mrhs(ctx, 0, link_prec, 32, batchf<SpinorF>(tmp, Vh, 32), kact, epi, br, false);
    }
    case 16: {
        BEpiCG<SpinorH, SpinorF> epi{batchf<SpinorH>(p, Vh, 16), batchf<SpinorH>(r, Vh, 16), batchf<SpinorF>(x, Vh, 32),
                                     ctx->bscal->alpha, &ctx->bscal->m4};
        return run_mrhs(ctx, 0, link_prec, 16, batchf<SpinorH>(tmp, Vh, 16), kact, epi, br, false);
    }
    }
    return set_err(ctx, HISQ_ERR_INVALID_ARG, "batched sloppy precision must be 32 or 16");
}

// out_j = D in_j on output parity par for the k fields of a block (slots
// 0..k-1 active, mrhs_set_identity), FP32 or FP16 storage; |out_j|^2 -> out[j]
hisq_status launch_mrhs_dslash_store(hisq_ctx *ctx, int par, int prec, const void *in, void *out, int k)
{
    const int Vh = ctx->g.Vh;
    BatchRed br = batch_red(ctx, BFIN_STORE);
    switch (prec) {
    case 32:
        return run_mrhs(ctx, par, 32, 32, batchf<SpinorF>(const_cast<void *>(in), Vh, 32), k,
                        BEpiStore<SpinorF>{batchf<SpinorF>(out, Vh, 32)}, br, false);
    case 16:
        return run_mrhs(ctx, par, 32, 16, batchf<SpinorH>(const_cast<void *>(in), Vh, 16), k,
                        BEpiStore<SpinorH>{batchf<SpinorH>(out, Vh, 16)}, br, false);
    }
    return set_err(ctx, HISQ_ERR_INVALID_ARG, "batched operator: precision must be 32 or 16");
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

// The persistent batched CG (k_bcg_persistent) for the kact active slots: up
// to max_iters iterations, stopping after the first iteration in which a
// right-hand side's |r|^2 leaves [lo2_h[j], hi2_h[j]] (host arrays by RHS id)
// and two more.
// Synchronous: on return *n_done iterations have run, its_rhs[j] (host, by RHS
// id) counts those of right-hand side j, and the batch scalars (rr, pp, alpha,
// beta, iter) are those of each one's last iteration; phase_s (nullable)
// accumulates the seconds of the D_oe and D_eo phases.  HISQ_ERR_TIMEOUT if a
// grid barrier ran out.  The launch shape is the batch's tuned one.
hisq_status launch_bcg_persistent(hisq_ctx *ctx, int prec, int link_prec, void *p, void *tmp, void *r, void *x,
                                  int kact, int max_iters, const double *lo2_h, const double *hi2_h, int *n_done,
                                  int *its_rhs, double *phase_s)
{
    const int Vh = ctx->g.Vh;
    if (link_prec != 32 || (ctx->long_recon != 12 && ctx->long_recon != 18))
        return set_err(ctx, HISQ_ERR_INVALID_ARG, "persistent batched CG: FP32 links with 18- or 12-real long links");
    if (prec != 32 && prec != 16) return set_err(ctx, HISQ_ERR_INVALID_ARG, "persistent batched CG: sloppy 32 or 16");
    if (kact < 1 || kact > kMaxBatch || max_iters < 1) return set_err(ctx, HISQ_ERR_INVALID_ARG, "persistent batched CG");
    // the shape the autotuner picks for this batch (tuned on an ordinary D_oe
    // launch the first time, which leaves nothing the persistent kernel reads)
    if (!ctx->tuned.count(mrhs_key(ctx, kact, prec))) {
        hisq_status st = launch_mrhs_dslash_tt(ctx, prec, link_prec, p, tmp, kact);
        if (st != HISQ_OK) return st;
    }
    MrhsShape sh;
    hisq_status st = mrhs_shape(ctx, kact, prec, &sh, false, nullptr);
    if (st != HISQ_OK) return st;
    if (sh.tma || sh.x2) return set_err(ctx, HISQ_ERR_INVALID_ARG, "persistent batched CG: register-kernel shapes only");
    const MrhsTile tl = sh.tile;
    const int threads = 32 * tl.nch * tl.nsg;
    const bool r12 = ctx->long_recon == 12;
    const LinksFvB Lo{ctx->links_f[1], Vh, r12 ? 1 : 2}, Le{ctx->links_f[0], Vh, r12 ? 1 : 2};
    const LinksF12 L12o{r12 ? ctx->links_f12[1] : nullptr, Vh}, L12e{r12 ? ctx->links_f12[0] : nullptr, Vh};
    const float c3 = float(ctx->long_scale);

    auto go = [&](auto kern, auto tagS) -> hisq_status {
        typedef decltype(tagS) S;
        int bps = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, threads, 0) != cudaSuccess || bps < 1) {
            cudaGetLastError();
            return set_err(ctx, HISQ_ERR_CUDA, "persistent batched CG: occupancy query");
        }
        const int grid = grid_for(ctx, long(Vh), 32 * tl.nsg, bps); // every block resident
        const size_t part_bytes = sizeof(double) * size_t(grid) * 3 * kMaxBatch;
        char *buf = (char *)get_buf(ctx, BUF_PERSIST,
                                    part_bytes + sizeof(double) * 2 * kMaxBatch + 64 + sizeof(int) * kMaxBatch);
        if (!buf) return HISQ_ERR_OOM;
        double *lo2 = (double *)(buf + part_bytes), *hi2 = lo2 + kMaxBatch;
        unsigned long long *ns = (unsigned long long *)(hi2 + kMaxBatch);
        int *done = (int *)(ns + 2);
        int *its_d = done + 2;
        HISQ_CUDA(cudaMemcpyAsync(lo2, lo2_h, sizeof(double) * kMaxBatch, cudaMemcpyHostToDevice, ctx->stream));
        HISQ_CUDA(cudaMemcpyAsync(hi2, hi2_h, sizeof(double) * kMaxBatch, cudaMemcpyHostToDevice, ctx->stream));
        HISQ_CUDA(cudaMemsetAsync(ns, 0, 2 * sizeof(unsigned long long), ctx->stream));
        // failure injection (tests): a zero wait limit, so every block that waits
        // at the first barrier gives up
        const bool inject = ctx->inject_wait_timeout;
        ctx->inject_wait_timeout = false;
        PersistArgs pa{(double *)buf, ctx->ticket + 48, ctx->wait_status_d, lo2, hi2, max_iters, ctx->bmonitor_d,
                       ctx->bmonitor_len, phase_s ? ns : nullptr, done, its_d, inject ? 0ull : kGridWaitNs};
        BatchF<S> P = batchf<S>(p, Vh, prec), T = batchf<S>(tmp, Vh, prec), Rr = batchf<S>(r, Vh, prec);
        BatchF<SpinorF> X = batchf<SpinorF>(x, Vh, 32);
        Geom g = ctx->g;
        float c3v = c3;
        BatchScalars *scal = ctx->bscal;
        MrhsTile tlv = tl;
        LinksFvB lo = Lo, le = Le;
        LinksF12 l12o = L12o, l12e = L12e;
        void *args[] = {&g, &lo, &le, &l12o, &l12e, &c3v, &P, &T, &Rr, &X, &scal, &tlv, &pa};
        cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(kern), dim3(grid), dim3(threads),
                                                    args, 0, ctx->stream);
        if (e != cudaSuccess) return cuda_err(ctx, e, "persistent batched CG launch");
        unsigned long long hns[2] = {0, 0};
        int hdone = 0;
        HISQ_CUDA(cudaMemcpyAsync(&hdone, done, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        HISQ_CUDA(cudaMemcpyAsync(hns, ns, sizeof hns, cudaMemcpyDeviceToHost, ctx->stream));
        HISQ_CUDA(cudaMemcpyAsync(its_rhs, its_d, sizeof(int) * kMaxBatch, cudaMemcpyDeviceToHost, ctx->stream));
        HISQ_CUDA(cudaStreamSynchronize(ctx->stream));
        if (*(volatile int *)ctx->wait_status_h != 0) {
            const int code = *ctx->wait_status_h;
            *ctx->wait_status_h = 0;
            return set_err(ctx, HISQ_ERR_TIMEOUT, "persistent batched CG: a grid barrier ran out (code %d)", code);
        }
        *n_done = hdone;
        if (phase_s) {
            phase_s[0] += double(hns[0]) * 1e-9;
            phase_s[1] += double(hns[1]) * 1e-9;
        }
        return HISQ_OK;
    };
    auto by_r = [&](auto tagS) -> hisq_status {
        typedef decltype(tagS) S;
        if (r12) {
            switch (sh.R) {
            case 2: return go(k_bcg_persistent<2, S, SpinorF, LinksF12, true>, S{});
            case 3: return go(k_bcg_persistent<3, S, SpinorF, LinksF12, true>, S{});
            default: return go(k_bcg_persistent<4, S, SpinorF, LinksF12, true>, S{});
            }
        }
        switch (sh.R) {
        case 2: return go(k_bcg_persistent<2, S, SpinorF, LinksF12, false>, S{});
        case 3: return go(k_bcg_persistent<3, S, SpinorF, LinksF12, false>, S{});
        default: return go(k_bcg_persistent<4, S, SpinorF, LinksF12, false>, S{});
        }
    };
    return prec == 16 ? by_r(SpinorH{}) : by_r(SpinorF{});
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
