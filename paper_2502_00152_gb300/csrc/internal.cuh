// internal.cuh -- shared device types of the HISQ library: complex colour
// vectors and matrices, lattice geometry on one parity, storage formats of
// colour vectors and of the gathered link fields, and the deterministic
// grid-wide reduction used by every norm and inner product.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/hisq.h"

namespace hisq {

// ------------------------------------------------------------------ complex
template <typename T>
struct Cplx {
    T re, im;
};

template <typename T>
__host__ __device__ __forceinline__ Cplx<T> cmul(Cplx<T> a, Cplx<T> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

// colour vector: 3 complex numbers
template <typename T>
struct CVec {
    T re[3], im[3];
    __host__ __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int i = 0; i < 3; i++) re[i] = im[i] = T(0);
    }
    __host__ __device__ __forceinline__ T norm2() const
    {
        T s = 0;
#pragma unroll
        for (int i = 0; i < 3; i++) s += re[i] * re[i] + im[i] * im[i];
        return s;
    }
};

// colour matrix, row major
template <typename T>
struct CMat {
    T re[9], im[9];
};

// acc += W v
template <typename T>
__device__ __forceinline__ void mv_acc(CVec<T> &acc, const CMat<T> &W, const CVec<T> &v)
{
#pragma unroll
    for (int i = 0; i < 3; i++) {
#pragma unroll
        for (int j = 0; j < 3; j++) {
            acc.re[i] = fma(W.re[3 * i + j], v.re[j], acc.re[i]);
            acc.re[i] = fma(-W.im[3 * i + j], v.im[j], acc.re[i]);
            acc.im[i] = fma(W.re[3 * i + j], v.im[j], acc.im[i]);
            acc.im[i] = fma(W.im[3 * i + j], v.re[j], acc.im[i]);
        }
    }
}

// acc += s * (W v), s real
template <typename T>
__device__ __forceinline__ void mv_acc_scaled(CVec<T> &acc, T s, const CMat<T> &W, const CVec<T> &v)
{
    CVec<T> t;
    t.zero();
    mv_acc(t, W, v);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        acc.re[i] = fma(s, t.re[i], acc.re[i]);
        acc.im[i] = fma(s, t.im[i], acc.im[i]);
    }
}

// third row of an SU(3) matrix from the first two: row2 = conj(row0 x row1)
template <typename T>
__device__ __forceinline__ void su3_third_row(CMat<T> &W)
{
    // (a x b)_k = a_{k+1} b_{k+2} - a_{k+2} b_{k+1}
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        T are1 = W.re[k1], aim1 = W.im[k1], are2 = W.re[k2], aim2 = W.im[k2];
        T bre1 = W.re[3 + k1], bim1 = W.im[3 + k1], bre2 = W.re[3 + k2], bim2 = W.im[3 + k2];
        T cre = (are1 * bre2 - aim1 * bim2) - (are2 * bre1 - aim2 * bim1);
        T cim = (are1 * bim2 + aim1 * bre2) - (are2 * bim1 + aim2 * bre1);
        W.re[6 + k] = cre;
        W.im[6 + k] = -cim;
    }
}

// ---------------------------------------------------------------- geometry
// Exact division of n < 2^31 by a constant d < 2^16 as a multiply and a
// shift: with 2^s >= d and M = floor(2^(32+s) / d) + 1, floor(n M / 2^(32+s))
// = floor(n / d), because the excess n (M - 2^(32+s)/d) / 2^(32+s) < 1/(2d)
// never carries past the next multiple of 1/d (Granlund & Montgomery, PLDI 1994).
struct FastDiv {
    unsigned long long M;
    int shift; // 32 + s
    int d;
};
inline FastDiv make_fastdiv(int d)
{
    int s = 0;
    while ((1 << s) < d) s++;
    return FastDiv{((1ull << (32 + s)) / unsigned(d)) + 1ull, 32 + s, d};
}
__host__ __device__ __forceinline__ int fdiv(int n, const FastDiv &f)
{
    return int((unsigned long long)unsigned(n) * f.M >> f.shift);
}

struct Geom {
    int X, Y, Z, T;
    int X2;          // X / 2
    int Vh;          // sites of one parity
    int V;
    int t_antiperiodic;
    int stride[4];   // 1, X, XY, XYZ (full-lattice site index)
    int *oob;        // device flag set by out-of-range indices (HISQ_BOUNDS_CHECK builds)
    FastDiv dX2, dY, dZ; // division by X/2, Y and Z (site coordinates)
};

// Index check of the bounds-checking build (-DHISQ_BOUNDS_CHECK): an index
// outside [0, n) sets the context's flag and is replaced by 0, so the access
// stays inside the array; the normal build compiles to the index itself.
#ifdef HISQ_BOUNDS_CHECK
__device__ __forceinline__ int checked_index(const Geom &g, int i, int n)
{
    if (i < 0 || i >= n) {
        if (g.oob) atomicOr(g.oob, 1);
        return 0;
    }
    return i;
}
#else
__device__ __forceinline__ int checked_index(const Geom &, int i, int) { return i; }
#endif

// coordinates of checkerboard site cb of parity `par` (cb = s >> 1)
__device__ __forceinline__ void cb_coords(const Geom &g, int par, int cb, int c[4])
{
    int r = fdiv(cb, g.dX2);
    const int xh = cb - r * g.X2;
    int q = fdiv(r, g.dY);
    c[1] = r - q * g.Y;
    r = q;
    q = fdiv(r, g.dZ);
    c[2] = r - q * g.Z;
    c[3] = q;
    c[0] = 2 * xh + ((par + c[1] + c[2] + c[3]) & 1);
}

__device__ __forceinline__ int dim_of(const Geom &g, int mu)
{
    return mu == 0 ? g.X : (mu == 1 ? g.Y : (mu == 2 ? g.Z : g.T));
}

// checkerboard index of the site c + d * mu_hat (periodic wrap); |d| <= 3 < L
// (selects instead of indexing by a loop variable keep c[] in registers)
__device__ __forceinline__ int coord_of(const int c[4], int mu)
{
    return mu == 0 ? c[0] : (mu == 1 ? c[1] : (mu == 2 ? c[2] : c[3]));
}

__device__ __forceinline__ int stride_of(const Geom &g, int mu)
{
    return mu == 0 ? 1 : (mu == 1 ? g.X : (mu == 2 ? g.X * g.Y : g.X * g.Y * g.Z));
}

__device__ __forceinline__ int nb_cb(const Geom &g, const int c[4], int s, int mu, int d)
{
    const int L = dim_of(g, mu);
    const int cm = coord_of(c, mu);
    int cn = cm + d;
    cn += (cn < 0) ? L : 0;
    cn -= (cn >= L) ? L : 0;
    return checked_index(g, (s + (cn - cm) * stride_of(g, mu)) >> 1, g.Vh);
}

__device__ __forceinline__ int full_site(const Geom &g, const int c[4])
{
    return c[0] + g.X * (c[1] + g.Y * (c[2] + g.Z * c[3]));
}

// staggered phase eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1})
__device__ __forceinline__ float stag_phase(int mu, const int c[4])
{
    int e = 0;
    if (mu > 0) e += c[0];
    if (mu > 1) e += c[1];
    if (mu > 2) e += c[2];
    return (e & 1) ? -1.f : 1.f;
}

// ----------------------------------------------------- colour-vector storage
// One parity of a colour field, Vh sites.
//  FP64: [3][Vh] double2                       48 B / site
//  FP32: [Vh] float4 (colours 0,1) then [Vh] float2 (colour 2)   24 B / site
//  FP16: [Vh] uint4 = 6 halves (re,im x 3) + FP32 scale          16 B / site
//  BF16: [3][Vh] bf16x2 (re,im), eigenvector storage only         12 B / site
//  FP16 x 2^e: [3][Vh] half2 (re,im), eigenvector storage only     12 B / site
//  DF64: [3][Vh] float4 (re hi, re lo, im hi, im lo), residuals only 48 B / site
inline size_t spinor_bytes(int prec, int Vh)
{
    return (prec == 64 || prec == HISQ_PREC_DF64) ? size_t(Vh) * 48
                      : (prec == 32 ? size_t(Vh) * 24
                                    : ((prec == HISQ_PREC_BF16 || prec == HISQ_PREC_HALF_EV) ? size_t(Vh) * 12
                                                                                            : size_t(Vh) * 16));
}

struct SpinorD {
    double2 *p;
    int Vh;
    typedef double real;
    __device__ __forceinline__ CVec<double> load(int i) const
    {
        CVec<double> v;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            double2 a = p[size_t(c) * Vh + i];
            v.re[c] = a.x;
            v.im[c] = a.y;
        }
        return v;
    }
    __device__ __forceinline__ void store(int i, const CVec<double> &v) const
    {
#pragma unroll
        for (int c = 0; c < 3; c++) p[size_t(c) * Vh + i] = make_double2(v.re[c], v.im[c]);
    }
};

struct SpinorF {
    float4 *a;
    float2 *b;
    int Vh;
    typedef float real;
    __device__ __forceinline__ CVec<float> load(int i) const
    {
        float4 u = a[i];
        float2 w = b[i];
        CVec<float> v;
        v.re[0] = u.x;
        v.im[0] = u.y;
        v.re[1] = u.z;
        v.im[1] = u.w;
        v.re[2] = w.x;
        v.im[2] = w.y;
        return v;
    }
    __device__ __forceinline__ void store(int i, const CVec<float> &v) const
    {
        a[i] = make_float4(v.re[0], v.im[0], v.re[1], v.im[1]);
        b[i] = make_float2(v.re[2], v.im[2]);
    }
};

struct SpinorH {
    uint4 *p;
    int Vh;
    typedef float real;
    __device__ __forceinline__ CVec<float> load(int i) const
    {
        uint4 u = p[i];
        const float s = __uint_as_float(u.w);
        __half2 h0 = *reinterpret_cast<__half2 *>(&u.x);
        __half2 h1 = *reinterpret_cast<__half2 *>(&u.y);
        __half2 h2 = *reinterpret_cast<__half2 *>(&u.z);
        float2 f0 = __half22float2(h0), f1 = __half22float2(h1), f2 = __half22float2(h2);
        CVec<float> v;
        v.re[0] = f0.x * s;
        v.im[0] = f0.y * s;
        v.re[1] = f1.x * s;
        v.im[1] = f1.y * s;
        v.re[2] = f2.x * s;
        v.im[2] = f2.y * s;
        return v;
    }
    __device__ __forceinline__ void store(int i, const CVec<float> &v) const
    {
        float m = 0.f;
#pragma unroll
        for (int c = 0; c < 3; c++) m = fmaxf(m, fmaxf(fabsf(v.re[c]), fabsf(v.im[c])));
        const float inv = m > 0.f ? 1.0f / m : 0.f;
        __half2 h0 = __floats2half2_rn(v.re[0] * inv, v.im[0] * inv);
        __half2 h1 = __floats2half2_rn(v.re[1] * inv, v.im[1] * inv);
        __half2 h2 = __floats2half2_rn(v.re[2] * inv, v.im[2] * inv);
        uint4 u;
        u.x = *reinterpret_cast<unsigned *>(&h0);
        u.y = *reinterpret_cast<unsigned *>(&h1);
        u.z = *reinterpret_cast<unsigned *>(&h2);
        u.w = __float_as_uint(m);
        p[i] = u;
    }
};

inline SpinorD make_spinorD(void *p, int Vh) { return SpinorD{(double2 *)p, Vh}; }
inline SpinorF make_spinorF(void *p, int Vh) { return SpinorF{(float4 *)p, (float2 *)((char *)p + size_t(Vh) * 16), Vh}; }
inline SpinorH make_spinorH(void *p, int Vh) { return SpinorH{(uint4 *)p, Vh}; }

// BF16 values, colour-major like FP64: the vector-major operand layout of the
// tensor-core deflation GEMM (K index = (colour * Vh + cb) * 2 + re/im)
struct SpinorB {
    __nv_bfloat162 *p;
    int Vh;
    typedef float real;
    __device__ __forceinline__ CVec<float> load(int i) const
    {
        CVec<float> v;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float2 f = __bfloat1622float2(p[size_t(c) * Vh + i]);
            v.re[c] = f.x;
            v.im[c] = f.y;
        }
        return v;
    }
    __device__ __forceinline__ void store(int i, const CVec<float> &v) const
    {
#pragma unroll
        for (int c = 0; c < 3; c++) p[size_t(c) * Vh + i] = __floats2bfloat162_rn(v.re[c], v.im[c]);
    }
};
inline SpinorB make_spinorB(void *p, int Vh) { return SpinorB{(__nv_bfloat162 *)p, Vh}; }

// FP16 eigenvector storage (HISQ_PREC_HALF_EV): FP16 values of v * 2^e,
// colour-major like BF16 (12 B per site), with one power-of-two scale 2^e for
// every site and vector, the smallest with 4^e >= 3 Vh.  A unit vector's
// entries (|v| <= 1) then stay below 2 sqrt(3 Vh), inside the FP16 range for
// every Vh below 3.5e8, and are O(1) on average; the scaling is exact, so the
// stored value is the FP16 rounding of the FP32 value times 2^e.  The layout is
// the tensor-core deflation operand as it is.
__host__ __device__ __forceinline__ int ev_half_exponent(int Vh)
{
    const unsigned N = 3u * unsigned(Vh); // >= 3
#ifdef __CUDA_ARCH__
    const int lg = 32 - __clz(int(N - 1u)); // ceil(log2 N)
#else
    const int lg = 32 - __builtin_clz(N - 1u);
#endif
    return (lg + 1) / 2;
}
__host__ __device__ __forceinline__ float pow2f(int e)
{
    // 2^e for -126 <= e <= 127, exact
    union {
        unsigned u;
        float f;
    } b;
    b.u = unsigned(127 + e) << 23;
    return b.f;
}

struct SpinorE {
    __half2 *p;
    int Vh;
    float s, inv; // 2^e and 2^-e
    typedef float real;
    __device__ __forceinline__ CVec<float> load(int i) const
    {
        CVec<float> v;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float2 f = __half22float2(p[size_t(c) * Vh + i]);
            v.re[c] = f.x * inv;
            v.im[c] = f.y * inv;
        }
        return v;
    }
    __device__ __forceinline__ void store(int i, const CVec<float> &v) const
    {
#pragma unroll
        for (int c = 0; c < 3; c++) p[size_t(c) * Vh + i] = __floats2half2_rn(v.re[c] * s, v.im[c] * s);
    }
};
__host__ __device__ inline SpinorE make_spinorE(void *p, int Vh)
{
    const int e = ev_half_exponent(Vh);
    return SpinorE{(__half2 *)p, Vh, pow2f(e), pow2f(-e)};
}

// accessor of the same storage type as S for another field
template <class S>
inline S make_like(void *p, int Vh);
template <>
inline SpinorD make_like<SpinorD>(void *p, int Vh) { return make_spinorD(p, Vh); }
template <>
inline SpinorF make_like<SpinorF>(void *p, int Vh) { return make_spinorF(p, Vh); }
template <>
inline SpinorH make_like<SpinorH>(void *p, int Vh) { return make_spinorH(p, Vh); }
template <>
inline SpinorB make_like<SpinorB>(void *p, int Vh) { return make_spinorB(p, Vh); }
template <>
inline SpinorE make_like<SpinorE>(void *p, int Vh) { return make_spinorE(p, Vh); }

// convert between accumulation types
template <typename To, typename From>
__device__ __forceinline__ CVec<To> cvt(const CVec<From> &v)
{
    CVec<To> o;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        o.re[c] = To(v.re[c]);
        o.im[c] = To(v.im[c]);
    }
    return o;
}

// ------------------------------------------------------- gathered links
// For every output parity p and output site cb the 16 hop matrices W_h are
// stored with the staggered phase, the boundary sign, the minus sign of the
// backward hops and the adjoint of the backward links folded in, so that
//   (D psi)(x) = sum_mu sum_{kind} [ W_fwd psi(x + n mu) + W_bwd psi(x - n mu) ]
// (kind 0: fat, n = 1; kind 1: long, n = 3).
//
// FP64 (recon 18): double2 [p][mu][kind][fwd,bwd][k=0..8][Vh]
// FP32 (recon 18): float4  [p][mu][kind][k=0..8][Vh], float4 = (fwd_k, bwd_k)
// FP32 long links with recon 12: float4 [p][mu][k=0..5][Vh] holding rows 0,1
//   of the SU(3) factor S of fwd and bwd; W = sign * long_scale * S, with
//   sign = +-eta_mu(x) * (boundary sign) recomputed from the coordinates.
// FP32 long links with recon 8: float4 [p][mu][q=0..3][Vh]: q = 0, 1 for fwd,
//   2, 3 for bwd, each pair (a2, a3) and (b1, arg a1, arg c1) of the SU(3)
//   factor (a = row 0, b = row 1, c = row 2); the rest follows from unitarity.
// FP16 (recon 18): uint2 [p][mu][kind][k=0..8][Vh], uint2 = (fwd_k, bwd_k) as
//   two half2; FP16 long links with recon 12: uint2 [p][mu][k=0..5][Vh].
struct LinksD {
    const double2 *base; // parity offset applied
    int Vh;
    typedef double real;
    __device__ __forceinline__ void load(int mu, int kind, int i, CMat<double> &f, CMat<double> &b) const
    {
        const double2 *q = base + size_t((mu * 2 + kind) * 2) * 9 * Vh + i;
#pragma unroll
        for (int k = 0; k < 9; k++) {
            double2 a = __ldcs(q + size_t(k) * Vh);
            double2 c = __ldcs(q + size_t(9 + k) * Vh);
            f.re[k] = a.x;
            f.im[k] = a.y;
            b.re[k] = c.x;
            b.im[k] = c.y;
        }
    }
};

struct LinksF {
    const float4 *base; // parity offset applied
    int Vh;
    typedef float real;
    __device__ __forceinline__ void load(int mu, int kind, int i, CMat<float> &f, CMat<float> &b) const
    {
        const float4 *q = base + size_t((mu * 2 + kind) * 9) * Vh + i;
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

struct LinksF12 { // long links only
    const float4 *base; // parity offset applied
    int Vh;
    __device__ __forceinline__ void load(int mu, int i, CMat<float> &f, CMat<float> &b) const
    {
        const float4 *q = base + size_t(mu * 6) * Vh + i;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            float4 a = __ldcs(q + size_t(k) * Vh);
            f.re[k] = a.x;
            f.im[k] = a.y;
            b.re[k] = a.z;
            b.im[k] = a.w;
        }
        su3_third_row(f);
        su3_third_row(b);
    }
};

// SU(3) matrix from 8 reals: row 0 = (a1, a2, a3), column 0 = (a1, b1, c1)
// with |a1|, |c1| from the unit norms of row 0 and column 0 and the phases of
// a1, c1 stored; the four remaining entries follow from U = conj(cofactors)
// (c = conj(a x b), b = conj(c x a)) solved for b2, b3, c2, c3, each over
// N = |a2|^2 + |a3|^2 = 1 - |a1|^2.
__device__ __forceinline__ void su3_from8(const float4 p0, const float4 p1, CMat<float> &W)
{
    const float a2r = p0.x, a2i = p0.y, a3r = p0.z, a3i = p0.w, b1r = p1.x, b1i = p1.y;
    const float N = a2r * a2r + a2i * a2i + a3r * a3r + a3i * a3i;
    const float ma1 = sqrtf(fmaxf(0.f, 1.f - N));
    const float mc1 = sqrtf(fmaxf(0.f, N - (b1r * b1r + b1i * b1i)));
    float sa, ca, sc, cc;
    sincosf(p1.z, &sa, &ca);
    sincosf(p1.w, &sc, &cc);
    const float a1r = ma1 * ca, a1i = ma1 * sa, c1r = mc1 * cc, c1i = mc1 * sc;
    const float iN = 1.f / N;
    // complex helpers on (re, im) pairs
    auto mul = [](float xr, float xi, float yr, float yi, float &zr, float &zi) {
        zr = xr * yr - xi * yi;
        zi = xr * yi + xi * yr;
    };
    float tr, ti, ur, ui;
    // b2 = -(conj(a1) a2 b1 + conj(a3) conj(c1)) / N
    mul(a1r, -a1i, a2r, a2i, tr, ti);
    mul(tr, ti, b1r, b1i, tr, ti);
    mul(a3r, -a3i, c1r, -c1i, ur, ui);
    const float b2r = -(tr + ur) * iN, b2i = -(ti + ui) * iN;
    // b3 = (conj(a2) conj(c1) - conj(a1) a3 b1) / N
    mul(a2r, -a2i, c1r, -c1i, ur, ui);
    mul(a1r, -a1i, a3r, a3i, tr, ti);
    mul(tr, ti, b1r, b1i, tr, ti);
    const float b3r = (ur - tr) * iN, b3i = (ui - ti) * iN;
    // c2 = (conj(a3) conj(b1) - conj(a1) a2 c1) / N
    mul(a3r, -a3i, b1r, -b1i, ur, ui);
    mul(a1r, -a1i, a2r, a2i, tr, ti);
    mul(tr, ti, c1r, c1i, tr, ti);
    const float c2r = (ur - tr) * iN, c2i = (ui - ti) * iN;
    // c3 = -(conj(a1) a3 c1 + conj(a2) conj(b1)) / N
    mul(a1r, -a1i, a3r, a3i, tr, ti);
    mul(tr, ti, c1r, c1i, tr, ti);
    mul(a2r, -a2i, b1r, -b1i, ur, ui);
    const float c3r = -(tr + ur) * iN, c3i = -(ti + ui) * iN;
    W.re[0] = a1r; W.im[0] = a1i; W.re[1] = a2r; W.im[1] = a2i; W.re[2] = a3r; W.im[2] = a3i;
    W.re[3] = b1r; W.im[3] = b1i; W.re[4] = b2r; W.im[4] = b2i; W.re[5] = b3r; W.im[5] = b3i;
    W.re[6] = c1r; W.im[6] = c1i; W.re[7] = c2r; W.im[7] = c2i; W.re[8] = c3r; W.im[8] = c3i;
}

struct LinksF8 { // long links only, 8 reals per SU(3) factor
    const float4 *base; // parity offset applied
    int Vh;
    __device__ __forceinline__ void load(int mu, int i, CMat<float> &f, CMat<float> &b) const
    {
        const float4 *q = base + size_t(mu * 4) * Vh + i;
        const float4 f0 = __ldcs(q), f1 = __ldcs(q + Vh), b0 = __ldcs(q + 2 * size_t(Vh)), b1 = __ldcs(q + 3 * size_t(Vh));
        su3_from8(f0, f1, f);
        su3_from8(b0, b1, b);
    }
};

// floats of compressed FP32 long links per output site and parity (0: none)
inline size_t long_f32_bytes_per_site(int recon) { return recon == 12 ? 4 * 6 * 16 : (recon == 8 ? 4 * 4 * 16 : 0); }

// ------------------------------------------------------ device scalars
// Scalars of the CG recurrences live on the device so that consecutive kernels
// of one iteration never wait for the host.
struct DevScalars {
    double rr;      // |r|^2 of the current iterate
    double rr_new;  // |r|^2 after the update
    double pp;      // |p|^2
    double tt;      // |D_oe p|^2
    double alpha, beta;
    double m4;      // 4 m^2
    double pad0;
    long long iter; // iterations done
    long long pad1;
    double slot[16]; // generic reduction results
};

enum FinishOp : int {
    FIN_STORE = 0,    // slot[i] = total_i
    FIN_CG_ALPHA = 1, // tt = total_0; alpha = rr / (m4 pp + tt)
    FIN_CG_BETA = 2,  // rr_new = total_0; beta = rr_new / rr; monitor[iter] = rr_new
    FIN_CG_P = 3      // pp = total_0; rr = rr_new; iter += 1
};

constexpr int kMaxRedVals = 8;

// ------------------------------------------------- multi right-hand sides
constexpr int kMaxBatch = 64;

// per right-hand-side CG scalars of a batched solve (indexed by RHS id)
struct BatchScalars {
    double rr[kMaxBatch], rr_new[kMaxBatch], pp[kMaxBatch], tt[kMaxBatch];
    double alpha[kMaxBatch], beta[kMaxBatch], out[kMaxBatch];
    double m4;
    long long iter;
    int kact;             // active right-hand sides
    int idx[kMaxBatch];   // slot -> RHS id
};

enum BatchFinishOp : int {
    BFIN_STORE = 0, // out[j] = total
    BFIN_ALPHA = 1, // tt[j] = total; alpha[j] = rr[j] / (m4 pp[j] + tt[j])
    BFIN_BETA = 2,  // rr_new[j] = total; beta[j] = rr_new[j] / rr[j]; monitor
    BFIN_P = 3      // pp[j] = total; rr[j] = rr_new[j]; iter += 1
};

struct BatchRed {
    double *partials;     // >= gridDim.x * kMaxBatch
    unsigned int *ticket;
    BatchScalars *scal;
    double *monitor;      // host-mapped [monitor_len][kMaxBatch]
    int monitor_len;
    int op;
};
constexpr int kRedThreads = 256;

struct RedArgs {
    double *partials;       // >= gridDim.x * nvals doubles
    unsigned int *ticket;   // zero between uses
    DevScalars *scal;
    double *monitor;        // host-mapped residual history (FIN_CG_BETA)
    int monitor_len;
    int op;
    int slot0;              // first slot for FIN_STORE
};

// Deterministic grid reduction of NV doubles: each block writes its partial
// sums, the last block to finish adds the partials in block order.
template <int NV>
__device__ __forceinline__ void grid_reduce(double (&v)[NV], const RedArgs &ra)
{
    __shared__ double sh[NV][32];
    __shared__ bool am_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; j++) {
        double x = v[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[j][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; j++) {
            double s = 0;
            for (int w = 0; w < nwarps; w++) s += sh[j][w];
            ra.partials[size_t(blockIdx.x) * NV + j] = s;
        }
        __threadfence();
        unsigned int t = atomicAdd(ra.ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double tot[NV];
#pragma unroll
    for (int j = 0; j < NV; j++) {
        double s = 0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
            s += ((volatile double *)ra.partials)[size_t(b) * NV + j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[j][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; j++) {
            double s = 0;
            for (int w = 0; w < nwarps; w++) s += sh[j][w];
            tot[j] = s;
        }
        DevScalars *S = ra.scal;
        switch (ra.op) {
        case FIN_STORE:
#pragma unroll
            for (int j = 0; j < NV; j++) S->slot[ra.slot0 + j] = tot[j];
            break;
        case FIN_CG_ALPHA:
            S->tt = tot[0];
            S->alpha = S->rr / (S->m4 * S->pp + tot[0]);
            break;
        case FIN_CG_BETA:
            S->rr_new = tot[0];
            S->beta = tot[0] / S->rr;
            if (ra.monitor) ra.monitor[S->iter % ra.monitor_len] = tot[0];
            break;
        case FIN_CG_P:
            S->pp = tot[0];
            S->rr = S->rr_new;
            S->iter += 1;
            break;
        }
        *ra.ticket = 0u;
        __threadfence();
    }
}

// ---------------------------------------------------------------- context
// persistent scratch buffers of a context, grown on demand
enum BufId : int {
    BUF_DEFL_PART = 0, // deflation projection partial sums
    BUF_DEFL_C,        // deflation coefficients (complex FP64)
    BUF_ETA_FULL,      // full-lattice FP64 source (host API)
    BUF_PSI_FULL,      // full-lattice FP64 solution (host API)
    BUF_ETA_E,
    BUF_ETA_O,
    BUF_Y,             // even-site right-hand side y_e
    BUF_XHI,           // FP64 solution accumulator
    BUF_RHI,           // FP64 true residual
    BUF_TMPHI,         // FP64 odd temporary
    BUF_PSI_O,
    BUF_XSL,           // sloppy solution increment
    BUF_RSL,
    BUF_P,
    BUF_TMP,           // sloppy odd temporary
    BUF_TEST_A,
    BUF_TEST_B,
    BUF_TEST_C,
    BUF_EIG_Y,         // Ritz rotation matrix (FP64)
    BUF_EIG_W,         // eigensolver work vectors
    BUF_B_Y,           // batched solve: k FP64 right-hand sides y_e
    BUF_B_XHI,
    BUF_B_RHI,
    BUF_B_XSL,
    BUF_B_RSL,
    BUF_B_P,
    BUF_B_TMP,
    BUF_B_DX,          // batched solve: deflation increments (FP64, 16-bit eigenvectors)
    BUF_B_F32,         // batched solve: three FP32 temporaries for A dx
    BUF_TC_WORK,       // tensor-core deflation: R' operands, scales, status
    BUF_TC_PART,       // projection partial tiles per K split
    BUF_TC_C,          // projected coefficients (FP64)
    BUF_TC_D,          // expansion operands
    BUF_NET_PART,      // network weight-gradient partial sums
    BUF_GUESS,         // even part of a caller's initial guess
    BUF_DF_X,          // double-float residual: x split into (hi, lo)
    BUF_DF_T,          // double-float residual: odd temporary D_oe x
    BUF_PERSIST,       // persistent batched CG: per-block partials, thresholds
    BUF_COUNT
};

struct EigenStore {
    int n = 0;            // stored eigenpairs
    int prec = 32;        // storage precision (32, 16, HISQ_PREC_BF16 or HISQ_PREC_HALF_EV)
    void *vecs = nullptr; // n vectors of spinor_bytes(prec, Vh)
    std::vector<double> eps; // massless eigenvalues, ascending
    double *eps_dev = nullptr; // device copy of eps, written when the pairs are stored
    unsigned version = 0;    // bumped whenever the stored pairs change
};

} // namespace hisq

struct hisq_ctx {
    hisq::Geom g;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    std::string err;
    double mass = -1;
    bool links_loaded = false;
    bool profile = false;
    mutable unsigned long long launches = 0; // kernels launched by this context
    double last_window[2] = {0, 0}; // Chebyshev window of the last eigensolve
    int long_recon = 18;
    double long_scale = 1.0;

    // gathered links; index [parity]
    double2 *links_d[2] = {nullptr, nullptr};  // FP64, 16 hops
    float4 *links_f[2] = {nullptr, nullptr};   // FP32: fat (+ long when recon 18)
    float4 *links_f12[2] = {nullptr, nullptr}; // FP32 long, recon 12
    uint2 *links_h[2] = {nullptr, nullptr};    // FP16: fat (+ long when recon 18)
    uint2 *links_h12[2] = {nullptr, nullptr};  // FP16 long, recon 12
    float4 *links_df[2] = {nullptr, nullptr};  // double-float split of links_d (built on first use)

    // reduction scratch
    double *partials = nullptr;
    unsigned int *ticket = nullptr;
    hisq::DevScalars *scal = nullptr;
    double *monitor_h = nullptr; // host-mapped
    double *monitor_d = nullptr;
    int monitor_len = 1 << 16;
    int max_red_blocks = 0;

    hisq::EigenStore eig;

    // batched solves
    hisq::BatchScalars *bscal = nullptr;
    double *bpartials = nullptr;
    double *bmonitor_h = nullptr; // host-mapped
    double *bmonitor_d = nullptr;
    int bmonitor_len = 4096;

    // status word of the bounded waits in the pipelined kernels (host-mapped;
    // non-zero: a wait ran out, the code says which)
    int *wait_status_h = nullptr;
    int *wait_status_d = nullptr;

    // host-side failure injection: allocations left before they fail (-1: off)
    long long alloc_fail_after = -1;
    // host-side failure injection: the next tensor-core deflation issues no copy
    // and gives up its waits after a few thousand polls (one-shot)
    bool inject_wait_timeout = false;

    // launch shapes chosen by the autotuner, by problem key
    std::map<unsigned long long, int> tuned;
    // a batched-operator launch shape chosen by the caller (0: autotuned)
    int mrhs_force_kind = 0, mrhs_force_R = 0, mrhs_force_budget = 0;

    // profiling of the FP64 operator (hisq_set_profiling): event pairs around
    // each FP64 Dslash launch, summed once their launches have completed
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> fp64_pending;
    std::vector<cudaEvent_t> fp64_pool;
    double fp64_seconds = 0;
    unsigned long long fp64_launches = 0;

    // scratch buffers (grown on demand)
    void *bufs[hisq::BUF_COUNT] = {};
    size_t buf_cap[hisq::BUF_COUNT] = {};
    size_t bytes = 0;
};

namespace hisq {

// verbosity from the HISQ_LOG environment variable (0 = silent)
int log_level();

// error helpers (api.cu)
hisq_status set_err(hisq_ctx *c, hisq_status s, const char *fmt, ...);
hisq_status cuda_err(hisq_ctx *c, cudaError_t e, const char *what);
void *dev_alloc(hisq_ctx *c, size_t bytes);
void dev_free(hisq_ctx *c, void *p, size_t bytes);
// persistent scratch buffer `id` of at least `bytes` (nullptr + error set on OOM)
void *get_buf(hisq_ctx *c, int id, size_t bytes);

#define HISQ_CUDA(call)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) return ::hisq::cuda_err(ctx, e_, #call);                  \
    } while (0)

// grid size for a grid-stride kernel over n items
inline int grid_for(const hisq_ctx *ctx, long n, int threads, int blocks_per_sm)
{
    ctx->launches++; // every grid-stride launch sizes its grid here
    long want = (n + threads - 1) / threads;
    long cap = long(ctx->num_sms) * blocks_per_sm;
    if (cap > ctx->max_red_blocks) cap = ctx->max_red_blocks;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return int(want);
}

// ------------------------------------------------------- CUDA graph replay
// The launches of one CG iteration are the same every iteration (all scalars
// live in device memory), so they are captured once into a CUDA graph and
// replayed: one cudaGraphLaunch instead of three kernel launches.  Up to four
// variants (slot = iteration mod 4) carry the per-iteration event records.
// Graphs are used only on a stream that can be captured (not the legacy or
// per-thread default stream) and can be switched off with HISQ_GRAPHS=0.
struct IterGraphs {
    cudaGraphExec_t exec[4] = {nullptr, nullptr, nullptr, nullptr};
    unsigned long long launches[4] = {0, 0, 0, 0};
    long long key = -1;
    void release()
    {
        for (int i = 0; i < 4; i++) {
            if (exec[i]) cudaGraphExecDestroy(exec[i]);
            exec[i] = nullptr;
        }
    }
    ~IterGraphs() { release(); }
};

bool graphs_enabled(const hisq_ctx *ctx);

// records `ev` on the context's stream, as a graph node while capturing
inline cudaError_t record_event(hisq_ctx *ctx, cudaEvent_t ev, bool capturing)
{
    return capturing ? cudaEventRecordWithFlags(ev, ctx->stream, cudaEventRecordExternal)
                     : cudaEventRecord(ev, ctx->stream);
}

// Enqueue `body(capturing)` through graph slot `slot`: captured on first use for
// the current `key`, replayed afterwards; run directly when graphs are off.
template <class F>
hisq_status graph_run(hisq_ctx *ctx, IterGraphs &G, int slot, long long key, F &&body)
{
    if (!graphs_enabled(ctx)) return body(false);
    if (key != G.key) {
        G.release();
        G.key = key;
    }
    if (!G.exec[slot]) {
        const unsigned long long l0 = ctx->launches;
        cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_err(ctx, e, "graph capture begin");
        hisq_status s = body(true);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(ctx->stream, &g);
        if (s != HISQ_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return cuda_err(ctx, e, "graph capture end");
        e = cudaGraphInstantiate(&G.exec[slot], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            G.exec[slot] = nullptr;
            return cuda_err(ctx, e, "graph instantiate");
        }
        G.launches[slot] = ctx->launches - l0;
        ctx->launches = l0; // counted when replayed
    }
    ctx->launches += G.launches[slot];
    cudaError_t e = cudaGraphLaunch(G.exec[slot], ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "graph launch");
    return HISQ_OK;
}

// ------------------------------------------------------------ autotuner
// Launch-shape autotuning: `launch(i)` enqueues candidate i (0 <= i < n) of an
// idempotent launch (same inputs, same outputs whichever shape runs it).  On
// the first call for `key` each candidate is run once to warm up and twice
// timed with CUDA events; the fastest index is kept in the context and used
// from then on.  Not while the stream is being captured (the default index is
// used then, and not remembered), nor with HISQ_TUNE=0.
bool tuning_enabled();

template <class F>
hisq_status autotune(hisq_ctx *ctx, unsigned long long key, int n, int dflt, F &&launch, int *chosen)
{
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) {
        *chosen = it->second;
        return HISQ_OK;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusActive;
    if (!tuning_enabled() || cs != cudaStreamCaptureStatusNone || n <= 1) {
        *chosen = dflt;
        if (cs == cudaStreamCaptureStatusNone) ctx->tuned[key] = dflt;
        return HISQ_OK;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cuda_err(ctx, cudaGetLastError(), "tuner event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_err(ctx, cudaGetLastError(), "tuner event");
    }
    int best = dflt;
    float best_ms = 1e30f;
    hisq_status st = HISQ_OK;
    for (int i = 0; i < n && st == HISQ_OK; i++) {
        st = launch(i);
        if (st != HISQ_OK) break;
        cudaEventRecord(e0, ctx->stream);
        st = launch(i);
        if (st == HISQ_OK) st = launch(i);
        cudaEventRecord(e1, ctx->stream);
        if (st != HISQ_OK) break;
        float ms = 0;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = cuda_err(ctx, cudaGetLastError(), "tuner timing");
            break;
        }
        if (log_level() > 1) fprintf(stderr, "[hisq] autotune key %llx: candidate %d: %.3f ms per launch\n", key, i, ms / 2);
        if (ms < best_ms) {
            best_ms = ms;
            best = i;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HISQ_OK) return st;
    if (log_level() > 0)
        fprintf(stderr, "[hisq] autotune key %llx: candidate %d of %d (%.3f ms per launch)\n", key, best, n,
                best_ms / 2);
    ctx->tuned[key] = best;
    *chosen = best;
    return HISQ_OK;
}

inline RedArgs red_args(hisq_ctx *ctx, int op, int slot0 = 0)
{
    RedArgs r;
    r.partials = ctx->partials;
    r.ticket = ctx->ticket;
    r.scal = ctx->scal;
    r.monitor = ctx->monitor_d;
    r.monitor_len = ctx->monitor_len;
    r.op = op;
    r.slot0 = slot0;
    return r;
}

// ---------------------------------------------------- launchers (kernels.cu)
// All fields are one parity, Vh sites, in the storage format of their precision.
// Host-layout FP64 full-lattice field <-> one parity of a device field.
hisq_status launch_gather_parity(hisq_ctx *ctx, const double *full, int parity, int prec, void *out);
hisq_status launch_scatter_parity(hisq_ctx *ctx, const void *in, int prec, int parity, double *full);
// precision conversion between parity fields (also copies when equal)
hisq_status launch_convert(hisq_ctx *ctx, const void *in, int prec_in, void *out, int prec_out);

// out = a*x + b*y + c*D(in)  on output parity `out_parity`; x, y nullable,
// all of precision `prec`, links of precision link_prec (64 or 32).
// If norm_slot >= 0 the squared norm of out is reduced into scal->slot[norm_slot].
// FP16 sloppy links, built from the FP32 gathered links on first use (ingest.cu)
hisq_status ensure_half_links(hisq_ctx *ctx);

// FP64 operator timing: fold completed event pairs into the sums (all: wait
// for every pending one); discard: drop them without summing
void fp64_prof_drain(hisq_ctx *ctx, bool all, bool discard = false);
hisq_status launch_dslash(hisq_ctx *ctx, int out_parity, int prec, int link_prec, const void *in,
                          void *out, double a, const void *x, double b, const void *y, double c,
                          int norm_slot);

// CG iteration kernels (sloppy precision `prec`, links `link_prec`, x in xprec)
hisq_status launch_cg_dslash_tt(hisq_ctx *ctx, int prec, int link_prec, const void *p, void *tmp);
hisq_status launch_cg_dslash_update(hisq_ctx *ctx, int prec, int link_prec, int xprec,
                                    const void *tmp, const void *p, void *x, void *r);
hisq_status launch_cg_p_update(hisq_ctx *ctx, int prec, const void *r, void *p);

// BLAS-1 on one parity
hisq_status launch_norm2(hisq_ctx *ctx, int prec, const void *x, int slot);
hisq_status launch_axpy_d(hisq_ctx *ctx, double a, const void *x, int xprec, double *y); // y(FP64) += a x
hisq_status launch_zero(hisq_ctx *ctx, void *x, int prec);
hisq_status launch_cdot(hisq_ctx *ctx, int prec, const void *x, const void *y, int slot); // <x,y> re,im
hisq_status launch_scale_axpby_d(hisq_ctx *ctx, double a, const double *x, double b, double *y); // y = a x + b y

// deflation (Eq. 4) over n stored vectors of precision vprec (32 or 16):
// c_i = v_i^dag b (b FP64 or FP32), x += coef * sum_i d_i v_i (x FP64 or FP32)
hisq_status launch_defl_project(hisq_ctx *ctx, int n, int vprec, const void *V, int bprec, const void *b,
                                double *c_dev /* n complex, FP64 */);
hisq_status launch_defl_expand(hisq_ctx *ctx, int n, int vprec, const void *V, const double *d_dev, double coef,
                               int xprec, void *x);
// d_i = c_i / (eps_i + shift) in place
hisq_status launch_defl_scale(hisq_ctx *ctx, int n, double *c_dev, const double *eps_dev, double shift);
// FP32 field helpers for the eigensolver
hisq_status launch_scale_f(hisq_ctx *ctx, double s, const void *in, void *out);
hisq_status launch_random_f(hisq_ctx *ctx, unsigned long long seed, void *out);
// basis rotation for the eigensolver, in place: v_j <- sum_i Y[i][j] v_i for
// j < k_out, real Y (k_in x k_out), through a tmp of k_out x chunk floats
hisq_status launch_rotate_inplace(hisq_ctx *ctx, int k_in, int k_out, void *V, const double *Y_dev, float *tmp,
                                  int chunk);

// batched operator (mrhs.cu): active right-hand sides from ctx->bscal->idx
hisq_status launch_mrhs_dslash_tt(hisq_ctx *ctx, int prec, int link_prec, void *p, void *tmp, int kact);
hisq_status launch_mrhs_dslash_update(hisq_ctx *ctx, int prec, int link_prec, void *tmp, void *p, void *x, void *r,
                                      int kact);
hisq_status launch_mrhs_p_update(hisq_ctx *ctx, int prec, void *r, void *p, int kact);
// blocks of k ordinary FP32 fields (eigensolver): slots 0..k-1 active, and
// out_j = a x_j + b y_j + c D(in_j) on output parity par (x, y nullable)
hisq_status mrhs_set_identity(hisq_ctx *ctx, int k);
hisq_status launch_mrhs_dslash_lin(hisq_ctx *ctx, int par, const void *in, void *out, double a, const void *x,
                                   double b, const void *y, double c, int k);
hisq_status launch_mrhs_dslash_store(hisq_ctx *ctx, int par, int prec, const void *in, void *out, int k);
hisq_status launch_bcg_persistent(hisq_ctx *ctx, int prec, int link_prec, void *p, void *tmp, void *r, void *x,
                                  int kact, int max_iters, const double *lo2_h, const double *hi2_h, int *n_done,
                                  int *its_rhs, double *phase_s);

// double-float operator (df64.cu): fields of HISQ_PREC_DF64 storage
hisq_status ensure_df_links(hisq_ctx *ctx);
hisq_status launch_to_df64(hisq_ctx *ctx, const double *in, void *out);        // FP64 -> (hi, lo)
hisq_status launch_dslash_df(hisq_ctx *ctx, int out_parity, const void *in, void *out); // out = D in
// out (FP64) = a x + b y + c D in (x, y FP64, nullable); |out|^2 -> slot if >= 0
hisq_status launch_dslash_df_xpay(hisq_ctx *ctx, int out_parity, const void *in, double *out, double a,
                                  const double *x, double b, const double *y, double c, int norm_slot);
// r = b - (4m^2 - D_eo D_oe) x on even fields, |r|^2 -> slot
hisq_status launch_residual_df(hisq_ctx *ctx, const double *b, const double *x, double *r, int slot);

// link ingest (ingest.cu)
hisq_status ingest_links(hisq_ctx *ctx, const double *fat_dev, const double *lng_dev, int recon,
                         double long_scale, double *max_unitarity_err);

} // namespace hisq
