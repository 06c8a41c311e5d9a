// Device-side bodies of the multigrid kernels, shared by the single-system
// kernels (tpmg_kernels.cu) and the batched persistent kernels
// (tpmg_batch.cu).  One thread owns one vertical column (or one cell) of one
// level; see tpmg_kernels.cu for the layout and the arithmetic.
#pragma once

#include <cuda_runtime.h>

#include "tpmg_internal.h"

namespace tpmg {

// ------------------------------------------------------------------ conversions
// FP64 <-> FP32 conversions in integer arithmetic.  A hardware conversion
// between the two formats issues on the FP64 pipe (ncu counts one FP64-pipe
// instruction per conversion), which the refinement's residual, cast and
// update kernels already keep busy; these run on the integer ALU instead and
// give the results IEEE 754 defines for the conversion.

// x * 2^s rounded to the nearest binary32 value, ties to even: binary32
// subnormals where the value is below 2^-126, +-0 below half the smallest
// subnormal, +-infinity from 2^128 (less half an ulp) up; infinities stay
// infinite and a NaN becomes a quiet NaN of the same sign.  The product is
// never formed, so no intermediate rounding happens.
static __device__ __noinline__ float f64_to_f32_rn_rare(unsigned hi, unsigned lo, int s)
{
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    const unsigned long long frac = ((unsigned long long)(hi & 0xFFFFFu) << 32) | lo;
    if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (frac ? 0x00400000u : 0u));
    // |x| = M 2^E with M < 2^53 (no implicit bit for a binary64 subnormal)
    unsigned long long M = e ? (frac | (1ULL << 52)) : frac;
    if (M == 0) return __uint_as_float(sign);
    int E = (e ? e : 1) - 1075 + s;
    const int lz = __clzll((long long)M) - 11;  // normalise: bit 52 set
    M <<= lz;
    E -= lz;
    const int ef = E + 52 + 127;  // biased binary32 exponent of M 2^E
    if (ef >= 255) return __uint_as_float(sign | 0x7F800000u);
    // keep the top 24 bits (normal) or fewer (subnormal result)
    const int shift = ef >= 1 ? 29 : 30 - ef;
    if (shift >= 54) return __uint_as_float(sign);  // below half the smallest subnormal
    const unsigned long long r = M >> shift, rem = M & ((1ULL << shift) - 1),
                             half = 1ULL << (shift - 1);
    const unsigned up = (rem > half || (rem == half && (r & 1ULL))) ? 1u : 0u;
    // normal: (ef - 1) << 23 plus r (implicit bit at 23) carries into the
    // exponent on rounding up; subnormal: r itself, 2^23 if it rounds up to
    // the smallest normal
    const unsigned bits = ef >= 1 ? ((unsigned)(ef - 1) << 23) + (unsigned)r + up
                                  : (unsigned)r + up;
    return __uint_as_float(sign | bits);
}

__device__ __forceinline__ float f64_to_f32_rn(double x, int s = 0)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    const int ef = e - 896 + s;  // 1023 - 127: the binary32 biased exponent
    if (e == 0 || e == 0x7FF || ef < 1 || ef > 254) return f64_to_f32_rn_rare(hi, lo, s);
    // normal in, normal out: 23 fraction bits kept, 29 rounded off
    const unsigned mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29), rem = lo & 0x1FFFFFFFu;
    const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (mant & 1u))) ? 1u : 0u;
    return __uint_as_float((hi & 0x80000000u) | ((((unsigned)ef << 23) | mant) + up));
}

// The binary64 value of a binary32 value (exact).
__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
    if (e - 1u < 254u)  // normal
        return __hiloint2double((int)(sign | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
    if (e == 0xFFu)  // infinity, or a quiet NaN of the same sign
        return __hiloint2double((int)(sign | 0x7FF00000u | (m ? 0x80000u | (m >> 3) : 0u)),
                                (int)(m << 29));
    if (m == 0) return __hiloint2double((int)sign, 0);
    // subnormal m 2^-149 = 1.f 2^(p - 149), p the position of m's top bit
    const int p = 31 - __clz((int)m);
    const unsigned long long f52 = (unsigned long long)(m ^ (1u << p)) << (52 - p);
    return __hiloint2double((int)(sign | ((unsigned)(p + 874) << 20) | (unsigned)(f52 >> 32)),
                            (int)(unsigned)f52);
}

// f = 2^s for a positive normal binary64 power of two f, else kNotPow2.
constexpr int kNotPow2 = 1 << 30;
__device__ __forceinline__ int pow2_exponent(double f)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(f);
    const int e = (int)((u >> 52) & 0x7FFu);
    return ((u & 0x800FFFFFFFFFFFFFULL) == 0 && e != 0 && e != 0x7FF) ? e - 1023 : kNotPow2;
}

// The binary32 rounding of x f (s = pow2_exponent(f)): in integer
// arithmetic when f is a power of two, else by the hardware conversion of
// the FP64 product.
__device__ __forceinline__ float scaled_to_f32(double x, double f, int s)
{
    return s != kNotPow2 ? f64_to_f32_rn(x, s) : (float)(x * f);
}

// ------------------------------------------------------------------ reductions
// Maximum of two magnitudes (values >= 0 or NaN): non-negative doubles order
// as their bit patterns read as unsigned integers, and a NaN sorts above
// +Inf, so the integer maximum of the sign-cleared patterns is the maximum
// with NaN propagated, taken on the integer pipe instead of FP64 compares.
__device__ __forceinline__ double max_mag(double a, double b)
{
    constexpr unsigned long long kAbs = 0x7fffffffffffffffULL;
    const unsigned long long ia = (unsigned long long)__double_as_longlong(a) & kAbs;
    const unsigned long long ib = (unsigned long long)__double_as_longlong(b) & kAbs;
    return __longlong_as_double((long long)(ia > ib ? ia : ib));
}

template <int OP>  // 0: sum, 1: maximum magnitude (max_mag)
__device__ __forceinline__ double warp_reduce(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double w = __shfl_down_sync(0xffffffffu, v, o);
        v = OP == 0 ? v + w : max_mag(v, w);
    }
    return v;
}

// Deterministic block reduction; every thread of the block must call it.
// The block's value goes to partial[slot].
template <int OP>
__device__ __forceinline__ void block_store_at(double v, double *partial, int slot)
{
    __shared__ double ws[32];
    v = warp_reduce<OP>(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        v = warp_reduce<OP>(v);
        if (lane == 0) partial[slot] = v;
    }
    __syncthreads();  // ws may be reused by the next call in the same block
}

template <int OP>
__device__ __forceinline__ void block_store(double v, double *partial)
{
    block_store_at<OP>(v, partial, blockIdx.x);
}

// ------------------------------------------------------------------ stencil
// Column loop of the stencil: y = H x (MODE 0) or b - H x (MODE 1) for one
// column; returns the column's contribution to sum(y*y) (MODE 1) or
// sum(x*y) (MODE 0) when RED.  Loads of layers k+1..k+DEPTH are in flight
// while layer k is computed (register pipeline).
template <typename T>
struct StencilLoads {
    T xc, tz, h, txc, txw, tyn, tys, xe, xw, xn, xs, b;
};

template <typename T, int MODE>
__device__ __forceinline__ void stencil_load(StencilLoads<T> &s, const LevelDev<T> &L,
                                             const T *__restrict__ b, const T *__restrict__ x,
                                             size_t o, int col, int ie, int iw, int nlon,
                                             bool hasN, bool hasS)
{
    s.xc = __ldg(x + o + col);
    s.tz = __ldg(L.tz + o + col);
    s.h = __ldg(L.h + o + col);
    s.txc = __ldg(L.tx + o + col);
    s.txw = __ldg(L.tx + o + iw);
    s.xe = __ldg(x + o + ie);
    s.xw = __ldg(x + o + iw);
    s.tyn = hasN ? __ldg(L.ty + o + col) : T(0);
    s.xn = hasN ? __ldg(x + o + col + nlon) : T(0);
    s.tys = hasS ? __ldg(L.ty + o + col - nlon) : T(0);
    s.xs = hasS ? __ldg(x + o + col - nlon) : T(0);
    if (MODE) s.b = __ldg(b + o + col);
}

// TO != T (T double, TO float): y receives the rounding of out * yscale (the
// FP64 residual handed to the FP32 inner solve; yscale a power of two),
// rounded in integer arithmetic (f64_to_f32_rn).  NARROW_MUL: the product is
// formed in TO after the rounding, exact for a yscale that is a normal TO
// value (one FP64 operation fewer per cell).  The reduction uses out.
// HSUM: L.h holds the horizontal diagonal h + the four horizontal couplings,
// and the horizontal terms are taken in sum form, dh x_c - sum T x_nb (four
// FMAs instead of four subtractions and four FMAs); the vertical couplings,
// up to ~1e6 times h, keep the difference form whose subtraction is exact
// for neighbouring values of a smooth column.
template <typename T, int MODE, bool RED, typename TO = T, bool NARROW_MUL = false,
          bool HSUM = false>
__device__ __forceinline__ T stencil_column(const LevelDev<T> &L, const T *__restrict__ b,
                                            const T *__restrict__ x, TO *__restrict__ y, int col,
                                            T yscale = T(1))
{
    constexpr int kDepth = sizeof(T) == 8 ? 2 : 4;
    const int nlon = L.nlon, nlat = L.nlat, nz = L.nz;
    const int ncol = nlon * nlat;
    T acc = 0;
    if (col < ncol) {
        const int j = col / nlon, i = col - j * nlon;
        const int ie = (i + 1 == nlon) ? col - i : col + 1;
        const int iw = (i == 0) ? col + nlon - 1 : col - 1;
        const bool hasN = j + 1 < nlat, hasS = j > 0;
        const size_t plane = (size_t)ncol;
        StencilLoads<T> st[kDepth];
#pragma unroll
        for (int d = 0; d < kDepth; ++d)
            if (d < nz)
                stencil_load<T, MODE>(st[d], L, b, x, (size_t)d * plane, col, ie, iw, nlon, hasN,
                                      hasS);
        T xdn = 0, tdn = 0;
        for (int k0 = 0; k0 < nz; k0 += kDepth) {
#pragma unroll
            for (int d = 0; d < kDepth; ++d) {
                const int k = k0 + d;
                if (k < nz) {
                    const StencilLoads<T> &c = st[d];
                    const T xc = c.xc;
                    const T xup = (k + 1 < nz) ? st[(d + 1) % kDepth].xc : T(0);
                    T v = c.h * xc;
                    if (HSUM) {
                        v = fma(-c.txc, c.xe, v);
                        v = fma(-c.txw, c.xw, v);
                        if (hasN) v = fma(-c.tyn, c.xn, v);
                        if (hasS) v = fma(-c.tys, c.xs, v);
                    } else {
                        v = fma(c.txc, xc - c.xe, v);
                        v = fma(c.txw, xc - c.xw, v);
                        if (hasN) v = fma(c.tyn, xc - c.xn, v);
                        if (hasS) v = fma(c.tys, xc - c.xs, v);
                    }
                    v = fma(c.tz, xc - xup, v);
                    v = fma(tdn, xc - xdn, v);
                    const T out = MODE ? c.b - v : v;
                    if constexpr (sizeof(TO) == sizeof(T))
                        y[(size_t)k * plane + col] = out;
                    else
                        y[(size_t)k * plane + col] = NARROW_MUL
                                                         ? f64_to_f32_rn(out) * (TO)yscale
                                                         : f64_to_f32_rn(out * yscale);
                    if (RED) acc = fma(out, MODE ? out : xc, acc);
                    xdn = xc;
                    tdn = c.tz;
                    if (k + kDepth < nz)
                        stencil_load<T, MODE>(st[d], L, b, x, (size_t)(k + kDepth) * plane, col, ie,
                                              iw, nlon, hasN, hasS);
                }
            }
        }
    }
    return acc;
}

// Column loop of q = H d_new with the conjugate-gradient direction update
// fused in: d_new = z + beta d_old (BZ: d_new = z) is formed on the fly at
// the cell and its four horizontal neighbours, written for the cell, and
// returned sum_k d_new q of the column (the CG inner product <d, H d>).  The
// values equal those of a separate direction update followed by the apply.
template <typename T>
struct DirLoads {
    T zc, dc, ze, de, zw, dw, zn, dn, zs, ds, tz, h, txc, txw, tyn, tys;
};

template <typename T, bool BZ>
__device__ __forceinline__ void dir_load(DirLoads<T> &s, const LevelDev<T> &L,
                                         const T *__restrict__ z, const T *__restrict__ dold,
                                         size_t o, int col, int ie, int iw, int nlon, bool hasN,
                                         bool hasS)
{
    s.zc = __ldg(z + o + col);
    s.ze = __ldg(z + o + ie);
    s.zw = __ldg(z + o + iw);
    s.zn = hasN ? __ldg(z + o + col + nlon) : T(0);
    s.zs = hasS ? __ldg(z + o + col - nlon) : T(0);
    if (!BZ) {
        s.dc = __ldg(dold + o + col);
        s.de = __ldg(dold + o + ie);
        s.dw = __ldg(dold + o + iw);
        s.dn = hasN ? __ldg(dold + o + col + nlon) : T(0);
        s.ds = hasS ? __ldg(dold + o + col - nlon) : T(0);
    }
    s.tz = __ldg(L.tz + o + col);
    s.h = __ldg(L.h + o + col);
    s.txc = __ldg(L.tx + o + col);
    s.txw = __ldg(L.tx + o + iw);
    s.tyn = hasN ? __ldg(L.ty + o + col) : T(0);
    s.tys = hasS ? __ldg(L.ty + o + col - nlon) : T(0);
}

template <typename T, bool BZ>
__device__ __forceinline__ T dir_apply_column(const LevelDev<T> &L, const T *__restrict__ z,
                                              const T *__restrict__ dold, T beta,
                                              T *__restrict__ dnew, T *__restrict__ q, int col)
{
    constexpr int kDepth = sizeof(T) == 8 ? 2 : 3;
    const int nlon = L.nlon, nlat = L.nlat, nz = L.nz;
    const int ncol = nlon * nlat;
    T acc = 0;
    if (col >= ncol) return acc;
    const int j = col / nlon, i = col - j * nlon;
    const int ie = (i + 1 == nlon) ? col - i : col + 1;
    const int iw = (i == 0) ? col + nlon - 1 : col - 1;
    const bool hasN = j + 1 < nlat, hasS = j > 0;
    const size_t plane = (size_t)ncol;
    auto dv = [&](T zv, T dvv) { return BZ ? zv : fma(beta, dvv, zv); };
    DirLoads<T> st[kDepth];
#pragma unroll
    for (int d = 0; d < kDepth; ++d)
        if (d < nz)
            dir_load<T, BZ>(st[d], L, z, dold, (size_t)d * plane, col, ie, iw, nlon, hasN, hasS);
    T xdn = 0, tdn = 0;
    for (int k0 = 0; k0 < nz; k0 += kDepth) {
#pragma unroll
        for (int d = 0; d < kDepth; ++d) {
            const int k = k0 + d;
            if (k < nz) {
                const DirLoads<T> &c = st[d];
                const DirLoads<T> &nx = st[(d + 1) % kDepth];
                const T xc = dv(c.zc, c.dc);
                const T xup = (k + 1 < nz) ? dv(nx.zc, nx.dc) : T(0);
                T v = c.h * xc;
                v = fma(c.txc, xc - dv(c.ze, c.de), v);
                v = fma(c.txw, xc - dv(c.zw, c.dw), v);
                if (hasN) v = fma(c.tyn, xc - dv(c.zn, c.dn), v);
                if (hasS) v = fma(c.tys, xc - dv(c.zs, c.ds), v);
                v = fma(c.tz, xc - xup, v);
                v = fma(tdn, xc - xdn, v);
                const size_t o = (size_t)k * plane + col;
                dnew[o] = xc;
                q[o] = v;
                acc = fma(v, xc, acc);
                xdn = xc;
                tdn = c.tz;
                if (k + kDepth < nz)
                    dir_load<T, BZ>(st[d], L, z, dold, (size_t)(k + kDepth) * plane, col, ie, iw,
                                    nlon, hasN, hasS);
            }
        }
    }
    return acc;
}

// One cell of the stencil (cell-parallel form).
template <typename T, int MODE>
__device__ __forceinline__ void stencil_cell(const LevelDev<T> &L, const T *__restrict__ b,
                                             const T *__restrict__ x, T *__restrict__ y, int col,
                                             int k)
{
    const int nlon = L.nlon, nlat = L.nlat, nz = L.nz;
    const int ncol = nlon * nlat;
    if (col >= ncol) return;
    const int j = col / nlon, i = col - j * nlon;
    const int ie = (i + 1 == nlon) ? col - i : col + 1;
    const int iw = (i == 0) ? col + nlon - 1 : col - 1;
    const size_t plane = (size_t)ncol;
    const size_t o = (size_t)k * plane;
    const T xc = __ldg(x + o + col);
    T v = __ldg(L.h + o + col) * xc;
    v = fma(__ldg(L.tx + o + col), xc - __ldg(x + o + ie), v);
    v = fma(__ldg(L.tx + o + iw), xc - __ldg(x + o + iw), v);
    if (j + 1 < nlat) v = fma(__ldg(L.ty + o + col), xc - __ldg(x + o + col + nlon), v);
    if (j > 0) v = fma(__ldg(L.ty + o + col - nlon), xc - __ldg(x + o + col - nlon), v);
    if (k + 1 < nz) v = fma(__ldg(L.tz + o + col), xc - __ldg(x + o + plane + col), v);
    if (k > 0) v = fma(__ldg(L.tz + o - plane + col), xc - __ldg(x + o - plane + col), v);
    y[o + col] = MODE ? __ldg(b + o + col) - v : v;
}

// ------------------------------------------------------------------ smoother
// One sweep of Eq. (1), u_out = (1 - omega) u_in + omega H_z^{-1}(b - dH u_in),
// with the column tridiagonal H_z (diagonal s_k + t_{k-1} + t_k, couplings
// -t_k, s_k = h + the four horizontal couplings) solved by elimination with
// pivots p_k = q_k + t_k, on the setup factors m_k = 1/p_k and dq_k = q_k/p_k:
//   forward   y_k = (v_k + t_{k-1} y_{k-1}) m_k,  v_k = b_k + sum_h T u_in,nb
//   backward  x_k = x_{k+1} + (y_k - dq_k x_{k+1})
// This is the sweep on a non-zero guess; sweeps from a zero guess are
// smooth_staged (large levels) and smooth_warp_column (small FP32 levels).
// The forward values y wait in shared memory for the backward sweep
// (blockDim x nz values).
//
// Shared memory caps residency at a few blocks of 128 columns per SM, so the
// loads of layers k+1..k+DEPTH are issued before layer k is computed (a
// register pipeline) to keep enough bytes in flight to cover HBM latency:
// deeper for FP32 (few registers per layer, HBM-bound), shallow for FP64
// (FP64-ALU-bound, twice the registers per value).
template <typename T>
struct SmoothDepth {
    static constexpr int value = sizeof(T) == 8 ? 3 : 6;  // forward: layers in flight
    static constexpr int back = sizeof(T) == 8 ? 4 : 12;  // backward (u_in, q/p, b)
};

template <typename T>
struct SmoothLoads {
    T b, tz, m, txc, txw, tyn, tys, ue, uw, un, us;
};

// L2 eviction-priority hints (ld.global.nc.L2::cache_hint with a
// createpolicy policy): the sweep with the fused inner product reads b again
// in its backward pass, so b is loaded evict_last and the read-once
// coefficient streams evict_first.
struct L2Hints {
    unsigned long long keep, stream;
};

__device__ __forceinline__ L2Hints make_l2_hints()
{
    L2Hints h;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(h.keep));
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(h.stream));
    return h;
}

template <typename T>
__device__ __forceinline__ T ld_hint(const T *p, unsigned long long pol);

template <>
__device__ __forceinline__ float ld_hint<float>(const float *p, unsigned long long pol)
{
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}

template <>
__device__ __forceinline__ double ld_hint<double>(const double *p, unsigned long long pol)
{
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}

// One layer's loads of the sweep.  HINT: b kept and the own-column
// coefficients streamed in L2 (the policies above).
template <typename T, bool HINT>
__device__ __forceinline__ void smooth_load(SmoothLoads<T> &s, const LevelDev<T> &L,
                                            const T *__restrict__ b, const T *__restrict__ uin,
                                            size_t o, int col, int ie, int iw, int nlon, bool hasN,
                                            bool hasS, L2Hints hp)
{
    if (HINT) {
        s.b = ld_hint(b + o + col, hp.keep);
        s.tz = ld_hint(L.tz + o + col, hp.stream);
        s.m = ld_hint(L.m + o + col, hp.stream);
        s.txc = ld_hint(L.tx + o + col, hp.stream);
        s.tyn = hasN ? ld_hint(L.ty + o + col, hp.stream) : T(0);
    } else {
        s.b = __ldg(b + o + col);
        s.tz = __ldg(L.tz + o + col);
        s.m = __ldg(L.m + o + col);
        s.txc = __ldg(L.tx + o + col);
        s.tyn = hasN ? __ldg(L.ty + o + col) : T(0);
    }
    s.txw = __ldg(L.tx + o + iw);
    s.tys = hasS ? __ldg(L.ty + o + col - nlon) : T(0);
    s.ue = __ldg(uin + o + ie);
    s.uw = __ldg(uin + o + iw);
    s.un = hasN ? __ldg(uin + o + col + nlon) : T(0);
    s.us = hasS ? __ldg(uin + o + col - nlon) : T(0);
}

// One column of the sweep.  smraw: this block's dynamic shared memory
// (nz * blockDim values of T).  DOT: also accumulate sum_k b_k u_out,k of
// the column into *dacc (the CG inner product <r, z> when the sweep is the
// last one of a V-cycle applied to r); the single-system DOT sweep (BACK ==
// 0) loads with the L2 hints and an 8-layer FP32 forward pipeline.  BACK > 0
// overrides the backward depth (the batched kernels, which hold their
// work-item descriptors in registers as well).
// YOUT: the forward values wait in the thread's own output column (read back
// from L2 and overwritten on the way back) instead of shared memory.
template <typename T, bool DOT = false, int BACK = 0, bool YOUT = false>
__device__ __forceinline__ void smooth_column(const LevelDev<T> &L, const T *__restrict__ b,
                                              const T *__restrict__ uin, T *__restrict__ uout,
                                              T omega, int col, unsigned char *smraw,
                                              T *dacc = nullptr)
{
    constexpr bool HINT = DOT && BACK == 0;
    constexpr int kDepth = (HINT && sizeof(T) == 4) ? 8 : SmoothDepth<T>::value;
    const L2Hints hp = HINT ? make_l2_hints() : L2Hints{};
    const int nlon = L.nlon, nlat = L.nlat, nz = L.nz;
    const int bd = blockDim.x, tid = threadIdx.x;
    T *ys = reinterpret_cast<T *>(smraw);
    const int ncol = nlon * nlat;
    if (col >= ncol) return;
    const int j = col / nlon, i = col - j * nlon;
    const int ie = (i + 1 == nlon) ? col - i : col + 1;
    const int iw = (i == 0) ? col + nlon - 1 : col - 1;
    const bool hasN = j + 1 < nlat, hasS = j > 0;
    const size_t plane = (size_t)ncol;

    SmoothLoads<T> st[kDepth];
#pragma unroll
    for (int d = 0; d < kDepth; ++d)
        if (d < nz)
            smooth_load<T, HINT>(st[d], L, b, uin, (size_t)d * plane, col, ie, iw, nlon, hasN,
                                 hasS, hp);

    T yprev = 0, tdn = 0;
    for (int k0 = 0; k0 < nz; k0 += kDepth) {
#pragma unroll
        for (int d = 0; d < kDepth; ++d) {
            const int k = k0 + d;
            if (k < nz) {
                SmoothLoads<T> &c = st[d];
                T v = c.b;
                v = fma(c.txc, c.ue, v);
                v = fma(c.txw, c.uw, v);
                v = fma(c.tyn, c.un, v);
                v = fma(c.tys, c.us, v);
                const T y = fma(tdn, yprev, v) * c.m;
                if (YOUT)
                    uout[(size_t)k * plane + col] = y;
                else
                    ys[(size_t)k * bd + tid] = y;
                yprev = y;
                tdn = c.tz;
                if (k + kDepth < nz)
                    smooth_load<T, HINT>(c, L, b, uin, (size_t)(k + kDepth) * plane, col, ie, iw,
                                         nlon, hasN, hasS, hp);
            }
        }
    }

    const T om1 = T(1) - omega;
    T xk = yprev;
    // backward sweep: prefetch u_in, q/p (and b) kBack layers ahead
    constexpr int kBack = BACK > 0 ? BACK : SmoothDepth<T>::back;
    T up[kBack], dqp[kBack], bp[kBack];
#pragma unroll
    for (int d = 0; d < kBack; ++d) {
        const int k = nz - 1 - d;
        if (k >= 0) {
            const size_t o = (size_t)k * plane + col;
            up[d] = __ldg(uin + o);
            dqp[d] = HINT ? ld_hint(L.dq + o, hp.stream) : __ldg(L.dq + o);
            bp[d] = DOT ? __ldg(b + o) : T(0);
        }
    }
    for (int k0 = nz - 1; k0 >= 0; k0 -= kBack) {
#pragma unroll
        for (int d = 0; d < kBack; ++d) {
            const int k = k0 - d;
            if (k >= 0) {
                const size_t o = (size_t)k * plane + col;
                if (k < nz - 1)
                    xk = xk + fma(-dqp[d], xk, YOUT ? uout[o] : ys[(size_t)k * bd + tid]);
                const T uo = fma(om1, up[d], omega * xk);
                uout[o] = uo;
                if (DOT) *dacc = fma(bp[d], uo, *dacc);
                const int kn = k - kBack;
                if (kn >= 0) {
                    const size_t on = (size_t)kn * plane + col;
                    up[d] = __ldg(uin + on);
                    dqp[d] = HINT ? ld_hint(L.dq + on, hp.stream) : __ldg(L.dq + on);
                    if (DOT) bp[d] = __ldg(b + on);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ warp sweep
// One column of the sweep of Eq. (1) solved by a whole warp, for the small
// coarse levels, where one thread per column leaves the GPU waiting on the
// 2 nz dependent steps of the column recurrences.  Lane l owns layers
// [l C, l C + C), C = ceil(nz / 32).  Both recurrences are first-order and
// linear, so they run as warp scans of affine maps:
//   forward   y_k = (v_k + t_{k-1} y_{k-1}) / p_k  = (t_{k-1}/p_k) y_{k-1} + v_k/p_k
//   backward  x_k = y_k + (1 - q_k/p_k) x_{k+1}      (x_nz = 0)
// Each lane composes the maps of its layers, a Kogge-Stone scan across the
// lanes gives each lane the value entering its layers, and the lane then
// re-runs its own layers with the serial formulas of smooth_column.  The
// values differ from the serial sweep only by rounding.  u_in is read with
// ordinary (coherent) loads, so a block may read what its own earlier sweep
// wrote after a block barrier.  All 32 lanes must call it with the same
// col < ncol.
constexpr int kWarpLayers = (kMaxLayers + 31) / 32;  // layers per lane at most
// CM: the layers per lane the code is unrolled for (ceil(nz / 32) <= CM <=
// kWarpLayers; the launchers take the smallest of 2, 3, kWarpLayers that
// holds the level, so no predicated-off layer slots are issued).

// The two scans of the warp sweep over one lane's layers k0 .. k0 + C - 1:
// v holds the right-hand sides v_k on entry and the column solution x_k of
// H_z x = v on return; tprev = t_{k0-1} (0 for the first lane).
template <typename T, int CM>
__device__ __forceinline__ void warp_column_scan(T (&v)[CM], const T (&tz)[CM], const T (&m)[CM],
                                                 const T (&dq)[CM], T tprev, int C, int k0,
                                                 int nz, int lane)
{
    // forward: this lane's map y_out = A y_in + Cy, then an inclusive scan
    T A = 1, Cy = 0, tp = tprev;
#pragma unroll
    for (int c = 0; c < CM; ++c) {
        if (c < C && k0 + c < nz) {
            const T a = tp * m[c];
            Cy = fma(a, Cy, v[c] * m[c]);
            A = a * A;
            tp = tz[c];
        }
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T A2 = __shfl_up_sync(0xffffffffu, A, off);
        const T C2 = __shfl_up_sync(0xffffffffu, Cy, off);
        if (lane >= off) {
            Cy = fma(A, C2, Cy);
            A = A * A2;
        }
    }
    T y = __shfl_up_sync(0xffffffffu, Cy, 1);
    if (lane == 0) y = T(0);
    tp = tprev;
#pragma unroll
    for (int c = 0; c < CM; ++c) {
        if (c < C && k0 + c < nz) {
            y = fma(tp, y, v[c]) * m[c];
            v[c] = y;  // v now holds y
            tp = tz[c];
        }
    }

    // backward: x_bottom = E x_above + F over this lane's layers, suffix scan
    T E = 1, F = 0;
#pragma unroll
    for (int c = CM - 1; c >= 0; --c) {
        if (c < C && k0 + c < nz) {
            const T e = T(1) - dq[c];
            F = fma(e, F, v[c]);
            E = e * E;
        }
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T E2 = __shfl_down_sync(0xffffffffu, E, off);
        const T F2 = __shfl_down_sync(0xffffffffu, F, off);
        if (lane + off < 32) {
            F = fma(E, F2, F);
            E = E * E2;
        }
    }
    T x = __shfl_down_sync(0xffffffffu, F, 1);
    if (lane == 31) x = T(0);
#pragma unroll
    for (int c = CM - 1; c >= 0; --c) {
        if (c < C && k0 + c < nz) {
            x = x + fma(-dq[c], x, v[c]);
            v[c] = x;  // v now holds x
        }
    }
}

template <typename T, bool ZERO, int CM = kWarpLayers>
__device__ __forceinline__ void smooth_warp_column(const LevelDev<T> &L, const T *__restrict__ b,
                                                   const T *uin, T *uout, T omega, int col,
                                                   int lane)
{
    const int nlon = L.nlon, nlat = L.nlat, nz = L.nz;
    const int j = col / nlon, i = col - j * nlon;
    const int ie = (i + 1 == nlon) ? col - i : col + 1;
    const int iw = (i == 0) ? col + nlon - 1 : col - 1;
    const bool hasN = j + 1 < nlat, hasS = j > 0;
    const size_t plane = (size_t)nlon * nlat;
    const int C = (nz + 31) / 32;
    const int k0 = lane * C;
    T v[CM], tz[CM], m[CM], dq[CM], u0[CM];
#pragma unroll
    for (int c = 0; c < CM; ++c) {
        const int k = k0 + c;
        v[c] = tz[c] = m[c] = dq[c] = u0[c] = T(0);
        if (c < C && k < nz) {
            const size_t o = (size_t)k * plane;
            T vv = __ldg(b + o + col);
            if (!ZERO) {
                vv = fma(__ldg(L.tx + o + col), uin[o + ie], vv);
                vv = fma(__ldg(L.tx + o + iw), uin[o + iw], vv);
                if (hasN) vv = fma(__ldg(L.ty + o + col), uin[o + col + nlon], vv);
                if (hasS) vv = fma(__ldg(L.ty + o + col - nlon), uin[o + col - nlon], vv);
                u0[c] = uin[o + col];
            }
            v[c] = vv;
            tz[c] = __ldg(L.tz + o + col);
            m[c] = __ldg(L.m + o + col);
            dq[c] = __ldg(L.dq + o + col);
        }
    }
    const T tprev = (k0 >= 1 && k0 - 1 < nz) ? __ldg(L.tz + (size_t)(k0 - 1) * plane + col) : T(0);
    warp_column_scan<T, CM>(v, tz, m, dq, tprev, C, k0, nz, lane);
    const T om1 = T(1) - omega;
#pragma unroll
    for (int c = 0; c < CM; ++c) {
        const int k = k0 + c;
        if (c < C && k < nz)
            uout[(size_t)k * plane + col] = ZERO ? omega * v[c] : fma(om1, u0[c], omega * v[c]);
    }
}

// The coarsest-level solve (sweeps of Eq. (1) from zero) by one block with
// the whole level in shared memory: b, t_z, 1/p, q/p,
// t_x, t_y and the two sweep vectors, each stored as [column][layer], so a
// lane's own layers are consecutive words (bank-conflict free for an odd
// layers-per-lane count).  The level is staged once from its [layer][column]
// arrays and the result written back once; the sweeps in between touch no
// global memory.  Same arithmetic, same order as the sweeps from global
// memory (smooth_warp_column).  Called by every thread of the block; sh:
// kCoarseShArrays * ncol * nz values of dynamic shared memory.
constexpr int kCoarseShArrays = 8;

template <typename T, int CM = kWarpLayers>
__device__ __forceinline__ void coarse_solve_sh(const LevelDev<T> &L, const T *__restrict__ b,
                                                T *__restrict__ out, T omega, int sweeps, T *sh)
{
    const int nlon = L.nlon, nlat = L.nlat, nz = L.nz;
    const int ncol = nlon * nlat, n = ncol * nz;
    T *sb = sh, *stz = sh + n, *sm = sh + 2 * n, *sdq = sh + 3 * n, *stx = sh + 4 * n,
      *sty = sh + 5 * n;
    T *cur = sh + 6 * n, *oth = sh + 7 * n;
    for (int g = threadIdx.x; g < n; g += blockDim.x) {
        const int k = g / ncol, c = g - k * ncol, o = c * nz + k;
        sb[o] = __ldg(b + g);
        stz[o] = __ldg(L.tz + g);
        sm[o] = __ldg(L.m + g);
        sdq[o] = __ldg(L.dq + g);
        stx[o] = __ldg(L.tx + g);
        sty[o] = __ldg(L.ty + g);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int C = (nz + 31) / 32, k0 = lane * C;
    const T om1 = T(1) - omega;
    for (int it = 0; it < sweeps; ++it) {
        for (int col = warp; col < ncol; col += nw) {
            const int j = col / nlon, i = col - j * nlon;
            const int ie = (i + 1 == nlon) ? col - i : col + 1;
            const int iw = (i == 0) ? col + nlon - 1 : col - 1;
            const bool hasN = j + 1 < nlat, hasS = j > 0;
            const int oc = col * nz, oe = ie * nz, ow = iw * nz;
            const int on = (col + nlon) * nz, os = (col - nlon) * nz;
            T v[CM], tz[CM], m[CM], dq[CM], u0[CM];
#pragma unroll
            for (int c = 0; c < CM; ++c) {
                const int k = k0 + c;
                v[c] = tz[c] = m[c] = dq[c] = u0[c] = T(0);
                if (c < C && k < nz) {
                    T vv = sb[oc + k];
                    if (it > 0) {
                        vv = fma(stx[oc + k], cur[oe + k], vv);
                        vv = fma(stx[ow + k], cur[ow + k], vv);
                        if (hasN) vv = fma(sty[oc + k], cur[on + k], vv);
                        if (hasS) vv = fma(sty[os + k], cur[os + k], vv);
                        u0[c] = cur[oc + k];
                    }
                    v[c] = vv;
                    tz[c] = stz[oc + k];
                    m[c] = sm[oc + k];
                    dq[c] = sdq[oc + k];
                }
            }
            const T tprev = (k0 >= 1 && k0 - 1 < nz) ? stz[oc + k0 - 1] : T(0);
            warp_column_scan<T, CM>(v, tz, m, dq, tprev, C, k0, nz, lane);
#pragma unroll
            for (int c = 0; c < CM; ++c) {
                const int k = k0 + c;
                if (c < C && k < nz)
                    oth[oc + k] = it == 0 ? omega * v[c] : fma(om1, u0[c], omega * v[c]);
            }
        }
        __syncthreads();  // the sweep is complete before the next one reads it
        T *t = cur;
        cur = oth;
        oth = t;
    }
    for (int g = threadIdx.x; g < n; g += blockDim.x) {
        const int k = g / ncol, c = g - k * ncol;
        out[g] = cur[c * nz + k];
    }
}

// ------------------------------------------------------------------ staged sweep
// Asynchronous global->shared copies (cp.async, 4 or 8 bytes per thread).
// Each thread stages and later reads only its own slots, so completion of
// its own copy groups (cp.async.wait_group) is the only synchronisation.
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

template <typename T>
__device__ __forceinline__ void stage(T *dst, const T *src)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte values");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "n"((int)sizeof(T))
                 : "memory");
}

__device__ __forceinline__ void stage_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__device__ __forceinline__ void stage_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Layers in flight per thread in the staged sweep, and values staged per
// layer: forward b, t_z, 1/p (+ t_x east/west, t_y north/south and the four
// horizontal neighbours of u_in unless the guess is zero); backward q/p
// (+ u_in, + b for the fused inner product).
constexpr int kRing = 8;

template <bool ZERO>
struct RingSlot {
    static constexpr int NV = ZERO ? 3 : 11;
    enum { B = 0, TZ = 1, M = 2, TXC = 3, TXW = 4, TYN = 5, TYS = 6, UE = 7, UW = 8, UN = 9, US = 10 };
};

// Shared memory of one block of the staged sweep: the ring and the forward
// values y (nz per column).
template <typename T, bool ZERO>
__host__ __device__ constexpr size_t ring_smem_bytes(int nz, int block)
{
    return ((size_t)kRing * RingSlot<ZERO>::NV + (size_t)nz) * (size_t)block * sizeof(T);
}

// One column of the sweep of Eq. (1) on precomputed factors (m = 1/p,
// dq = q/p), the same arithmetic in the same order as smooth_column, with
// every load staged kRing layers ahead through shared memory by cp.async
// (the copies hold no registers, so the depth of the pipeline is not left to
// register allocation).  Horizontal neighbours missing at the poles read as 0
// (their slots are zeroed once and never staged).
template <typename T, bool ZERO, bool DOT = false>
__device__ __forceinline__ void smooth_staged(const LevelDev<T> &L, const T *__restrict__ b,
                                              const T *__restrict__ uin, T *__restrict__ uout,
                                              T omega, int col, unsigned char *smraw,
                                              T *dacc = nullptr)
{
    using S = RingSlot<ZERO>;
    constexpr int NV = S::NV;
    const int nlon = L.nlon, nlat = L.nlat, nz = L.nz;
    const int ncol = nlon * nlat;
    if (col >= ncol) return;
    const int bd = blockDim.x;
    T *ring = reinterpret_cast<T *>(smraw) + threadIdx.x;  // [kRing][NV][bd]
    T *ys = reinterpret_cast<T *>(smraw) + (size_t)kRing * NV * bd + threadIdx.x;  // [nz][bd]
    const int j = col / nlon, i = col - j * nlon;
    const int ie = (i + 1 == nlon) ? col - i : col + 1;
    const int iw = (i == 0) ? col + nlon - 1 : col - 1;
    const bool hasN = j + 1 < nlat, hasS = j > 0;
    const size_t plane = (size_t)ncol;

    // sources of the next layer to stage (advanced by one plane per layer)
    const T *pb = b + col, *pt = L.tz + col, *pm = L.m + col;
    const T *ptc = L.tx + col, *ptw = L.tx + iw;
    const T *pyn = L.ty + col, *pys = hasS ? L.ty + col - nlon : pyn;
    const T *ub = ZERO ? b : uin;  // u_in is not read from a zero guess
    const T *pue = ub + ie, *puw = ub + iw;
    const T *pun = hasN ? ub + col + nlon : pue, *pus = hasS ? ub + col - nlon : pue;
    if (!ZERO) {
        for (int d = 0; d < kRing; ++d) {
            T *sl = ring + (size_t)d * NV * bd;
            if (!hasN) sl[S::TYN * bd] = sl[S::UN * bd] = T(0);
            if (!hasS) sl[S::TYS * bd] = sl[S::US * bd] = T(0);
        }
    }
    auto issue = [&](int slot) {
        T *sl = ring + (size_t)slot * NV * bd;
        stage(sl + S::B * bd, pb);
        stage(sl + S::TZ * bd, pt);
        stage(sl + S::M * bd, pm);
        pb += plane;
        pt += plane;
        pm += plane;
        if (!ZERO) {
            stage(sl + S::TXC * bd, ptc);
            stage(sl + S::TXW * bd, ptw);
            stage(sl + S::UE * bd, pue);
            stage(sl + S::UW * bd, puw);
            if (hasN) {
                stage(sl + S::TYN * bd, pyn);
                stage(sl + S::UN * bd, pun);
            }
            if (hasS) {
                stage(sl + S::TYS * bd, pys);
                stage(sl + S::US * bd, pus);
            }
            ptc += plane;
            ptw += plane;
            pyn += plane;
            pys += plane;
            pue += plane;
            puw += plane;
            pun += plane;
            pus += plane;
        }
    };
    for (int d = 0; d < kRing; ++d) {
        if (d < nz) issue(d);
        stage_commit();
    }
    T yprev = 0, tdn = 0;
    int slot = 0;
    for (int k = 0; k < nz; ++k) {
        stage_wait<kRing - 1>();  // layer k has landed
        const T *sl = ring + (size_t)slot * NV * bd;
        T v = sl[S::B * bd];
        if (!ZERO) {
            v = fma(sl[S::TXC * bd], sl[S::UE * bd], v);
            v = fma(sl[S::TXW * bd], sl[S::UW * bd], v);
            v = fma(sl[S::TYN * bd], sl[S::UN * bd], v);
            v = fma(sl[S::TYS * bd], sl[S::US * bd], v);
        }
        const T y = fma(tdn, yprev, v) * sl[S::M * bd];
        tdn = sl[S::TZ * bd];
        ys[(size_t)k * bd] = y;
        yprev = y;
        if (k + kRing < nz) issue(slot);
        stage_commit();
        slot = (slot + 1 == kRing) ? 0 : slot + 1;
    }
    stage_wait<0>();

    // backward sweep: stage q/p (+ u_in, + b) of layers nz-1, nz-2, ...
    const size_t top = (size_t)(nz - 1) * plane + col;
    const T *qq = L.dq + top, *qu = (ZERO ? b : uin) + top, *qb = b + top;
    auto issue_back = [&](int sl_) {
        T *sl = ring + (size_t)sl_ * NV * bd;
        stage(sl, qq);
        qq -= plane;
        if (!ZERO) {
            stage(sl + bd, qu);
            qu -= plane;
        }
        if (DOT) {
            stage(sl + 2 * bd, qb);
            qb -= plane;
        }
    };
    for (int d = 0; d < kRing; ++d) {
        if (nz - 1 - d >= 0) issue_back(d);
        stage_commit();
    }
    const T om1 = T(1) - omega;
    T xk = yprev;
    T *uo_p = uout + top;
    slot = 0;
    for (int k = nz - 1; k >= 0; --k) {
        stage_wait<kRing - 1>();
        const T *sl = ring + (size_t)slot * NV * bd;
        if (k < nz - 1) xk = xk + fma(-sl[0], xk, ys[(size_t)k * bd]);
        const T uo = ZERO ? omega * xk : fma(om1, sl[bd], omega * xk);
        *uo_p = uo;
        uo_p -= plane;
        if (DOT) *dacc = fma(sl[2 * bd], uo, *dacc);
        if (k - kRing >= 0) issue_back(slot);
        stage_commit();
        slot = (slot + 1 == kRing) ? 0 : slot + 1;
    }
    stage_wait<0>();
}

// ------------------------------------------------------------------ transfers
// Restriction R = P^T as a gather: coarse (I, J, k) sums, over the fine rows
// listed for J with their latitude weights, the fine residuals at longitudes
// 2I-1, 2I, 2I+1, 2I+2 (mod nlon) with weights 1/4, 3/4, 3/4, 1/4.
// Bilinear prolongation and correction: fine cell 2I adds
// sum_a w_a (3/4 e[J_a, I] + 1/4 e[J_a, I-1]) and 2I+1 adds
// sum_a w_a (3/4 e[J_a, I] + 1/4 e[J_a, I+1]) (periodic in longitude).

// Layers k0 <= k < k1 of one coarse column of the restriction: the row
// list of J (at most kMaxRestrictRows fine rows, checked at setup) and the
// longitude indices are read once, then every layer issues its loads
// independently of the others, one layer per loop trip (unrolling the
// layer loop costs 8 registers and runs 20-25 % slower at 1536 x 1152 and
// 768 x 726 columns).  The sum over the row list runs in its (ascending
// fine-row) order.
template <typename T>
__device__ __forceinline__ void restrict_layers(const LevelDev<T> &F, const LinkDev &K,
                                                const T *__restrict__ r, T *__restrict__ bc,
                                                int col, int k0, int k1)
{
    const int nf = F.nlon, nc = nf / 2;
    const int ncol_c = nc * K.nlat_c;
    if (col >= ncol_c) return;
    const int J = col / nc, I = col - J * nc;
    const int i0 = 2 * I, i1 = 2 * I + 1;
    const int im = (i0 == 0) ? nf - 1 : i0 - 1;
    const int ip = (i1 + 1 == nf) ? 0 : i1 + 1;
    const int p0 = __ldg(K.rptr + J), cnt = __ldg(K.rptr + J + 1) - p0;
    const size_t plane_f = (size_t)nf * F.nlat, plane_c = (size_t)ncol_c;
    int off[kMaxRestrictRows];
    T w[kMaxRestrictRows];
#pragma unroll
    for (int a = 0; a < kMaxRestrictRows; ++a) {
        off[a] = a < cnt ? __ldg(K.rrow + p0 + a) * nf : 0;
        w[a] = a < cnt ? (T)__ldg(K.rw + p0 + a) : T(0);
    }
    const T q1 = T(0.25), q3 = T(0.75);
#pragma unroll 1
    for (int k = k0; k < k1; ++k) {
        const T *rk = r + (size_t)k * plane_f;
        T acc = 0;
#pragma unroll
        for (int a = 0; a < kMaxRestrictRows; ++a) {
            if (a < cnt) {
                const T *row = rk + off[a];
                acc = fma(w[a],
                          fma(q1, __ldg(row + im) + __ldg(row + ip),
                              q3 * (__ldg(row + i0) + __ldg(row + i1))),
                          acc);
            }
        }
        bc[(size_t)k * plane_c + col] = acc;
    }
}

// Layers k0 <= k < k1 of one pair of fine columns (t = j * nlon/2 + I) of
// the prolongation and correction, the row links read once.
template <typename T>
__device__ __forceinline__ void prolong_layers(const LevelDev<T> &F, const LinkDev &K,
                                               const T *__restrict__ ec, T *__restrict__ u, int t,
                                               int k0, int k1)
{
    const int nf = F.nlon, nc = nf / 2;
    const int npair = nc * F.nlat;
    if (t >= npair) return;
    const int j = t / nc, I = t - j * nc;
    const int Im = (I == 0) ? nc - 1 : I - 1;
    const int Ip = (I + 1 == nc) ? 0 : I + 1;
    const int Ja = __ldg(K.j0 + j), Jb = __ldg(K.j1 + j);
    const size_t plane_c = (size_t)nc * K.nlat_c, plane_f = (size_t)nf * F.nlat;
    const T q1 = T(0.25), q3 = T(0.75);
    const T wa = (T)__ldg(K.w0 + j);
    const T wb = Jb >= 0 ? (T)__ldg(K.w1 + j) : T(0);
    const size_t oa = (size_t)Ja * nc, ob = (size_t)(Jb >= 0 ? Jb : Ja) * nc;
    const size_t of = (size_t)j * nf + 2 * I;
#pragma unroll 1
    for (int k = k0; k < k1; ++k) {
        const T *ek = ec + (size_t)k * plane_c;
        const T *ea = ek + oa;
        const T ca = __ldg(ea + I);
        T a0 = wa * fma(q3, ca, q1 * __ldg(ea + Im));
        T a1 = wa * fma(q3, ca, q1 * __ldg(ea + Ip));
        if (Jb >= 0) {
            const T *eb = ek + ob;
            const T cb = __ldg(eb + I);
            a0 = fma(wb, fma(q3, cb, q1 * __ldg(eb + Im)), a0);
            a1 = fma(wb, fma(q3, cb, q1 * __ldg(eb + Ip)), a1);
        }
        T *uk = u + (size_t)k * plane_f + of;
        uk[0] += a0;
        uk[1] += a1;
    }
}

// ------------------------------------------------------------------ residual + restriction
template <typename T>
struct Pair;
template <>
struct Pair<float> {
    using type = float2;
};
template <>
struct Pair<double> {
    using type = double2;
};

template <typename T>
__device__ __forceinline__ typename Pair<T>::type ld_pair(const T *p)
{
    return __ldg(reinterpret_cast<const typename Pair<T>::type *>(p));
}


// b_c = R (b - H u) on one layer k, for a band of kRRBand coarse rows
// [Jb, Je) and one coarse column per lane: lanes 1..30 of a warp own coarse
// columns 30 w .. 30 w + 29 (w: the warp's index along longitude), lanes 0
// and 31 carry the neighbouring columns (periodic).  A lane walks the fine
// rows of the band's gather lists northward and, per row, forms
//   * the residual of its fine columns 2I and 2I+1: the stencil of
//     stencil_column with the same operations in the same order, the outer
//     east/west values and the west face coupling taken from the adjacent
//     lanes;
//   * the longitude sum of the restriction, 1/4 r[2I-1] + 3/4 (r[2I] +
//     r[2I+1]) + 1/4 r[2I+2], the outer residuals from the adjacent lanes;
//   * its latitude contributions w0 (row j0) and w1 (row j1) of the
//     prolongation links (R = P^T) to the at most three coarse rows still
//     open, storing a coarse row once its last listed fine row has passed.
// Each coarse value is the sum restrict_layers forms over the residual
// stencil_column writes, term for term and in the same order, so the result
// equals the two kernels' exactly; the residual never reaches memory.  The
// fine rows shared by two bands are computed in both.  All 32 lanes of the
// warp call it (whole warps past the last column return together); b, u and
// the coefficient arrays aligned to two values.
// PRE: u is the sweep of Eq. (1) from zero, u = omega H_z^{-1} b, whose
// residual is (1 - omega) b plus the four horizontal couplings of u (H_z u =
// omega b cancels everything else; om1 = 1 - omega): the same walk without
// h, t_z and the layers above and below, terms added east, west, north,
// south.
template <typename T, bool PRE = false>
__device__ __forceinline__ void resid_restrict_band(const LevelDev<T> &F, const LinkDev &K,
                                                    const T *__restrict__ b,
                                                    const T *__restrict__ u, T *__restrict__ bc,
                                                    int warp, int lane, int Jb, int k,
                                                    T om1 = T(0), int band = kRRBand)
{
    using P2 = typename Pair<T>::type;
    constexpr unsigned kAll = 0xffffffffu;
    const int nf = F.nlon, nc = nf / 2, nlat = F.nlat, nz = F.nz, ncJ = K.nlat_c;
    const int Iown = warp * kRROwned + lane - 1;
    const bool owned = lane >= 1 && lane <= kRROwned && Iown < nc;
    int I = Iown < 0 ? Iown + nc : (Iown >= nc ? Iown - nc : Iown);
    if (I >= nc) I = nc - 1;  // past the east neighbour of the last column: unused
    const int Je = min(ncJ, Jb + band);
    const size_t plane = (size_t)nf * nlat, plane_c = (size_t)nc * ncJ;
    const size_t o = (size_t)k * plane + 2 * I;
    const bool up = k + 1 < nz, dn = k > 0;
    const T *uk = u + o, *bk = b + o, *hk = F.h + o, *txk = F.tx + o, *tyk = F.ty + o;
    const T *tzk = F.tz + o;
    const T *uu = up ? uk + plane : uk, *ud = dn ? uk - plane : uk, *tzd = dn ? tzk - plane : tzk;
    T *out = bc + (size_t)k * plane_c + (owned ? Iown : 0);
    const int jfirst = __ldg(K.rrow + __ldg(K.rptr + Jb));
    const int jlast = __ldg(K.rrow + __ldg(K.rptr + Je) - 1);
    const T q1 = T(0.25), q3 = T(0.75);
    int Jlo = Jb;                                          // lowest open coarse row
    int lastlo = __ldg(K.rrow + __ldg(K.rptr + Jlo + 1) - 1);  // its last fine row
    T a0 = 0, a1 = 0, a2 = 0;                              // rows Jlo, Jlo + 1, Jlo + 2
    P2 zero;
    zero.x = zero.y = T(0);
    P2 Us = jfirst > 0 ? ld_pair(uk + (size_t)(jfirst - 1) * nf) : zero;
    P2 Tys = jfirst > 0 ? ld_pair(tyk + (size_t)(jfirst - 1) * nf) : zero;
    P2 Uc = ld_pair(uk + (size_t)jfirst * nf);
    // The FP32 PRE form has little arithmetic per row to cover its loads, so
    // it issues the next row's loads (u and t_y one row north, b and t_x on
    // the row) before combining this one: two rows in flight per thread.  The
    // full residual, and FP64 (ALU-bound), keep one row.
    constexpr bool kAhead = PRE && sizeof(T) == 4;
    P2 nUn = zero, nB = zero, nTX = zero, nTYN = zero;
    if (kAhead) {
        const size_t o0 = (size_t)jfirst * nf;
        nUn = jfirst + 1 < nlat ? ld_pair(uk + o0 + nf) : zero;
        nB = ld_pair(bk + o0);
        nTX = ld_pair(txk + o0);
        nTYN = jfirst + 1 < nlat ? ld_pair(tyk + o0) : zero;
    }
#pragma unroll 1
    for (int j = jfirst; j <= jlast; ++j) {
        const bool hasN = j + 1 < nlat, hasS = j > 0;
        const size_t oj = (size_t)j * nf;
        P2 Un, B, TX, TYN;
        if (kAhead) {
            Un = nUn;
            B = nB;
            TX = nTX;
            TYN = nTYN;
            if (j < jlast) {
                const size_t o1 = oj + nf;
                const bool n1 = j + 2 < nlat;
                nUn = n1 ? ld_pair(uk + o1 + nf) : zero;
                nB = ld_pair(bk + o1);
                nTX = ld_pair(txk + o1);
                nTYN = n1 ? ld_pair(tyk + o1) : zero;
            }
        } else {
            Un = hasN ? ld_pair(uk + oj + nf) : zero;
            B = ld_pair(bk + oj);
            TX = ld_pair(txk + oj);
            TYN = hasN ? ld_pair(tyk + oj) : zero;
        }
        const T uw = __shfl_up_sync(kAll, Uc.y, 1);    // u[2I-1]
        const T ue = __shfl_down_sync(kAll, Uc.x, 1);  // u[2I+2]
        const T txw = __shfl_up_sync(kAll, TX.y, 1);   // t_x[2I-1], west face of 2I
        T r0, r1;
        if (PRE) {
            r0 = om1 * B.x;
            r0 = fma(TX.x, Uc.y, r0);
            r0 = fma(txw, uw, r0);
            if (hasN) r0 = fma(TYN.x, Un.x, r0);
            if (hasS) r0 = fma(Tys.x, Us.x, r0);
            r1 = om1 * B.y;
            r1 = fma(TX.y, ue, r1);
            r1 = fma(TX.x, Uc.x, r1);
            if (hasN) r1 = fma(TYN.y, Un.y, r1);
            if (hasS) r1 = fma(Tys.y, Us.y, r1);
        } else {
            const P2 Hh = ld_pair(hk + oj), TZ = ld_pair(tzk + oj);
            const P2 TZD = dn ? ld_pair(tzd + oj) : zero;
            const P2 UU = up ? ld_pair(uu + oj) : zero;
            const P2 UD = dn ? ld_pair(ud + oj) : zero;
            T v0 = Hh.x * Uc.x;
            v0 = fma(TX.x, Uc.x - Uc.y, v0);
            v0 = fma(txw, Uc.x - uw, v0);
            if (hasN) v0 = fma(TYN.x, Uc.x - Un.x, v0);
            if (hasS) v0 = fma(Tys.x, Uc.x - Us.x, v0);
            v0 = fma(TZ.x, Uc.x - UU.x, v0);
            v0 = fma(TZD.x, Uc.x - UD.x, v0);
            T v1 = Hh.y * Uc.y;
            v1 = fma(TX.y, Uc.y - ue, v1);
            v1 = fma(TX.x, Uc.y - Uc.x, v1);
            if (hasN) v1 = fma(TYN.y, Uc.y - Un.y, v1);
            if (hasS) v1 = fma(Tys.y, Uc.y - Us.y, v1);
            v1 = fma(TZ.y, Uc.y - UU.y, v1);
            v1 = fma(TZD.y, Uc.y - UD.y, v1);
            r0 = B.x - v0;
            r1 = B.y - v1;
        }
        const T rw = __shfl_up_sync(kAll, r1, 1);    // r[2I-1]
        const T re = __shfl_down_sync(kAll, r0, 1);  // r[2I+2]
        const T sv = fma(q1, rw + re, q3 * (r0 + r1));
        while (j > lastlo) {  // Jlo has all its rows
            if (owned) out[(size_t)Jlo * nc] = a0;
            a0 = a1;
            a1 = a2;
            a2 = T(0);
            ++Jlo;
            lastlo = Jlo < Je ? __ldg(K.rrow + __ldg(K.rptr + Jlo + 1) - 1) : 0x7fffffff;
        }
        const int J0 = __ldg(K.j0 + j), J1 = __ldg(K.j1 + j);
        if (J0 >= Jb && J0 < Je) {
            const T w = (T)__ldg(K.w0 + j);
            const int d = J0 - Jlo;
            if (d == 0) a0 = fma(w, sv, a0);
            else if (d == 1) a1 = fma(w, sv, a1);
            else a2 = fma(w, sv, a2);
        }
        if (J1 >= Jb && J1 < Je) {
            const T w = (T)__ldg(K.w1 + j);
            const int d = J1 - Jlo;
            if (d == 0) a0 = fma(w, sv, a0);
            else if (d == 1) a1 = fma(w, sv, a1);
            else a2 = fma(w, sv, a2);
        }
        Us = Uc;
        Uc = Un;
        Tys = TYN;
    }
    while (Jlo < Je) {
        if (owned) out[(size_t)Jlo * nc] = a0;
        a0 = a1;
        a1 = a2;
        a2 = T(0);
        ++Jlo;
    }
}

}  // namespace tpmg
