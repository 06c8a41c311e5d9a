// Device-side bodies of the multigrid kernels, shared by the single-system
// kernels (tpmg_kernels.cu) and the batched persistent kernels
// (tpmg_batch.cu).  One thread owns one vertical column (or one cell) of one
// level; see tpmg_kernels.cu for the layout and the arithmetic.
#pragma once

#include <cuda_runtime.h>

#include "tpmg_internal.h"

namespace tpmg {

// ------------------------------------------------------------------ reductions
template <int OP>  // 0: sum, 1: max
__device__ __forceinline__ double warp_reduce(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double w = __shfl_down_sync(0xffffffffu, v, o);
        v = OP == 0 ? v + w : fmax(v, w);
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
// sum(x*y) (MODE 0) when RED.
template <typename T, int MODE, bool RED>
__device__ __forceinline__ T stencil_column(const LevelDev<T> &L, const T *__restrict__ b,
                                            const T *__restrict__ x, T *__restrict__ y, int col)
{
    const int nlon = L.nlon, nlat = L.nlat, nz = L.nz;
    const int ncol = nlon * nlat;
    T acc = 0;
    if (col < ncol) {
        const int j = col / nlon, i = col - j * nlon;
        const int ie = (i + 1 == nlon) ? col - i : col + 1;
        const int iw = (i == 0) ? col + nlon - 1 : col - 1;
        const bool hasN = j + 1 < nlat, hasS = j > 0;
        const size_t plane = (size_t)ncol;
        T xdn = 0, tdn = 0;
        T xc = x[col];
        for (int k = 0; k < nz; ++k) {
            const size_t o = (size_t)k * plane;
            const T xup = (k + 1 < nz) ? x[o + plane + col] : T(0);
            const T tup = L.tz[o + col];
            T v = L.h[o + col] * xc;
            v = fma(L.tx[o + col], xc - x[o + ie], v);
            v = fma(L.tx[o + iw], xc - x[o + iw], v);
            if (hasN) v = fma(L.ty[o + col], xc - x[o + col + nlon], v);
            if (hasS) v = fma(L.ty[o + col - nlon], xc - x[o + col - nlon], v);
            v = fma(tup, xc - xup, v);
            v = fma(tdn, xc - xdn, v);
            const T out = MODE ? b[o + col] - v : v;
            y[o + col] = out;
            if (RED) acc = fma(out, MODE ? out : xc, acc);
            xdn = xc;
            xc = xup;
            tdn = tup;
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
// pivots p_k = q_k + t_k:
//   forward   y_k = (v_k + t_{k-1} y_{k-1}) / p_k
//   backward  x_k = x_{k+1} + (y_k - (q_k / p_k) x_{k+1})
// PRE: 1/p_k and q_k/p_k read from the setup factors; otherwise
// q_k = s_k + t_{k-1} q_{k-1}/p_{k-1} is formed on the fly.  The forward
// values y (and q/p on the fly) wait in shared memory for the backward sweep:
// blockDim x nz values per array.
//
// Shared memory caps residency at ~3 blocks of 128 columns per SM, so the
// loads of layers k+1..k+DEPTH are issued before layer k is computed (a
// register pipeline) to keep enough bytes in flight to cover HBM latency:
// deeper for the FP32 sweeps (few registers per layer, HBM-bound), shallow
// for FP64 (FP64-ALU-bound, twice the registers per value).
template <typename T, bool ZERO>
struct SmoothDepth {
    static constexpr int value = sizeof(T) == 8 ? (ZERO ? 4 : 3) : (ZERO ? 4 : 6);
};

template <typename T>
struct SmoothLoads {
    T b, tz, m, h, txc, txw, tyn, tys, ue, uw, un, us;
};

template <typename T, bool ZERO, bool PRE>
__device__ __forceinline__ void smooth_load(SmoothLoads<T> &s, const LevelDev<T> &L,
                                            const T *__restrict__ b, const T *__restrict__ uin,
                                            size_t o, int col, int ie, int iw, int nlon, bool hasN,
                                            bool hasS)
{
    s.b = __ldg(b + o + col);
    s.tz = __ldg(L.tz + o + col);
    if (PRE) s.m = __ldg(L.m + o + col);
    if (!PRE) s.h = __ldg(L.h + o + col);
    if (!ZERO || !PRE) {
        s.txc = __ldg(L.tx + o + col);
        s.txw = __ldg(L.tx + o + iw);
        s.tyn = hasN ? __ldg(L.ty + o + col) : T(0);
        s.tys = hasS ? __ldg(L.ty + o + col - nlon) : T(0);
    }
    if (!ZERO) {
        s.ue = __ldg(uin + o + ie);
        s.uw = __ldg(uin + o + iw);
        s.un = hasN ? __ldg(uin + o + col + nlon) : T(0);
        s.us = hasS ? __ldg(uin + o + col - nlon) : T(0);
    }
}

// One column of the sweep.  smraw: this block's dynamic shared memory
// (nz * blockDim values of T per stored array).
template <typename T, bool ZERO, bool PRE>
__device__ __forceinline__ void smooth_column(const LevelDev<T> &L, const T *__restrict__ b,
                                              const T *__restrict__ uin, T *__restrict__ uout,
                                              T omega, int col, unsigned char *smraw)
{
    constexpr int kDepth = SmoothDepth<T, ZERO>::value;
    const int nlon = L.nlon, nlat = L.nlat, nz = L.nz;
    const int bd = blockDim.x, tid = threadIdx.x;
    T *ys = reinterpret_cast<T *>(smraw);
    T *ds = ys + (size_t)nz * bd;
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
            smooth_load<T, ZERO, PRE>(st[d], L, b, uin, (size_t)d * plane, col, ie, iw, nlon,
                                      hasN, hasS);

    T yprev = 0, tdn = 0, dprev = 0;
    for (int k0 = 0; k0 < nz; k0 += kDepth) {
#pragma unroll
        for (int d = 0; d < kDepth; ++d) {
            const int k = k0 + d;
            if (k < nz) {
                SmoothLoads<T> &c = st[d];
                T v = c.b;
                if (!ZERO) {
                    v = fma(c.txc, c.ue, v);
                    v = fma(c.txw, c.uw, v);
                    v = fma(c.tyn, c.un, v);
                    v = fma(c.tys, c.us, v);
                }
                const T tup = c.tz;
                T y;
                if (PRE) {
                    y = fma(tdn, yprev, v) * c.m;
                } else {
                    const T s = c.h + c.txc + c.txw + c.tyn + c.tys;
                    const T q = (k == 0) ? s : fma(tdn, dprev, s);
                    const T inv = T(1) / (q + tup);
                    y = fma(tdn, yprev, v) * inv;
                    dprev = q * inv;
                    ds[(size_t)k * bd + tid] = dprev;
                }
                ys[(size_t)k * bd + tid] = y;
                yprev = y;
                tdn = tup;
                if (k + kDepth < nz)
                    smooth_load<T, ZERO, PRE>(c, L, b, uin, (size_t)(k + kDepth) * plane, col, ie,
                                              iw, nlon, hasN, hasS);
            }
        }
    }

    const T om1 = T(1) - omega;
    T xk = yprev;
    // backward sweep: prefetch u_in (and the precomputed q/p) kDepth layers ahead
    T up[kDepth], dqp[kDepth];
#pragma unroll
    for (int d = 0; d < kDepth; ++d) {
        const int k = nz - 1 - d;
        if (k >= 0) {
            const size_t o = (size_t)k * plane + col;
            up[d] = ZERO ? T(0) : __ldg(uin + o);
            dqp[d] = PRE ? __ldg(L.dq + o) : T(0);
        }
    }
    for (int k0 = nz - 1; k0 >= 0; k0 -= kDepth) {
#pragma unroll
        for (int d = 0; d < kDepth; ++d) {
            const int k = k0 - d;
            if (k >= 0) {
                const size_t o = (size_t)k * plane + col;
                if (k < nz - 1) {
                    const T dqk = PRE ? dqp[d] : ds[(size_t)k * bd + tid];
                    xk = xk + fma(-dqk, xk, ys[(size_t)k * bd + tid]);
                }
                uout[o] = ZERO ? omega * xk : fma(om1, up[d], omega * xk);
                const int kn = k - kDepth;
                if (kn >= 0) {
                    const size_t on = (size_t)kn * plane + col;
                    if (!ZERO) up[d] = __ldg(uin + on);
                    if (PRE) dqp[d] = __ldg(L.dq + on);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ transfers
// Restriction R = P^T as a gather: coarse (I, J, k) sums, over the fine rows
// listed for J with their latitude weights, the fine residuals at longitudes
// 2I-1, 2I, 2I+1, 2I+2 (mod nlon) with weights 1/4, 3/4, 3/4, 1/4.
// One coarse cell (col, k) of the restriction.
template <typename T>
__device__ __forceinline__ void restrict_cell(const LevelDev<T> &F, const LinkDev &K,
                                              const T *__restrict__ r, T *__restrict__ bc, int col,
                                              int k)
{
    const int nf = F.nlon, nc = nf / 2;
    const int ncol_c = nc * K.nlat_c;
    if (col >= ncol_c) return;
    const int J = col / nc, I = col - J * nc;
    const int i0 = 2 * I, i1 = 2 * I + 1;
    const int im = (i0 == 0) ? nf - 1 : i0 - 1;
    const int ip = (i1 + 1 == nf) ? 0 : i1 + 1;
    const size_t plane_f = (size_t)nf * F.nlat, plane_c = (size_t)ncol_c;
    const int p0 = __ldg(K.rptr + J), p1 = __ldg(K.rptr + J + 1);
    const T q1 = T(0.25), q3 = T(0.75);
    const T *rk = r + (size_t)k * plane_f;
    T acc = 0;
    for (int p = p0; p < p1; ++p) {
        const T *row = rk + (size_t)__ldg(K.rrow + p) * nf;
        const T w = (T)__ldg(K.rw + p);
        acc = fma(w, fma(q1, __ldg(row + im) + __ldg(row + ip), q3 * (__ldg(row + i0) + __ldg(row + i1))),
                  acc);
    }
    bc[(size_t)k * plane_c + col] = acc;
}

// Bilinear prolongation and correction: fine cell 2I adds
// sum_a w_a (3/4 e[J_a, I] + 1/4 e[J_a, I-1]) and 2I+1 adds
// sum_a w_a (3/4 e[J_a, I] + 1/4 e[J_a, I+1]) (periodic in longitude).
// One pair of fine cells (t = j * nlon/2 + I, layer k) of the prolongation.
template <typename T>
__device__ __forceinline__ void prolong_pair(const LevelDev<T> &F, const LinkDev &K,
                                             const T *__restrict__ ec, T *__restrict__ u, int t,
                                             int k)
{
    const int nf = F.nlon, nc = nf / 2;
    const int npair = nc * F.nlat;
    if (t >= npair) return;
    const int j = t / nc, I = t - j * nc;
    const int Im = (I == 0) ? nc - 1 : I - 1;
    const int Ip = (I + 1 == nc) ? 0 : I + 1;
    const int Ja = __ldg(K.j0 + j), Jb = __ldg(K.j1 + j);
    const size_t plane_c = (size_t)nc * K.nlat_c;
    const T q1 = T(0.25), q3 = T(0.75);
    const T *ek = ec + (size_t)k * plane_c;
    const T *ea = ek + (size_t)Ja * nc;
    const T wa = (T)__ldg(K.w0 + j);
    const T ca = __ldg(ea + I);
    T a0 = wa * fma(q3, ca, q1 * __ldg(ea + Im));
    T a1 = wa * fma(q3, ca, q1 * __ldg(ea + Ip));
    if (Jb >= 0) {
        const T *eb = ek + (size_t)Jb * nc;
        const T wb = (T)__ldg(K.w1 + j);
        const T cb = __ldg(eb + I);
        a0 = fma(wb, fma(q3, cb, q1 * __ldg(eb + Im)), a0);
        a1 = fma(wb, fma(q3, cb, q1 * __ldg(eb + Ip)), a1);
    }
    T *uk = u + (size_t)k * nf * F.nlat + (size_t)j * nf + 2 * I;
    uk[0] += a0;
    uk[1] += a1;
}

}  // namespace tpmg
