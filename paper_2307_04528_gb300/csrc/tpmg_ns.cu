// Kernels of the nonsymmetric (directed-coupling) operator: the solve kernels in FP64
// and FP32, the setup kernels in FP64.
//
// Every face carries two couplings, one for each row it enters (the row's
// own coupling to its east / north / upper neighbour, and the neighbour
// row's coupling back).  A kernel sees one operator through an NsView: H
// reads (h, tx, ty, tz, txr, tyr, tzr), H^T the same arrays swapped with the
// column sums h^T as mass, so one set of kernels applies, smooths and
// coarsens both, and the transposed apply is a transposed-stencil read of
// H's own arrays.  Layout and traversal as the symmetric kernels: fields
// [nz][nlat][nlon], one thread per column walking the layers (the column
// solve of Eq. (1) is sequential in k), longitude fastest so that a warp's
// loads of one layer are one coalesced segment.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "tpmg_internal.h"

namespace tpmg {
namespace {

// Columns per block of the sweep.
constexpr int kNsSmoothBlock = 64;
constexpr int kNsCellBlock = 256;

struct Col {
    int j, i, ie, iw;
    bool hasN, hasS;
};

__device__ __forceinline__ Col col_of(int col, int nlon, int nlat)
{
    Col c;
    c.j = col / nlon;
    c.i = col - c.j * nlon;
    c.ie = (c.i + 1 == nlon) ? col - c.i : col + 1;
    c.iw = (c.i == 0) ? col + nlon - 1 : col - 1;
    c.hasN = c.j + 1 < nlat;
    c.hasS = c.j > 0;
    return c;
}

// (A x)_c = h x_c + e (x_c - x_E) + w[W] (x_c - x_W) + n (x_c - x_N)
//           + s[S] (x_c - x_S) + u (x_c - x_U) + d[D] (x_c - x_D)
// The loads of layers k+1 .. k+kStDepth-1 are in flight while layer k is
// combined (a register pipeline, as the symmetric stencil's).
constexpr int kStDepth = 2;

template <typename T>
struct StLoads {
    T xc, h, e, w, n, s, u, d, xe, xw, xn, xs, b;
};

template <typename T, int MODE>
__device__ __forceinline__ void st_load(StLoads<T> &L, const NsView<T> &V, const T *__restrict__ b,
                                        const T *__restrict__ x, size_t o, int col, const Col &c,
                                        int nlon)
{
    L.xc = __ldg(x + o + col);
    L.h = __ldg(V.h + o + col);
    L.e = __ldg(V.e + o + col);
    L.w = __ldg(V.w + o + c.iw);
    L.u = __ldg(V.u + o + col);
    L.d = __ldg(V.d + o + col);
    L.xe = __ldg(x + o + c.ie);
    L.xw = __ldg(x + o + c.iw);
    L.n = c.hasN ? __ldg(V.n + o + col) : T(0);
    L.xn = c.hasN ? __ldg(x + o + col + nlon) : T(0);
    L.s = c.hasS ? __ldg(V.s + o + col - nlon) : T(0);
    L.xs = c.hasS ? __ldg(x + o + col - nlon) : T(0);
    if (MODE) L.b = __ldg(b + o + col);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kBlock)
k_ns_stencil(NsView<T> V, const T *__restrict__ b, const T *__restrict__ x, T *__restrict__ y)
{
    const int nlon = V.nlon, nlat = V.nlat, nz = V.nz, ncol = nlon * nlat;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const Col c = col_of(col, nlon, nlat);
    const size_t plane = (size_t)ncol;
    StLoads<T> st[kStDepth];
#pragma unroll
    for (int q = 0; q < kStDepth; ++q)
        if (q < nz) st_load<T, MODE>(st[q], V, b, x, (size_t)q * plane, col, c, nlon);
    T xdn = 0, ddn = 0;
    for (int k0 = 0; k0 < nz; k0 += kStDepth) {
#pragma unroll
        for (int q = 0; q < kStDepth; ++q) {
            const int k = k0 + q;
            if (k < nz) {
                const StLoads<T> &L = st[q];
                const T xc = L.xc;
                T v = L.h * xc;
                v = fma(L.e, xc - L.xe, v);
                v = fma(L.w, xc - L.xw, v);
                if (c.hasN) v = fma(L.n, xc - L.xn, v);
                if (c.hasS) v = fma(L.s, xc - L.xs, v);
                if (k + 1 < nz) v = fma(L.u, xc - st[(q + 1) % kStDepth].xc, v);
                if (k > 0) v = fma(ddn, xc - xdn, v);
                y[(size_t)k * plane + col] = MODE ? L.b - v : v;
                ddn = L.d;  // coupling of the row above back to this layer
                xdn = xc;
                if (k + kStDepth < nz)
                    st_load<T, MODE>(st[q], V, b, x, (size_t)(k + kStDepth) * plane, col, c, nlon);
            }
        }
    }
}

// r = (1 - omega) b + e u_E + w[W] u_W + n u_N + s[S] u_S
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_ns_presmooth_resid(NsView<T> V, const T *__restrict__ b, const T *__restrict__ u, T om1,
                     T *__restrict__ r)
{
    const int nlon = V.nlon, nlat = V.nlat, ncol = nlon * nlat;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const Col c = col_of(col, nlon, nlat);
    const size_t plane = (size_t)ncol;
    for (int k = 0; k < V.nz; ++k) {
        const size_t o = (size_t)k * plane;
        T v = om1 * __ldg(b + o + col);
        v = fma(__ldg(V.e + o + col), __ldg(u + o + c.ie), v);
        v = fma(__ldg(V.w + o + c.iw), __ldg(u + o + c.iw), v);
        if (c.hasN) v = fma(__ldg(V.n + o + col), __ldg(u + o + col + nlon), v);
        if (c.hasS) v = fma(__ldg(V.s + o + col - nlon), __ldg(u + o + col - nlon), v);
        r[o + col] = v;
    }
}

// One sweep of Eq. (1) on a column: forward y_k = (v_k + l_k y_{k-1}) / p_k
// with l_k = d[k-1] (the row's coupling to the layer below) and v = b plus the
// horizontal couplings of u_in; backward x_k = x_{k+1} + (y_k - (q_k/p_k)
// x_{k+1}); u_out = (1 - omega) u_in + omega x.  With a guess, register
// pipelines of kFwdDepth layers forward and kBackDepth backward (3.61 -> 2.53
// ms at 1536x1152x70).  The forward values wait in the thread's own column
// of u_out, which the backward pass overwrites (the reads hit L2): without a
// shared-memory buffer the block count is no longer capped at 6 per SM
// (1536x1152x70: 2.53 -> 2.33 ms with a guess, 1.60 -> 1.18 ms from zero).
// No block barrier: a thread past the last column returns at once.
constexpr int kFwdDepth = 3;
constexpr int kBackDepth = 4;

template <typename T>
struct SmLoads {
    T b, e, w, n, s, ue, uw, un, us, m, d;
};

template <typename T>
__device__ __forceinline__ void sm_load(SmLoads<T> &L, const NsView<T> &V, const T *__restrict__ b,
                                        const T *__restrict__ uin, size_t o, int col,
                                        const Col &c, int nlon)
{
    L.b = __ldg(b + o + col);
    L.m = __ldg(V.m + o + col);
    L.d = __ldg(V.d + o + col);
    L.e = __ldg(V.e + o + col);
    L.w = __ldg(V.w + o + c.iw);
    L.ue = __ldg(uin + o + c.ie);
    L.uw = __ldg(uin + o + c.iw);
    L.n = c.hasN ? __ldg(V.n + o + col) : T(0);
    L.un = c.hasN ? __ldg(uin + o + col + nlon) : T(0);
    L.s = c.hasS ? __ldg(V.s + o + col - nlon) : T(0);
    L.us = c.hasS ? __ldg(uin + o + col - nlon) : T(0);
}

// The sweep from zero (3 loads per layer) as a plain walk: with the forward
// values in shared memory it ran 1.59 ms at 1536x1152x70 against 1.82-1.94
// ms with 4-12 layers of loads in flight (FP64).
template <typename T>
__global__ void __launch_bounds__(kNsSmoothBlock)
k_ns_smooth0(NsView<T> V, const T *__restrict__ b, T *__restrict__ uout, T omega)
{
    const int ncol = V.nlon * V.nlat, nz = V.nz;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const size_t plane = (size_t)ncol;
    T yprev = 0, ldn = 0;
    for (int k = 0; k < nz; ++k) {
        const size_t o = (size_t)k * plane + col;
        const T y = fma(ldn, yprev, __ldg(b + o)) * __ldg(V.m + o);
        uout[o] = y;  // forward value, overwritten on the way back
        yprev = y;
        ldn = __ldg(V.d + o);
    }
    T xk = yprev;
    for (int k = nz - 1; k >= 0; --k) {
        const size_t o = (size_t)k * plane + col;
        if (k < nz - 1) xk = xk + fma(-__ldg(V.dq + o), xk, uout[o]);
        uout[o] = omega * xk;
    }
}

template <typename T>
__global__ void __launch_bounds__(kNsSmoothBlock)
k_ns_smooth(NsView<T> V, const T *__restrict__ b, const T *__restrict__ uin, T *__restrict__ uout,
            T omega)
{
    const int nlon = V.nlon, nlat = V.nlat, nz = V.nz, ncol = nlon * nlat;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const Col c = col_of(col, nlon, nlat);
    const size_t plane = (size_t)ncol;
    SmLoads<T> st[kFwdDepth];
#pragma unroll
    for (int q = 0; q < kFwdDepth; ++q)
        if (q < nz) sm_load<T>(st[q], V, b, uin, (size_t)q * plane, col, c, nlon);
    T yprev = 0, ldn = 0;
    for (int k0 = 0; k0 < nz; k0 += kFwdDepth) {
#pragma unroll
        for (int q = 0; q < kFwdDepth; ++q) {
            const int k = k0 + q;
            if (k < nz) {
                const SmLoads<T> &L = st[q];
                T v = L.b;
                v = fma(L.e, L.ue, v);
                v = fma(L.w, L.uw, v);
                v = fma(L.n, L.un, v);
                v = fma(L.s, L.us, v);
                const T y = fma(ldn, yprev, v) * L.m;
                uout[(size_t)k * plane + col] = y;  // forward value
                yprev = y;
                ldn = L.d;
                if (k + kFwdDepth < nz)
                    sm_load<T>(st[q], V, b, uin, (size_t)(k + kFwdDepth) * plane, col, c, nlon);
            }
        }
    }
    const T om1 = T(1) - omega;
    T xk = yprev;
    T dqp[kBackDepth], up[kBackDepth];
#pragma unroll
    for (int q = 0; q < kBackDepth; ++q) {
        const int k = nz - 1 - q;
        if (k >= 0) {
            dqp[q] = __ldg(V.dq + (size_t)k * plane + col);
            up[q] = __ldg(uin + (size_t)k * plane + col);
        }
    }
    for (int k0 = nz - 1; k0 >= 0; k0 -= kBackDepth) {
#pragma unroll
        for (int q = 0; q < kBackDepth; ++q) {
            const int k = k0 - q;
            if (k >= 0) {
                const size_t o = (size_t)k * plane + col;
                if (k < nz - 1) xk = xk + fma(-dqp[q], xk, uout[o]);
                uout[o] = fma(om1, up[q], omega * xk);
                const int kn = k - kBackDepth;
                if (kn >= 0) {
                    const size_t on = (size_t)kn * plane + col;
                    dqp[q] = __ldg(V.dq + on);
                    up[q] = __ldg(uin + on);
                }
            }
        }
    }
}

// Column factors: s = h + e + w[W] + n + s[S]; q_0 = s_0, q_k = s_k + l_k
// q_{k-1} / p_{k-1} (l_k = d[k-1]), p_k = q_k + u_k; m = 1/p, dq = q/p.
__global__ void __launch_bounds__(kBlock)
k_ns_column_lu(NsView<double> V, double *__restrict__ m, double *__restrict__ dq)
{
    const int nlon = V.nlon, nlat = V.nlat, ncol = nlon * nlat;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const Col c = col_of(col, nlon, nlat);
    const size_t plane = (size_t)ncol;
    double qp = 0.0, pp = 1.0, ldn = 0.0;
    for (int k = 0; k < V.nz; ++k) {
        const size_t o = (size_t)k * plane;
        double sv = V.h[o + col] + V.e[o + col] + V.w[o + c.iw] + V.n[o + col];
        if (c.hasS) sv += V.s[o + col - nlon];
        const double q = (k == 0) ? sv : sv + ldn * qp / pp;
        const double p = q + V.u[o + col];
        m[o + col] = 1.0 / p;
        dq[o + col] = q / p;
        qp = q;
        pp = p;
        ldn = V.d[o + col];
    }
}

// h^T = h + (e - w) + (w[W] - e[W]) + (n - s) + (s[S] - n[S]) + (u - d) + (d[D] - u[D])
// of the forward view (e, n, u = tx, ty, tz; w, s, d = txr, tyr, tzr).
__global__ void __launch_bounds__(kNsCellBlock)
k_ns_colmass(NsView<double> V, double *__restrict__ hT)
{
    const int nlon = V.nlon, nlat = V.nlat, ncol = nlon * nlat;
    const size_t n = (size_t)ncol * V.nz;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int k = (int)(idx / ncol), col = (int)(idx - (size_t)k * ncol);
    const Col c = col_of(col, nlon, nlat);
    const size_t o = (size_t)k * ncol;
    double v = V.h[idx] + (V.e[idx] - V.w[idx]);
    v = v + (V.w[o + c.iw] - V.e[o + c.iw]);
    v = v + (V.n[idx] - V.s[idx]);
    if (c.hasS) v = v + (V.s[idx - nlon] - V.n[idx - nlon]);
    v = v + (V.u[idx] - V.d[idx]);
    if (k > 0) v = v + (V.d[idx - ncol] - V.u[idx - ncol]);
    hT[idx] = v;
}

// One thread per coarse column walks the layers: sums over the 2 x cnt
// children, the east faces of the odd fine columns, the top child row's
// north faces; lon faces x sx, lat faces x sy[J] (0 on the last row).
__global__ void __launch_bounds__(kBlock)
k_ns_coarsen(NsView<double> F, LinkDev K, double sx, double *__restrict__ hc, double *__restrict__ ec,
             double *__restrict__ nc_, double *__restrict__ uc, double *__restrict__ wc,
             double *__restrict__ sc, double *__restrict__ dc)
{
    const int nf = F.nlon, nci = nf / 2;
    const int ncol_c = nci * K.nlat_c;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol_c) return;
    const int J = col / nci, I = col - J * nci;
    const int j0 = K.cfirst[J], cnt = K.ccnt[J], top = j0 + cnt - 1;
    const size_t plane_f = (size_t)nf * F.nlat, plane_c = (size_t)ncol_c;
    const bool last = J == K.nlat_c - 1;
    const double sy = last ? 0.0 : K.sy[J];
    for (int k = 0; k < F.nz; ++k) {
        const size_t of = (size_t)k * plane_f;
        double hs = 0, us = 0, ds = 0, es = 0, ws = 0;
        for (int j = j0; j <= top; ++j) {
            const size_t a = of + (size_t)j * nf + 2 * I;
            hs += F.h[a];
            hs += F.h[a + 1];
            if (uc) {
                us += F.u[a];
                us += F.u[a + 1];
                ds += F.d[a];
                ds += F.d[a + 1];
                es += F.e[a + 1];
                ws += F.w[a + 1];
            }
        }
        const size_t oc = (size_t)k * plane_c + col;
        hc[oc] = hs;
        if (!uc) continue;
        const size_t t = of + (size_t)top * nf + 2 * I;
        double ns = 0, ss = 0;
        ns += F.n[t];
        ns += F.n[t + 1];
        ss += F.s[t];
        ss += F.s[t + 1];
        uc[oc] = us;
        dc[oc] = ds;
        ec[oc] = es * sx;
        wc[oc] = ws * sx;
        nc_[oc] = last ? 0.0 : ns * sy;
        sc[oc] = last ? 0.0 : ss * sy;
    }
}

__device__ __forceinline__ bool ok_coupling(double t) { return t >= 0.0 && isfinite(t); }

// bits: 1 h <= 0 or non-finite, 2 a coupling < 0 or non-finite, 4 a non-zero
// pole or top face
__global__ void __launch_bounds__(kNsCellBlock)
k_ns_validate(NsView<double> V, int *__restrict__ flag)
{
    const int ncol = V.nlon * V.nlat;
    const size_t n = (size_t)ncol * V.nz;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int k = (int)(idx / ncol), col = (int)(idx - (size_t)k * ncol);
    const int j = col / V.nlon;
    int bits = 0;
    const double h = V.h[idx];
    if (!(h > 0.0) || !isfinite(h)) bits |= 1;
    const double e = V.e[idx], nn = V.n[idx], u = V.u[idx];
    const double w = V.w[idx], s = V.s[idx], d = V.d[idx];
    if (!ok_coupling(e) || !ok_coupling(nn) || !ok_coupling(u) || !ok_coupling(w) ||
        !ok_coupling(s) || !ok_coupling(d))
        bits |= 2;
    if (j == V.nlat - 1 && (nn != 0.0 || s != 0.0)) bits |= 4;
    if (k == V.nz - 1 && (u != 0.0 || d != 0.0)) bits |= 4;
    if (bits) atomicOr(flag, bits);
}

__global__ void __launch_bounds__(kNsCellBlock)
k_ns_positive(const double *__restrict__ a, size_t n, int *__restrict__ flag)
{
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const double v = a[idx];
    if (!(v > 0.0) || !isfinite(v)) atomicOr(flag, 8);
}

// dL/dtheta = -lam^T (dH/dtheta) x per array entry
__global__ void __launch_bounds__(kNsCellBlock)
k_ns_coeff_grad(int nlon, int nlat, int nz, const double *__restrict__ lam,
                const double *__restrict__ x, double *__restrict__ gh, double *__restrict__ gtx,
                double *__restrict__ gty, double *__restrict__ gtz, double *__restrict__ gtxr,
                double *__restrict__ gtyr, double *__restrict__ gtzr)
{
    const int ncol = nlon * nlat;
    const size_t n = (size_t)ncol * nz;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int k = (int)(idx / ncol), col = (int)(idx - (size_t)k * ncol);
    const Col c = col_of(col, nlon, nlat);
    const size_t o = (size_t)k * ncol;
    const double lc = lam[idx], xc = x[idx];
    if (gh) gh[idx] = -lc * xc;
    const double le = lam[o + c.ie], xe = x[o + c.ie];
    if (gtx) gtx[idx] = -lc * (xc - xe);
    if (gtxr) gtxr[idx] = -le * (xe - xc);
    if (c.hasN) {
        const double ln = lam[idx + nlon], xn = x[idx + nlon];
        if (gty) gty[idx] = -lc * (xc - xn);
        if (gtyr) gtyr[idx] = -ln * (xn - xc);
    } else {
        if (gty) gty[idx] = 0.0;
        if (gtyr) gtyr[idx] = 0.0;
    }
    if (k + 1 < nz) {
        const double lu = lam[idx + ncol], xu = x[idx + ncol];
        if (gtz) gtz[idx] = -lc * (xc - xu);
        if (gtzr) gtzr[idx] = -lu * (xu - xc);
    } else {
        if (gtz) gtz[idx] = 0.0;
        if (gtzr) gtzr[idx] = 0.0;
    }
}

template <typename T>
int col_blocks(const NsView<T> &V, int block)
{
    return (V.nlon * V.nlat + block - 1) / block;
}

unsigned cell_blocks(size_t n) { return (unsigned)((n + kNsCellBlock - 1) / kNsCellBlock); }

}  // namespace

template <typename T>
cudaError_t launch_ns_stencil(const NsView<T> &V, int mode, const T *b, const T *x, T *y,
                              cudaStream_t s)
{
    if (mode)
        k_ns_stencil<T, 1><<<col_blocks(V, kBlock), kBlock, 0, s>>>(V, b, x, y);
    else
        k_ns_stencil<T, 0><<<col_blocks(V, kBlock), kBlock, 0, s>>>(V, b, x, y);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ns_presmooth_resid(const NsView<T> &V, const T *b, const T *u, double omega,
                                      T *r, cudaStream_t s)
{
    k_ns_presmooth_resid<T><<<col_blocks(V, kBlock), kBlock, 0, s>>>(V, b, u, T(1.0 - omega), r);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ns_smooth(const NsView<T> &V, const T *b, const T *u_in, T *u_out,
                             double omega, cudaStream_t s)
{
    const int grid = col_blocks(V, kNsSmoothBlock);
    if (u_in)
        k_ns_smooth<T><<<grid, kNsSmoothBlock, 0, s>>>(V, b, u_in, u_out, (T)omega);
    else
        k_ns_smooth0<T><<<grid, kNsSmoothBlock, 0, s>>>(V, b, u_out, (T)omega);
    return cudaGetLastError();
}

#define TPMG_NS_INSTANTIATE(T)                                                                \
    template cudaError_t launch_ns_stencil<T>(const NsView<T> &, int, const T *, const T *, T *, \
                                              cudaStream_t);                                  \
    template cudaError_t launch_ns_presmooth_resid<T>(const NsView<T> &, const T *, const T *, \
                                                      double, T *, cudaStream_t);             \
    template cudaError_t launch_ns_smooth<T>(const NsView<T> &, const T *, const T *, T *,     \
                                             double, cudaStream_t);
TPMG_NS_INSTANTIATE(double)
TPMG_NS_INSTANTIATE(float)
#undef TPMG_NS_INSTANTIATE

cudaError_t launch_ns_column_lu(const NsView<double> &V, double *m, double *dq, cudaStream_t s)
{
    k_ns_column_lu<<<col_blocks(V, kBlock), kBlock, 0, s>>>(V, m, dq);
    return cudaGetLastError();
}

cudaError_t launch_ns_colmass(const NsView<double> &V, double *hT, cudaStream_t s)
{
    const size_t n = (size_t)V.nlon * V.nlat * V.nz;
    k_ns_colmass<<<cell_blocks(n), kNsCellBlock, 0, s>>>(V, hT);
    return cudaGetLastError();
}

cudaError_t launch_ns_coarsen(const NsView<double> &F, const LinkDev &K, double sx, double *h,
                              double *e, double *n, double *u, double *w, double *sv, double *d,
                              cudaStream_t s)
{
    const int ncol_c = (F.nlon / 2) * K.nlat_c;
    k_ns_coarsen<<<(ncol_c + kBlock - 1) / kBlock, kBlock, 0, s>>>(F, K, sx, h, e, n, u, w, sv,
                                                                   d);
    return cudaGetLastError();
}

cudaError_t launch_ns_validate(const NsView<double> &V, int *flag, cudaStream_t s)
{
    const size_t n = (size_t)V.nlon * V.nlat * V.nz;
    k_ns_validate<<<cell_blocks(n), kNsCellBlock, 0, s>>>(V, flag);
    return cudaGetLastError();
}

cudaError_t launch_ns_positive(const double *a, size_t n, int *flag, cudaStream_t s)
{
    k_ns_positive<<<cell_blocks(n), kNsCellBlock, 0, s>>>(a, n, flag);
    return cudaGetLastError();
}

cudaError_t launch_ns_coeff_grad(int nlon, int nlat, int nz, const double *lam, const double *x,
                                 double *gh, double *gtx, double *gty, double *gtz,
                                 double *gtxr, double *gtyr, double *gtzr, cudaStream_t s)
{
    const size_t n = (size_t)nlon * nlat * nz;
    k_ns_coeff_grad<<<cell_blocks(n), kNsCellBlock, 0, s>>>(nlon, nlat, nz, lam, x, gh, gtx, gty,
                                                            gtz, gtxr, gtyr, gtzr);
    return cudaGetLastError();
}

}  // namespace tpmg
