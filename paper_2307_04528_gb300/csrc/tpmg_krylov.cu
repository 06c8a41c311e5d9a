// Vector steps of the BiCGStab outer iteration (van der Vorst's stabilised
// bi-conjugate gradients with right preconditioning): the comparison solver
// of Section 1 (BiCGStab preconditioned by the vertical line relaxation of
// Eq. (1)) and its multigrid-preconditioned variant, in FP64 and FP32.
//
// Every scalar of the iteration lives on the device (BicgScalars) and is
// formed by one-block finalize kernels from per-block partial sums in a fixed
// order, so an iteration issues no host synchronisation until its residual
// norm is read.  Grid-stride kernels on one wave of full occupancy, like the
// conjugate-gradient vector kernels.
#include <cuda_runtime.h>

#include "tpmg_device.cuh"
#include "tpmg_internal.h"

namespace tpmg {

// FP32 forms on 16-byte vectors (four elements per load and store, the same
// arithmetic per element; partial sums grouped by vector) for lengths that
// are multiples of 4 on 16-byte aligned vectors, as the conjugate-gradient
// vector kernels.
namespace {

struct F4 {
    float v[4];
};

__device__ __forceinline__ F4 ld4(const float *p, size_t i)
{
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p) + i);
    return {{q.x, q.y, q.z, q.w}};
}

__device__ __forceinline__ F4 ld4w(const float *p, size_t i)  // a vector this kernel writes
{
    const float4 q = reinterpret_cast<const float4 *>(p)[i];
    return {{q.x, q.y, q.z, q.w}};
}

__device__ __forceinline__ void st4(float *p, size_t i, const F4 &a)
{
    reinterpret_cast<float4 *>(p)[i] = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}

bool f4_ok(size_t n, const void *a, const void *b, const void *c = nullptr,
           const void *d = nullptr, const void *e = nullptr, const void *f = nullptr,
           const void *g = nullptr)
{
    return n % 4 == 0 && ((uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d |
                          (uintptr_t)e | (uintptr_t)f | (uintptr_t)g) % 16 == 0;
}

#define TPMG_GRID_LOOP4(n4)                                                               \
    _Pragma("unroll 2") for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;   \
                             c < (n4); c += (size_t)gridDim.x * blockDim.x)

template <bool FIRST>
__global__ void __launch_bounds__(kBlock)
k_bicg_dir_f4(float *__restrict__ p, const float *__restrict__ r, const float *__restrict__ v,
              size_t n4, const BicgScalars *sc)
{
    const float beta = FIRST ? 0.f : (float)sc->beta, omega = FIRST ? 0.f : (float)sc->omega;
    TPMG_GRID_LOOP4(n4)
    {
        const F4 rv = ld4(r, c);
        if (FIRST) {
            st4(p, c, rv);
        } else {
            const F4 vv = ld4(v, c);
            F4 pv = ld4w(p, c);
#pragma unroll
            for (int q = 0; q < 4; ++q) pv.v[q] = fmaf(beta, fmaf(-omega, vv.v[q], pv.v[q]), rv.v[q]);
            st4(p, c, pv);
        }
    }
}

__global__ void __launch_bounds__(kBlock)
k_bicg_s_f4(float *__restrict__ sv, const float *__restrict__ r, const float *__restrict__ v,
            size_t n4, const BicgScalars *sc)
{
    const float alpha = (float)sc->alpha;
    TPMG_GRID_LOOP4(n4)
    {
        const F4 rv = ld4(r, c), vv = ld4(v, c);
        F4 o;
#pragma unroll
        for (int q = 0; q < 4; ++q) o.v[q] = fmaf(-alpha, vv.v[q], rv.v[q]);
        st4(sv, c, o);
    }
}

__global__ void __launch_bounds__(kBlock)
k_dot2_f4(const float *__restrict__ t, const float *__restrict__ sv, size_t n4, double *pa,
          double *pb)
{
    float a = 0, b = 0;
    TPMG_GRID_LOOP4(n4)
    {
        const F4 tv = ld4(t, c), s4 = ld4(sv, c);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            a = fmaf(tv.v[q], s4.v[q], a);
            b = fmaf(tv.v[q], tv.v[q], b);
        }
    }
    block_store<0>((double)a, pa);
    block_store<0>((double)b, pb);
}

__global__ void __launch_bounds__(kBlock)
k_bicg_update_f4(float *__restrict__ x, float *__restrict__ r, const float *__restrict__ ph,
                 const float *__restrict__ sh, const float *__restrict__ sv,
                 const float *__restrict__ t, const float *__restrict__ rh, size_t n4,
                 const BicgScalars *sc, double *pa, double *pb)
{
    const float alpha = (float)sc->alpha, omega = (float)sc->omega;
    float a = 0, b = 0;
    TPMG_GRID_LOOP4(n4)
    {
        F4 xv = ld4w(x, c);
        const F4 p4 = ld4(ph, c), s4 = ld4(sh, c), v4 = ld4(sv, c), t4 = ld4(t, c),
                 h4 = ld4(rh, c);
        F4 rv;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            xv.v[q] = fmaf(omega, s4.v[q], fmaf(alpha, p4.v[q], xv.v[q]));
            rv.v[q] = fmaf(-omega, t4.v[q], v4.v[q]);
            a = fmaf(rv.v[q], rv.v[q], a);
            b = fmaf(h4.v[q], rv.v[q], b);
        }
        st4(x, c, xv);
        st4(r, c, rv);
    }
    block_store<0>((double)a, pa);
    block_store<0>((double)b, pb);
}

#undef TPMG_GRID_LOOP4

}  // namespace

// p = r (first iteration) or p = r + beta (p - omega v)
template <typename T, bool FIRST>
__global__ void __launch_bounds__(kBlock)
k_bicg_dir(T *__restrict__ p, const T *__restrict__ r, const T *__restrict__ v, size_t n,
           const BicgScalars *sc)
{
    const T beta = FIRST ? T(0) : (T)sc->beta, omega = FIRST ? T(0) : (T)sc->omega;
#pragma unroll 4
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x)
        p[c] = FIRST ? r[c] : fma(beta, fma(-omega, v[c], p[c]), r[c]);
}

template <typename T>
cudaError_t launch_bicg_dir(T *p, const T *r, const T *v, size_t n, const BicgScalars *sc,
                            bool first, cudaStream_t s)
{
    const int g = vec_grid(n);
    if constexpr (sizeof(T) == 4) {
        if (f4_ok(n, p, r, v)) {
            if (first) k_bicg_dir_f4<true><<<g, kBlock, 0, s>>>(p, r, v, n / 4, sc);
            else k_bicg_dir_f4<false><<<g, kBlock, 0, s>>>(p, r, v, n / 4, sc);
            return cudaGetLastError();
        }
    }
    if (first) k_bicg_dir<T, true><<<g, kBlock, 0, s>>>(p, r, v, n, sc);
    else k_bicg_dir<T, false><<<g, kBlock, 0, s>>>(p, r, v, n, sc);
    return cudaGetLastError();
}

// s = r - alpha v
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_bicg_s(T *__restrict__ sv, const T *__restrict__ r, const T *__restrict__ v, size_t n,
         const BicgScalars *sc)
{
    const T alpha = (T)sc->alpha;
#pragma unroll 4
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x)
        sv[c] = fma(-alpha, v[c], r[c]);
}

template <typename T>
cudaError_t launch_bicg_s(T *sv, const T *r, const T *v, size_t n, const BicgScalars *sc,
                          cudaStream_t s)
{
    if constexpr (sizeof(T) == 4) {
        if (f4_ok(n, sv, r, v)) {
            k_bicg_s_f4<<<vec_grid(n), kBlock, 0, s>>>(sv, r, v, n / 4, sc);
            return cudaGetLastError();
        }
    }
    k_bicg_s<T><<<vec_grid(n), kBlock, 0, s>>>(sv, r, v, n, sc);
    return cudaGetLastError();
}

// Per-block sums of <t, s> (pa) and <t, t> (pb).
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_dot2(const T *__restrict__ t, const T *__restrict__ sv, size_t n, double *pa, double *pb)
{
    T a = 0, b = 0;
#pragma unroll 4
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x) {
        const T tv = t[c];
        a = fma(tv, sv[c], a);
        b = fma(tv, tv, b);
    }
    block_store<0>((double)a, pa);
    block_store<0>((double)b, pb);
}

template <typename T>
int launch_dot2(const T *t, const T *sv, size_t n, double *pa, double *pb, cudaStream_t s)
{
    const int g = vec_grid(n);
    if constexpr (sizeof(T) == 4) {
        if (f4_ok(n, t, sv)) {
            k_dot2_f4<<<g, kBlock, 0, s>>>(t, sv, n / 4, pa, pb);
            return g;
        }
    }
    k_dot2<T><<<g, kBlock, 0, s>>>(t, sv, n, pa, pb);
    return g;
}

// x += alpha ph + omega sh; r = s - omega t; per-block sums of <r, r> (pa)
// and <rh, r> (pb).
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_bicg_update(T *__restrict__ x, T *__restrict__ r, const T *__restrict__ ph,
              const T *__restrict__ sh, const T *__restrict__ sv, const T *__restrict__ t,
              const T *__restrict__ rh, size_t n, const BicgScalars *sc, double *pa, double *pb)
{
    const T alpha = (T)sc->alpha, omega = (T)sc->omega;
    T a = 0, b = 0;
#pragma unroll 4
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x) {
        x[c] = fma(omega, sh[c], fma(alpha, ph[c], x[c]));
        const T rv = fma(-omega, t[c], sv[c]);
        r[c] = rv;
        a = fma(rv, rv, a);
        b = fma(rh[c], rv, b);
    }
    block_store<0>((double)a, pa);
    block_store<0>((double)b, pb);
}

template <typename T>
int launch_bicg_update(T *x, T *r, const T *ph, const T *sh, const T *sv, const T *t,
                       const T *rh, size_t n, const BicgScalars *sc, double *pa, double *pb,
                       cudaStream_t s)
{
    const int g = vec_grid(n);
    if constexpr (sizeof(T) == 4) {
        if (f4_ok(n, x, r, ph, sh, sv, t, rh)) {
            k_bicg_update_f4<<<g, kBlock, 0, s>>>(x, r, ph, sh, sv, t, rh, n / 4, sc, pa, pb);
            return g;
        }
    }
    k_bicg_update<T><<<g, kBlock, 0, s>>>(x, r, ph, sh, sv, t, rh, n, sc, pa, pb);
    return g;
}

// Fixed-order sums of n partials of pa (and pb) and the scalar step `op`:
//   BICG_START   rr = sum pa; rho = rr (the shadow residual is r itself)
//   BICG_ALPHA   rv = sum pa; alpha = rho / rv  (rv = 0: breakdown)
//   BICG_OMEGA   ts = sum pa, tt = sum pb; omega = ts / tt (tt = 0: omega = 0,
//                the preconditioned s vanished and x takes alpha ph alone)
//   BICG_NEXT    rr = sum pa, rho_new = sum pb; beta = (rho_new / rho)
//                (alpha / omega); rho = rho_new  (rho_new = 0 or omega = 0: breakdown)
__device__ __forceinline__ double block_sum(const double *__restrict__ p, int n)
{
    __shared__ double ws[32];
    double v = 0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) v += p[c];
    v = warp_reduce<0>(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    v = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
    v = warp_reduce<0>(v);  // every warp forms the same total
    __syncthreads();        // ws is reused by the next call
    return v;
}

__global__ void __launch_bounds__(1024)
k_bicg_finalize(const double *__restrict__ pa, const double *__restrict__ pb, int n,
                BicgScalars *sc, int op)
{
    const double a = block_sum(pa, n);
    const double b = (op == BICG_OMEGA || op == BICG_NEXT) ? block_sum(pb, n) : 0.0;
    if (threadIdx.x != 0) return;
    switch (op) {
    case BICG_START:
        sc->rr = a;
        sc->rho = a;
        sc->brk = 0.0;
        break;
    case BICG_ALPHA:
        sc->rv = a;
        if (a != 0.0) {
            sc->alpha = sc->rho / a;
        } else {
            sc->alpha = 0.0;
            sc->brk = 1.0;
        }
        break;
    case BICG_OMEGA:
        sc->ts = a;
        sc->tt = b;
        sc->omega = b != 0.0 ? a / b : 0.0;
        break;
    case BICG_NEXT:
        sc->rr = a;
        if (b != 0.0 && sc->omega != 0.0 && sc->rho != 0.0) {
            sc->beta = (b / sc->rho) * (sc->alpha / sc->omega);
        } else {
            sc->beta = 0.0;
            sc->brk = 1.0;
        }
        sc->rho = b;
        break;
    }
}

cudaError_t launch_bicg_finalize(const double *pa, const double *pb, int n, BicgScalars *sc,
                                 int op, cudaStream_t s)
{
    k_bicg_finalize<<<1, 1024, 0, s>>>(pa, pb, n, sc, op);
    return cudaGetLastError();
}

// x *= f
template <typename T>
__global__ void __launch_bounds__(kBlock) k_scale(T *__restrict__ x, T f, size_t n)
{
#pragma unroll 4
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x)
        x[c] *= f;
}

template <typename T>
cudaError_t launch_scale(T *x, double f, size_t n, cudaStream_t s)
{
    k_scale<T><<<vec_grid(n), kBlock, 0, s>>>(x, (T)f, n);
    return cudaGetLastError();
}

// Per-block maxima of (h + the four horizontal couplings) / h: its inverse
// over the level bounds the spectrum of H_z^{-1} H from below.
__global__ void __launch_bounds__(kBlock) k_hz_ratio(LevelDev<double> L, double *partial)
{
    const int nlon = L.nlon, nlat = L.nlat;
    const size_t plane = (size_t)nlon * nlat, n = plane * L.nz;
    double m = 0;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x) {
        const size_t col = c % plane;
        const int j = (int)(col / nlon), i = (int)(col - (size_t)j * nlon);
        const size_t iw = (i == 0) ? c + nlon - 1 : c - 1;
        double hor = L.tx[c] + L.tx[iw];
        if (j + 1 < nlat) hor += L.ty[c];
        if (j > 0) hor += L.ty[c - nlon];
        m = max_mag(m, (L.h[c] + hor) / L.h[c]);
    }
    block_store<1>(m, partial);
}

int launch_hz_ratio(const LevelDev<double> &L, double *partial, cudaStream_t s)
{
    const int g = vec_grid((size_t)L.nlon * L.nlat * L.nz);
    k_hz_ratio<<<g, kBlock, 0, s>>>(L, partial);
    return g;
}

// One Chebyshev step of the coarsest-level solve: x += d, then
// d = c1 d + c2 z (first: d = c2 z, x untouched).
template <typename T, bool FIRST>
__global__ void __launch_bounds__(kBlock)
k_cheb_step(T *__restrict__ x, T *__restrict__ d, const T *__restrict__ z, T c1, T c2, size_t n)
{
#pragma unroll 4
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x) {
        if (FIRST) {
            d[c] = c2 * z[c];
        } else {
            const T dv = d[c];
            x[c] += dv;
            d[c] = fma(c1, dv, c2 * z[c]);
        }
    }
}

template <typename T>
cudaError_t launch_cheb_step(T *x, T *d, const T *z, double c1, double c2, size_t n, bool first,
                             cudaStream_t s)
{
    const int g = vec_grid(n);
    if (first) k_cheb_step<T, true><<<g, kBlock, 0, s>>>(x, d, z, (T)c1, (T)c2, n);
    else k_cheb_step<T, false><<<g, kBlock, 0, s>>>(x, d, z, (T)c1, (T)c2, n);
    return cudaGetLastError();
}

#define TPMG_KRYLOV_INST(T)                                                                     \
    template cudaError_t launch_bicg_dir<T>(T *, const T *, const T *, size_t,                  \
                                            const BicgScalars *, bool, cudaStream_t);           \
    template cudaError_t launch_bicg_s<T>(T *, const T *, const T *, size_t, const BicgScalars *, \
                                          cudaStream_t);                                        \
    template int launch_dot2<T>(const T *, const T *, size_t, double *, double *, cudaStream_t); \
    template int launch_bicg_update<T>(T *, T *, const T *, const T *, const T *, const T *,     \
                                       const T *, size_t, const BicgScalars *, double *,         \
                                       double *, cudaStream_t);                                  \
    template cudaError_t launch_scale<T>(T *, double, size_t, cudaStream_t);                   \
    template cudaError_t launch_cheb_step<T>(T *, T *, const T *, double, double, size_t, bool, \
                                             cudaStream_t);

TPMG_KRYLOV_INST(double)
TPMG_KRYLOV_INST(float)

}  // namespace tpmg
