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
