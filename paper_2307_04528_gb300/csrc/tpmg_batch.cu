// Batched persistent kernels for ensembles of independent systems.
//
// Every step of the V-cycle (and every fine-level vector operation of the
// conjugate-gradient iteration) is issued once for the whole ensemble: a
// persistent grid walks a precomputed work list of (participant, tile)
// items, where a participant is one level of one system with its own
// shape and vectors.  Items are assigned to blocks by a fixed stride, so
// every sum is formed in the same order on every run.  Systems whose
// activity flag is 0 (converged) are skipped.  The per-column and per-cell
// arithmetic is the single-system code of tpmg_device.cuh.
#include <cuda_runtime.h>

#include "tpmg_device.cuh"
#include "tpmg_internal.h"

namespace tpmg {

template <typename T, bool ZERO>
__global__ void __launch_bounds__(kBlock, 4) k_bsmooth(const BOp<T> *__restrict__ ops, const BItem *__restrict__ items,
                          int nitems, T omega, const int *__restrict__ active)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BItem item = items[it];
        const BOp<T> &op = ops[item.op];
        if (active && !active[op.sys]) continue;
        const int col = item.tile * blockDim.x + threadIdx.x;
        if (ZERO)
            smooth_staged<T, true>(op.L, op.a, nullptr, op.y, omega, col, smraw);
        else
            smooth_column<T, false, true>(op.L, op.a, op.x, op.y, omega, col, smraw);
    }
}

template <typename T>
cudaError_t launch_bsmooth(const BOp<T> *ops, const BItem *items, int nitems, bool zero,
                           double omega, const int *active, int grid, int block, int nzmax,
                           cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    if (zero) {
        const size_t smem = ring_smem_bytes<T, true>(nzmax, block);
        k_bsmooth<T, true><<<grid, block, smem, s>>>(ops, items, nitems, (T)omega, active);
    } else {
        const size_t smem = (size_t)nzmax * block * sizeof(T);
        k_bsmooth<T, false><<<grid, block, smem, s>>>(ops, items, nitems, (T)omega, active);
    }
    return cudaGetLastError();
}

cudaError_t bsmooth_prepare()
{
    cudaError_t e;
    int dev = 0, lim = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
        cudaSuccess)
        return e;
    const void *kernels[] = {(const void *)k_bsmooth<double, true>, (const void *)k_bsmooth<double, false>,
                             (const void *)k_bsmooth<float, true>, (const void *)k_bsmooth<float, false>};
    for (const void *k : kernels)
        if ((e = set_dynamic_smem_limit(k, lim)) != cudaSuccess) return e;
    return cudaSuccess;
}

template <typename T, int KIND>
__global__ void __launch_bounds__(kBlock)
k_bcells(const BOp<T> *__restrict__ ops, const BItem *__restrict__ items, int nitems,
         const int *__restrict__ active)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BItem item = items[it];
        const BOp<T> &op = ops[item.op];
        if (active && !active[op.sys]) continue;
        const int k = item.tile / op.nblk;
        const int c = (item.tile - k * op.nblk) * blockDim.x + threadIdx.x;
        if (KIND == 0) {
            if (c < op.L.nlon * op.L.nlat) stencil_cell<T, 1>(op.L, op.a, op.x, op.y, c, k);
        } else if (KIND == 1) {
            restrict_cell<T>(op.L, op.K, op.a, op.y, c, k);
        } else {
            prolong_pair<T>(op.L, op.K, op.a, op.y, c, k);
        }
    }
}

template <typename T>
cudaError_t launch_bcells(int kind, const BOp<T> *ops, const BItem *items, int nitems,
                          const int *active, int grid, cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    if (kind == 0) k_bcells<T, 0><<<grid, kBlock, 0, s>>>(ops, items, nitems, active);
    else if (kind == 1) k_bcells<T, 1><<<grid, kBlock, 0, s>>>(ops, items, nitems, active);
    else k_bcells<T, 2><<<grid, kBlock, 0, s>>>(ops, items, nitems, active);
    return cudaGetLastError();
}

template <typename T, int MODE>
__global__ void __launch_bounds__(kBlock)
k_bstencil_red(const BOp<T> *__restrict__ ops, const BItem *__restrict__ items, int nitems,
               double *__restrict__ partial, const int *__restrict__ active)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BItem item = items[it];
        const BOp<T> &op = ops[item.op];
        if (active && !active[op.sys]) continue;
        const T acc = stencil_column<T, MODE, true>(op.L, op.a, op.x, op.y,
                                                    item.tile * blockDim.x + threadIdx.x);
        block_store_at<0>((double)acc, partial, it);
    }
}

template <typename T>
cudaError_t launch_bstencil_red(int mode, const BOp<T> *ops, const BItem *items, int nitems,
                                double *partial, const int *active, int grid, cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    if (mode) k_bstencil_red<T, 1><<<grid, kBlock, 0, s>>>(ops, items, nitems, partial, active);
    else k_bstencil_red<T, 0><<<grid, kBlock, 0, s>>>(ops, items, nitems, partial, active);
    return cudaGetLastError();
}

// Vector ops; item.tile = chunk index within the system's vector.
//   BV_DOT:    partial = sum a*b
//   BV_UPDATE: a += alpha c; b -= alpha d; partial = sum b*b   (x, r, dir, Adir)
//   BV_DIR:    a = b + beta c                                 (dir_out, z, dir_in)
//   BV_DIR0:   a = b
//   BV_ADD:    a += b
//   BV_MAXABS: partial = max |a|
template <typename T, int OP>
__global__ void __launch_bounds__(kBlock)
k_bvec(const BVec<T> *__restrict__ vs, const BItem *__restrict__ items, int nitems,
       const CgScalars *__restrict__ sc, double *__restrict__ partial,
       const int *__restrict__ active)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BItem item = items[it];
        const BVec<T> &v = vs[item.op];
        if (active && !active[v.sys]) continue;
        const size_t c0 = (size_t)item.tile * kVecChunk;
        const size_t c1 = c0 + kVecChunk < v.n ? c0 + kVecChunk : v.n;
        double acc = 0;
        T tacc = 0;
        const T alpha = (OP == BV_UPDATE) ? (T)sc[v.sys].alpha : T(0);
        const T beta = (OP == BV_DIR) ? (T)sc[v.sys].beta : T(0);
        for (size_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            if (OP == BV_DOT) {
                tacc = fma(v.a[c], v.b[c], tacc);
            } else if (OP == BV_UPDATE) {
                v.a[c] = fma(alpha, v.c[c], v.a[c]);
                const T rv = fma(-alpha, v.d[c], v.b[c]);
                v.b[c] = rv;
                tacc = fma(rv, rv, tacc);
            } else if (OP == BV_DIR) {
                v.a[c] = fma(beta, v.c[c], v.b[c]);
            } else if (OP == BV_DIR0) {
                v.a[c] = v.b[c];
            } else if (OP == BV_ADD) {
                v.a[c] += v.b[c];
            } else {
                const double m = fabs((double)v.a[c]);
                acc = (m > acc || m != m) ? m : acc;
            }
        }
        if (OP == BV_DOT || OP == BV_UPDATE) block_store_at<0>((double)tacc, partial, it);
        if (OP == BV_MAXABS) block_store_at<1>(acc, partial, it);
    }
}

template <typename T>
cudaError_t launch_bvec(int op, const BVec<T> *v, const BItem *items, int nitems,
                        const CgScalars *sc, double *partial, const int *active, int grid,
                        cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    switch (op) {
    case BV_DOT: k_bvec<T, BV_DOT><<<grid, kBlock, 0, s>>>(v, items, nitems, sc, partial, active); break;
    case BV_UPDATE: k_bvec<T, BV_UPDATE><<<grid, kBlock, 0, s>>>(v, items, nitems, sc, partial, active); break;
    case BV_DIR: k_bvec<T, BV_DIR><<<grid, kBlock, 0, s>>>(v, items, nitems, sc, partial, active); break;
    case BV_DIR0: k_bvec<T, BV_DIR0><<<grid, kBlock, 0, s>>>(v, items, nitems, sc, partial, active); break;
    case BV_ADD: k_bvec<T, BV_ADD><<<grid, kBlock, 0, s>>>(v, items, nitems, sc, partial, active); break;
    default: k_bvec<T, BV_MAXABS><<<grid, kBlock, 0, s>>>(v, items, nitems, sc, partial, active); break;
    }
    return cudaGetLastError();
}

template <int MODE>
__global__ void __launch_bounds__(kBlock)
k_bmix(const BMix *__restrict__ vs, const BItem *__restrict__ items, int nitems,
       const double *__restrict__ sdata, const int *__restrict__ active)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BItem item = items[it];
        const BMix &v = vs[item.op];
        if (active && !active[v.sys]) continue;
        const double f = sdata[v.sys];
        const size_t c0 = (size_t)item.tile * kVecChunk;
        const size_t c1 = c0 + kVecChunk < v.n ? c0 + kVecChunk : v.n;
        for (size_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
            if (MODE == 0) v.r32[c] = (float)(v.r[c] * f);
            else v.x[c] = fma(f, (double)v.e32[c], v.x[c]);
        }
    }
}

cudaError_t launch_bmix(int mode, const BMix *v, const BItem *items, int nitems,
                        const double *sdata, const int *active, int grid, cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    if (mode == 0) k_bmix<0><<<grid, kBlock, 0, s>>>(v, items, nitems, sdata, active);
    else k_bmix<1><<<grid, kBlock, 0, s>>>(v, items, nitems, sdata, active);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256)
k_bfinalize(const double *__restrict__ partial, const int *__restrict__ off, CgScalars *sc,
            int which, int op, const int *__restrict__ active)
{
    const int sys = blockIdx.x;
    if (active && !active[sys]) return;
    const int p0 = off[sys], p1 = off[sys + 1];
    double v = 0;
    for (int c = p0 + threadIdx.x; c < p1; c += blockDim.x)
        v = op == 3 ? ((partial[c] > v || partial[c] != partial[c]) ? partial[c] : v) : v + partial[c];
    __shared__ double ws[8];
    v = op == 3 ? warp_reduce<1>(v) : warp_reduce<0>(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        v = op == 3 ? warp_reduce<1>(v) : warp_reduce<0>(v);
        if (lane == 0) {
            CgScalars &S = sc[sys];
            reinterpret_cast<double *>(&S)[which] = v;
            if (op == 1) S.alpha = S.rz / v;
            if (op == 2) {
                S.beta = v / S.rz;
                S.rz = v;
            }
        }
    }
}

cudaError_t launch_bfinalize(const double *partial, const int *off, int nsys, CgScalars *sc,
                             int which, int op, const int *active, cudaStream_t s)
{
    k_bfinalize<<<nsys, 256, 0, s>>>(partial, off, sc, which, op, active);
    return cudaGetLastError();
}

#define TPMG_BINST(T)                                                                           \
    template cudaError_t launch_bsmooth<T>(const BOp<T> *, const BItem *, int, bool, double,      \
                                           const int *, int, int, int, cudaStream_t);             \
    template cudaError_t launch_bcells<T>(int, const BOp<T> *, const BItem *, int, const int *,   \
                                          int, cudaStream_t);                                     \
    template cudaError_t launch_bstencil_red<T>(int, const BOp<T> *, const BItem *, int,          \
                                                double *, const int *, int, cudaStream_t);        \
    template cudaError_t launch_bvec<T>(int, const BVec<T> *, const BItem *, int,                 \
                                        const CgScalars *, double *, const int *, int, cudaStream_t);

TPMG_BINST(double)
TPMG_BINST(float)

}  // namespace tpmg
