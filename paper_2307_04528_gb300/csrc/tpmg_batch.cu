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

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "tpmg_device.cuh"
#include "tpmg_internal.h"

namespace tpmg {

// Blocks of `kernel` the whole GPU holds at once (persistent grid for the
// column-walk work lists), cached per kernel and block size.
static int resident_grid(const void *kernel, int block, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_pair(kernel, block);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int dev = 0, sms = 1, per_sm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess)
        return 152;
    const int g = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    cache[key] = g;
    return g;
}

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
            smooth_column<T>(op.L, op.a, op.x, op.y, omega, col, smraw);
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

template <typename T>
__global__ void __launch_bounds__(kBlock, 4) k_bsmooth_dot(const BOp<T> *__restrict__ ops, const BItem *__restrict__ items,
                              int nitems, T omega, const int *__restrict__ active,
                              double *__restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BItem item = items[it];
        const BOp<T> &op = ops[item.op];
        if (active && !active[op.sys]) continue;
        T acc = 0;
        smooth_column<T, true, 6>(op.L, op.a, op.x, op.y, omega,
                                               item.tile * blockDim.x + threadIdx.x, smraw, &acc);
        block_store_at<0>((double)acc, partial, it);
    }
}

template <typename T>
cudaError_t launch_bsmooth_dot(const BOp<T> *ops, const BItem *items, int nitems, double omega,
                               const int *active, int grid, int block, int nzmax,
                               double *partial, cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    const size_t smem = (size_t)nzmax * block * sizeof(T);
    k_bsmooth_dot<T><<<grid, block, smem, s>>>(ops, items, nitems, (T)omega, active, partial);
    return cudaGetLastError();
}

// One system's coarsest-level solve per block (coarse_solve_sh).
template <typename T>
__global__ void __launch_bounds__(kCoarseSolveThreads)
k_bcoarse_solve(const BOp<T> *__restrict__ ops, T omega, int sweeps,
                const int *__restrict__ active)
{
    const BOp<T> &op = ops[blockIdx.x];
    if (active && !active[op.sys]) return;
    extern __shared__ __align__(16) unsigned char sh_raw[];
    coarse_solve_sh<T>(op.L, op.a, op.y, omega, sweeps, reinterpret_cast<T *>(sh_raw));
}

template <typename T>
cudaError_t launch_bcoarse_solve(const BOp<T> *ops, int nops, double omega, int sweeps,
                                 const int *active, size_t smem, cudaStream_t s)
{
    if (nops <= 0) return cudaSuccess;
    k_bcoarse_solve<T><<<nops, kCoarseSolveThreads, smem, s>>>(ops, (T)omega, sweeps, active);
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
                             (const void *)k_bsmooth<float, true>, (const void *)k_bsmooth<float, false>,
                             (const void *)k_bsmooth_dot<double>, (const void *)k_bsmooth_dot<float>,
                             (const void *)k_bcoarse_solve<double>, (const void *)k_bcoarse_solve<float>};
    for (const void *k : kernels)
        if ((e = set_dynamic_smem_limit(k, lim)) != cudaSuccess) return e;
    return cudaSuccess;
}

template <typename T, int KIND>
__global__ void __launch_bounds__(kBlock)
k_bcells(const BOp<T> *__restrict__ ops, const BItem *__restrict__ items, int nitems,
         const int *__restrict__ active, T om1)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BItem item = items[it];
        const BOp<T> &op = ops[item.op];
        if (active && !active[op.sys]) continue;
        if (KIND >= 3) {  // fused residual + restriction: tile = (band * nz + k) * nblk + xb
            const int xb = item.tile % op.nblk, rest = item.tile / op.nblk;
            const int k = rest % op.L.nz, band = rest / op.L.nz;
            const int warp = (xb * blockDim.x + threadIdx.x) >> 5;
            if (warp * kRROwned < op.L.nlon / 2)  // whole warps
                resid_restrict_band<T, KIND == 4>(op.L, op.K, op.a, op.x, op.y, warp,
                                                  threadIdx.x & 31, band * kRRBand, k, om1);
            continue;
        }
        const int zc = item.tile / op.nblk;
        const int c = (item.tile - zc * op.nblk) * blockDim.x + threadIdx.x;
        const int k0 = zc * op.kz, k1 = min(op.L.nz, k0 + op.kz);
        if (KIND == 0) {
            if (op.kz >= op.L.nz) {
                stencil_column<T, 1, false>(op.L, op.a, op.x, op.y, c);
            } else if (c < op.L.nlon * op.L.nlat) {
                for (int k = k0; k < k1; ++k) stencil_cell<T, 1>(op.L, op.a, op.x, op.y, c, k);
            }
        } else if (KIND == 1) {
            restrict_layers<T>(op.L, op.K, op.a, op.y, c, k0, k1);
        } else {
            prolong_layers<T>(op.L, op.K, op.a, op.y, c, k0, k1);
        }
    }
}

template <typename T>
cudaError_t launch_bcells(int kind, const BOp<T> *ops, const BItem *items, int nitems,
                          const int *active, int grid, cudaStream_t s, double omega)
{
    if (nitems <= 0) return cudaSuccess;
    const void *k = kind == 0   ? (const void *)k_bcells<T, 0>
                    : kind == 1 ? (const void *)k_bcells<T, 1>
                    : kind == 2 ? (const void *)k_bcells<T, 2>
                    : kind == 3 ? (const void *)k_bcells<T, 3>
                                : (const void *)k_bcells<T, 4>;
    grid = std::min(grid, resident_grid(k, kBlock, 0));
    const T om1 = T(1) - (T)omega;
    if (kind == 0) k_bcells<T, 0><<<grid, kBlock, 0, s>>>(ops, items, nitems, active, om1);
    else if (kind == 1) k_bcells<T, 1><<<grid, kBlock, 0, s>>>(ops, items, nitems, active, om1);
    else if (kind == 2) k_bcells<T, 2><<<grid, kBlock, 0, s>>>(ops, items, nitems, active, om1);
    else if (kind == 3) k_bcells<T, 3><<<grid, kBlock, 0, s>>>(ops, items, nitems, active, om1);
    else k_bcells<T, 4><<<grid, kBlock, 0, s>>>(ops, items, nitems, active, om1);
    return cudaGetLastError();
}

template <typename T, bool BZ>
__global__ void __launch_bounds__(kBlock)
k_bdir_apply(const BOp<T> *__restrict__ ops, const BItem *__restrict__ items, int nitems,
             const CgScalars *__restrict__ sc, double *__restrict__ partial,
             const int *__restrict__ active)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BItem item = items[it];
        const BOp<T> &op = ops[item.op];
        if (active && !active[op.sys]) continue;
        const T beta = BZ ? T(0) : (T)sc[op.sys].beta;
        const T acc = dir_apply_column<T, BZ>(op.L, op.a, op.x, beta, op.y, op.w,
                                              item.tile * blockDim.x + threadIdx.x);
        block_store_at<0>((double)acc, partial, it);
    }
}

template <typename T>
cudaError_t launch_bdir_apply(bool bz, const BOp<T> *ops, const BItem *items, int nitems,
                              const CgScalars *sc, double *partial, const int *active, int grid,
                              cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    if (bz) {
        grid = std::min(grid, resident_grid((const void *)k_bdir_apply<T, true>, kBlock, 0));
        k_bdir_apply<T, true><<<grid, kBlock, 0, s>>>(ops, items, nitems, sc, partial, active);
    } else {
        grid = std::min(grid, resident_grid((const void *)k_bdir_apply<T, false>, kBlock, 0));
        k_bdir_apply<T, false><<<grid, kBlock, 0, s>>>(ops, items, nitems, sc, partial, active);
    }
    return cudaGetLastError();
}

template <bool NARROW>
__global__ void __launch_bounds__(kBlock)
k_bresid_cast(const BResid32 *__restrict__ ops, const BItem *__restrict__ items, int nitems,
              const double *__restrict__ sdata, double *__restrict__ partial,
              const int *__restrict__ active)
{
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BItem item = items[it];
        const BResid32 &op = ops[item.op];
        if (active && !active[op.sys]) continue;
        const double acc = stencil_column<double, 1, true, float, NARROW>(
            op.L, op.b, op.x, op.r32, item.tile * blockDim.x + threadIdx.x, sdata[op.sys]);
        block_store_at<0>(acc, partial, it);
    }
}

cudaError_t launch_bresid_cast(bool narrow, const BResid32 *ops, const BItem *items, int nitems,
                               const double *sdata, double *partial, const int *active, int grid,
                               cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    if (narrow) {
        grid = std::min(grid, resident_grid((const void *)k_bresid_cast<true>, kBlock, 0));
        k_bresid_cast<true><<<grid, kBlock, 0, s>>>(ops, items, nitems, sdata, partial, active);
    } else {
        grid = std::min(grid, resident_grid((const void *)k_bresid_cast<false>, kBlock, 0));
        k_bresid_cast<false><<<grid, kBlock, 0, s>>>(ops, items, nitems, sdata, partial, active);
    }
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
    if (mode) {
        grid = std::min(grid, resident_grid((const void *)k_bstencil_red<T, 1>, kBlock, 0));
        k_bstencil_red<T, 1><<<grid, kBlock, 0, s>>>(ops, items, nitems, partial, active);
    } else {
        grid = std::min(grid, resident_grid((const void *)k_bstencil_red<T, 0>, kBlock, 0));
        k_bstencil_red<T, 0><<<grid, kBlock, 0, s>>>(ops, items, nitems, partial, active);
    }
    return cudaGetLastError();
}

// Vector ops; item.tile = chunk index within the system's vector.
//   BV_DOT:    partial = sum a*b
//   BV_UPDATE: a += alpha c; b -= alpha d; partial = sum b*b   (x, r, dir, Adir)
//   BV_DIR:    a = b + beta c                                 (dir_out, z, dir_in)
//   BV_DIR0:   a = b
//   BV_ADD:    a += b
//   BV_MAXABS: partial = max |a|
// The chunk loop takes the vectors as restrict-qualified arguments, so the
// loads of later elements are not held behind the stores of earlier ones.
template <typename T, int OP>
__device__ __forceinline__ double bvec_chunk(T *__restrict__ a, T *__restrict__ b,
                                             const T *__restrict__ c, const T *__restrict__ d,
                                             size_t c0, size_t c1, T alpha, T beta)
{
    double acc = 0;
    T tacc = 0;
#pragma unroll 4
    for (size_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
        if (OP == BV_DOT) {
            tacc = fma(a[i], b[i], tacc);
        } else if (OP == BV_UPDATE) {
            a[i] = fma(alpha, c[i], a[i]);
            const T rv = fma(-alpha, d[i], b[i]);
            b[i] = rv;
            tacc = fma(rv, rv, tacc);
        } else if (OP == BV_DIR) {
            a[i] = fma(beta, c[i], b[i]);
        } else if (OP == BV_DIR0) {
            a[i] = b[i];
        } else if (OP == BV_ADD) {
            a[i] += b[i];
        } else {
            acc = max_mag(acc, (double)a[i]);  // NaN propagates
        }
    }
    return OP == BV_MAXABS ? acc : (double)tacc;
}

// The FP32 chunk on 16-byte vectors (chunks are multiples of kBlock values;
// lengths and bases checked by the caller): the same arithmetic per
// element, four elements per load and store.
template <int OP>
__device__ __forceinline__ double bvec_chunk_f4(float *__restrict__ a, float *__restrict__ b,
                                                const float *__restrict__ c,
                                                const float *__restrict__ d, size_t c0, size_t c1,
                                                float alpha, float beta)
{
    float4 *a4 = reinterpret_cast<float4 *>(a);
    float4 *b4 = reinterpret_cast<float4 *>(b);
    const float4 *c4 = reinterpret_cast<const float4 *>(c);
    const float4 *d4 = reinterpret_cast<const float4 *>(d);
    double acc = 0;
    float tacc = 0;
#pragma unroll 2
    for (size_t i = c0 / 4 + threadIdx.x; i < c1 / 4; i += blockDim.x) {
        if (OP == BV_DOT) {
            const float4 x = a4[i], y = b4[i];
            tacc = fmaf(x.x, y.x, tacc);
            tacc = fmaf(x.y, y.y, tacc);
            tacc = fmaf(x.z, y.z, tacc);
            tacc = fmaf(x.w, y.w, tacc);
        } else if (OP == BV_UPDATE) {
            float4 x = a4[i], r = b4[i];
            const float4 dv = c4[i], q = d4[i];
            x.x = fmaf(alpha, dv.x, x.x);
            x.y = fmaf(alpha, dv.y, x.y);
            x.z = fmaf(alpha, dv.z, x.z);
            x.w = fmaf(alpha, dv.w, x.w);
            r.x = fmaf(-alpha, q.x, r.x);
            r.y = fmaf(-alpha, q.y, r.y);
            r.z = fmaf(-alpha, q.z, r.z);
            r.w = fmaf(-alpha, q.w, r.w);
            a4[i] = x;
            b4[i] = r;
            tacc = fmaf(r.x, r.x, tacc);
            tacc = fmaf(r.y, r.y, tacc);
            tacc = fmaf(r.z, r.z, tacc);
            tacc = fmaf(r.w, r.w, tacc);
        } else if (OP == BV_DIR) {
            const float4 z = b4[i], dv = c4[i];
            a4[i] = make_float4(fmaf(beta, dv.x, z.x), fmaf(beta, dv.y, z.y),
                                fmaf(beta, dv.z, z.z), fmaf(beta, dv.w, z.w));
        } else if (OP == BV_DIR0) {
            a4[i] = b4[i];
        } else if (OP == BV_ADD) {
            float4 x = a4[i];
            const float4 y = b4[i];
            x.x += y.x;
            x.y += y.y;
            x.z += y.z;
            x.w += y.w;
            a4[i] = x;
        } else {
            const float4 x = a4[i];
            acc = max_mag(acc, (double)x.x);  // NaN propagates
            acc = max_mag(acc, (double)x.y);
            acc = max_mag(acc, (double)x.z);
            acc = max_mag(acc, (double)x.w);
        }
    }
    return OP == BV_MAXABS ? acc : (double)tacc;
}

__device__ __forceinline__ bool f4_chunk(const void *a, const void *b, const void *c,
                                         const void *d, size_t c0, size_t c1)
{
    return ((uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d) % 16 == 0 && c0 % 4 == 0 &&
           c1 % 4 == 0;
}

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
        const size_t c0 = (size_t)item.tile * v.chunk;
        const size_t c1 = c0 + v.chunk < v.n ? c0 + v.chunk : v.n;
        const T alpha = (OP == BV_UPDATE) ? (T)sc[v.sys].alpha : T(0);
        const T beta = (OP == BV_DIR) ? (T)sc[v.sys].beta : T(0);
        double acc;
        if constexpr (sizeof(T) == 4) {
            acc = f4_chunk(v.a, v.b, v.c, v.d, c0, c1)
                      ? bvec_chunk_f4<OP>(v.a, v.b, v.c, v.d, c0, c1, alpha, beta)
                      : bvec_chunk<T, OP>(v.a, v.b, v.c, v.d, c0, c1, alpha, beta);
        } else {
            acc = bvec_chunk<T, OP>(v.a, v.b, v.c, v.d, c0, c1, alpha, beta);
        }
        if (OP == BV_DOT || OP == BV_UPDATE) block_store_at<0>(acc, partial, it);
        if (OP == BV_MAXABS) block_store_at<1>(acc, partial, it);
    }
}

template <typename T>
cudaError_t launch_bvec(int op, const BVec<T> *v, const BItem *items, int nitems,
                        const CgScalars *sc, double *partial, const int *active, int grid,
                        cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    grid = std::min(grid, resident_grid((const void *)k_bvec<T, BV_UPDATE>, kBlock, 0));
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
__device__ __forceinline__ void bmix_chunk(double *__restrict__ x, const double *__restrict__ r,
                                           float *__restrict__ r32, const float *__restrict__ e32,
                                           size_t c0, size_t c1, double f)
{
    const int sx = MODE == 0 ? pow2_exponent(f) : kNotPow2;
    if (f4_chunk(x, r, r32, e32, c0, c1)) {  // four values per load and store
#pragma unroll 2
        for (size_t i = c0 / 4 + threadIdx.x; i < c1 / 4; i += blockDim.x) {
            if (MODE == 0) {
                const double2 a = reinterpret_cast<const double2 *>(r)[2 * i];
                const double2 b = reinterpret_cast<const double2 *>(r)[2 * i + 1];
                reinterpret_cast<float4 *>(r32)[i] =
                    make_float4(scaled_to_f32(a.x, f, sx), scaled_to_f32(a.y, f, sx),
                                scaled_to_f32(b.x, f, sx), scaled_to_f32(b.y, f, sx));
            } else {
                const float4 e = reinterpret_cast<const float4 *>(e32)[i];
                double2 a = reinterpret_cast<double2 *>(x)[2 * i];
                double2 b = reinterpret_cast<double2 *>(x)[2 * i + 1];
                a.x = fma(f, f32_to_f64(e.x), a.x);
                a.y = fma(f, f32_to_f64(e.y), a.y);
                b.x = fma(f, f32_to_f64(e.z), b.x);
                b.y = fma(f, f32_to_f64(e.w), b.y);
                reinterpret_cast<double2 *>(x)[2 * i] = a;
                reinterpret_cast<double2 *>(x)[2 * i + 1] = b;
            }
        }
        return;
    }
#pragma unroll 4
    for (size_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        if (MODE == 0) r32[c] = scaled_to_f32(r[c], f, sx);
        else x[c] = fma(f, f32_to_f64(e32[c]), x[c]);
    }
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
        const size_t c0 = (size_t)item.tile * v.chunk;
        const size_t c1 = c0 + v.chunk < v.n ? c0 + v.chunk : v.n;
        bmix_chunk<MODE>(v.x, v.r, v.r32, v.e32, c0, c1, sdata[v.sys]);
    }
}

cudaError_t launch_bmix(int mode, const BMix *v, const BItem *items, int nitems,
                        const double *sdata, const int *active, int grid, cudaStream_t s)
{
    if (nitems <= 0) return cudaSuccess;
    grid = std::min(grid, resident_grid((const void *)k_bmix<1>, kBlock, 0));
    if (mode == 0) k_bmix<0><<<grid, kBlock, 0, s>>>(v, items, nitems, sdata, active);
    else k_bmix<1><<<grid, kBlock, 0, s>>>(v, items, nitems, sdata, active);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256)
k_bfinalize(const double *__restrict__ partial, const int *__restrict__ beg,
            const int *__restrict__ end, CgScalars *sc, int which, int op,
            const int *__restrict__ active)
{
    const int sys = blockIdx.x;
    if (active && !active[sys]) return;
    const int p0 = beg[sys], p1 = end[sys];
    double v = 0;
    for (int c = p0 + threadIdx.x; c < p1; c += blockDim.x)
        v = op == 3 ? max_mag(v, partial[c]) : v + partial[c];
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

cudaError_t launch_bfinalize(const double *partial, const int *beg, const int *end, int nsys,
                             CgScalars *sc, int which, int op, const int *active, cudaStream_t s)
{
    k_bfinalize<<<nsys, 256, 0, s>>>(partial, beg, end, sc, which, op, active);
    return cudaGetLastError();
}

#define TPMG_BINST(T)                                                                           \
    template cudaError_t launch_bcoarse_solve<T>(const BOp<T> *, int, double, int, const int *,  \
                                                 size_t, cudaStream_t);                          \
    template cudaError_t launch_bsmooth<T>(const BOp<T> *, const BItem *, int, bool, double,      \
                                           const int *, int, int, int, cudaStream_t);             \
    template cudaError_t launch_bsmooth_dot<T>(const BOp<T> *, const BItem *, int, double,        \
                                               const int *, int, int, int, double *, cudaStream_t); \
    template cudaError_t launch_bcells<T>(int, const BOp<T> *, const BItem *, int, const int *,   \
                                          int, cudaStream_t, double);                             \
    template cudaError_t launch_bstencil_red<T>(int, const BOp<T> *, const BItem *, int,          \
                                                double *, const int *, int, cudaStream_t);        \
    template cudaError_t launch_bvec<T>(int, const BVec<T> *, const BItem *, int,                 \
                                        const CgScalars *, double *, const int *, int, cudaStream_t); \
    template cudaError_t launch_bdir_apply<T>(bool, const BOp<T> *, const BItem *, int,           \
                                              const CgScalars *, double *, const int *, int,      \
                                              cudaStream_t);

TPMG_BINST(double)
TPMG_BINST(float)

}  // namespace tpmg
