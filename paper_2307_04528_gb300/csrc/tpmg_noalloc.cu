// Residual and relative residual norm with no device allocation at all.
//
// Some callers cannot allocate device memory when they need this check: a
// forecast model that hands the library its fields from a device pool it
// owns and forbids any other cudaMalloc (an allocation can synchronise the
// device and fragments the pool), or host code in C or Fortran that has no
// device allocator to pass a workspace from.  For them this file keeps the
// reduction scratch in a file-scope __device__ array that lives as long as
// the library is loaded, and needs neither a handle nor a workspace.
//
// Limits and sharing: the array holds the per-block partial sums of at most
// kMaxBlocks blocks of kThreads columns, so grids beyond
// kMaxBlocks * kThreads columns (nlon * nlat) are rejected.  Every call on a
// device uses the same array and leaves its contents behind; calls that
// overlap on the GPU (two streams, or two host threads) race on it.
//
// The coefficients are not validated here (mg_setup does that for a handle);
// the operator is the one mg_setup accepts: the model-top coupling
// tz[nz-1] is never read, as the top face carries no flux.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/tpmg.h"
#include "tpmg_handle.h"
#include "tpmg_internal.h"

namespace {

constexpr int kThreads = 128;
constexpr int kMaxBlocks = 16384;  // 2 x 16384 partials + 2 results = 256 KB + 16 B

// partial[0 .. kMaxBlocks): sum r^2 per block; partial[kMaxBlocks ..): sum b^2;
// result at [2 kMaxBlocks], [2 kMaxBlocks + 1].
static __device__ __align__(256) double g_noalloc_scratch[2 * kMaxBlocks + 2];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

int err(int code, const char *msg)
{
    tpmg::set_last_error(msg);
    return code;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void block_sum2(double a, double b, double *pa, double *pb)
{
    __shared__ double wa[32], wb[32];
    a = warp_sum(a);
    b = warp_sum(b);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        wa[w] = a;
        wb[w] = b;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        a = lane < nw ? wa[lane] : 0.0;
        b = lane < nw ? wb[lane] : 0.0;
        a = warp_sum(a);
        b = warp_sum(b);
        if (lane == 0) {
            *pa = a;
            *pb = b;
        }
    }
}

// r = b - H x in flux form (one thread per column, k innermost), with the
// per-block sums of r^2 and b^2 written to the scratch array.
__global__ void __launch_bounds__(kThreads)
k_residual_norm_static(int nlon, int nlat, int nz, const double *__restrict__ tx,
                       const double *__restrict__ ty, const double *__restrict__ tz,
                       const double *__restrict__ h, const double *__restrict__ b,
                       const double *__restrict__ x, double *__restrict__ r, double *scratch)
{
    const int ncol = nlon * nlat;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    double rr = 0, bb = 0;
    if (col < ncol) {
        const int j = col / nlon, i = col - j * nlon;
        const int ie = (i + 1 == nlon) ? col - i : col + 1;
        const int iw = (i == 0) ? col + nlon - 1 : col - 1;
        const size_t plane = (size_t)ncol;
        double xdn = 0, tdn = 0, xc = x[col];
        for (int k = 0; k < nz; ++k) {
            const size_t o = (size_t)k * plane;
            const double xup = (k + 1 < nz) ? x[o + plane + col] : 0.0;
            const double tup = (k + 1 < nz) ? tz[o + col] : 0.0;  // no flux through the top
            double v = h[o + col] * xc;
            v = fma(tx[o + col], xc - x[o + ie], v);
            v = fma(tx[o + iw], xc - x[o + iw], v);
            if (j + 1 < nlat) v = fma(ty[o + col], xc - x[o + col + nlon], v);
            if (j > 0) v = fma(ty[o + col - nlon], xc - x[o + col - nlon], v);
            v = fma(tup, xc - xup, v);
            v = fma(tdn, xc - xdn, v);
            const double bv = b[o + col];
            const double rv = bv - v;
            r[o + col] = rv;
            rr = fma(rv, rv, rr);
            bb = fma(bv, bv, bb);
            xdn = xc;
            xc = xup;
            tdn = tup;
        }
    }
    block_sum2(rr, bb, scratch + blockIdx.x, scratch + kMaxBlocks + blockIdx.x);
}

// Fixed-order sum of the partials; result[0] = sum r^2, result[1] = sum b^2.
__global__ void __launch_bounds__(1024) k_finalize_static(int nblocks, double *scratch)
{
    double a = 0, b = 0;
    for (int c = threadIdx.x; c < nblocks; c += blockDim.x) {
        a += scratch[c];
        b += scratch[kMaxBlocks + c];
    }
    double *res = scratch + 2 * kMaxBlocks;
    block_sum2(a, b, res, res + 1);
}

// Device address of the scratch array on the current device, looked up once
// per device (the symbol's host-side name is not a device address).
int scratch_for_current_device(double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(MG_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return err(MG_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return err(MG_ERR_CUDA, cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return MG_OK;
}

}  // namespace

extern "C" int mg_residual_norm_noalloc(const mg_grid *grid, const mg_coeffs *coeffs,
                                        const double *b, const double *x, double *r,
                                        double *rel_out, void *stream)
{
    if (!grid || !coeffs || !b || !x || !r || !rel_out || !coeffs->tx || !coeffs->ty ||
        !coeffs->tz || !coeffs->h)
        return err(MG_ERR_ARG, "null argument");
    if (grid->nlon < 1 || grid->nlat < 1 || grid->nz < 1)
        return err(MG_ERR_ARG, "grid extents must be positive");
    const long long ncol = (long long)grid->nlon * grid->nlat;
    const long long nblocks = (ncol + kThreads - 1) / kThreads;
    if (nblocks > kMaxBlocks) {
        char buf[160];
        snprintf(buf, sizeof buf, "nlon*nlat = %lld columns exceeds the static scratch limit of "
                 "%d columns", ncol, kMaxBlocks * kThreads);
        return err(MG_ERR_ARG, buf);
    }
    double *scratch = nullptr;
    int st = scratch_for_current_device(&scratch);
    if (st != MG_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // A launch that fails (no kernel image, a bad stream) must not let the
    // copy below return the previous call's result from the shared array.
    k_residual_norm_static<<<(int)nblocks, kThreads, 0, s>>>(
        grid->nlon, grid->nlat, grid->nz, coeffs->tx, coeffs->ty, coeffs->tz, coeffs->h, b, x, r,
        scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return err(MG_ERR_CUDA, cudaGetErrorString(e));
    k_finalize_static<<<1, 1024, 0, s>>>((int)nblocks, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return err(MG_ERR_CUDA, cudaGetErrorString(e));
    tpmg::g_launches.fetch_add(2, std::memory_order_relaxed);
    double res[2] = {0, 0};
    e = cudaMemcpyAsync(res, scratch + 2 * kMaxBlocks, sizeof res, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return err(MG_ERR_CUDA, cudaGetErrorString(e));
    if (!std::isfinite(res[0]) || !std::isfinite(res[1]))
        return err(MG_ERR_NONFINITE, "non-finite norm");
    const double rel = res[1] > 0 ? std::sqrt(res[0] / res[1]) : std::sqrt(res[0]);
    if (!std::isfinite(rel)) return err(MG_ERR_NONFINITE, "non-finite norm");
    *rel_out = rel;
    return MG_OK;
}
