// CUDA kernels of the tensor-product multigrid (sm_103a).
//
// Data layout: every field is [nz][nlat][nlon], longitude fastest.  One
// thread owns one vertical column (i, j) and walks k, so at every k the
// threads of a warp touch consecutive addresses (coalesced, one 128-byte
// line per warp per array in FP32, two in FP64).  Horizontal neighbours
// (i +- 1, j +- 1) are re-reads of lines that neighbouring threads of the
// same or an adjacent block load, served by L1/L2.  The V-cycle's fused
// residual + restriction is the exception: a thread walks the fine rows of a
// latitude band on one layer (k_resid_restrict), because the restriction
// gathers across rows, not along the column.
//
// The path is HBM-bound in FP32 and FP64-ALU-bound in FP64 on GB300
// (~2 DFMA/clk/SM), so the FP64 kernels minimise FP64 operations: the
// smoother takes the Jacobi arrangement of Eq. (1) (no vertical fluxes, ~10
// FP64 ops per cell) and reads precomputed column factors.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "tpmg_device.cuh"
#include "tpmg_internal.h"

namespace tpmg {

// SM count of the device (set at setup; sizes the work split of the
// cell-parallel transfers).
static int g_sms = 152;

// ------------------------------------------------------------------ stencil
// mode 0: y = H x;  mode 1: y = b - H x.  Flux form
//   (H x)_c = h_c x_c + sum_f T_f (x_c - x_nb(f)).
template <typename T, int MODE, bool RED>
__global__ void __launch_bounds__(kBlock)
k_stencil(LevelDev<T> L, const T *__restrict__ b, const T *__restrict__ x, T *__restrict__ y,
          double *__restrict__ partial, const int *__restrict__ flag)
{
    if (flag && !*flag) return;
    const T acc = stencil_column<T, MODE, RED>(L, b, x, y, blockIdx.x * blockDim.x + threadIdx.x);
    if (RED) block_store<0>((double)acc, partial);
}

// d_new = z + beta d_old and q = H d_new in one pass (beta from the CG
// scalars; BZ: first direction d_new = z), with the block sums of <d_new, q>.
template <typename T, bool BZ>
__global__ void __launch_bounds__(kBlock)
k_dir_apply(LevelDev<T> L, const T *__restrict__ z, const T *__restrict__ dold,
            const CgScalars *__restrict__ sc, T *__restrict__ dnew, T *__restrict__ q,
            double *__restrict__ partial, const int *__restrict__ flag)
{
    if (flag && !*flag) return;
    const T beta = BZ ? T(0) : (T)sc->beta;
    const T acc = dir_apply_column<T, BZ>(L, z, dold, beta, dnew, q,
                                          blockIdx.x * blockDim.x + threadIdx.x);
    block_store<0>((double)acc, partial);
}

template <typename T>
int launch_dir_apply(const LevelDev<T> &L, const T *z, const T *d_old, const CgScalars *sc,
                     T *d_new, T *q, double *partial, cudaStream_t s, const int *flag)
{
    if constexpr (sizeof(T) == 4) {
        const int g = launch_dir_apply_tma(L, z, d_old, sc, d_new, q, partial, s, flag);
        if (g >= 0) return g;
    }
    const int ncol = L.nlon * L.nlat;
    const int grid = (ncol + kBlock - 1) / kBlock;
    if (d_old == nullptr)
        k_dir_apply<T, true><<<grid, kBlock, 0, s>>>(L, z, d_old, sc, d_new, q, partial, flag);
    else
        k_dir_apply<T, false><<<grid, kBlock, 0, s>>>(L, z, d_old, sc, d_new, q, partial, flag);
    return grid;
}

// r32 = (float)((b - H x) * inv_scale) with the FP64 residual and the block
// sums of ||b - H x||^2 (the outer step of the mixed-precision refinement:
// no FP64 residual vector is stored).
template <bool NARROW_MUL>
__global__ void __launch_bounds__(kBlock)
k_resid_cast(LevelDev<double> L, const double *__restrict__ b, const double *__restrict__ x,
             float *__restrict__ r32, double inv_scale, double *__restrict__ partial)
{
    const double acc = stencil_column<double, 1, true, float, NARROW_MUL, true>(
        L, b, x, r32, blockIdx.x * blockDim.x + threadIdx.x, inv_scale);
    block_store<0>(acc, partial);
}

// dh = h + the four horizontal couplings of each cell (pole faces carry none).
__global__ void __launch_bounds__(kBlock) k_hdiag(LevelDev<double> L, double *__restrict__ dh)
{
    const int nlon = L.nlon, nlat = L.nlat;
    const size_t plane = (size_t)nlon * nlat, n = plane * L.nz;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x) {
        const size_t col = c % plane;
        const int j = (int)(col / nlon), i = (int)(col - (size_t)j * nlon);
        const size_t iw = (i == 0) ? c + nlon - 1 : c - 1;
        double d = L.h[c] + L.tx[c];
        d += L.tx[iw];
        if (j + 1 < nlat) d += L.ty[c];
        if (j > 0) d += L.ty[c - nlon];
        dh[c] = d;
    }
}

cudaError_t launch_hdiag(const LevelDev<double> &L, double *dh, cudaStream_t s)
{
    const size_t n = (size_t)L.nlon * L.nlat * L.nz;
    const size_t g = std::min((n + (size_t)kBlock * 8 - 1) / ((size_t)kBlock * 8),
                              (size_t)g_sms * 16);
    k_hdiag<<<(int)std::max<size_t>(g, 1), kBlock, 0, s>>>(L, dh);
    return cudaGetLastError();
}

// The refinement's residual: L.h must hold the horizontal diagonal
// (launch_hdiag), the horizontal terms taken in sum form (stencil_column,
// HSUM).
int launch_residual_cast(const LevelDev<double> &L, const double *b, const double *x, float *r32,
                         double inv_scale, double *partial, cudaStream_t s)
{
    const int ncol = L.nlon * L.nlat;
    const int grid = (ncol + kBlock - 1) / kBlock;
    // Scaling after the rounding to float is exact while the residual's
    // significant entries are normal floats: |r| <= ||r|| < 2^10 / inv_scale
    // stays below 2^110, and entries down to 2^-56 ||r|| stay above 2^-126.
    const bool narrow = inv_scale >= 0x1p-100 && inv_scale <= 0x1p60;
    if (narrow) k_resid_cast<true><<<grid, kBlock, 0, s>>>(L, b, x, r32, inv_scale, partial);
    else k_resid_cast<false><<<grid, kBlock, 0, s>>>(L, b, x, r32, inv_scale, partial);
    return grid;
}

// Cell-parallel variant (one thread per cell, grid = column blocks x layers)
// for levels with too few columns to fill the GPU with column loops.
template <typename T, int MODE>
__global__ void __launch_bounds__(kBlock)
k_stencil_cells(LevelDev<T> L, const T *__restrict__ b, const T *__restrict__ x, T *__restrict__ y,
                const int *__restrict__ flag)
{
    if (flag && !*flag) return;
    stencil_cell<T, MODE>(L, b, x, y, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y);
}

// below this many columns the column loops cannot fill the GPU
constexpr int kCellParallelColumns = 32768;

template <typename T>
int launch_stencil(const LevelDev<T> &L, int mode, const T *b, const T *x, T *y, double *partial,
                   cudaStream_t s, const int *flag)
{
    const int ncol = L.nlon * L.nlat;
    const int grid = (ncol + kBlock - 1) / kBlock;
    if (!partial && ncol < kCellParallelColumns) {
        const dim3 g2(grid, L.nz);
        if (mode) k_stencil_cells<T, 1><<<g2, kBlock, 0, s>>>(L, b, x, y, flag);
        else k_stencil_cells<T, 0><<<g2, kBlock, 0, s>>>(L, b, x, y, flag);
        return 0;
    }
    if (partial) {
        if (mode) k_stencil<T, 1, true><<<grid, kBlock, 0, s>>>(L, b, x, y, partial, flag);
        else k_stencil<T, 0, true><<<grid, kBlock, 0, s>>>(L, b, x, y, partial, flag);
        return grid;
    }
    if (mode) k_stencil<T, 1, false><<<grid, kBlock, 0, s>>>(L, b, x, y, nullptr, flag);
    else k_stencil<T, 0, false><<<grid, kBlock, 0, s>>>(L, b, x, y, nullptr, flag);
    return 0;
}

// ------------------------------------------------------------------ smoother
// One sweep of Eq. (1), u_out = (1 - omega) u_in + omega H_z^{-1}(b - dH u_in),
// with the column tridiagonal H_z (diagonal s_k + t_{k-1} + t_k, couplings
// -t_k, s_k = h + the four horizontal couplings) solved by elimination with
// pivots p_k = q_k + t_k:
//   forward   y_k = (v_k + t_{k-1} y_{k-1}) / p_k
//   backward  x_k = x_{k+1} + (y_k - (q_k / p_k) x_{k+1})
// on the setup factors 1/p_k and q_k/p_k.  The forward values y wait in
// shared memory for the backward sweep (blockDim x nz values).
//
// Sweeps from a zero guess (the pre-smoother of every level) read four
// streams per cell (b, t_z, 1/p, q/p) and are staged through shared memory
// by cp.async, kRing layers ahead (smooth_staged); sweeps on a non-zero guess
// read eleven values per cell, and the register pipeline of smooth_column
// keeps more of them in flight than a shared-memory ring of the same depth
// would at its occupancy.
// FP64 sweeps on a guess keep their forward values in the output column:
// 90 registers allow 5 blocks per SM, shared memory for nz x 128 doubles
// only 3.  (FP32 is register-limited at 4 blocks either way, and its
// forward values are better kept out of DRAM.)
template <typename T>
constexpr bool kYOut = sizeof(T) == 8;

template <typename T>
__global__ void __launch_bounds__(kBlock)
k_smooth(LevelDev<T> L, const T *__restrict__ b, const T *__restrict__ uin, T *__restrict__ uout,
         T omega, const int *__restrict__ flag)
{
    if (flag && !*flag) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    smooth_column<T, false, 0, kYOut<T>>(L, b, uin, uout, omega,
                                         blockIdx.x * blockDim.x + threadIdx.x, smraw);
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
k_smooth0(LevelDev<T> L, const T *__restrict__ b, T *__restrict__ uout, T omega,
          const int *__restrict__ flag)
{
    if (flag && !*flag) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    smooth_staged<T, true>(L, b, nullptr, uout, omega, blockIdx.x * blockDim.x + threadIdx.x,
                           smraw);
}

// The last sweep of a V-cycle applied to r, with the block sums of
// <r, u_out> (the CG inner product) written to partial[block].
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_smooth_dot(LevelDev<T> L, const T *__restrict__ b, const T *__restrict__ uin,
             T *__restrict__ uout, T omega, double *__restrict__ partial,
             const int *__restrict__ flag)
{
    if (flag && !*flag) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    T acc = 0;
    smooth_column<T, true, 0, kYOut<T>>(L, b, uin, uout, omega,
                                        blockIdx.x * blockDim.x + threadIdx.x, smraw, &acc);
    block_store<0>((double)acc, partial);
}

template <typename T>
int launch_smooth_dot(const LevelDev<T> &L, const T *b, const T *u_in, T *u_out, double omega,
                      double *partial, cudaStream_t s, const int *flag)
{
    const size_t smem = kYOut<T> ? 0 : (size_t)L.nz * kBlock * sizeof(T);
    const int ncol = L.nlon * L.nlat;
    const int grid = (ncol + kBlock - 1) / kBlock;
    k_smooth_dot<T><<<grid, kBlock, smem, s>>>(L, b, u_in, u_out, (T)omega, partial, flag);
    return grid;
}

// One warp per column (smooth_warp_column), for levels small enough that
// the serial column recurrences would dominate.
template <typename T, bool ZERO, int CM>
__global__ void __launch_bounds__(kBlock)
k_smooth_warp(LevelDev<T> L, const T *__restrict__ b, const T *uin, T *uout, T omega,
              const int *__restrict__ flag)
{
    if (flag && !*flag) return;
    const int col = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (col >= L.nlon * L.nlat) return;  // whole warps
    smooth_warp_column<T, ZERO, CM>(L, b, uin, uout, omega, col, threadIdx.x & 31);
}

// Layers per lane the warp sweeps are unrolled for (smooth_warp_column):
// the smallest of 2, 3 and kWarpLayers that holds nz layers in 32 lanes.
static inline int warp_layers_for(int nz) { return nz <= 64 ? 2 : nz <= 96 ? 3 : kWarpLayers; }

// f.template operator()<CM>() for the CM of nz.
template <typename F>
static inline auto with_warp_layers(int nz, F &&f)
{
    switch (warp_layers_for(nz)) {
    case 2: return f(std::integral_constant<int, 2>{});
    case 3: return f(std::integral_constant<int, 3>{});
    default: return f(std::integral_constant<int, kWarpLayers>{});
    }
}

// The coarsest-level solve (Section 2.3's simple iteration: `sweeps`
// block-Jacobi sweeps from a zero guess) as one block: the warps share the
// columns, a block barrier separates the sweeps, and the sweeps alternate
// between out and scratch so that the last one lands in out.

template <typename T, int CM>
__global__ void __launch_bounds__(kCoarseSolveThreads)
k_coarse_solve(LevelDev<T> L, const T *__restrict__ b, T *out, T *scratch, T omega, int sweeps,
               const int *__restrict__ flag)
{
    if (flag && !*flag) return;
    const int ncol = L.nlon * L.nlat;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T *cur = (sweeps % 2 == 1) ? out : scratch;
    T *oth = (cur == out) ? scratch : out;
    for (int c = warp; c < ncol; c += nw)
        smooth_warp_column<T, true, CM>(L, b, nullptr, cur, omega, c, lane);
    for (int it = 1; it < sweeps; ++it) {
        __syncthreads();  // the previous sweep is visible to the whole block
        for (int c = warp; c < ncol; c += nw)
            smooth_warp_column<T, false, CM>(L, b, cur, oth, omega, c, lane);
        T *t = cur;
        cur = oth;
        oth = t;
    }
}

// The same solve with the whole level in shared memory (coarse_solve_sh).
template <typename T, int CM>
__global__ void __launch_bounds__(kCoarseSolveThreads)
k_coarse_solve_sh(LevelDev<T> L, const T *__restrict__ b, T *__restrict__ out, T omega, int sweeps,
                  const int *__restrict__ flag)
{
    if (flag && !*flag) return;
    extern __shared__ __align__(16) unsigned char sh_raw[];
    coarse_solve_sh<T, CM>(L, b, out, omega, sweeps, reinterpret_cast<T *>(sh_raw));
}

// Opt-in shared memory per block (set by smooth_prepare).
static int g_smem_optin = 48 * 1024;

size_t coarse_sh_bytes(int ncol, int nz, size_t value_bytes)
{
    return (size_t)kCoarseShArrays * ncol * nz * value_bytes;
}

bool coarse_sh_fits(int ncol, int nz, size_t value_bytes)
{
    return coarse_sh_bytes(ncol, nz, value_bytes) <= (size_t)g_smem_optin;
}

// FP32 levels with at most this many cells take the warp sweep (larger
// ones do not fit L2, where the warp's strided column loads cost sectors).
constexpr size_t kWarpSweepCells = (size_t)1 << 17;
// Coarsest levels with at most this many columns take the one-block solve.
constexpr int kCoarseSolveColumns = 2048;

// FP32 only: the scans cost about twice the FP64 operations of the serial
// sweep, and the FP64 sweeps are bound by FP64 arithmetic.
bool coarse_solve_fits(int nlon, int nlat, size_t value_bytes)
{
    return value_bytes == 4 && nlon * nlat <= kCoarseSolveColumns;
}

template <typename T>
cudaError_t launch_coarse_solve(const LevelDev<T> &L, const T *b, T *out, T *scratch, double omega,
                                int sweeps, cudaStream_t s)
{
    const size_t sh = coarse_sh_bytes(L.nlon * L.nlat, L.nz, sizeof(T));
    const bool in_sh = sweeps >= 1 && coarse_sh_fits(L.nlon * L.nlat, L.nz, sizeof(T));
    with_warp_layers(L.nz, [&](auto cm) {
        constexpr int CM = decltype(cm)::value;
        if (in_sh)
            k_coarse_solve_sh<T, CM><<<1, kCoarseSolveThreads, sh, s>>>(L, b, out, (T)omega,
                                                                        sweeps, nullptr);
        else
            k_coarse_solve<T, CM><<<1, kCoarseSolveThreads, 0, s>>>(L, b, out, scratch,
                                                                    (T)omega, sweeps, nullptr);
        return 0;
    });
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_smooth(const LevelDev<T> &L, const T *b, const T *u_in, T *u_out, double omega,
                          cudaStream_t s, const int *flag)
{
    const int ncol = L.nlon * L.nlat;
    const int grid = (ncol + kBlock - 1) / kBlock;
    if constexpr (sizeof(T) == 4) {
        if ((size_t)ncol * L.nz <= kWarpSweepCells) {
            const int wgrid = (int)(((size_t)ncol * 32 + kBlock - 1) / kBlock);
            with_warp_layers(L.nz, [&](auto cm) {
                constexpr int CM = decltype(cm)::value;
                if (u_in == nullptr)
                    k_smooth_warp<T, true, CM><<<wgrid, kBlock, 0, s>>>(L, b, nullptr, u_out,
                                                                        (T)omega, flag);
                else
                    k_smooth_warp<T, false, CM><<<wgrid, kBlock, 0, s>>>(L, b, u_in, u_out,
                                                                         (T)omega, flag);
                return 0;
            });
            return cudaGetLastError();
        }
    }
    if (u_in == nullptr) {
        const size_t smem = ring_smem_bytes<T, true>(L.nz, kBlock);
        k_smooth0<T><<<grid, kBlock, smem, s>>>(L, b, u_out, (T)omega, flag);
    } else {
        const size_t smem = kYOut<T> ? 0 : (size_t)L.nz * kBlock * sizeof(T);
        k_smooth<T><<<grid, kBlock, smem, s>>>(L, b, u_in, u_out, (T)omega, flag);
    }
    return cudaGetLastError();
}

// Allow a kernel the opt-in shared memory per block (lim) less its static
// shared memory as dynamic shared memory.
cudaError_t set_dynamic_smem_limit(const void *kernel, int lim)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                lim - (int)a.sharedSizeBytes);
}

// Set the dynamic shared-memory limit of every smoother kernel to the
// opt-in maximum (must precede stream capture) and record the SM count.
cudaError_t smooth_prepare()
{
    cudaError_t e;
    int dev = 0, sms = 0, lim = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
        cudaSuccess)
        return e;
    if (sms > 0) g_sms = sms;
    if (lim > 0) g_smem_optin = lim;
    const void *kernels[] = {(const void *)k_smooth<double>,     (const void *)k_smooth<float>,
                             (const void *)k_smooth0<double>,    (const void *)k_smooth0<float>,
                             (const void *)k_smooth_dot<double>, (const void *)k_smooth_dot<float>,
                             (const void *)k_coarse_solve_sh<double, 2>,
                             (const void *)k_coarse_solve_sh<double, 3>,
                             (const void *)k_coarse_solve_sh<double, kWarpLayers>,
                             (const void *)k_coarse_solve_sh<float, 2>,
                             (const void *)k_coarse_solve_sh<float, 3>,
                             (const void *)k_coarse_solve_sh<float, kWarpLayers>};
    for (const void *k : kernels)
        if ((e = set_dynamic_smem_limit(k, lim)) != cudaSuccess) return e;
    return cudaSuccess;
}

// Largest dynamic shared memory one smoother block of kBlock columns needs
// for nz layers (checked against the device limit at setup).
size_t smooth_smem_bytes(int nz, size_t value_bytes)
{
    const size_t ring = value_bytes == 8 ? ring_smem_bytes<double, true>(nz, kBlock)
                                         : ring_smem_bytes<float, true>(nz, kBlock);
    const size_t plain = (size_t)nz * kBlock * value_bytes;
    return ring > plain ? ring : plain;
}

// ------------------------------------------------------------------ transfers
// Restriction R = P^T as a gather, one thread per coarse cell (grid: coarse
// column blocks x layers): coarse (I, J, k) sums, over the fine rows listed
// for J with their latitude weights, the fine residuals at longitudes 2I-1,
// 2I, 2I+1, 2I+2 (mod nlon) with weights 1/4, 3/4, 3/4, 1/4.
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_restrict(LevelDev<T> F, LinkDev K, const T *__restrict__ r, T *__restrict__ bc, int kz,
           const int *__restrict__ flag)
{
    if (flag && !*flag) return;
    const int k0 = blockIdx.y * kz;
    restrict_layers<T>(F, K, r, bc, blockIdx.x * blockDim.x + threadIdx.x, k0,
                       min(F.nz, k0 + kz));
}

// Residual and restriction fused (resid_restrict_band): grid x = warps of
// kRROwned coarse columns, y = layers, z = bands of `band` coarse rows
// (kRRBand; fewer on levels too small to fill the GPU, shortening the serial
// row walk of each warp at the cost of forming band-edge rows twice).  With
// the layers before the bands in launch order, the blocks of one band at
// neighbouring layers run together and share the planes above and below in
// L2 (bands before layers: 0.662 instead of 0.614 ms at 1536 x 1152 x 70).
// PRE: u is the sweep from zero (the residual's presmoothing form).  band0:
// first band of this launch (more than 65535 bands take several launches).
// The FP32 PRE form runs at 12 blocks per SM (40 registers): its band walk
// is latency-bound, and the extra resident warps outweigh a few spilled bytes.
template <typename T, bool PRE>
__global__ void __launch_bounds__(kBlock, (PRE && sizeof(T) == 4) ? 12 : 0)
k_resid_restrict(LevelDev<T> F, LinkDev K, const T *__restrict__ b, const T *__restrict__ u,
                 T *__restrict__ bc, T om1, int band0, int band, const int *__restrict__ flag)
{
    if (flag && !*flag) return;
    const int warp = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (warp * kRROwned >= F.nlon / 2) return;  // whole warps
    resid_restrict_band<T, PRE>(F, K, b, u, bc, warp, threadIdx.x & 31,
                                (band0 + (int)blockIdx.z) * band, blockIdx.y, om1, band);
}

bool resid_restrict_fits(const void *b, const void *u, size_t value_bytes)
{
    return (uintptr_t)b % (2 * value_bytes) == 0 && (uintptr_t)u % (2 * value_bytes) == 0;
}

// Coarse rows per band of the fused residual + restriction: the widest
// band (of kRRBand, 4, 2, 1) whose warps still make two waves of 48 per SM.
template <typename T>
int rr_band(const LevelDev<T> &F, const LinkDev &K)
{
    const long long warps = (F.nlon / 2 + kRROwned - 1) / kRROwned;
    int band = kRRBand;
    while (band > 1 && warps * F.nz * ((K.nlat_c + band - 1) / band) < 2LL * 48 * g_sms)
        band /= 2;
    return band;
}

template <typename T>
cudaError_t launch_resid_restrict(const LevelDev<T> &F, const LinkDev &K, const T *b, const T *u,
                                  T *bc, cudaStream_t s, const int *flag, bool presmooth,
                                  double omega)
{
    const int nc = F.nlon / 2;
    const int warps = (nc + kRROwned - 1) / kRROwned;
    const int band = rr_band(F, K);
    const int bands = (K.nlat_c + band - 1) / band;
    const T om1 = T(1) - (T)omega;
    for (int band0 = 0; band0 < bands; band0 += 65535) {  // grid z limit
        const dim3 grid((warps * 32 + kBlock - 1) / kBlock, F.nz, std::min(65535, bands - band0));
        if (presmooth)
            k_resid_restrict<T, true><<<grid, kBlock, 0, s>>>(F, K, b, u, bc, om1, band0, band,
                                                              flag);
        else
            k_resid_restrict<T, false><<<grid, kBlock, 0, s>>>(F, K, b, u, bc, om1, band0, band,
                                                               flag);
    }
    return cudaGetLastError();
}

// Layers per thread of the cell-parallel transfers: enough column-layer
// blocks for two waves of 16 blocks on every SM, and at most 16 layers.

static int layers_per_thread(size_t columns, int nz)
{
    const size_t target = (size_t)g_sms * 16 * kBlock * 2;
    size_t kz = columns * (size_t)nz / target;
    if (kz < 1) kz = 1;
    if (kz > 16) kz = 16;
    return (int)kz;
}

template <typename T>
cudaError_t launch_restrict(const LevelDev<T> &F, const LinkDev &K, const T *r, T *bc,
                            cudaStream_t s, const int *flag)
{
    const int ncol_c = (F.nlon / 2) * K.nlat_c;
    const int kz = layers_per_thread(ncol_c, F.nz);
    const dim3 grid((ncol_c + kBlock - 1) / kBlock, (F.nz + kz - 1) / kz);
    k_restrict<T><<<grid, kBlock, 0, s>>>(F, K, r, bc, kz, flag);
    return cudaGetLastError();
}

// Bilinear prolongation and correction, one thread per pair of fine cells
// (i = 2I, 2I+1) over a range of layers: fine cell 2I adds sum_a w_a
// (3/4 e[J_a, I] + 1/4 e[J_a, I-1]) and 2I+1 adds sum_a w_a (3/4 e[J_a, I] +
// 1/4 e[J_a, I+1]) (periodic in longitude); three coarse loads per coarse
// row serve both.
template <typename T>
__global__ void __launch_bounds__(kBlock)
k_prolong_add(LevelDev<T> F, LinkDev K, const T *__restrict__ ec, T *__restrict__ u, int kz,
              const int *__restrict__ flag)
{
    if (flag && !*flag) return;
    const int k0 = blockIdx.y * kz;
    prolong_layers<T>(F, K, ec, u, blockIdx.x * blockDim.x + threadIdx.x, k0, min(F.nz, k0 + kz));
}

template <typename T>
cudaError_t launch_prolong_add(const LevelDev<T> &F, const LinkDev &K, const T *ec, T *u,
                               cudaStream_t s, const int *flag)
{
    const int npair = (F.nlon / 2) * F.nlat;
    const int kz = layers_per_thread(npair, F.nz);
    const dim3 grid((npair + kBlock - 1) / kBlock, (F.nz + kz - 1) / kz);
    k_prolong_add<T><<<grid, kBlock, 0, s>>>(F, K, ec, u, kz, flag);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ vectors
// Grid of the vector kernels: one wave of full occupancy (16 blocks of 128
// threads per SM) striding over the vector, at least 8 elements per thread;
// a grid-stride stream of this shape runs at the copy rate, where one block
// per few elements spends its time starting blocks.
static inline int red_grid(size_t n)
{
    size_t g = (n + (size_t)kBlock * 8 - 1) / ((size_t)kBlock * 8);
    const size_t wave = (size_t)g_sms * 16;
    if (g > wave) g = wave;
    if (g < 1) g = 1;
    if (g > (size_t)kReduceSlots) g = kReduceSlots;
    return (int)g;
}

int vec_grid(size_t n) { return red_grid(n); }

template <typename T>
int dir_apply_partials(const LevelDev<T> &L, const T *z, const T *d_old, const T *d_new,
                       const T *q)
{
    if constexpr (sizeof(T) == 4) {
        const int g = dir_apply_tma_grid(L, z, d_old, d_new, q);
        if (g >= 0) return g;
    }
    return (L.nlon * L.nlat + kBlock - 1) / kBlock;
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
k_dot(const T *__restrict__ a, const T *__restrict__ b, size_t n, double *partial)
{
    T acc = 0;
#pragma unroll 4
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x)
        acc = fma(a[c], b[c], acc);
    block_store<0>((double)acc, partial);
}

// 16-byte vector forms of the FP32 vector kernels (four elements per load
// and store; the same arithmetic per element, the partial sums grouped by
// vector), for lengths that are multiples of 4 on 16-byte aligned vectors:
// the one-element loops issued four times the instructions and left the CG
// update at ~0.79 of HBM (mixed solve 84.7 -> 82.6 ms with the vector form).
static bool vec4_ok(size_t n, const void *a, const void *b = nullptr, const void *c = nullptr,
                    const void *d = nullptr)
{
    return n % 4 == 0 && ((uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d) % 16 == 0;
}

__global__ void __launch_bounds__(kBlock)
k_dot_f4(const float4 *__restrict__ a, const float4 *__restrict__ b, size_t n4, double *partial)
{
    float acc = 0.f;
#pragma unroll 2
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n4;
         c += (size_t)gridDim.x * blockDim.x) {
        const float4 x = __ldg(a + c), y = __ldg(b + c);
        acc = fmaf(x.x, y.x, acc);
        acc = fmaf(x.y, y.y, acc);
        acc = fmaf(x.z, y.z, acc);
        acc = fmaf(x.w, y.w, acc);
    }
    block_store<0>((double)acc, partial);
}

template <typename T>
int launch_dot(const T *a, const T *b, size_t n, double *partial, cudaStream_t s)
{
    const int g = red_grid(n);
    if constexpr (sizeof(T) == 4) {
        if (vec4_ok(n, a, b)) {
            k_dot_f4<<<g, kBlock, 0, s>>>(reinterpret_cast<const float4 *>(a),
                                          reinterpret_cast<const float4 *>(b), n / 4, partial);
            return g;
        }
    }
    k_dot<T><<<g, kBlock, 0, s>>>(a, b, n, partial);
    return g;
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_maxabs(const T *__restrict__ a, size_t n, double *partial)
{
    double m = 0;
#pragma unroll 4
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x)
        m = max_mag(m, (double)a[c]);  // NaN propagates
    block_store<1>(m, partial);
}

template <typename T>
int launch_maxabs(const T *a, size_t n, double *partial, cudaStream_t s)
{
    const int g = red_grid(n);
    k_maxabs<T><<<g, kBlock, 0, s>>>(a, n, partial);
    return g;
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
k_cg_update(T *__restrict__ x, T *__restrict__ r, const T *__restrict__ d, const T *__restrict__ Ad,
            size_t n, const CgScalars *sc, double *partial)
{
    const T alpha = (T)sc->alpha;
    T acc = 0;
#pragma unroll 4
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x) {
        x[c] = fma(alpha, d[c], x[c]);
        const T rv = fma(-alpha, Ad[c], r[c]);
        r[c] = rv;
        acc = fma(rv, rv, acc);
    }
    block_store<0>((double)acc, partial);
}

__global__ void __launch_bounds__(kBlock)
k_cg_update_f4(float4 *__restrict__ x, float4 *__restrict__ r, const float4 *__restrict__ d,
               const float4 *__restrict__ Ad, size_t n4, const CgScalars *sc,
               double *partial)
{
    const float alpha = (float)sc->alpha;
    float acc = 0.f;
#pragma unroll 2
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n4;
         c += (size_t)gridDim.x * blockDim.x) {
        float4 xv = x[c], rv = r[c];
        const float4 dv = __ldg(d + c), qv = __ldg(Ad + c);
        xv.x = fmaf(alpha, dv.x, xv.x);
        xv.y = fmaf(alpha, dv.y, xv.y);
        xv.z = fmaf(alpha, dv.z, xv.z);
        xv.w = fmaf(alpha, dv.w, xv.w);
        rv.x = fmaf(-alpha, qv.x, rv.x);
        rv.y = fmaf(-alpha, qv.y, rv.y);
        rv.z = fmaf(-alpha, qv.z, rv.z);
        rv.w = fmaf(-alpha, qv.w, rv.w);
        x[c] = xv;
        r[c] = rv;
        acc = fmaf(rv.x, rv.x, acc);
        acc = fmaf(rv.y, rv.y, acc);
        acc = fmaf(rv.z, rv.z, acc);
        acc = fmaf(rv.w, rv.w, acc);
    }
    block_store<0>((double)acc, partial);
}

template <typename T>
int launch_cg_update(T *x, T *r, const T *d, const T *Ad, size_t n, const CgScalars *sc,
                     double *partial, cudaStream_t s)
{
    const int g = red_grid(n);
    if constexpr (sizeof(T) == 4) {
        if (vec4_ok(n, x, r, d, Ad)) {
            k_cg_update_f4<<<g, kBlock, 0, s>>>(
                reinterpret_cast<float4 *>(x), reinterpret_cast<float4 *>(r),
                reinterpret_cast<const float4 *>(d), reinterpret_cast<const float4 *>(Ad), n / 4,
                sc, partial);
            return g;
        }
    }
    k_cg_update<T><<<g, kBlock, 0, s>>>(x, r, d, Ad, n, sc, partial);
    return g;
}

template <typename T, bool BZ>
__global__ void __launch_bounds__(kBlock)
k_cg_direction(const T *__restrict__ z, const T *__restrict__ din, T *__restrict__ dout, size_t n,
               const CgScalars *sc)
{
    const T beta = BZ ? T(0) : (T)sc->beta;
#pragma unroll 4
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x)
        dout[c] = BZ ? z[c] : fma(beta, din[c], z[c]);
}

template <bool BZ>
__global__ void __launch_bounds__(kBlock)
k_cg_direction_f4(const float4 *__restrict__ z, const float4 *__restrict__ din,
                  float4 *__restrict__ dout, size_t n4, const CgScalars *sc)
{
    const float beta = BZ ? 0.f : (float)sc->beta;
#pragma unroll 2
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n4;
         c += (size_t)gridDim.x * blockDim.x) {
        const float4 zv = __ldg(z + c);
        if (BZ) {
            dout[c] = zv;
        } else {
            const float4 dv = din[c];
            dout[c] = make_float4(fmaf(beta, dv.x, zv.x), fmaf(beta, dv.y, zv.y),
                                  fmaf(beta, dv.z, zv.z), fmaf(beta, dv.w, zv.w));
        }
    }
}

template <typename T>
cudaError_t launch_cg_direction(const T *z, const T *d_in, T *d_out, size_t n, const CgScalars *sc,
                                bool beta_zero, cudaStream_t s)
{
    const int g = red_grid(n);
    if constexpr (sizeof(T) == 4) {
        if (vec4_ok(n, z, d_in, d_out)) {
            const float4 *z4 = reinterpret_cast<const float4 *>(z);
            const float4 *di = reinterpret_cast<const float4 *>(d_in);
            float4 *dw = reinterpret_cast<float4 *>(d_out);
            if (beta_zero) k_cg_direction_f4<true><<<g, kBlock, 0, s>>>(z4, di, dw, n / 4, sc);
            else k_cg_direction_f4<false><<<g, kBlock, 0, s>>>(z4, di, dw, n / 4, sc);
            return cudaGetLastError();
        }
    }
    if (beta_zero) k_cg_direction<T, true><<<g, kBlock, 0, s>>>(z, d_in, d_out, n, sc);
    else k_cg_direction<T, false><<<g, kBlock, 0, s>>>(z, d_in, d_out, n, sc);
    return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_add(T *__restrict__ x, const T *__restrict__ e, size_t n)
{
#pragma unroll 4
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x)
        x[c] += e[c];
}

template <typename T>
cudaError_t launch_add(T *x, const T *e, size_t n, cudaStream_t s)
{
    k_add<T><<<red_grid(n), kBlock, 0, s>>>(x, e, n);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kBlock)
k_cast_scaled(const double *__restrict__ r, float *__restrict__ r32, double inv, size_t n)
{
    const int sx = pow2_exponent(inv);
#pragma unroll 4
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x)
        r32[c] = scaled_to_f32(r[c], inv, sx);
}

__global__ void __launch_bounds__(kBlock)
k_cast_scaled_v4(const double2 *__restrict__ r, float4 *__restrict__ r32, double inv, size_t n4)
{
    const int sx = pow2_exponent(inv);
#pragma unroll 2
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n4;
         c += (size_t)gridDim.x * blockDim.x) {
        const double2 a = __ldg(r + 2 * c), b = __ldg(r + 2 * c + 1);
        r32[c] = make_float4(scaled_to_f32(a.x, inv, sx), scaled_to_f32(a.y, inv, sx),
                             scaled_to_f32(b.x, inv, sx), scaled_to_f32(b.y, inv, sx));
    }
}

cudaError_t launch_cast_scaled(const double *r, float *r32, double inv_scale, size_t n,
                               cudaStream_t s)
{
    if (vec4_ok(n, r, r32))
        k_cast_scaled_v4<<<red_grid(n), kBlock, 0, s>>>(reinterpret_cast<const double2 *>(r),
                                                         reinterpret_cast<float4 *>(r32),
                                                         inv_scale, n / 4);
    else
        k_cast_scaled<<<red_grid(n), kBlock, 0, s>>>(r, r32, inv_scale, n);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kBlock)
k_update_mixed(double *__restrict__ x, const float *__restrict__ e, double scale, size_t n)
{
#pragma unroll 4
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x)
        x[c] = fma(scale, f32_to_f64(e[c]), x[c]);
}

__global__ void __launch_bounds__(kBlock)
k_update_mixed_v4(double2 *__restrict__ x, const float4 *__restrict__ e, double scale, size_t n4)
{
#pragma unroll 2
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n4;
         c += (size_t)gridDim.x * blockDim.x) {
        const float4 ev = __ldg(e + c);
        double2 a = x[2 * c], b = x[2 * c + 1];
        a.x = fma(scale, f32_to_f64(ev.x), a.x);
        a.y = fma(scale, f32_to_f64(ev.y), a.y);
        b.x = fma(scale, f32_to_f64(ev.z), b.x);
        b.y = fma(scale, f32_to_f64(ev.w), b.y);
        x[2 * c] = a;
        x[2 * c + 1] = b;
    }
}

cudaError_t launch_update_mixed(double *x, const float *e, double scale, size_t n, cudaStream_t s)
{
    if (vec4_ok(n, x, e))
        k_update_mixed_v4<<<red_grid(n), kBlock, 0, s>>>(reinterpret_cast<double2 *>(x),
                                                          reinterpret_cast<const float4 *>(e),
                                                          scale, n / 4);
    else
        k_update_mixed<<<red_grid(n), kBlock, 0, s>>>(x, e, scale, n);
    return cudaGetLastError();
}

// Fixed-order final reduction of per-block partials and the CG scalar update.
__global__ void __launch_bounds__(1024)
k_finalize(const double *__restrict__ partial, int n, CgScalars *sc, int which, int op)
{
    __shared__ double ws[32];
    double v = 0;
    for (int c = threadIdx.x; c < n; c += blockDim.x)
        v = op == 3 ? max_mag(v, partial[c]) : v + partial[c];
    if (op == 3) v = warp_reduce<1>(v);
    else v = warp_reduce<0>(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        if (op == 3) v = warp_reduce<1>(v);
        else v = warp_reduce<0>(v);
        if (lane == 0) {
            double *slots = reinterpret_cast<double *>(sc);
            slots[which] = v;
            // a zero denominator only follows an exact solution (r = 0): the
            // step and the new direction's history are then zero
            if (op == 1) sc->alpha = v != 0.0 ? sc->rz / v : 0.0;
            if (op == 2) {
                sc->beta = sc->rz != 0.0 ? v / sc->rz : 0.0;
                sc->rz = v;
            }
        }
    }
}

cudaError_t launch_finalize(const double *partial, int n, CgScalars *sc, int which, int op,
                            cudaStream_t s)
{
    k_finalize<<<1, 1024, 0, s>>>(partial, n, sc, which, op);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ setup
// Error bits: 1 h <= 0 or non-finite; 2 T < 0 or non-finite; 4 non-zero pole/top face.
__global__ void __launch_bounds__(kBlock) k_validate(LevelDev<double> L, int *flag)
{
    const size_t n = (size_t)L.nz * L.nlat * L.nlon;
    const size_t plane = (size_t)L.nlat * L.nlon;
    int bits = 0;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x) {
        const double h = L.h[c], tx = L.tx[c], ty = L.ty[c], tz = L.tz[c];
        if (!(h > 0.0) || !isfinite(h)) bits |= 1;
        if (!(tx >= 0.0) || !isfinite(tx) || !(ty >= 0.0) || !isfinite(ty) || !(tz >= 0.0) ||
            !isfinite(tz))
            bits |= 2;
        const size_t k = c / plane;
        const size_t j = (c - k * plane) / L.nlon;
        if (j + 1 == (size_t)L.nlat && ty != 0.0) bits |= 4;
        if (k + 1 == (size_t)L.nz && tz != 0.0) bits |= 4;
    }
    if (bits) atomicOr(flag, bits);
}

cudaError_t launch_validate(const LevelDev<double> &L, int *flag, cudaStream_t s)
{
    const size_t n = (size_t)L.nz * L.nlat * L.nlon;
    k_validate<<<red_grid(n), kBlock, 0, s>>>(L, flag);
    return cudaGetLastError();
}

// Coarse coefficients (rediscretisation of the same flux form on the coarse
// cells): h and tz summed over the children; the coarse east face sums the
// fine east faces of the children at i = 2I+1 (times sx = 1/2, the ratio of
// the centre distances); the coarse north face sums the north faces of the
// top child row (times sy[J]); the north-pole face is zero.
__global__ void __launch_bounds__(kBlock)
k_coarsen(LevelDev<double> F, LinkDev K, double sx, double *__restrict__ txc,
          double *__restrict__ tyc, double *__restrict__ tzc, double *__restrict__ hc)
{
    const int nf = F.nlon, nc = nf / 2;
    const int ncol_c = nc * K.nlat_c;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol_c) return;
    const int J = col / nc, I = col - J * nc;
    const int j0 = K.cfirst[J], cnt = K.ccnt[J], top = j0 + cnt - 1;
    const size_t plane_f = (size_t)nf * F.nlat, plane_c = (size_t)ncol_c;
    for (int k = 0; k < F.nz; ++k) {
        const size_t of = (size_t)k * plane_f;
        double hs = 0, zs = 0, xs = 0;
        for (int j = j0; j <= top; ++j) {
            const size_t a = of + (size_t)j * nf + 2 * I;
            hs += F.h[a];
            hs += F.h[a + 1];
            zs += F.tz[a];
            zs += F.tz[a + 1];
            xs += F.tx[a + 1];
        }
        const size_t t = of + (size_t)top * nf + 2 * I;
        double ys = 0;
        ys += F.ty[t];
        ys += F.ty[t + 1];
        const size_t oc = (size_t)k * plane_c + col;
        hc[oc] = hs;
        tzc[oc] = zs;
        txc[oc] = xs * sx;
        tyc[oc] = (J == K.nlat_c - 1) ? 0.0 : ys * K.sy[J];
    }
}

cudaError_t launch_coarsen(const LevelDev<double> &F, const LinkDev &K, double sx, double *txc,
                           double *tyc, double *tzc, double *hc, cudaStream_t s)
{
    const int ncol_c = (F.nlon / 2) * K.nlat_c;
    k_coarsen<<<(ncol_c + kBlock - 1) / kBlock, kBlock, 0, s>>>(F, K, sx, txc, tyc, tzc, hc);
    return cudaGetLastError();
}

// Column factors: q_0 = s_0, q_k = s_k + t_{k-1} q_{k-1} / p_{k-1}, p_k = q_k + t_k;
// store m = 1/p and dq = q/p.
__global__ void __launch_bounds__(kBlock)
k_column_lu(LevelDev<double> L, double *__restrict__ m, double *__restrict__ dq)
{
    const int nlon = L.nlon, nlat = L.nlat;
    const int ncol = nlon * nlat;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const int j = col / nlon, i = col - j * nlon;
    const int iw = (i == 0) ? col + nlon - 1 : col - 1;
    const size_t plane = (size_t)ncol;
    double qp = 0, pp = 1, tdn = 0;
    for (int k = 0; k < L.nz; ++k) {
        const size_t o = (size_t)k * plane;
        double s = L.h[o + col] + L.tx[o + col] + L.tx[o + iw] + L.ty[o + col];
        if (j > 0) s += L.ty[o + col - nlon];
        const double q = (k == 0) ? s : s + tdn * qp / pp;
        const double tup = L.tz[o + col];
        const double p = q + tup;
        m[o + col] = 1.0 / p;
        dq[o + col] = q / p;
        qp = q;
        pp = p;
        tdn = tup;
    }
}

cudaError_t launch_column_lu(const LevelDev<double> &L, double *m, double *dq, cudaStream_t s)
{
    const int ncol = L.nlon * L.nlat;
    k_column_lu<<<(ncol + kBlock - 1) / kBlock, kBlock, 0, s>>>(L, m, dq);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kBlock)
k_to_float(const double *__restrict__ in, float *__restrict__ out, double scale, size_t n)
{
    const int sx = pow2_exponent(scale);
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
         c += (size_t)gridDim.x * blockDim.x)
        out[c] = scaled_to_f32(in[c], scale, sx);
}

cudaError_t launch_to_float(const double *in, float *out, double scale, size_t n, cudaStream_t s)
{
    k_to_float<<<red_grid(n), kBlock, 0, s>>>(in, out, scale, n);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ gradient
__global__ void __launch_bounds__(kBlock)
k_coeff_grad(int nlon, int nlat, int nz, const double *__restrict__ lam,
             const double *__restrict__ x, double *gh, double *gtx, double *gty, double *gtz)
{
    const int ncol = nlon * nlat;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncol) return;
    const int j = col / nlon, i = col - j * nlon;
    const int ie = (i + 1 == nlon) ? col - i : col + 1;
    const size_t plane = (size_t)ncol;
    for (int k = 0; k < nz; ++k) {
        const size_t o = (size_t)k * plane + col;
        const double l = lam[o], xv = x[o];
        if (gh) gh[o] = -l * xv;
        if (gtx) {
            const size_t e = (size_t)k * plane + ie;
            gtx[o] = -(l - lam[e]) * (xv - x[e]);
        }
        if (gty) gty[o] = (j + 1 < nlat) ? -(l - lam[o + nlon]) * (xv - x[o + nlon]) : 0.0;
        if (gtz) gtz[o] = (k + 1 < nz) ? -(l - lam[o + plane]) * (xv - x[o + plane]) : 0.0;
    }
}

cudaError_t launch_coeff_grad(int nlon, int nlat, int nz, const double *lam, const double *x,
                              double *gh, double *gtx, double *gty, double *gtz, cudaStream_t s)
{
    const int ncol = nlon * nlat;
    k_coeff_grad<<<(ncol + kBlock - 1) / kBlock, kBlock, 0, s>>>(nlon, nlat, nz, lam, x, gh, gtx,
                                                                gty, gtz);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ instantiations
#define TPMG_INST(T)                                                                              \
    template int launch_stencil<T>(const LevelDev<T> &, int, const T *, const T *, T *, double *, \
                                   cudaStream_t, const int *);                                    \
    template cudaError_t launch_smooth<T>(const LevelDev<T> &, const T *, const T *, T *, double,  \
                                          cudaStream_t, const int *);                             \
    template int launch_smooth_dot<T>(const LevelDev<T> &, const T *, const T *, T *, double,      \
                                      double *, cudaStream_t, const int *);                       \
    template cudaError_t launch_resid_restrict<T>(const LevelDev<T> &, const LinkDev &, const T *, \
                                                  const T *, T *, cudaStream_t, const int *, bool, \
                                                  double);                                        \
    template int rr_band<T>(const LevelDev<T> &, const LinkDev &);                                 \
    template cudaError_t launch_restrict<T>(const LevelDev<T> &, const LinkDev &, const T *, T *,  \
                                            cudaStream_t, const int *);                           \
    template cudaError_t launch_prolong_add<T>(const LevelDev<T> &, const LinkDev &, const T *,    \
                                               T *, cudaStream_t, const int *);                   \
    template int launch_dot<T>(const T *, const T *, size_t, double *, cudaStream_t);             \
    template int launch_maxabs<T>(const T *, size_t, double *, cudaStream_t);                     \
    template int launch_cg_update<T>(T *, T *, const T *, const T *, size_t, const CgScalars *,    \
                                     double *, cudaStream_t);                                     \
    template cudaError_t launch_cg_direction<T>(const T *, const T *, T *, size_t,                \
                                                const CgScalars *, bool, cudaStream_t);           \
    template cudaError_t launch_add<T>(T *, const T *, size_t, cudaStream_t);                    \
    template cudaError_t launch_coarse_solve<T>(const LevelDev<T> &, const T *, T *, T *, double, \
                                                int, cudaStream_t);                               \
    template int launch_dir_apply<T>(const LevelDev<T> &, const T *, const T *, const CgScalars *, \
                                     T *, T *, double *, cudaStream_t, const int *);            \
    template int dir_apply_partials<T>(const LevelDev<T> &, const T *, const T *, const T *,      \
                                       const T *);

TPMG_INST(double)
TPMG_INST(float)

}  // namespace tpmg
