// The FP32 direction update + apply of the conjugate-gradient iteration
// (q = H d, d = z + beta d_old, <d, q>) with its layer planes staged by the
// Tensor Memory Accelerator (cp.async.bulk.tensor into shared memory,
// completion on mbarriers), for the levels large enough to be bound by HBM
// bandwidth.
//
// A block owns a tile of TI x TJ columns (one consumer thread per column)
// and walks the layers.  One extra warp of the block is the producer: for
// each layer its lane 0 issues the bulk copies of every array's plane tile
// into a stage of a ring in shared memory (the coefficients of the tile,
// t_x with the column west of it, t_y with the row south of it, and the
// vectors read at the horizontal neighbours with a one-cell halo), as soon
// as the consumer warps have released that stage; the consumers wait for a
// stage's bytes, compute, and release it (mbarriers both ways, no block-wide
// barrier per layer).  The copies hold no registers, so many layers of loads
// are in flight per block at a few dozen registers per thread, and one
// instruction moves a plane tile where the register pipeline issued one load
// per value.
//
// Tensor maps are 3-D [nz][nlat][nlon] views of each array, encoded on the
// host per launch.  The box of a halo'd array starts 4 values west of the
// tile (a 16-byte aligned x coordinate, as the bulk copies require) and one
// row south; rows beyond the poles and longitudes beyond the ends of the
// grid arrive as zeros, and the periodic neighbours across the longitude
// seam (the first and last columns of the grid) are read with plain loads.
// Every value enters the arithmetic in the same operation and order as in
// the register-pipeline kernel (dir_apply_column in tpmg_device.cuh), so the
// outputs are equal bit for bit; only the grouping of the fused inner
// product's partial sums follows the tiles.
//
// Throughput of these staged column walks grows with the columns resident
// per SM (each layer step costs a near-fixed latency), so the ring is kept
// small.  The same staging of the block-Jacobi sweep of Eq. (1) did not beat
// its register-pipeline kernel: its forward values must wait for the
// backward pass (in shared memory they cap residency; kept in L2 through
// the output array, the sweep with its fused inner product still ran at
// 0.96 ms against 0.82 ms at 1536 x 1152 x 70), so the sweeps keep the
// register pipeline.  Nor did the sweep from a zero guess: its layer of a
// 32 x 8 tile is only 3 KB (b, t_z, 1/p; 1 KB of q/p on the way back), a
// ring handoff takes ~3 us under load, and the forward values (70 KB per
// tile) leave room for two blocks of eight stages per SM, ~50 KB in flight:
// 1.17 ms against 0.48 ms for the per-thread cp.async ring, which keeps
// each thread's own copies in flight with no handoff between warps.
//
// Waits on the mbarriers are bounded: a thread that gives up records it in
// a device flag (MG_ERR_TIMEOUT at the end of a solve) and raises an abort
// flag in shared memory that ends every other wait of the block; the
// producer then waits (bounded) for its own copies in flight before the
// block leaves its shared memory.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "tpmg_device.cuh"
#include "tpmg_internal.h"

namespace tpmg {

namespace {

constexpr int TI = 32;                     // tile width (longitudes), one warp
constexpr unsigned kWaitSpins = 1u << 22;  // bounded mbarrier wait

__device__ int g_tma_timeouts;  // threads that gave up waiting on a copy

__host__ __device__ constexpr int al128(int b) { return (b + 127) / 128 * 128; }

__device__ __forceinline__ uint32_t saddr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void bar_expect(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait that also gives up once another thread of the block has
// given up (*abort set); a thread whose own wait runs out records it.
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    for (unsigned it = 0; it < kWaitSpins; ++it) {
        if (bar_try(bar, parity)) return true;
        if ((it & 63u) == 63u && *abort) return false;
    }
    if (!*abort) atomicAdd(&g_tma_timeouts, 1);
    *abort = 1;
    return false;
}

// A consumer warp has finished reading a stage: one arrival per warp.
__device__ __forceinline__ void bar_release(uint64_t *bar)
{
    __syncwarp();
    if ((threadIdx.x & 31) == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

// Bulk tensor copy of the box at (x, y, z) into shared memory; with a
// 64-bit L2 eviction policy when pol != 0.
__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *map, int x, int y, int z,
                                         uint64_t *bar, unsigned long long pol = 0)
{
    if (pol)
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
            ".L2::cache_hint [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(saddr(dst)),
            "l"(map), "r"(x), "r"(y), "r"(z), "r"(saddr(bar)), "l"(pol)
            : "memory");
    else
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(saddr(dst)),
            "l"(map), "r"(x), "r"(y), "r"(z), "r"(saddr(bar))
            : "memory");
}

// Ring protocol.  Warp NC of the block is the producer, warps 0..NC-1
// consume.  Stage s has a `full` barrier (one arrival: the producer's
// expect_tx; completes when the stage's bytes have landed) and an `empty`
// barrier (NC arrivals: each consumer warp once it has read the stage).  The
// n-th use of a stage (n = 0, 1, ...) waits on full with parity n & 1; the
// producer refills the stage once empty has completed phase n - 1.
template <int S>
struct Ring {
    uint64_t full[S], empty[S];
    int abort;
};

template <int S>
__device__ __forceinline__ void ring_init(Ring<S> *R, int nc)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            bar_init(&R->full[s], 1);
            bar_init(&R->empty[s], (unsigned)nc);
        }
        R->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

// The producer (lane 0 of the producer warp): `uses` stage uses in order,
// issue(n, s) arming full[s] and issuing the n-th use's copies.  After an
// abort it lets the last copy issued into each stage land (bounded) before
// the block leaves its shared memory.
template <int S, typename Issue>
__device__ __forceinline__ void produce(Ring<S> *R, int uses, Issue issue)
{
    int issued[S];
    for (int s = 0; s < S; ++s) issued[s] = 0;
    bool ok = true;
    for (int n = 0; n < uses; ++n) {
        const int s = n % S, use = n / S;
        if (use > 0 && !bar_wait(&R->empty[s], (uint32_t)((use - 1) & 1), &R->abort)) {
            ok = false;
            break;
        }
        issue(n, s);
        ++issued[s];
    }
    if (!ok)
        for (int s = 0; s < S; ++s)
            if (issued[s] > 0)
                for (unsigned it = 0; it < kWaitSpins; ++it)
                    if (bar_try(&R->full[s], (uint32_t)((issued[s] - 1) & 1))) break;
}

// ------------------------------------------------------------------ maps
typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        cudaGetLastError();
    });
    return fn;
}

// 3-D FP32 view [nz][nlat][nlon] of p with a bx x by x 1 box.
bool encode(CUtensorMap *m, const float *p, int nlon, int nlat, int nz, int bx, int by)
{
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nlon, (cuuint64_t)nlat, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nlon * 4, (cuuint64_t)nlon * nlat * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1}, es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(p), dims, strides, box,
               es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Levels that take the staged kernels: HBM-bound sizes, rows of whole
// 16-byte groups (the strides of a tensor map), 16-byte aligned arrays.
bool usable(const LevelDev<float> &L, std::initializer_list<const void *> ptrs)
{
    if ((long long)L.nlon * L.nlat < kTmaMinColumns || L.nlon % 4 || L.nz > kMaxLayers)
        return false;
    for (const void *p : ptrs)
        if (p && !aligned16(p)) return false;
    return encoder() != nullptr;
}

// Sum over the consumer threads (warps 0..nc-1) of v into partial[blockIdx.x];
// every thread of the block calls it (the producer warp with v = 0).
__device__ __forceinline__ void block_sum_store(double v, double *partial)
{
    block_store<0>(v, partial);
}

// ------------------------------------------------------------------ direction update + apply
// Tile 32 x 8 columns: 8 consumer warps and a producer warp; ring of
// kDirStages layers.
constexpr int kDirTJ = 8, kDirConsumers = kDirTJ, kDirThreads = TI * (kDirTJ + 1),
              kDirStages = 6;
constexpr int kXW = TI + 8;                 // halo box width: i0-4 .. i0+TI+3
constexpr int kTXW = TI + 4;                // t_x box width: i0-4 .. i0+TI-1

template <bool BZ>
struct DirStage {
    static constexpr int XH = kDirTJ + 2, TYH = kDirTJ + 1;
    static constexpr int Z = 0, D = Z + al128(kXW * XH * 4);
    static constexpr int TX = D + (BZ ? 0 : al128(kXW * XH * 4));
    static constexpr int TY = TX + al128(kTXW * kDirTJ * 4);
    static constexpr int TZ = TY + al128(TI * TYH * 4);
    static constexpr int H = TZ + al128(TI * kDirTJ * 4);
    static constexpr int BYTES = H + al128(TI * kDirTJ * 4);
    static constexpr unsigned TX_BYTES =
        (kXW * XH * (BZ ? 1 : 2) + kTXW * kDirTJ + TI * TYH + 2 * TI * kDirTJ) * 4;
    static constexpr size_t SMEM = (size_t)kDirStages * BYTES + 128 + sizeof(Ring<kDirStages>);
};

struct DirMaps {
    CUtensorMap z, d, tx, ty, tz, h;
};

template <bool BZ>
__global__ void __launch_bounds__(kDirThreads)
k_dir_apply_tma(const __grid_constant__ DirMaps M, LevelDev<float> L, const float *__restrict__ z,
                const float *__restrict__ dold, const CgScalars *__restrict__ sc,
                float *__restrict__ dnew, float *__restrict__ q, double *__restrict__ partial,
                const int *__restrict__ flag)
{
    using St = DirStage<BZ>;
    constexpr int S = kDirStages;
    if (flag && !*flag) return;
    extern __shared__ unsigned char smraw[];
    unsigned char *sm = smraw + ((128u - (saddr(smraw) & 127u)) & 127u);
    Ring<S> *R = reinterpret_cast<Ring<S> *>(sm + S * St::BYTES);
    const int nlon = L.nlon, nlat = L.nlat, nz = L.nz;
    const int ntx = (nlon + TI - 1) / TI;
    const int i0 = (blockIdx.x % ntx) * TI, j0 = (blockIdx.x / ntx) * kDirTJ;
    const int warp = threadIdx.x >> 5;
    ring_init(R, kDirConsumers);
    float acc = 0.f;
    if (warp == kDirConsumers) {  // producer
        if ((threadIdx.x & 31) == 0)
            produce<S>(R, nz, [&](int k, int s) {
                unsigned char *st = sm + s * St::BYTES;
                uint64_t *bar = &R->full[s];
                bar_expect(bar, St::TX_BYTES);
                tma_load(st + St::Z, &M.z, i0 - 4, j0 - 1, k, bar);
                if (!BZ) tma_load(st + St::D, &M.d, i0 - 4, j0 - 1, k, bar);
                tma_load(st + St::TX, &M.tx, i0 - 4, j0, k, bar);
                tma_load(st + St::TY, &M.ty, i0, j0 - 1, k, bar);
                tma_load(st + St::TZ, &M.tz, i0, j0, k, bar);
                tma_load(st + St::H, &M.h, i0, j0, k, bar);
            });
    } else {  // consumers: one column each
        const int ti = threadIdx.x % TI, tj = warp;
        const int i = i0 + ti, j = j0 + tj;
        const bool inside = i < nlon && j < nlat;
        const bool hasN = j + 1 < nlat, hasS = j > 0;
        const size_t plane = (size_t)nlon * nlat;
        const size_t col = (size_t)j * nlon + i;
        const float beta = BZ ? 0.f : (float)sc->beta;
        auto dv = [&](float zv, float dvv) { return BZ ? zv : fmaf(beta, dvv, zv); };
        const int cx = ti + 4, cy = tj + 1;  // own cell in the halo boxes
        const int c = cy * kXW + cx, t = tj * TI + ti;
        float xdn = 0.f, tdn = 0.f;
        for (int k = 0; k < nz; ++k) {
            const int s = k % S;
            if (!bar_wait(&R->full[s], (k / S) & 1, &R->abort)) break;
            // the layer above: its stage is the next one (released after it)
            if (k + 1 < nz && !bar_wait(&R->full[(k + 1) % S], ((k + 1) / S) & 1, &R->abort))
                break;
            const unsigned char *st = sm + s * St::BYTES;
            const float *Z = (const float *)(st + St::Z), *D = (const float *)(st + St::D);
            const float *TX = (const float *)(st + St::TX), *TY = (const float *)(st + St::TY);
            if (inside) {
                const float xc = dv(Z[c], BZ ? 0.f : D[c]);
                float xe = dv(Z[c + 1], BZ ? 0.f : D[c + 1]);
                float xw = dv(Z[c - 1], BZ ? 0.f : D[c - 1]);
                float txw = TX[tj * kTXW + cx - 1];
                const size_t o = (size_t)k * plane + col;
                if (i == 0) {  // periodic neighbour across the seam
                    xw = dv(__ldg(z + o + nlon - 1), BZ ? 0.f : __ldg(dold + o + nlon - 1));
                    txw = __ldg(L.tx + o + nlon - 1);
                }
                if (i + 1 == nlon) xe = dv(__ldg(z + o - i), BZ ? 0.f : __ldg(dold + o - i));
                float xup = 0.f;
                if (k + 1 < nz) {
                    const unsigned char *nx = sm + ((k + 1) % S) * St::BYTES;
                    xup = dv(((const float *)(nx + St::Z))[c],
                             BZ ? 0.f : ((const float *)(nx + St::D))[c]);
                }
                float v = ((const float *)(st + St::H))[t] * xc;
                v = fmaf(TX[tj * kTXW + cx], xc - xe, v);
                v = fmaf(txw, xc - xw, v);
                if (hasN)
                    v = fmaf(TY[(tj + 1) * TI + ti], xc - dv(Z[c + kXW], BZ ? 0.f : D[c + kXW]), v);
                if (hasS)
                    v = fmaf(TY[tj * TI + ti], xc - dv(Z[c - kXW], BZ ? 0.f : D[c - kXW]), v);
                const float tz = ((const float *)(st + St::TZ))[t];
                v = fmaf(tz, xc - xup, v);
                v = fmaf(tdn, xc - xdn, v);
                dnew[o] = xc;
                q[o] = v;
                acc = fmaf(v, xc, acc);
                xdn = xc;
                tdn = tz;
            }
            bar_release(&R->empty[s]);
        }
    }
    block_sum_store(R->abort ? 0.0 : (double)acc, partial);
}

}  // namespace

// ------------------------------------------------------------------ launchers
int dir_apply_tma_grid(const LevelDev<float> &L, const void *z, const void *d_old,
                       const void *d_new, const void *q)
{
    if (!usable(L, {z, d_old, d_new, q, L.tx, L.ty, L.tz, L.h})) return -1;
    const int grid = ((L.nlon + TI - 1) / TI) * ((L.nlat + kDirTJ - 1) / kDirTJ);
    return grid <= kReduceSlots ? grid : -1;
}

int launch_dir_apply_tma(const LevelDev<float> &L, const float *z, const float *d_old,
                         const CgScalars *sc, float *d_new, float *q, double *partial,
                         cudaStream_t s, const int *flag)
{
    const int grid = dir_apply_tma_grid(L, z, d_old, d_new, q);
    if (grid < 0) return -1;
    DirMaps M;
    const int nl = L.nlon, nt = L.nlat, nz = L.nz;
    const int XH = kDirTJ + 2;
    if (!encode(&M.z, z, nl, nt, nz, kXW, XH) ||
        (d_old && !encode(&M.d, d_old, nl, nt, nz, kXW, XH)) ||
        !encode(&M.tx, L.tx, nl, nt, nz, kTXW, kDirTJ) ||
        !encode(&M.ty, L.ty, nl, nt, nz, TI, kDirTJ + 1) ||
        !encode(&M.tz, L.tz, nl, nt, nz, TI, kDirTJ) || !encode(&M.h, L.h, nl, nt, nz, TI, kDirTJ))
        return -1;
    if (!d_old) M.d = M.z;
    if (d_old)
        k_dir_apply_tma<false><<<grid, kDirThreads, DirStage<false>::SMEM, s>>>(
            M, L, z, d_old, sc, d_new, q, partial, flag);
    else
        k_dir_apply_tma<true><<<grid, kDirThreads, DirStage<true>::SMEM, s>>>(
            M, L, z, d_old, sc, d_new, q, partial, flag);
    return grid;  // launch errors are left for the caller's cudaGetLastError
}

// The staged kernels' occupancy is set by their shared memory: ask for the
// largest shared-memory carveout so that as many blocks as fit are resident.
template <typename K>
static cudaError_t prepare_kernel(K kernel, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

cudaError_t tma_prepare()
{
    if (!encoder()) return cudaSuccess;  // no tensor maps: the register kernels run
    cudaError_t e = prepare_kernel(k_dir_apply_tma<false>, DirStage<false>::SMEM);
    if (e == cudaSuccess) e = prepare_kernel(k_dir_apply_tma<true>, DirStage<true>::SMEM);
    return e;
}

int tma_timeouts(cudaStream_t s, bool reset)
{
    int v = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_tma_timeouts, sizeof v, 0, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return -1;
    if (v && reset) {
        const int zero = 0;
        cudaMemcpyToSymbolAsync(g_tma_timeouts, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, s);
    }
    return v;
}

}  // namespace tpmg
