// Internal interface between the host driver (tpmg_api.cpp) and the CUDA
// kernels (tpmg_kernels.cu).  Not part of the public C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace tpmg {

// One multigrid level in one precision.  All pointers are device pointers
// into the caller's workspace, [nz][nlat][nlon] unless noted.
template <typename T>
struct LevelDev {
    int nlon, nlat, nz;
    const T *tx, *ty, *tz, *h;  // coefficients (FP32 copies are scaled by a power of two)
    const T *m;                 // 1 / p_k, pivot inverse of the column tridiagonal
    const T *dq;                // q_k / p_k, p_k = q_k + tz_k (row-sum form of the pivot)
};

// Links from level l to level l+1 (device arrays, sizes in comments).
struct LinkDev {
    int nlat_c;                 // coarse rows
    const int *j0;              // [nlat]   prolongation: fine row j takes w0*row j0
    const double *w0;           // [nlat]
    const int *j1;              // [nlat]   + w1*row j1 (j1 = -1: none)
    const double *w1;           // [nlat]
    const int *rptr;            // [nlat_c+1] restriction: coarse row J gathers rows
    const int *rrow;            //            rrow[rptr[J]..rptr[J+1]) with weights rw
    const double *rw;
    const int *cfirst;          // [nlat_c] first fine row of coarse row J
    const int *ccnt;            // [nlat_c] 1 or 2 fine rows
    const double *sy;           // [nlat_c] coarse north-face distance ratio
};

// Device-side scalars of a conjugate-gradient iteration.
struct CgScalars {
    double rz, rz_new, dAd, rr, alpha, beta, maxabs, pad;
};

// Device-side scalars of a BiCGStab iteration (brk: a breakdown was met).
struct BicgScalars {
    double rho, alpha, omega, beta, rv, ts, tt, rr, brk, pad;
};
enum { BICG_START = 0, BICG_ALPHA = 1, BICG_OMEGA = 2, BICG_NEXT = 3 };

constexpr int kBlock = 128;          // threads per block, one column per thread
constexpr int kMaxLayers = 192;      // MG_MAX_NZ of the C ABI (checked in tpmg_api.cpp)
constexpr int kMaxRestrictRows = 4;  // fine rows per coarse row of the restriction (checked at setup)
constexpr int kCoarseSolveThreads = 1024;  // one-block coarsest-level solve: 32 warps (FP32 only)
// Fused residual + restriction: coarse rows per band, coarse columns owned
// by a warp (lanes 1..30; lanes 0 and 31 carry the neighbours).
constexpr int kRRBand = 8;
constexpr int kRROwned = 30;
constexpr int kReduceSlots = 65536;  // per-block partial sums kept in the workspace

// ---- launchers (tpmg_kernels.cu); all asynchronous on `s` -----------------
// flag (device int, may be null): when it reads 0 the launch does nothing
// (a converged system of a batch).
//
// y = H x (mode 0) or y = b - H x (mode 1).  If `partial` != null each block
// writes sum(y*y) (mode 1) or sum(x*y) (mode 0) to partial[block]; returns
// the number of blocks written (0 if partial == null).
template <typename T>
int launch_stencil(const LevelDev<T> &L, int mode, const T *b, const T *x, T *y,
                   double *partial, cudaStream_t s, const int *flag = nullptr);

// d_new = z + beta d_old (beta read from sc; d_old == nullptr: d_new = z) and
// q = H d_new in one pass, with per-block partial sums of <d_new, q>; returns
// the number of partial sums.
template <typename T>
int launch_dir_apply(const LevelDev<T> &L, const T *z, const T *d_old, const CgScalars *sc,
                     T *d_new, T *q, double *partial, cudaStream_t s, const int *flag = nullptr);

// One smoother sweep of Eq. (1) in the arrangement
//   u_out = (1 - omega) u_in + omega H_z^{-1} (b - dH u_in)
// (u_in == nullptr: zero initial guess).
template <typename T>
cudaError_t launch_smooth(const LevelDev<T> &L, const T *b, const T *u_in, T *u_out,
                          double omega, cudaStream_t s, const int *flag = nullptr);

// The coarsest-level solve: `sweeps` sweeps from a zero guess in one
// one-block launch (result in out; scratch: a second level vector), for
// coarsest levels where coarse_solve_fits(nlon, nlat, sizeof value).
bool coarse_solve_fits(int nlon, int nlat, size_t value_bytes);
template <typename T>
cudaError_t launch_coarse_solve(const LevelDev<T> &L, const T *b, T *out, T *scratch, double omega,
                                int sweeps, cudaStream_t s);

// The same sweep (non-zero guess) writing the block sums of <b, u_out> to
// partial[block]; returns the number of blocks.
template <typename T>
int launch_smooth_dot(const LevelDev<T> &L, const T *b, const T *u_in, T *u_out, double omega,
                      double *partial, cudaStream_t s, const int *flag = nullptr);

// Raise the dynamic shared-memory limit of the smoother kernels (once per
// process and device, before any stream capture).
cudaError_t smooth_prepare();
// dynamic shared memory a kernel may use: lim less its static shared memory
cudaError_t set_dynamic_smem_limit(const void *kernel, int lim);
// dynamic shared memory of the largest smoother block for nz layers of
// value_bytes-wide values
size_t smooth_smem_bytes(int nz, size_t value_bytes);

// b_c = R (b - H u) in one pass; b and u aligned to two values
// (resid_restrict_fits).
bool resid_restrict_fits(const void *b, const void *u, size_t value_bytes);
// presmooth: u is the sweep of Eq. (1) from zero with this omega, and the
// residual is taken as (1 - omega) b plus u's horizontal couplings.
template <typename T>
cudaError_t launch_resid_restrict(const LevelDev<T> &F, const LinkDev &K, const T *b, const T *u,
                                  T *bc, cudaStream_t s, const int *flag = nullptr,
                                  bool presmooth = false, double omega = 0.0);
// Coarse rows per band of its row walk: kRRBand, fewer on levels too small
// to fill the GPU (the same sums in the same order whatever the band).
template <typename T>
int rr_band(const LevelDev<T> &F, const LinkDev &K);
template <typename T>
cudaError_t launch_restrict(const LevelDev<T> &F, const LinkDev &K, const T *r, T *bc,
                            cudaStream_t s, const int *flag = nullptr);

template <typename T>
cudaError_t launch_prolong_add(const LevelDev<T> &F, const LinkDev &K, const T *ec, T *u,
                               cudaStream_t s, const int *flag = nullptr);

// Sum `n` partials in a fixed order into slots[which]; then (op) update
// the CG scalars: 0 plain store, 1 alpha = rz / dAd, 2 beta = rz_new / rz
// and rz = rz_new, 3 max instead of sum.
cudaError_t launch_finalize(const double *partial, int n, CgScalars *sc, int which, int op,
                            cudaStream_t s);

// partial dot products: sum(a*b) per block.
template <typename T>
int launch_dot(const T *a, const T *b, size_t n, double *partial, cudaStream_t s);

// per-block max |a|
template <typename T>
int launch_maxabs(const T *a, size_t n, double *partial, cudaStream_t s);

// x += alpha d; r -= alpha Ad; partial sum(r*r).  alpha from sc->alpha.
template <typename T>
int launch_cg_update(T *x, T *r, const T *d, const T *Ad, size_t n, const CgScalars *sc,
                     double *partial, cudaStream_t s);

// d_out = z + beta d_in (beta from sc->beta; beta_zero: d_out = z).
template <typename T>
cudaError_t launch_cg_direction(const T *z, const T *d_in, T *d_out, size_t n,
                                const CgScalars *sc, bool beta_zero, cudaStream_t s);

// Grid of the vector kernels for n elements (one wave of full occupancy).
int vec_grid(size_t n);

// ---- TMA-staged FP32 direction update + apply (tpmg_tma.cu) ---------------
// Levels of at least kTmaMinColumns columns (and rows of whole 16-byte
// groups, 16-byte aligned arrays) take the staged kernel; the launcher
// returns -1 when a level or buffer does not suit it (the caller then runs
// the register-pipeline kernel), else the number of blocks (and partial
// sums) launched.
constexpr long long kTmaMinColumns = 1LL << 18;
int dir_apply_tma_grid(const LevelDev<float> &L, const void *z, const void *d_old,
                       const void *d_new, const void *q);
int launch_dir_apply_tma(const LevelDev<float> &L, const float *z, const float *d_old,
                         const CgScalars *sc, float *d_new, float *q, double *partial,
                         cudaStream_t s, const int *flag);
// Shared-memory limits of the staged kernel (once per process and device,
// before any stream capture).
cudaError_t tma_prepare();
// Threads of the staged kernel that gave up waiting on a copy since the
// last reset (-1 if the flag could not be read).  Synchronises s.
int tma_timeouts(cudaStream_t s, bool reset);
// Partial sums launch_dir_apply writes for these arguments.
template <typename T>
int dir_apply_partials(const LevelDev<T> &L, const T *z, const T *d_old, const T *d_new,
                       const T *q);

// ---- BiCGStab vector steps (tpmg_krylov.cu); scalars read from sc ----
// p = r (first) or p = r + beta (p - omega v)
template <typename T>
cudaError_t launch_bicg_dir(T *p, const T *r, const T *v, size_t n, const BicgScalars *sc,
                            bool first, cudaStream_t s);
// s = r - alpha v
template <typename T>
cudaError_t launch_bicg_s(T *sv, const T *r, const T *v, size_t n, const BicgScalars *sc,
                          cudaStream_t s);
// per-block <t, s> into pa and <t, t> into pb; returns the number of blocks
template <typename T>
int launch_dot2(const T *t, const T *sv, size_t n, double *pa, double *pb, cudaStream_t s);
// x += alpha ph + omega sh; r = s - omega t; per-block <r, r> (pa), <rh, r> (pb)
template <typename T>
int launch_bicg_update(T *x, T *r, const T *ph, const T *sh, const T *sv, const T *t,
                       const T *rh, size_t n, const BicgScalars *sc, double *pa, double *pb,
                       cudaStream_t s);
// fixed-order sums of the partials and the scalar step op (BICG_*)
cudaError_t launch_bicg_finalize(const double *pa, const double *pb, int n, BicgScalars *sc,
                                 int op, cudaStream_t s);
// x *= f
template <typename T>
cudaError_t launch_scale(T *x, double f, size_t n, cudaStream_t s);
// per-block maxima of (h + horizontal couplings) / h over the level
int launch_hz_ratio(const LevelDev<double> &L, double *partial, cudaStream_t s);
// Chebyshev step: x += d, d = c1 d + c2 z (first: d = c2 z)
template <typename T>
cudaError_t launch_cheb_step(T *x, T *d, const T *z, double c1, double c2, size_t n, bool first,
                             cudaStream_t s);

// x += e (same precision)
template <typename T>
cudaError_t launch_add(T *x, const T *e, size_t n, cudaStream_t s);

// dh = h + the four horizontal couplings (the refinement residual's diagonal).
cudaError_t launch_hdiag(const LevelDev<double> &L, double *dh, cudaStream_t s);
// r32 = (float)((b - H x) * inv_scale) and ||b - H x||^2 partial sums, L.h
// replaced by the horizontal diagonal (launch_hdiag); returns the number of
// partial sums.
int launch_residual_cast(const LevelDev<double> &L, const double *b, const double *x, float *r32,
                         double inv_scale, double *partial, cudaStream_t s);
// r32 = (float)(r64 * inv_scale)
cudaError_t launch_cast_scaled(const double *r, float *r32, double inv_scale, size_t n,
                               cudaStream_t s);
// x64 += scale * (double)e32
cudaError_t launch_update_mixed(double *x, const float *e, double scale, size_t n,
                                cudaStream_t s);

// ---- setup ----
// Validate fine coefficients; ORs error bits into *flag (device int).
cudaError_t launch_validate(const LevelDev<double> &L, int *flag, cudaStream_t s);
// Coarse coefficients of level l+1 from level l (sums; lon faces x sx, lat faces x sy[J]).
cudaError_t launch_coarsen(const LevelDev<double> &F, const LinkDev &K, double sx, double *txc,
                           double *tyc, double *tzc, double *hc, cudaStream_t s);
// Column factors (m, dq) of every column of a level, in FP64.
cudaError_t launch_column_lu(const LevelDev<double> &L, double *m, double *dq, cudaStream_t s);
// FP32 copies: out = (float)(scale * in) for coefficients; m32 = (float)(m / scale);
// dq32 = (float)dq.
cudaError_t launch_to_float(const double *in, float *out, double scale, size_t n, cudaStream_t s);

// Coefficient gradient (see mg_coeff_grad); outputs may be null.
cudaError_t launch_coeff_grad(int nlon, int nlat, int nz, const double *lam, const double *x,
                              double *gh, double *gtx, double *gty, double *gtz, cudaStream_t s);

// ---- batched ensemble (tpmg_batch.cu) -----------------------------------------
// One participant of a batched step: one level of one system and the vectors
// the step reads and writes.
template <typename T>
struct BOp {
    LevelDev<T> L;   // the level (the fine level of a transfer)
    LinkDev K;       // link to the next coarser level (transfers)
    const T *a;      // right-hand side / source
    const T *x;      // second input (smoother u_in, nullptr = zero guess; stencil x)
    T *y;            // output
    T *w;            // second output (direction update + apply: H d)
    int sys;         // system index (activity flag, per-system reductions)
    int nblk;        // thread blocks per layer range (column tiles)
    int kz;          // layers per work item (residual, transfers); nz: whole columns
};

// FP64 residual of one system handed to its FP32 inner solve (scaled).
struct BResid32 {
    LevelDev<double> L;
    const double *b, *x;
    float *r32;
    int sys, nblk;
};

// A work item: participant `op`, tile `tile` (a column block, or
// layer * nblk + column block for the cell-parallel kernels).
struct BItem {
    int op, tile;
};

// One fine-level vector operation of one system (roles depend on the kernel).
template <typename T>
struct BVec {
    T *a, *b, *c, *d;
    size_t n, chunk;  // length; elements per work item
    int sys, nchunk;
};

// FP64 <-> FP32 transfer of the mixed-precision refinement of one system.
struct BMix {
    double *x;          // FP64 solution (update)
    const double *r;    // FP64 residual (cast)
    float *r32;         // FP32 right-hand side of the inner solve (cast)
    const float *e32;   // FP32 correction (update)
    size_t n, chunk;    // length; elements per work item
    int sys, nchunk;
};

// Elements per vector work item: the batch's total length split into about
// kVecItems items (enough per resident block to balance the load), at least
// kVecChunkMin, a multiple of kBlock.
constexpr int kVecChunkMin = kBlock * 16;
constexpr int kVecItems = 16384;

enum { BV_DOT = 0, BV_UPDATE = 1, BV_DIR = 2, BV_DIR0 = 3, BV_ADD = 4, BV_MAXABS = 5 };

template <typename T>
cudaError_t launch_bsmooth(const BOp<T> *ops, const BItem *items, int nitems, bool zero,
                           double omega, const int *active, int grid, int block, int nzmax,
                           cudaStream_t s);
// kind: 0 residual y = a - H x, 1 restriction, 2 prolongation (cell pairs), 3 residual and
// restriction fused (y = R (a - H x), resid_restrict_band), 4 the same after a sweep from
// zero with this omega (the presmoothing form); an item is a column tile over op.kz layers
// (op.kz == nz: column walk of the residual), for kinds 3 and 4 a (band, layer, warp block)
// tile with op.nblk warp blocks along longitude
template <typename T>
cudaError_t launch_bcells(int kind, const BOp<T> *ops, const BItem *items, int nitems,
                          const int *active, int grid, cudaStream_t s, double omega = 0.0);
// Column-loop stencil with one partial sum per item (mode 1: residual + sum r^2;
// mode 0: apply + sum x*y).
template <typename T>
cudaError_t launch_bstencil_red(int mode, const BOp<T> *ops, const BItem *items, int nitems,
                                double *partial, const int *active, int grid, cudaStream_t s);
// Direction update + apply for every system (item = column tile, one partial
// per item): op.y = op.a + beta_sys op.x (bz: op.y = op.a), op.w = H op.y,
// partial = sum op.y * op.w.
template <typename T>
cudaError_t launch_bdir_apply(bool bz, const BOp<T> *ops, const BItem *items, int nitems,
                              const CgScalars *sc, double *partial, const int *active, int grid,
                              cudaStream_t s);
// r32 = (float)((b - H x) * sdata[sys]) in FP64 with the partial sums of
// |b - H x|^2 (item = column tile); narrow: the scaling after the rounding.
cudaError_t launch_bresid_cast(bool narrow, const BResid32 *ops, const BItem *items, int nitems,
                               const double *sdata, double *partial, const int *active, int grid,
                               cudaStream_t s);
// Vector kernels over per-system chunks; per-item partials where the op reduces.
template <typename T>
cudaError_t launch_bvec(int op, const BVec<T> *v, const BItem *items, int nitems,
                        const CgScalars *sc, double *partial, const int *active, int grid,
                        cudaStream_t s);
// mode 0: r32 = (float)(r * sdata[sys]); mode 1: x += sdata[sys] * (double)e32
cudaError_t launch_bmix(int mode, const BMix *v, const BItem *items, int nitems,
                        const double *sdata, const int *active, int grid, cudaStream_t s);
// Per-system fixed-order sum of partial[beg[s] .. end[s]) into sc[s] (ops
// as launch_finalize; op 3 = max); inactive systems are skipped.
cudaError_t launch_bfinalize(const double *partial, const int *beg, const int *end, int nsys,
                             CgScalars *sc, int which, int op, const int *active, cudaStream_t s);
// The last sweep of the batched V-cycle with <b, u_out> fused: one partial
// sum per item (block_store_at), as launch_bsmooth otherwise.
template <typename T>
cudaError_t launch_bsmooth_dot(const BOp<T> *ops, const BItem *items, int nitems, double omega,
                               const int *active, int grid, int block, int nzmax,
                               double *partial, cudaStream_t s);
cudaError_t bsmooth_prepare();
// The coarsest-level solve of several systems, one block each with its level
// in shared memory (coarse_solve_sh); op.a = b, op.y = out.  smem: the
// largest coarse_sh_bytes of the ops.
template <typename T>
cudaError_t launch_bcoarse_solve(const BOp<T> *ops, int nops, double omega, int sweeps,
                                 const int *active, size_t smem, cudaStream_t s);
// Shared memory of the one-block coarsest-level solve, and whether it fits.
size_t coarse_sh_bytes(int ncol, int nz, size_t value_bytes);
bool coarse_sh_fits(int ncol, int nz, size_t value_bytes);

// ---- nonsymmetric operator (tpmg_ns.cu), FP64 ----------------------------
// One operator of the directed flux form as a kernel sees it: the mass h and,
// per face, the row's own coupling to its east / north / upper neighbour
// (e, n, u, read at the cell) and the coupling of the row beyond the face
// back to the cell (w, s, d, read at the west / south / lower neighbour's
// face index).  H: (h, tx, ty, tz, txr, tyr, tzr); H^T: (h^T, txr, tyr,
// tzr, tx, ty, tz).  m, dq: the view's column factors 1/p and q/p.  FP32
// views hold the FP64 arrays scaled by one power of two (m by its inverse).
template <typename T>
struct NsView {
    int nlon, nlat, nz;
    const T *h, *e, *n, *u, *w, *s, *d;
    const T *m, *dq;
};

// y = A x (mode 0) or b - A x (mode 1) in the directed flux form.
template <typename T>
cudaError_t launch_ns_stencil(const NsView<T> &V, int mode, const T *b, const T *x, T *y,
                              cudaStream_t s);
// r = (1 - omega) b plus the four horizontal couplings of u (the residual
// after one sweep from zero, u = omega A_z^{-1} b).
template <typename T>
cudaError_t launch_ns_presmooth_resid(const NsView<T> &V, const T *b, const T *u, double omega,
                                      T *r, cudaStream_t s);
// One sweep of Eq. (1), u_out = (1 - omega) u_in + omega A_z^{-1}(b - dA u_in)
// (u_in == nullptr: zero guess).
template <typename T>
cudaError_t launch_ns_smooth(const NsView<T> &V, const T *b, const T *u_in, T *u_out,
                             double omega, cudaStream_t s);
// Column factors of a view (FP64).
cudaError_t launch_ns_column_lu(const NsView<double> &V, double *m, double *dq, cudaStream_t s);
// h^T = h + sum over the six faces of (row coupling - column coupling) of H
// (the forward view).
cudaError_t launch_ns_colmass(const NsView<double> &V, double *hT, cudaStream_t s);
// Coarse arrays of the next level from a fine view (R10 for both couplings
// of a face, masses summed); null outputs are skipped.
cudaError_t launch_ns_coarsen(const NsView<double> &F, const LinkDev &K, double sx, double *h,
                              double *e, double *n, double *u, double *w, double *sv, double *d,
                              cudaStream_t s);
// Validation of the fine arrays (bits as launch_validate) and of a mass
// array (bit 8: h^T <= 0 or non-finite).
cudaError_t launch_ns_validate(const NsView<double> &V, int *flag, cudaStream_t s);
cudaError_t launch_ns_positive(const double *a, size_t n, int *flag, cudaStream_t s);
// Gradient of the seven arrays (outputs may be null).
cudaError_t launch_ns_coeff_grad(int nlon, int nlat, int nz, const double *lam, const double *x,
                                 double *gh, double *gtx, double *gty, double *gtz,
                                 double *gtxr, double *gtyr, double *gtzr, cudaStream_t s);

// Set the thread-local message mg_last_error() returns.
void set_last_error(const char *msg);

}  // namespace tpmg
