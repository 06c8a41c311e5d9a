/*
 * tpmg.h -- C ABI of the GB300 tensor-product multigrid library (libtpmg.so).
 *
 * Solves H u = b for the pressure-correction system of the paper (Section 2:
 * a sparse discrete operator of Laplacian type) on a cell-centred
 * latitude-longitude grid of nz layers, nlat latitude rows and nlon
 * longitudes, with the tensor-product multigrid of Sections 2.1-2.3: a
 * vertical line (block-Jacobi) smoother, Eq. (1); horizontal-only coarsening
 * with conditional semi-coarsening in latitude (Section 2.2); a V-cycle
 * (Section 2, Fig. 1) with a simple iterative coarsest-level solve
 * (Section 2.3).
 *
 * Conventions
 *   Layout. Every field is a dense array [nz][nlat][nlon] (C order, index
 *     (k*nlat + j)*nlon + i), longitude fastest.  Face coefficients:
 *       tx[k,j,i] couples cells (i, i+1 mod nlon)  (periodic longitude)
 *       ty[k,j,i] couples rows  (j, j+1); ty[:, nlat-1, :] must be 0 (pole)
 *       tz[k,j,i] couples layers (k, k+1); tz[nz-1] must be 0 (model top)
 *       h [k,j,i] Helmholtz (diagonal) term, > 0
 *     (H u)_c = h_c u_c + sum over the six faces of T_f (u_c - u_nb(f)).
 *   Memory. Unless stated otherwise, pointers are DEVICE pointers on the
 *     current CUDA device.  The library allocates no device memory: the
 *     caller passes one device workspace (size from mg_workspace_bytes) to
 *     mg_setup and keeps it alive until mg_destroy.  The handle itself is
 *     host memory owned by the library.
 *   Streams. `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Every call is stream-ordered; only the calls that
 *     return host scalars (solves, norms, mg_setup's validation) synchronise
 *     the stream.
 *   Errors. Every int-returning call returns an mg_status; no call aborts,
 *     traps or throws.  mg_last_error() returns a thread-local message for
 *     the last failing call on this thread.
 */
#ifndef TPMG_H
#define TPMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MG_OK = 0,
    MG_ERR_ARG = 1,            /* bad shape, null pointer, level out of range */
    MG_ERR_COEFF = 2,          /* h <= 0, T < 0, non-finite, or a non-zero pole/top face */
    MG_ERR_NONFINITE = 3,      /* NaN/Inf met in a right-hand side or residual */
    MG_ERR_NOT_CONVERGED = 4,  /* maxit reached before the tolerance */
    MG_ERR_DIVERGED = 5,       /* residual grew beyond 1e3 x its start */
    MG_ERR_TIMEOUT = 6,        /* a bounded device wait (TMA-staged kernel) gave up */
    MG_ERR_CUDA = 7,           /* a CUDA runtime call failed */
    MG_ERR_WORKSPACE = 8       /* workspace too small or misaligned */
} mg_status;

enum { MG_METHOD_CG = 0, MG_METHOD_STATIONARY = 1, MG_METHOD_BICGSTAB = 2,
       MG_METHOD_BICGSTAB_LINE = 3 };
enum { MG_PREC_FP64 = 0, MG_PREC_FP32 = 1 };
enum { MG_COARSE_JACOBI = 0, MG_COARSE_PCG = 1, MG_COARSE_CHEBYSHEV = 2 };

typedef struct mg_handle mg_handle;

typedef struct {
    int nlon;   /* longitudes; divisible by 2^(levels-1); >= 4 */
    int nlat;   /* latitude rows; even (mirror-symmetric hemispheres); >= 2 */
    int nz;     /* layers; 1 <= nz <= MG_MAX_NZ */
} mg_grid;

#define MG_MAX_NZ 192

typedef struct {
    const double *tx, *ty, *tz, *h;   /* device, [nz][nlat][nlon], FP64 */
} mg_coeffs;

typedef struct {
    int levels;        /* 0: coarsen down to the coarsest level (nlon >= 4 there);
                          4 is the shallow hierarchy of Section 2.3; -1: coarsen until a
                          level's largest (sum of horizontal couplings) / h is at most
                          iso_ratio (at most as deep as 0; the workspace is sized for that
                          depth; single systems only) */
    int nu1, nu2;      /* pre/post smoothing sweeps (V(1,1) default) */
    int coarse_iters;  /* block-Jacobi sweeps on the coarsest level (12) */
    int method;        /* outer iteration: MG_METHOD_CG (V-cycle-preconditioned CG,
                          default), MG_METHOD_STATIONARY (x <- x + V(b - H x), Section 2),
                          MG_METHOD_BICGSTAB (BiCGStab preconditioned by the V-cycle), or
                          MG_METHOD_BICGSTAB_LINE (BiCGStab preconditioned by line_sweeps
                          sweeps of Eq. (1) from zero: the solver of Section 1 that the
                          multigrid replaced; only the fine level takes part).
                          BiCGStab: single systems only (mg_batch_setup rejects it). */
    int mixed;         /* 1: also build the FP32 hierarchy for mg_solve_mixed */
    int maxit;         /* outer iterations (200) */
    int inner_maxit;   /* mixed: FP32 iterations per FP64 refinement step (12) */
    double omega;      /* Eq. (1) relaxation factor (0.85) */
    double alpha_c;    /* Section 2.2 anisotropy threshold for merging rows (0.6) */
    double inner_tol;  /* mixed: FP32 relative tolerance per refinement step (5e-4; loosened
                          when the outer target needs less) */
    int coarse_method; /* coarsest-level solve from zero (Section 2.3's simple iteration on
                          the coarsest grid): MG_COARSE_JACOBI, coarse_iters block-Jacobi
                          sweeps (default; V stays a fixed linear operator), or MG_COARSE_PCG,
                          coarse_iters iterations of CG preconditioned by the column solves
                          (for shallow hierarchies; V then depends nonlinearly on its input,
                          which the stationary method tolerates; CG usually does), or
                          MG_COARSE_CHEBYSHEV, coarse_iters Chebyshev steps on the
                          column-solve preconditioner over [mu, 2], mu = min over the level
                          of h / (h + the horizontal couplings), a bound of the spectrum of
                          H_z^{-1} H (a fixed polynomial: V stays linear).  Single systems
                          only: mg_batch_setup takes MG_COARSE_JACOBI alone. */
    int line_sweeps;   /* MG_METHOD_BICGSTAB_LINE: sweeps of Eq. (1) per preconditioner
                          application (1) */
    double iso_ratio;  /* levels = -1: the largest (sum of the horizontal couplings) / h
                          the coarsest level may keep (6.25: four faces at Section 2.3's
                          nu^2 / 4^3 = 1.56) */
} mg_params;

typedef struct {
    int iterations;         /* outer iterations (V-cycles or refinement steps) */
    int inner_iterations;   /* mixed: total FP32 iterations */
    double rel_res;         /* final ||b - H x||_2 / ||b||_2 (FP64) */
    double *history;        /* HOST array (may be NULL): rel. residual per outer step */
    int history_cap;        /* capacity of history */
    int history_len;        /* entries written */
} mg_stats;

/* Fill *p with the defaults listed above.  Never fails. */
void mg_default_params(mg_params *p);

/* Bytes of device workspace mg_setup needs for this grid and these
 * parameters (256-byte aligned start required).  MG_ERR_ARG on a bad grid. */
int mg_workspace_bytes(const mg_grid *grid, const mg_params *params, size_t *bytes);

/* Build the hierarchy (Sections 2.1-2.3): copy the fine coefficients into
 * the workspace (the caller may free them afterwards), validate them
 * (MG_ERR_COEFF), build the conditional semi-coarsening row maps
 * (Section 2.2), assemble the coarse operators, factor every column
 * tridiagonal of every level (FP64, and FP32 when params->mixed).
 * Synchronises `stream` once.  On failure *out is NULL. */
int mg_setup(const mg_grid *grid, const mg_coeffs *coeffs, const mg_params *params,
             void *workspace, size_t ws_bytes, void *stream, mg_handle **out);

/* Release the handle (host memory only; the workspace stays the caller's). */
void mg_destroy(mg_handle *h);

/* y = H x on the fine level (Section 2).  x, y: device FP64 fields. */
int mg_apply(mg_handle *h, const double *x, double *y, void *stream);

/* e = V r: one V(nu1, nu2)-cycle from a zero initial guess (Section 2,
 * Fig. 1).  r, e: device FP64 fine-level fields; r is not modified. */
int mg_vcycle(mg_handle *h, const double *r, double *e, void *stream);

/* The same V-cycle in either precision: prec MG_PREC_FP64 (as mg_vcycle) or
 * MG_PREC_FP32, the FP32 hierarchy the inner solve of mg_solve_mixed uses
 * (needs params->mixed = 1; its coefficients are the FP64 ones scaled by
 * mg_fp32_scale, so e approximates (c H)^{-1} r).  r, e: device fields of
 * that precision on the fine level, distinct; r is not modified.  Uses the
 * handle's level work vectors: calls on one handle must not overlap. */
int mg_vcycle_prec(mg_handle *h, int prec, const void *r, void *e, void *stream);

/* Solve H x = b to ||b - H x||_2 <= tol ||b||_2 in FP64 (Section 2).
 * x: in = initial guess, out = solution.  stats may be NULL.  Returns
 * MG_OK, MG_ERR_NOT_CONVERGED (x holds the last iterate), MG_ERR_NONFINITE
 * or MG_ERR_DIVERGED.  Synchronises once per iteration (one scalar). */
int mg_solve(mg_handle *h, const double *b, double *x, double tol, mg_stats *stats,
             void *stream);

/* Same system, FP32 multigrid inside FP64 iterative refinement (Section 1:
 * single-precision solves): FP64 residual, norms and update; FP32 storage
 * and arithmetic in the smoother, residual and transfers of the inner
 * solve.  Needs params->mixed = 1 at setup (else MG_ERR_ARG).  x: in =
 * initial guess, out = solution. */
int mg_solve_mixed(mg_handle *h, const double *b, double *x, double tol, mg_stats *stats,
                   void *stream);

/* Solve H x = b entirely in single precision, as a model that runs its
 * solver in FP32 would (Section 1: single-precision solves, where Krylov
 * methods can stall at tight tolerances): FP32 storage and arithmetic in
 * every vector, operator and preconditioner step (the FP32 hierarchy of
 * params->mixed = 1, else MG_ERR_ARG), inner products accumulated in FP64,
 * the configured method.  b, x: device FP32 fields (x: in = initial guess,
 * out = solution).  The residuals in stats are FP32 ones relative to
 * ||b||; a tolerance below the FP32 floor of this operator ends with
 * MG_ERR_NOT_CONVERGED (x the last iterate) or MG_ERR_DIVERGED. */
int mg_solve_single(mg_handle *h, const float *b, float *x, double tol, mg_stats *stats,
                    void *stream);

/* Coefficient gradient of a loss L(x) through H x = b (differentiable
 * solve), given the adjoint lambda = H^{-T} dL/dx (H is symmetric, so
 * lambda comes from mg_solve on dL/dx) and the solution x:
 *   gh  = -lambda * x
 *   gtx = -(lambda_c - lambda_e)(x_c - x_e)  (east faces; same for gty/gtz)
 * All device FP64 fields; any of the outputs may be NULL. */
int mg_coeff_grad(mg_handle *h, const double *lambda, const double *x,
                  double *gh, double *gtx, double *gty, double *gtz, void *stream);

/* ---- per-level kernels (the V-cycle's steps), for checking and profiling.
 * `prec` selects the FP64 or FP32 hierarchy; pointers are device arrays of
 * that precision with the level's shape (mg_level_shape). */

/* Shape of level l (0 = finest) and the number of levels. */
int mg_num_levels(const mg_handle *h);
int mg_level_shape(const mg_handle *h, int level, int *nlon, int *nlat, int *nz);

/* Copy level l's coefficients (FP64) into caller device arrays (any NULL). */
int mg_level_coeffs(mg_handle *h, int level, double *tx, double *ty, double *tz,
                    double *hh, void *stream);

/* y = H_l x (prec: MG_PREC_FP64 or MG_PREC_FP32; FP32 acts on the scaled
 * copies, see mg_fp32_scale). */
int mg_level_apply(mg_handle *h, int level, int prec, const void *x, void *y, void *stream);

/* r = b - H_l u, H_l in the flux form of Section 2's operator (the
 * Helmholtz term plus T_f (u_c - u_nb) over the six faces). */
int mg_level_residual(mg_handle *h, int level, int prec, const void *b, const void *u,
                      void *r, void *stream);

/* out = the V-cycle's coarsest-level solve applied to b (the configured
 * coarse_method and coarse_iters, from a zero guess), on the coarsest level
 * (b, out: its shape, distinct).  Uses the handle's coarsest-level work
 * vectors: calls on one handle must not overlap. */
int mg_coarse_solve(mg_handle *h, int prec, const void *b, void *out, void *stream);

/* bc = R_l (b - H_l u): the residual restricted to level l+1 in one pass
 * (Section 2's V-cycle: restrict the residual to the coarse grid), the
 * residual itself never stored (the FP32 V-cycle's form after more than one
 * pre-smoothing sweep; equal term for term to mg_level_residual followed by
 * mg_level_restrict).  b, u: level l;
 * bc: level l+1, aliasing neither.  Buffers not aligned to two values take
 * the two passes through the handle's level-l residual vector (calls on one
 * handle must not overlap).  MG_ERR_ARG on the coarsest level. */
int mg_level_residual_restrict(mg_handle *h, int level, int prec, const void *b, const void *u,
                               void *bc, void *stream);

/* bc = R_l ((1 - omega) b + the horizontal couplings of u): the restricted
 * residual b - H_l u for u the sweep of Eq. (1) from zero on b, u = omega
 * H_z^{-1} b, written without the column couplings H_z u = omega b cancels
 * (the V-cycle's form when nu1 = 1).  b, u: level l; bc: level l+1.
 * Unaligned b or u are first copied into the handle's level-l work vectors
 * (calls on one handle must not overlap).  MG_ERR_ARG on the coarsest level. */
int mg_level_presmooth_restrict(mg_handle *h, int level, int prec, const void *b, const void *u,
                                void *bc, void *stream);

/* One smoother sweep of Eq. (1) on level l:
 *   u_out = u_in + omega H_z^{-1} (b - H u_in), evaluated as
 *   (1 - omega) u_in + omega H_z^{-1} (b - dH u_in).
 * u_in == NULL means the zero initial guess.  u_out must not alias u_in. */
int mg_level_smooth(mg_handle *h, int level, int prec, const void *b, const void *u_in,
                    void *u_out, void *stream);

/* out = `sweeps` sweeps of Eq. (1) on level l from the zero guess (b, out:
 * the level's shape, distinct).  On the coarsest level with sweeps =
 * coarse_iters this is the V-cycle's coarsest-level solve (Section 2.3: a
 * simple iteration on the coarsest grid), run as one launch when the level
 * is small enough; elsewhere one launch per sweep.  Uses the handle's level
 * scratch vector: calls on one handle must not overlap.  MG_ERR_ARG for
 * sweeps outside 1..1000 or aliased buffers. */
int mg_level_relax(mg_handle *h, int level, int prec, int sweeps, const void *b, void *out,
                   void *stream);

/* The same sweep (u_in != NULL) also returning *dot = <b, u_out> (host
 * double; FP64 accumulation of per-column sums): the last sweep of a V-cycle
 * with the conjugate-gradient inner product <r, z> fused in.  Synchronises. */
int mg_level_smooth_dot(mg_handle *h, int level, int prec, const void *b, const void *u_in,
                        void *u_out, double *dot, void *stream);

/* The fused step of the conjugate-gradient iteration preconditioned by the
 * V-cycle (Section 2's multigrid as a preconditioner) on level l:
 *   d_new = z + beta d_old  (d_old == NULL: d_new = z),  q = H_l d_new,
 * and *dot = <d_new, q> (host double; FP64 accumulation of per-block sums).
 * z, d_old, d_new, q: device arrays of the level's shape and precision,
 * d_new and q distinct from the inputs.  Uses the handle's scalar and
 * partial-sum storage: calls on one handle must not overlap.  Synchronises. */
int mg_level_dir_apply(mg_handle *h, int level, int prec, const void *z, const void *d_old,
                       double beta, void *d_new, void *q, double *dot, void *stream);

/* bc = R r: restriction from level l to l+1 (R = P^T; the coarse grid of
 * Section 2.2: longitude halved, latitude rows merged where the anisotropy
 * allows). */
int mg_level_restrict(mg_handle *h, int level, int prec, const void *r, void *bc,
                      void *stream);

/* u += P ec: bilinear horizontal prolongation from level l+1 to level l
 * (the coarse-grid correction of Section 2's V-cycle). */
int mg_level_prolong_add(mg_handle *h, int level, int prec, const void *ec, void *u,
                         void *stream);

/* The power-of-two factor c by which the FP32 coefficient copies are
 * scaled (FP32 level l holds c * coefficients); 0 when not built. */
double mg_fp32_scale(const mg_handle *h);

/* The precision changes of the mixed-precision refinement (Section 1:
 * single-precision multigrid; the outer residual and the update in double
 * precision), on n device values, stream-ordered, no handle needed.
 * mg_cast_fp32: y[i] = x[i] * scale rounded to the nearest FP32 value, ties
 *   to even (FP32 subnormals kept, +-0 below half the smallest one, +-inf
 *   from the overflow threshold; the FP32 right-hand side of an inner solve,
 *   scale the reciprocal of its power-of-two normalisation).  x and y must
 *   not overlap.
 * mg_update_fp64: x[i] += scale * e[i] in FP64 (one rounding: the product
 *   of a power-of-two scale and an FP32 value is exact).
 * scale must be finite and non-zero (MG_ERR_ARG); n = 0 is a no-op.  With a
 * power-of-two scale the conversions run in integer arithmetic, off the FP64
 * pipe, with the IEEE 754 results. */
int mg_cast_fp32(const double *x, float *y, double scale, size_t n, void *stream);
int mg_update_fp64(double *x, const float *e, double scale, size_t n, void *stream);

/* ---- batched ensemble of independent systems.
 * n systems of possibly different shapes share one device workspace and the
 * same parameters; every V-cycle step and fine-level vector operation of all
 * systems is one persistent-kernel launch over a precomputed work list of
 * (system level, column tile), the batched V-cycle is replayed from one CUDA
 * graph, and converged systems are switched off by device-side flags.
 * mg_batch_setup autotunes the smoother's column-tile width and persistent
 * grid on the batch itself (mg_batch_tuning reports them); the other steps
 * run on persistent grids of as many blocks as the GPU holds at once. */
typedef struct mg_batch mg_batch;

/* Workspace bytes for n systems with these grids and common params. */
int mg_batch_workspace_bytes(int n, const mg_grid *grids, const mg_params *params,
                             size_t *bytes);

/* Set up the n hierarchies (as mg_setup, each from coeffs[i]) and the batched
 * work lists, then autotune.  Synchronises `stream`.  On failure *out = NULL. */
int mg_batch_setup(int n, const mg_grid *grids, const mg_coeffs *coeffs,
                   const mg_params *params, void *workspace, size_t ws_bytes, void *stream,
                   mg_batch **out);

/* Release the batch (host memory; the workspace stays the caller's). */
void mg_batch_destroy(mg_batch *b);

/* The handle of system i (owned by the batch; valid until mg_batch_destroy). */
int mg_batch_handle(mg_batch *b, int i, mg_handle **out);

/* Launch shapes: the tuned smoother column-tile width (threads per block)
 * and persistent grid; cell_grid and vec_grid are upper bounds of the
 * cell-type and vector steps' grids (each launch takes the smaller of the
 * bound and the kernel's resident grid). */
int mg_batch_tuning(const mg_batch *b, int *smooth_block, int *smooth_grid, int *cell_grid,
                    int *vec_grid);

/* Solve all systems: b[i], x[i] are HOST arrays of n device pointers (FP64
 * fields of system i; x[i] in = initial guess, out = solution), each to
 * ||b_i - H_i x_i|| <= tol ||b_i||.  mixed = 1: FP32 multigrid inside FP64
 * refinement (needs params->mixed at setup); 0: FP64.  stats (n entries) and
 * status (n ints) may be NULL.  Returns MG_OK when every system converged,
 * else the first failing status. */
int mg_batch_solve(mg_batch *b, const double *const *bs, double *const *xs, double tol,
                   int mixed, mg_stats *stats, int *status, void *stream);

/* ---- measurement hooks (off by default; no effect on results).
 * When profiling is on (on = 1: fine-level launches only; on = 2: every
 * level), each kernel launch of this handle is bracketed by CUDA events on
 * its stream (events created by mg_profile_enable, freed by
 * mg_profile_enable(h, 0) or mg_destroy).  mg_profile_read returns, for the
 * launches of kernel class `kind` on `level` in precision `prec`, the launch
 * count and the summed event time in ms (synchronises on the events).
 * kind: 0 smoother (non-zero guess), 1 smoother (zero guess), 2 residual,
 * 3 apply, 4 restriction, 5 prolongation, 6 vector/reduction kernels. */
/* ---- nonsymmetric operator (directed couplings) and its transpose.
 * Section 1 names BiCGStab as the solver of the operational Helmholtz
 * problem, which is nonsymmetric.  In this form every face carries two
 * couplings, one for each row it enters:
 *   tx[c]: row c's coupling to its east neighbour E;  txr[c]: row E's coupling to c
 *   ty[c], tyr[c]: the same across c's north face;    tz[c], tzr[c]: across c's upper face
 *   (H u)_c = h_c u_c + tx[c](u_c - u_E) + txr[W](u_c - u_W) + ty[c](u_c - u_N)
 *             + tyr[S](u_c - u_S) + tz[c](u_c - u_U) + tzr[D](u_c - u_D)
 * with W, S, D the west, south and lower neighbours.  h is H's row sum.
 * H^T has the two couplings of every face swapped and the column sums
 *   h^T_c = h_c + sum over c's six faces of (row coupling - column coupling)
 * as its mass.  txr = tx, tyr = ty, tzr = tz is mg_setup's symmetric
 * operator.  Requirements (else MG_ERR_COEFF): h > 0 and h^T > 0 (H
 * diagonally dominant by rows and by columns), couplings finite and >= 0,
 * pole and top faces 0 in all six coupling arrays.
 * Hierarchy: Section 2.2's grid hierarchy (depends on the grid only), each
 * of a face's two couplings coarsened by mg_setup's rule, masses summed;
 * H^T's hierarchy is built by the same rule from H^T (its couplings are
 * H's swapped, its masses the sums of the fine column sums).  A call with
 * transpose = 1 works on H^T's hierarchy; its sweeps solve the transposed
 * column systems.
 * FP64, and with params->mixed = 1 also an FP32 copy of both hierarchies
 * for mg_ns_solve_mixed.  params: method MG_METHOD_STATIONARY or
 * MG_METHOD_BICGSTAB (V-cycle-preconditioned; CG and the line-relaxed
 * BiCGStab are rejected), coarse_method MG_COARSE_JACOBI, levels >= 0; the
 * other fields as for mg_setup (MG_ERR_ARG otherwise). */
typedef struct mg_ns_handle mg_ns_handle;

typedef struct {
    const double *h, *tx, *ty, *tz, *txr, *tyr, *tzr;   /* device, [nz][nlat][nlon], FP64 */
} mg_ns_coeffs;

/* Workspace bytes mg_ns_setup needs (256-byte aligned start). */
int mg_ns_workspace_bytes(const mg_grid *grid, const mg_params *params, size_t *bytes);

/* Copy the seven arrays into the workspace, validate them, build both
 * hierarchies and factor every column system of both.  Synchronises
 * `stream`.  On failure *out is NULL. */
int mg_ns_setup(const mg_grid *grid, const mg_ns_coeffs *coeffs, const mg_params *params,
                void *workspace, size_t ws_bytes, void *stream, mg_ns_handle **out);

/* Release the handle (host memory only). */
void mg_ns_destroy(mg_ns_handle *h);

/* y = H x (transpose 0) or y = H^T x (transpose 1) on the fine level; the
 * transposed apply reads H's own arrays at the transposed positions (the
 * couplings into c from its neighbours' rows) with h^T as its mass.  x, y:
 * distinct device FP64 fields. */
int mg_ns_apply(mg_ns_handle *h, int transpose, const double *x, double *y, void *stream);

/* e = V r: one V(nu1, nu2) cycle from zero of H or of H^T (Section 2).  r, e:
 * distinct device FP64 fine-level fields; r is not modified.  Uses the
 * handle's level vectors: calls on one handle must not overlap. */
int mg_ns_vcycle(mg_ns_handle *h, int transpose, const double *r, double *e, void *stream);

/* Solve H x = b (transpose 0) or H^T x = b (transpose 1) to
 * ||b - A x||_2 <= tol ||b||_2 with the configured method.  x: in =
 * initial guess, out = solution.  Returns as mg_solve. */
int mg_ns_solve(mg_ns_handle *h, int transpose, const double *b, double *x, double tol,
                mg_stats *stats, void *stream);

/* The same solves with FP32 multigrid inside FP64 iterative refinement
 * (Section 1's single-precision solves, as mg_solve_mixed): FP64 residual
 * b - A x, norms and update; the configured method (stationary or BiCGStab
 * with the V-cycle) in FP32 on the FP32 copy of H's or H^T's hierarchy
 * (params->mixed = 1 at setup, else MG_ERR_ARG; its arrays are the FP64 ones
 * scaled by mg_ns_fp32_scale) for at most params->inner_maxit iterations per
 * refinement step.  x: in = initial guess, out = solution.  Returns as
 * mg_solve; stats->inner_iterations counts the FP32 iterations. */
int mg_ns_solve_mixed(mg_ns_handle *h, int transpose, const double *b, double *x, double tol,
                      mg_stats *stats, void *stream);

/* e = V r of H or H^T in either precision: prec MG_PREC_FP64 (as
 * mg_ns_vcycle) or MG_PREC_FP32 (the FP32 hierarchy; e approximates
 * (c A)^{-1} r, c = mg_ns_fp32_scale).  r, e: distinct device fields of that
 * precision; calls on one handle must not overlap. */
int mg_ns_vcycle_prec(mg_ns_handle *h, int transpose, int prec, const void *r, void *e,
                      void *stream);

/* The power of two the FP32 arrays are scaled by (0 without them). */
double mg_ns_fp32_scale(const mg_ns_handle *h);

/* Gradient of a loss L(x) through H x = b with respect to the seven arrays,
 * given x and lambda = H^{-T} dL/dx (mg_ns_solve with transpose = 1):
 * dL/dtheta = -lambda^T (dH/dtheta) x, i.e.
 *   gh = -lambda_c x_c,  gtx = -lambda_c (x_c - x_E),  gtxr = -lambda_E (x_E - x_c)
 * and likewise north and up; 0 on the pole and top faces.  Device FP64
 * fields; any output may be NULL. */
int mg_ns_coeff_grad(mg_ns_handle *h, const double *lambda, const double *x, double *gh,
                     double *gtx, double *gty, double *gtz, double *gtxr, double *gtyr,
                     double *gtzr, void *stream);

/* Levels and their shapes (as mg_num_levels / mg_level_shape). */
int mg_ns_num_levels(const mg_ns_handle *h);
int mg_ns_level_shape(const mg_ns_handle *h, int level, int *nlon, int *nlat, int *nz);

/* Copies of level `level`'s arrays of H (transpose 0) or of H^T
 * (transpose 1: h^T and the couplings as H^T sees them) into device FP64
 * fields of the level's shape; a NULL output is skipped. */
int mg_ns_level_coeffs(mg_ns_handle *h, int level, int transpose, double *h_out, double *tx,
                       double *ty, double *tz, double *txr, double *tyr, double *tzr,
                       void *stream);

/* One sweep of Eq. (1) on a level of H or H^T in FP64 or (prec
 * MG_PREC_FP32, mixed handles) on the FP32 hierarchy:
 * u_out = (1 - omega) u_in + omega A_z^{-1} (b - dA u_in), u_in NULL = zero
 * guess.  Device fields of that precision and the level's shape; u_out
 * distinct from u_in and b. */
int mg_ns_level_smooth(mg_ns_handle *h, int level, int transpose, int prec, const void *b,
                       const void *u_in, void *u_out, void *stream);

int mg_profile_enable(mg_handle *h, int on);
int mg_profile_read(mg_handle *h, int kind, int level, int prec, int *launches, double *ms);

/* Residual without any device allocation.  Computes r = b - H x on the fine
 * grid given directly by `coeffs` (no handle, no workspace) and returns
 * *rel_out = ||r||_2 / ||b||_2 (||r||_2 if b = 0) on the host.  The paper
 * has no counterpart: this exists for callers that cannot allocate device
 * memory when they need the check -- a forecast model that owns every
 * device buffer through its own pool and forbids further cudaMalloc, or C
 * or Fortran host code with no device allocator for a workspace.
 * The reduction scratch is a file-scope __device__ array of 256 KB that
 * every GPU loading the library keeps until exit; grids with more than
 * 16384 * 128 = 2,097,152 columns (nlon * nlat) are rejected (MG_ERR_ARG).
 * The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and leave their partial sums in it: calls that
 * overlap on the GPU (other streams, other host threads) race.  Calls
 * cudaMalloc/cudaFree never.  The coefficients are not validated (mg_setup
 * does that for a handle); the operator is the one mg_setup accepts, the
 * top-face coupling tz[nz-1] not being read.  b, x, r: device FP64 fields;
 * rel_out: host.  MG_ERR_NONFINITE when either norm is NaN or Inf,
 * MG_ERR_CUDA when a launch or the copy fails (*rel_out is then left as it
 * was).  Synchronises `stream`. */
int mg_residual_norm_noalloc(const mg_grid *grid, const mg_coeffs *coeffs, const double *b,
                             const double *x, double *r, double *rel_out, void *stream);

/* Kernel launches issued by this library in this process so far. */
unsigned long long mg_launch_count(void);

/* Thread-local message of the last error on this thread ("" if none). */
const char *mg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TPMG_H */
