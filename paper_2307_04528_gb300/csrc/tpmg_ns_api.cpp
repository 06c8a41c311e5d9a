// Host driver of the nonsymmetric operator (C ABI mg_ns_*): the hierarchies
// of H and of H^T on Section 2.2's grid hierarchy, the V-cycle of either
// (Section 2), the stationary iteration and BiCGStab (Section 1's solver for
// the nonsymmetric problem, here preconditioned by the V-cycle), and the
// coefficient gradient of the seven arrays.  FP64 throughout.
//
// Workspace layout (carved with 256-byte alignment from the caller's buffer):
// per level the seven arrays of H, the column sums h^T, the column factors of
// H and of H^T, the V-cycle vectors and the level's row links; then the
// fine-level solver vectors, the reduction partials and the device scalars.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/tpmg.h"
#include "tpmg_handle.h"
#include "tpmg_internal.h"

using namespace tpmg;

namespace {

struct NsLevel {
    int nlon = 0, nlat = 0, nz = 0;
    size_t n = 0;
    double *h = nullptr, *tx = nullptr, *ty = nullptr, *tz = nullptr;
    double *txr = nullptr, *tyr = nullptr, *tzr = nullptr, *hT = nullptr;
    double *m = nullptr, *dq = nullptr, *mT = nullptr, *dqT = nullptr;
    double *b = nullptr, *u = nullptr, *w = nullptr, *r = nullptr;
    LinkHost link;
    LinkDev linkdev{};
};

}  // namespace

struct mg_ns_handle {
    mg_grid grid{};
    mg_params p{};
    int L = 0;
    std::vector<NsLevel> lev;
    // fine-level solver vectors (BiCGStab: r, r^, p, p^, v, s, s^, t; the
    // stationary iteration: r and the correction e)
    double *r = nullptr, *rh = nullptr, *pv = nullptr, *ph = nullptr, *v = nullptr;
    double *sv = nullptr, *sh = nullptr, *t = nullptr, *e = nullptr;
    double *partial = nullptr;
    CgScalars *sc = nullptr;
    BicgScalars *bsc = nullptr;
    int *flag = nullptr;
};

namespace {

#define NRUN(expr)                                                                          \
    do {                                                                                    \
        const cudaError_t e_ = (expr);                                                      \
        g_launches.fetch_add(1, std::memory_order_relaxed);                                 \
        if (e_ != cudaSuccess)                                                              \
            return fail(MG_ERR_CUDA, "kernel launch (%s:%d): %s", __FILE__, __LINE__,       \
                        cudaGetErrorString(e_));                                            \
    } while (0)

struct Bump {
    char *base;
    size_t off = 0;
    explicit Bump(void *b) : base((char *)b) {}
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

NsView view(const NsLevel &v, bool tr)
{
    if (!tr) return {v.nlon, v.nlat, v.nz, v.h, v.tx, v.ty, v.tz, v.txr, v.tyr, v.tzr, v.m, v.dq};
    return {v.nlon, v.nlat, v.nz, v.hT, v.txr, v.tyr, v.tzr, v.tx, v.ty, v.tz, v.mT, v.dqT};
}

LevelDev<double> shape_of(const NsLevel &v)
{
    return {v.nlon, v.nlat, v.nz, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
}

int ns_check(const mg_grid *g, const mg_params *p)
{
    if (!g || !p) return fail(MG_ERR_ARG, "null grid or params");
    if (p->method != MG_METHOD_STATIONARY && p->method != MG_METHOD_BICGSTAB)
        return fail(MG_ERR_ARG, "nonsymmetric solves take MG_METHOD_STATIONARY or "
                                "MG_METHOD_BICGSTAB (method %d)", p->method);
    if (p->coarse_method != MG_COARSE_JACOBI)
        return fail(MG_ERR_ARG, "nonsymmetric hierarchy: coarse_method MG_COARSE_JACOBI only");
    if (p->mixed) return fail(MG_ERR_ARG, "nonsymmetric hierarchy: FP64 only (mixed = 0)");
    if (p->levels < 0) return fail(MG_ERR_ARG, "nonsymmetric hierarchy: levels >= 0");
    return MG_OK;
}

// Shapes and row links of every level: the grid hierarchy of the symmetric
// planner (it depends on the grid and the parameters only).
int ns_plan(mg_ns_handle *H, const mg_grid *g, const mg_params *p)
{
    CHK(ns_check(g, p));
    mg_handle *tmp = nullptr;
    size_t bytes = 0;
    CHK(handle_plan(g, p, nullptr, &bytes, &tmp));
    H->grid = *g;
    H->p = *p;
    H->L = tmp->L;
    H->lev.assign(H->L, NsLevel{});
    for (int l = 0; l < H->L; ++l) {
        NsLevel &v = H->lev[l];
        v.nlon = tmp->lev[l].nlon;
        v.nlat = tmp->lev[l].nlat;
        v.nz = tmp->lev[l].nz;
        v.n = tmp->lev[l].n;
        v.link = tmp->lev[l].link;
    }
    mg_destroy(tmp);
    return MG_OK;
}

size_t ns_carve(mg_ns_handle *H, void *base)
{
    Bump cv(base);
    for (int l = 0; l < H->L; ++l) {
        NsLevel &v = H->lev[l];
        const size_t n = v.n;
        for (double **a : {&v.h, &v.tx, &v.ty, &v.tz, &v.txr, &v.tyr, &v.tzr, &v.hT, &v.m, &v.dq,
                           &v.mT, &v.dqT, &v.u, &v.w, &v.r})
            *a = cv.take<double>(n);
        if (l > 0) v.b = cv.take<double>(n);
        if (l + 1 < H->L) {
            const LinkHost &K = v.link;
            LinkDev &D = v.linkdev;
            D.nlat_c = K.nlat_c;
            D.j0 = cv.take<int>(K.j0.size());
            D.w0 = cv.take<double>(K.w0.size());
            D.j1 = cv.take<int>(K.j1.size());
            D.w1 = cv.take<double>(K.w1.size());
            D.rptr = cv.take<int>(K.rptr.size());
            D.rrow = cv.take<int>(K.rrow.size());
            D.rw = cv.take<double>(K.rw.size());
            D.cfirst = cv.take<int>(K.cfirst.size());
            D.ccnt = cv.take<int>(K.ccnt.size());
            D.sy = cv.take<double>(K.sy.size());
        }
    }
    const size_t n0 = H->lev[0].n;
    for (double **a : {&H->r, &H->rh, &H->pv, &H->ph, &H->v, &H->sv, &H->sh, &H->t, &H->e})
        *a = cv.take<double>(n0);
    H->partial = cv.take<double>(kReduceSlots);
    H->sc = cv.take<CgScalars>(1);
    H->bsc = cv.take<BicgScalars>(1);
    H->flag = cv.take<int>(4);
    return cv.off + 256;
}

template <typename V>
int upload(const V &host, const void *dst, cudaStream_t s)
{
    if (host.empty()) return MG_OK;
    CU(cudaMemcpyAsync(const_cast<void *>(dst), host.data(), host.size() * sizeof(host[0]),
                       cudaMemcpyHostToDevice, s));
    return MG_OK;
}

int ns_setup(mg_ns_handle *H, const mg_ns_coeffs *co, void *ws, size_t ws_bytes, cudaStream_t s)
{
    const size_t need = ns_carve(H, nullptr);
    if (!ws) return fail(MG_ERR_WORKSPACE, "null workspace");
    if ((uintptr_t)ws % 256) return fail(MG_ERR_WORKSPACE, "workspace not 256-byte aligned");
    if (ws_bytes < need)
        return fail(MG_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, need);
    ns_carve(H, ws);
    NsLevel &f = H->lev[0];
    const size_t bytes0 = f.n * sizeof(double);
    const double *src[7] = {co->h, co->tx, co->ty, co->tz, co->txr, co->tyr, co->tzr};
    double *dst[7] = {f.h, f.tx, f.ty, f.tz, f.txr, f.tyr, f.tzr};
    for (int a = 0; a < 7; ++a)
        CU(cudaMemcpyAsync(dst[a], src[a], bytes0, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemsetAsync(H->flag, 0, 4 * sizeof(int), s));
    NRUN(launch_ns_validate(view(f, false), H->flag, s));
    NRUN(launch_ns_colmass(view(f, false), f.hT, s));
    NRUN(launch_ns_positive(f.hT, f.n, H->flag, s));
    int flag = 0;
    CU(cudaMemcpyAsync(&flag, H->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (flag)
        return fail(MG_ERR_COEFF, "invalid coefficients (bits %d: 1 h<=0/non-finite, 2 coupling<0/"
                                  "non-finite, 4 non-zero pole or top face, 8 column sum <= 0)",
                    flag);
    for (int l = 0; l < H->L; ++l) {
        NsLevel &v = H->lev[l];
        if (l + 1 < H->L) {
            const LinkHost &K = v.link;
            const LinkDev &D = v.linkdev;
            CHK(upload(K.j0, D.j0, s));
            CHK(upload(K.w0, D.w0, s));
            CHK(upload(K.j1, D.j1, s));
            CHK(upload(K.w1, D.w1, s));
            CHK(upload(K.rptr, D.rptr, s));
            CHK(upload(K.rrow, D.rrow, s));
            CHK(upload(K.rw, D.rw, s));
            CHK(upload(K.cfirst, D.cfirst, s));
            CHK(upload(K.ccnt, D.ccnt, s));
            CHK(upload(K.sy, D.sy, s));
            NsLevel &c = H->lev[l + 1];
            // H's coarse arrays; H^T's coarse couplings are these swapped, so
            // only its mass (the sums of the column sums) is formed apart
            NRUN(launch_ns_coarsen(view(v, false), D, 0.5, c.h, c.tx, c.ty, c.tz, c.txr, c.tyr,
                                   c.tzr, s));
            NRUN(launch_ns_coarsen(view(v, true), D, 0.5, c.hT, nullptr, nullptr, nullptr,
                                   nullptr, nullptr, nullptr, s));
        }
        NRUN(launch_ns_column_lu(view(v, false), v.m, v.dq, s));
        NRUN(launch_ns_column_lu(view(v, true), v.mT, v.dqT, s));
        // the uploads above read pageable host vectors: finish before they go away
        CU(cudaStreamSynchronize(s));
    }
    return MG_OK;
}

// `count` sweeps of Eq. (1) ending in `end`, alternating with `other`: from
// zero (start == nullptr) or from the iterate in `start`, which must be
// `other` for an odd count and `end` for an even one (a sweep never writes
// its own input).
int ns_sweeps(const NsView &V, const double *b, const double *start, int count, double *end,
              double *other, double omega, cudaStream_t s)
{
    if (count <= 0) return fail(MG_ERR_ARG, "no sweeps");
    double *cur;
    int left = count;
    if (!start) {
        cur = (count % 2 == 1) ? end : other;
        NRUN(launch_ns_smooth(V, b, nullptr, cur, omega, s));
        --left;
    } else {
        if (start != ((count % 2 == 1) ? other : end))
            return fail(MG_ERR_ARG, "sweep buffers out of parity");
        cur = const_cast<double *>(start);
    }
    for (; left > 0; --left) {
        double *next = (cur == end) ? other : end;
        NRUN(launch_ns_smooth(V, b, cur, next, omega, s));
        cur = next;
    }
    return MG_OK;
}

// One V(nu1, nu2) cycle from zero on level l of H (tr false) or H^T: out =
// V b.  The pre-smoothed iterate is placed so that the nu2 post-sweeps end
// in `out` (no copies); restriction and prolongation are the symmetric
// path's (they depend on the grid only).
int ns_vcycle_level(mg_ns_handle *H, int l, bool tr, const double *b, double *out, cudaStream_t s)
{
    NsLevel &v = H->lev[l];
    const NsView V = view(v, tr);
    const double om = H->p.omega;
    const int nu1 = H->p.nu1, nu2 = H->p.nu2;
    if (l == H->L - 1) return ns_sweeps(V, b, nullptr, H->p.coarse_iters, out, v.w, om, s);
    // the pre-smoothed iterate lives where nu2 post-sweeps alternating with
    // v.w end in out: v.w for odd nu2, out for even
    double *pre = (nu2 % 2 == 1) ? v.w : out;
    CHK(ns_sweeps(V, b, nullptr, nu1, pre, pre == out ? v.w : out, om, s));
    if (nu1 == 1)
        NRUN(launch_ns_presmooth_resid(V, b, pre, om, v.r, s));
    else
        NRUN(launch_ns_stencil(V, 1, b, pre, v.r, s));
    NsLevel &c = H->lev[l + 1];
    NRUN(launch_restrict<double>(shape_of(v), v.linkdev, v.r, c.b, s));
    CHK(ns_vcycle_level(H, l + 1, tr, c.b, c.u, s));
    NRUN(launch_prolong_add<double>(shape_of(v), v.linkdev, c.u, pre, s));
    if (nu2 > 0) CHK(ns_sweeps(V, b, pre, nu2, out, v.w, om, s));
    return MG_OK;
}

bool bad(double v) { return !(v == v) || std::isinf(v); }

// <a, b> into the scalar slot `which` of sc and back to the host.
int ns_dot(mg_ns_handle *H, const double *a, const double *b, double *out, cudaStream_t s)
{
    const size_t n = H->lev[0].n;
    const int nb = launch_dot<double>(a, b, n, H->partial, s);
    NRUN(cudaGetLastError());
    NRUN(launch_finalize(H->partial, nb, H->sc, S_RR, 0, s));
    CU(cudaMemcpyAsync(out, reinterpret_cast<double *>(H->sc) + S_RR, sizeof(double),
                       cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return MG_OK;
}

struct Record {
    std::vector<double> *hist;
    double bn;
    int *its;
    double *rel;
    void operator()(double rr, int it) const
    {
        *rel = bn > 0 ? std::sqrt(rr) / bn : 0.0;
        if (hist) hist->push_back(*rel);
        *its = it;
    }
};

int ns_stationary(mg_ns_handle *H, bool tr, const double *b, double *x, double tol, int maxit,
                  const Record &rec, double bb, cudaStream_t s)
{
    const NsView A = view(H->lev[0], tr);
    const size_t n = H->lev[0].n;
    const double bn = std::sqrt(bb);
    double rr0 = -1;
    for (int it = 0;; ++it) {
        NRUN(launch_ns_stencil(A, 1, b, x, H->r, s));
        double rr = 0;
        CHK(ns_dot(H, H->r, H->r, &rr, s));
        if (bad(rr)) return fail(MG_ERR_NONFINITE, "non-finite residual");
        if (rr0 < 0) rr0 = rr;
        rec(rr, it);
        if (std::sqrt(rr) <= tol * bn) return MG_OK;
        if (it >= maxit)
            return fail(MG_ERR_NOT_CONVERGED, "not converged after %d iterations (rel %.3e)", it,
                        *rec.rel);
        if (rr > 1e6 * rr0) return fail(MG_ERR_DIVERGED, "residual grew to %.3e", *rec.rel);
        CHK(ns_vcycle_level(H, 0, tr, H->r, H->e, s));
        NRUN(launch_add<double>(x, H->e, n, s));
    }
}

int read_bicg(mg_ns_handle *H, double *rr, double *brk, cudaStream_t s)
{
    double v[2] = {0, 0};
    CU(cudaMemcpyAsync(v, &H->bsc->rr, sizeof v, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    *rr = v[0];
    *brk = v[1];
    return MG_OK;
}

// BiCGStab right-preconditioned by the V-cycle (the iteration of the
// symmetric driver's solve_bicgstab): restarts from the true residual with
// r^ = r when the recursive residual meets the tolerance or on a breakdown.
int ns_bicgstab(mg_ns_handle *H, bool tr, const double *b, double *x, double tol, int maxit,
                const Record &rec, double bb, cudaStream_t s)
{
    const NsView A = view(H->lev[0], tr);
    const size_t n = H->lev[0].n;
    BicgScalars *sc = H->bsc;
    double *pa = H->partial, *pb = H->partial + kReduceSlots / 2;
    const double bn = std::sqrt(bb);
    int its = 0;
    double rr0 = -1;
    while (true) {
        double rr = 0, brk = 0;
        NRUN(launch_ns_stencil(A, 1, b, x, H->r, s));
        int nb = launch_dot<double>(H->r, H->r, n, pa, s);
        NRUN(cudaGetLastError());
        NRUN(launch_bicg_finalize(pa, nullptr, nb, sc, BICG_START, s));
        CHK(read_bicg(H, &rr, &brk, s));
        if (bad(rr)) return fail(MG_ERR_NONFINITE, "non-finite residual");
        if (rr0 < 0) rr0 = rr;
        rec(rr, its);
        if (std::sqrt(rr) <= tol * bn) return MG_OK;
        if (its >= maxit)
            return fail(MG_ERR_NOT_CONVERGED, "not converged after %d iterations (rel %.3e)", its,
                        *rec.rel);
        if (rr > 1e6 * rr0) return fail(MG_ERR_DIVERGED, "residual grew to %.3e", *rec.rel);
        NRUN(launch_bicg_dir<double>(H->rh, H->r, nullptr, n, sc, true, s));  // r^ = r
        bool first = true;
        while (its < maxit) {
            ++its;
            NRUN(launch_bicg_dir<double>(H->pv, H->r, H->v, n, sc, first, s));
            first = false;
            CHK(ns_vcycle_level(H, 0, tr, H->pv, H->ph, s));
            NRUN(launch_ns_stencil(A, 0, nullptr, H->ph, H->v, s));
            nb = launch_dot<double>(H->rh, H->v, n, pa, s);
            NRUN(cudaGetLastError());
            NRUN(launch_bicg_finalize(pa, nullptr, nb, sc, BICG_ALPHA, s));
            NRUN(launch_bicg_s<double>(H->sv, H->r, H->v, n, sc, s));
            CHK(ns_vcycle_level(H, 0, tr, H->sv, H->sh, s));
            NRUN(launch_ns_stencil(A, 0, nullptr, H->sh, H->t, s));
            nb = launch_dot2<double>(H->t, H->sv, n, pa, pb, s);
            NRUN(cudaGetLastError());
            NRUN(launch_bicg_finalize(pa, pb, nb, sc, BICG_OMEGA, s));
            nb = launch_bicg_update<double>(x, H->r, H->ph, H->sh, H->sv, H->t, H->rh, n, sc, pa,
                                            pb, s);
            NRUN(cudaGetLastError());
            NRUN(launch_bicg_finalize(pa, pb, nb, sc, BICG_NEXT, s));
            CHK(read_bicg(H, &rr, &brk, s));
            if (bad(rr)) return fail(MG_ERR_NONFINITE, "non-finite residual");
            if (std::sqrt(rr) <= tol * bn || its >= maxit || brk != 0.0) break;
            rec(rr, its);
            if (rr > 1e6 * rr0) return fail(MG_ERR_DIVERGED, "residual grew to %.3e", *rec.rel);
        }
    }
}

int level_ok(const mg_ns_handle *H, int level)
{
    if (!H) return fail(MG_ERR_ARG, "null handle");
    if (level < 0 || level >= H->L) return fail(MG_ERR_ARG, "level %d out of range", level);
    return MG_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" int mg_ns_workspace_bytes(const mg_grid *grid, const mg_params *params, size_t *bytes)
{
    if (!bytes) return fail(MG_ERR_ARG, "null bytes");
    mg_ns_handle tmp;
    CHK(ns_plan(&tmp, grid, params));
    *bytes = ns_carve(&tmp, nullptr);
    return MG_OK;
}

extern "C" int mg_ns_setup(const mg_grid *grid, const mg_ns_coeffs *coeffs,
                           const mg_params *params, void *workspace, size_t ws_bytes,
                           void *stream, mg_ns_handle **out)
{
    if (!out) return fail(MG_ERR_ARG, "null out");
    *out = nullptr;
    if (!coeffs || !coeffs->h || !coeffs->tx || !coeffs->ty || !coeffs->tz || !coeffs->txr ||
        !coeffs->tyr || !coeffs->tzr)
        return fail(MG_ERR_ARG, "null coefficient pointer");
    mg_ns_handle *H = new mg_ns_handle;
    int st = ns_plan(H, grid, params);
    if (st == MG_OK) st = ns_setup(H, coeffs, workspace, ws_bytes, (cudaStream_t)stream);
    if (st != MG_OK) {
        delete H;
        return st;
    }
    *out = H;
    return MG_OK;
}

extern "C" void mg_ns_destroy(mg_ns_handle *h) { delete h; }

extern "C" int mg_ns_apply(mg_ns_handle *H, int transpose, const double *x, double *y,
                           void *stream)
{
    CHK(level_ok(H, 0));
    if (!x || !y || x == y) return fail(MG_ERR_ARG, "null or aliased vectors");
    const cudaStream_t s = (cudaStream_t)stream;
    NRUN(launch_ns_stencil(view(H->lev[0], transpose != 0), 0, nullptr, x, y, s));
    return MG_OK;
}

extern "C" int mg_ns_vcycle(mg_ns_handle *H, int transpose, const double *r, double *e,
                            void *stream)
{
    CHK(level_ok(H, 0));
    if (!r || !e || r == e) return fail(MG_ERR_ARG, "null or aliased vectors");
    return ns_vcycle_level(H, 0, transpose != 0, r, e, (cudaStream_t)stream);
}

extern "C" int mg_ns_solve(mg_ns_handle *H, int transpose, const double *b, double *x,
                           double tol, mg_stats *st, void *stream)
{
    CHK(level_ok(H, 0));
    if (!b || !x || b == x) return fail(MG_ERR_ARG, "null or aliased vectors");
    if (!(tol > 0.0)) return fail(MG_ERR_ARG, "tol must be > 0");
    const cudaStream_t s = (cudaStream_t)stream;
    double bb = 0;
    CHK(ns_dot(H, b, b, &bb, s));
    if (bad(bb)) return fail(MG_ERR_NONFINITE, "non-finite right-hand side");
    std::vector<double> hist;
    int its = 0;
    double rel = 0;
    const Record rec{&hist, std::sqrt(bb), &its, &rel};
    const bool tr = transpose != 0;
    int rc = H->p.method == MG_METHOD_STATIONARY
                 ? ns_stationary(H, tr, b, x, tol, H->p.maxit, rec, bb, s)
                 : ns_bicgstab(H, tr, b, x, tol, H->p.maxit, rec, bb, s);
    if (st) {
        st->iterations = its;
        st->inner_iterations = 0;
        st->rel_res = rel;
        st->history_len = 0;
        if (st->history && st->history_cap > 0) {
            const int m = std::min<int>(st->history_cap, (int)hist.size());
            std::copy(hist.begin(), hist.begin() + m, st->history);
            st->history_len = m;
        }
    }
    return rc;
}

extern "C" int mg_ns_coeff_grad(mg_ns_handle *H, const double *lam, const double *x, double *gh,
                                double *gtx, double *gty, double *gtz, double *gtxr,
                                double *gtyr, double *gtzr, void *stream)
{
    CHK(level_ok(H, 0));
    if (!lam || !x) return fail(MG_ERR_ARG, "null lambda or x");
    const NsLevel &f = H->lev[0];
    NRUN(launch_ns_coeff_grad(f.nlon, f.nlat, f.nz, lam, x, gh, gtx, gty, gtz, gtxr, gtyr, gtzr,
                              (cudaStream_t)stream));
    return MG_OK;
}

extern "C" int mg_ns_num_levels(const mg_ns_handle *H) { return H ? H->L : 0; }

extern "C" int mg_ns_level_shape(const mg_ns_handle *H, int level, int *nlon, int *nlat,
                                 int *nz)
{
    CHK(level_ok(H, level));
    const NsLevel &v = H->lev[level];
    if (nlon) *nlon = v.nlon;
    if (nlat) *nlat = v.nlat;
    if (nz) *nz = v.nz;
    return MG_OK;
}

extern "C" int mg_ns_level_coeffs(mg_ns_handle *H, int level, int transpose, double *h_out,
                                  double *tx, double *ty, double *tz, double *txr, double *tyr,
                                  double *tzr, void *stream)
{
    CHK(level_ok(H, level));
    const NsLevel &v = H->lev[level];
    const NsView V = view(v, transpose != 0);
    const cudaStream_t s = (cudaStream_t)stream;
    const double *src[7] = {V.h, V.e, V.n, V.u, V.w, V.s, V.d};
    double *dst[7] = {h_out, tx, ty, tz, txr, tyr, tzr};
    for (int a = 0; a < 7; ++a)
        if (dst[a])
            CU(cudaMemcpyAsync(dst[a], src[a], v.n * sizeof(double), cudaMemcpyDeviceToDevice,
                               s));
    return MG_OK;
}

extern "C" int mg_ns_level_smooth(mg_ns_handle *H, int level, int transpose, const double *b,
                                  const double *u_in, double *u_out, void *stream)
{
    CHK(level_ok(H, level));
    if (!b || !u_out || u_out == u_in || u_out == b)
        return fail(MG_ERR_ARG, "null or aliased vectors");
    NRUN(launch_ns_smooth(view(H->lev[level], transpose != 0), b, u_in, u_out, H->p.omega,
                          (cudaStream_t)stream));
    return MG_OK;
}
