// Host driver of the nonsymmetric operator (C ABI mg_ns_*): the hierarchies
// of H and of H^T on Section 2.2's grid hierarchy, the V-cycle of either
// (Section 2), the stationary iteration and BiCGStab (Section 1's solver for
// the nonsymmetric problem, here preconditioned by the V-cycle), the
// mixed-precision form (FP32 multigrid inside FP64 refinement, Section 1's
// single-precision remark) and the coefficient gradient of the seven arrays.
//
// Workspace layout (carved with 256-byte alignment from the caller's buffer):
// per level the seven arrays of H, the column sums h^T, the column factors of
// H and of H^T, the V-cycle vectors and the level's row links, and with
// params->mixed their FP32 copies; then the fine-level solver vectors of
// each precision, the reduction partials and the device scalars.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/tpmg.h"
#include "tpmg_handle.h"
#include "tpmg_internal.h"

using namespace tpmg;

namespace {

template <typename T>
struct NsArrays {  // one level's arrays in one precision
    T *h = nullptr, *tx = nullptr, *ty = nullptr, *tz = nullptr;
    T *txr = nullptr, *tyr = nullptr, *tzr = nullptr, *hT = nullptr;
    T *m = nullptr, *dq = nullptr, *mT = nullptr, *dqT = nullptr;
    T *b = nullptr, *u = nullptr, *w = nullptr, *r = nullptr;  // V-cycle vectors
};

struct NsLevel {
    int nlon = 0, nlat = 0, nz = 0;
    size_t n = 0;
    NsArrays<double> d;
    NsArrays<float> f;  // FP32 copies (params->mixed)
    LinkHost link;
    LinkDev linkdev{};
};

// Fine-level solver vectors of one precision (BiCGStab: r, r^, p, p^, v, s,
// s^, t; the stationary iteration: r and the correction e; x: the inner
// solution of the mixed form).
template <typename T>
struct NsKrylov {
    T *r = nullptr, *rh = nullptr, *pv = nullptr, *ph = nullptr, *v = nullptr;
    T *sv = nullptr, *sh = nullptr, *t = nullptr, *e = nullptr, *x = nullptr;
};

}  // namespace

struct mg_ns_handle {
    mg_grid grid{};
    mg_params p{};
    int L = 0;
    std::vector<NsLevel> lev;
    NsKrylov<double> k64;
    NsKrylov<float> k32;
    double scale32 = 0.0;  // the FP32 arrays hold scale32 x the FP64 ones
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

template <typename T>
NsArrays<T> &arr(NsLevel &v);
template <>
NsArrays<double> &arr<double>(NsLevel &v) { return v.d; }
template <>
NsArrays<float> &arr<float>(NsLevel &v) { return v.f; }

template <typename T>
NsKrylov<T> &kry(mg_ns_handle *H);
template <>
NsKrylov<double> &kry<double>(mg_ns_handle *H) { return H->k64; }
template <>
NsKrylov<float> &kry<float>(mg_ns_handle *H) { return H->k32; }

template <typename T>
NsView<T> view(NsLevel &l, bool tr)
{
    const NsArrays<T> &v = arr<T>(l);
    if (!tr) return {l.nlon, l.nlat, l.nz, v.h, v.tx, v.ty, v.tz, v.txr, v.tyr, v.tzr, v.m, v.dq};
    return {l.nlon, l.nlat, l.nz, v.hT, v.txr, v.tyr, v.tzr, v.tx, v.ty, v.tz, v.mT, v.dqT};
}

template <typename T>
LevelDev<T> shape_of(const NsLevel &v)
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
    if (p->levels < 0) return fail(MG_ERR_ARG, "nonsymmetric hierarchy: levels >= 0");
    if (p->mixed && (p->inner_maxit < 1 || !(p->inner_tol > 0.0)))
        return fail(MG_ERR_ARG, "invalid inner-solve parameters");
    return MG_OK;
}

// Shapes and row links of every level: the grid hierarchy of the symmetric
// planner (it depends on the grid and the parameters only).
int ns_plan(mg_ns_handle *H, const mg_grid *g, const mg_params *p)
{
    CHK(ns_check(g, p));
    mg_handle *tmp = nullptr;
    size_t bytes = 0;
    mg_params q = *p;
    q.mixed = 0;  // the planner only lays out shapes and links here
    CHK(handle_plan(g, &q, nullptr, &bytes, &tmp));
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

template <typename T>
void carve_arrays(Bump &cv, NsArrays<T> &a, size_t n, bool coarse)
{
    for (T **p : {&a.h, &a.tx, &a.ty, &a.tz, &a.txr, &a.tyr, &a.tzr, &a.hT, &a.m, &a.dq, &a.mT,
                  &a.dqT, &a.u, &a.w, &a.r})
        *p = cv.take<T>(n);
    // the right-hand side: coarse levels, and the FP32 fine level (the inner
    // solve's r / sc)
    if (coarse || sizeof(T) == 4) a.b = cv.take<T>(n);
}

template <typename T>
void carve_krylov(Bump &cv, NsKrylov<T> &k, size_t n)
{
    for (T **p : {&k.r, &k.rh, &k.pv, &k.ph, &k.v, &k.sv, &k.sh, &k.t, &k.e, &k.x})
        *p = cv.take<T>(n);
}

size_t ns_carve(mg_ns_handle *H, void *base)
{
    Bump cv(base);
    const bool mixed = H->p.mixed != 0;
    for (int l = 0; l < H->L; ++l) {
        NsLevel &v = H->lev[l];
        carve_arrays<double>(cv, v.d, v.n, l > 0);
        if (mixed) carve_arrays<float>(cv, v.f, v.n, l > 0);
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
    carve_krylov<double>(cv, H->k64, n0);
    if (mixed) carve_krylov<float>(cv, H->k32, n0);
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

// max |a| over n values into *out (synchronises)
int ns_maxabs(mg_ns_handle *H, const double *a, size_t n, double *out, cudaStream_t s)
{
    const int nb = launch_maxabs<double>(a, n, H->partial, s);
    NRUN(cudaGetLastError());
    NRUN(launch_finalize(H->partial, nb, H->sc, S_MAX, 3, s));
    CU(cudaMemcpyAsync(out, reinterpret_cast<double *>(H->sc) + S_MAX, sizeof(double),
                       cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return MG_OK;
}

// FP32 copies of every level: the arrays scaled by one power of two that
// brings the largest to O(1) (exact; FP32's range then holds the column
// solves' products), the factors 1/p by its inverse, q/p as they are.
int ns_setup_fp32(mg_ns_handle *H, cudaStream_t s)
{
    double big = 0;
    for (NsLevel &v : H->lev)
        for (const double *a : {v.d.h, v.d.hT, v.d.tx, v.d.ty, v.d.tz, v.d.txr, v.d.tyr, v.d.tzr}) {
            double m = 0;
            CHK(ns_maxabs(H, a, v.n, &m, s));
            big = std::max(big, m);
        }
    if (!(big > 0) || !std::isfinite(big)) return fail(MG_ERR_COEFF, "bad coefficient range");
    int ex = 0;
    std::frexp(big, &ex);
    H->scale32 = std::ldexp(1.0, -ex);
    for (NsLevel &v : H->lev) {
        const NsArrays<double> &d = v.d;
        const NsArrays<float> &f = v.f;
        const double *src[8] = {d.h, d.hT, d.tx, d.ty, d.tz, d.txr, d.tyr, d.tzr};
        float *dst[8] = {f.h, f.hT, f.tx, f.ty, f.tz, f.txr, f.tyr, f.tzr};
        for (int a = 0; a < 8; ++a) NRUN(launch_to_float(src[a], dst[a], H->scale32, v.n, s));
        NRUN(launch_to_float(d.m, f.m, 1.0 / H->scale32, v.n, s));
        NRUN(launch_to_float(d.mT, f.mT, 1.0 / H->scale32, v.n, s));
        NRUN(launch_to_float(d.dq, f.dq, 1.0, v.n, s));
        NRUN(launch_to_float(d.dqT, f.dqT, 1.0, v.n, s));
    }
    CU(cudaStreamSynchronize(s));
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
    double *dst[7] = {f.d.h, f.d.tx, f.d.ty, f.d.tz, f.d.txr, f.d.tyr, f.d.tzr};
    for (int a = 0; a < 7; ++a)
        CU(cudaMemcpyAsync(dst[a], src[a], bytes0, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemsetAsync(H->flag, 0, 4 * sizeof(int), s));
    NRUN(launch_ns_validate(view<double>(f, false), H->flag, s));
    NRUN(launch_ns_colmass(view<double>(f, false), f.d.hT, s));
    NRUN(launch_ns_positive(f.d.hT, f.n, H->flag, s));
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
            NRUN(launch_ns_coarsen(view<double>(v, false), D, 0.5, c.d.h, c.d.tx, c.d.ty, c.d.tz,
                                   c.d.txr, c.d.tyr, c.d.tzr, s));
            NRUN(launch_ns_coarsen(view<double>(v, true), D, 0.5, c.d.hT, nullptr, nullptr,
                                   nullptr, nullptr, nullptr, nullptr, s));
        }
        NRUN(launch_ns_column_lu(view<double>(v, false), v.d.m, v.d.dq, s));
        NRUN(launch_ns_column_lu(view<double>(v, true), v.d.mT, v.d.dqT, s));
        // the uploads above read pageable host vectors: finish before they go away
        CU(cudaStreamSynchronize(s));
    }
    if (H->p.mixed) CHK(ns_setup_fp32(H, s));
    return MG_OK;
}

// `count` sweeps of Eq. (1) ending in `end`, alternating with `other`: from
// zero (start == nullptr) or from the iterate in `start`, which must be
// `other` for an odd count and `end` for an even one (a sweep never writes
// its own input).
template <typename T>
int ns_sweeps(const NsView<T> &V, const T *b, const T *start, int count, T *end, T *other,
              double omega, cudaStream_t s)
{
    if (count <= 0) return fail(MG_ERR_ARG, "no sweeps");
    T *cur;
    int left = count;
    if (!start) {
        cur = (count % 2 == 1) ? end : other;
        NRUN(launch_ns_smooth<T>(V, b, nullptr, cur, omega, s));
        --left;
    } else {
        if (start != ((count % 2 == 1) ? other : end))
            return fail(MG_ERR_ARG, "sweep buffers out of parity");
        cur = const_cast<T *>(start);
    }
    for (; left > 0; --left) {
        T *next = (cur == end) ? other : end;
        NRUN(launch_ns_smooth<T>(V, b, cur, next, omega, s));
        cur = next;
    }
    return MG_OK;
}

// One V(nu1, nu2) cycle from zero on level l of H (tr false) or H^T, in
// either precision: out = V b.  The pre-smoothed iterate is placed so that
// the nu2 post-sweeps end in `out` (no copies); restriction and prolongation
// are the symmetric path's (they depend on the grid only).
template <typename T>
int ns_vcycle_level(mg_ns_handle *H, int l, bool tr, const T *b, T *out, cudaStream_t s)
{
    NsLevel &v = H->lev[l];
    NsArrays<T> &a = arr<T>(v);
    const NsView<T> V = view<T>(v, tr);
    const double om = H->p.omega;
    const int nu1 = H->p.nu1, nu2 = H->p.nu2;
    if (l == H->L - 1) return ns_sweeps<T>(V, b, nullptr, H->p.coarse_iters, out, a.w, om, s);
    // the pre-smoothed iterate lives where nu2 post-sweeps alternating with
    // a.w end in out: a.w for odd nu2, out for even
    T *pre = (nu2 % 2 == 1) ? a.w : out;
    CHK(ns_sweeps<T>(V, b, nullptr, nu1, pre, pre == out ? a.w : out, om, s));
    if (nu1 == 1)
        NRUN(launch_ns_presmooth_resid<T>(V, b, pre, om, a.r, s));
    else
        NRUN(launch_ns_stencil<T>(V, 1, b, pre, a.r, s));
    NsLevel &c = H->lev[l + 1];
    NsArrays<T> &ca = arr<T>(c);
    NRUN(launch_restrict<T>(shape_of<T>(v), v.linkdev, a.r, ca.b, s));
    CHK(ns_vcycle_level<T>(H, l + 1, tr, ca.b, ca.u, s));
    NRUN(launch_prolong_add<T>(shape_of<T>(v), v.linkdev, ca.u, pre, s));
    if (nu2 > 0) CHK(ns_sweeps<T>(V, b, pre, nu2, out, a.w, om, s));
    return MG_OK;
}

bool bad(double v) { return !(v == v) || std::isinf(v); }

// <a, b> into the scalar slot S_RR of sc and back to the host.
template <typename T>
int ns_dot(mg_ns_handle *H, const T *a, const T *b, double *out, cudaStream_t s)
{
    const size_t n = H->lev[0].n;
    const int nb = launch_dot<T>(a, b, n, H->partial, s);
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

// x <- x + V(b - A x).  inner: x enters as zero and the FP32 residual b - A x
// decides (the inner solve of the mixed form).
template <typename T>
int ns_stationary(mg_ns_handle *H, bool tr, const T *b, T *x, double tol, int maxit,
                  const Record &rec, double bb, cudaStream_t s)
{
    NsLevel &f = H->lev[0];
    const NsView<T> A = view<T>(f, tr);
    NsKrylov<T> &k = kry<T>(H);
    const size_t n = f.n;
    const double bn = std::sqrt(bb);
    double rr0 = -1;
    for (int it = 0;; ++it) {
        NRUN(launch_ns_stencil<T>(A, 1, b, x, k.r, s));
        double rr = 0;
        CHK(ns_dot<T>(H, k.r, k.r, &rr, s));
        if (bad(rr)) return fail(MG_ERR_NONFINITE, "non-finite residual");
        if (rr0 < 0) rr0 = rr;
        rec(rr, it);
        if (std::sqrt(rr) <= tol * bn) return MG_OK;
        if (it >= maxit)
            return fail(MG_ERR_NOT_CONVERGED, "not converged after %d iterations (rel %.3e)", it,
                        *rec.rel);
        if (rr > 1e6 * rr0) return fail(MG_ERR_DIVERGED, "residual grew to %.3e", *rec.rel);
        CHK(ns_vcycle_level<T>(H, 0, tr, k.r, k.e, s));
        NRUN(launch_add<T>(x, k.e, n, s));
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
// inner: x enters as zero (r = b without a stencil) and the recursive
// residual decides (the FP64 outer residual is the check).
template <typename T>
int ns_bicgstab(mg_ns_handle *H, bool tr, const T *b, T *x, double tol, int maxit,
                const Record &rec, double bb, cudaStream_t s, bool inner = false)
{
    NsLevel &f = H->lev[0];
    const NsView<T> A = view<T>(f, tr);
    NsKrylov<T> &k = kry<T>(H);
    const size_t n = f.n;
    BicgScalars *sc = H->bsc;
    double *pa = H->partial, *pb = H->partial + kReduceSlots / 2;
    const double bn = std::sqrt(bb);
    int its = 0;
    double rr0 = -1;
    bool first_outer = true;
    while (true) {
        double rr = 0, brk = 0;
        if (inner && first_outer)
            NRUN(launch_bicg_dir<T>(k.r, b, nullptr, n, sc, true, s));  // r = b
        else
            NRUN(launch_ns_stencil<T>(A, 1, b, x, k.r, s));
        first_outer = false;
        int nb = launch_dot<T>(k.r, k.r, n, pa, s);
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
        NRUN(launch_bicg_dir<T>(k.rh, k.r, nullptr, n, sc, true, s));  // r^ = r
        bool first = true;
        while (its < maxit) {
            ++its;
            NRUN(launch_bicg_dir<T>(k.pv, k.r, k.v, n, sc, first, s));
            first = false;
            CHK(ns_vcycle_level<T>(H, 0, tr, k.pv, k.ph, s));
            NRUN(launch_ns_stencil<T>(A, 0, nullptr, k.ph, k.v, s));
            nb = launch_dot<T>(k.rh, k.v, n, pa, s);
            NRUN(cudaGetLastError());
            NRUN(launch_bicg_finalize(pa, nullptr, nb, sc, BICG_ALPHA, s));
            NRUN(launch_bicg_s<T>(k.sv, k.r, k.v, n, sc, s));
            CHK(ns_vcycle_level<T>(H, 0, tr, k.sv, k.sh, s));
            NRUN(launch_ns_stencil<T>(A, 0, nullptr, k.sh, k.t, s));
            nb = launch_dot2<T>(k.t, k.sv, n, pa, pb, s);
            NRUN(cudaGetLastError());
            NRUN(launch_bicg_finalize(pa, pb, nb, sc, BICG_OMEGA, s));
            nb = launch_bicg_update<T>(x, k.r, k.ph, k.sh, k.sv, k.t, k.rh, n, sc, pa, pb, s);
            NRUN(cudaGetLastError());
            NRUN(launch_bicg_finalize(pa, pb, nb, sc, BICG_NEXT, s));
            CHK(read_bicg(H, &rr, &brk, s));
            if (bad(rr)) return fail(MG_ERR_NONFINITE, "non-finite residual");
            if (std::sqrt(rr) <= tol * bn || its >= maxit || brk != 0.0) {
                if (inner && brk == 0.0) {
                    rec(rr, its);
                    return std::sqrt(rr) <= tol * bn ? MG_OK : MG_ERR_NOT_CONVERGED;
                }
                break;
            }
            rec(rr, its);
            if (rr > 1e6 * rr0) return fail(MG_ERR_DIVERGED, "residual grew to %.3e", *rec.rel);
        }
    }
}

template <typename T>
int ns_solve_impl(mg_ns_handle *H, bool tr, const T *b, T *x, double tol, int maxit,
                  const Record &rec, double bb, cudaStream_t s, bool inner)
{
    if (H->p.method == MG_METHOD_STATIONARY)
        return ns_stationary<T>(H, tr, b, x, tol, maxit, rec, bb, s);
    return ns_bicgstab<T>(H, tr, b, x, tol, maxit, rec, bb, s, inner);
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
    NRUN(launch_ns_stencil<double>(view<double>(H->lev[0], transpose != 0), 0, nullptr, x, y, s));
    return MG_OK;
}

extern "C" int mg_ns_vcycle(mg_ns_handle *H, int transpose, const double *r, double *e,
                            void *stream)
{
    CHK(level_ok(H, 0));
    if (!r || !e || r == e) return fail(MG_ERR_ARG, "null or aliased vectors");
    return ns_vcycle_level<double>(H, 0, transpose != 0, r, e, (cudaStream_t)stream);
}

extern "C" int mg_ns_vcycle_prec(mg_ns_handle *H, int transpose, int prec, const void *r,
                                 void *e, void *stream)
{
    CHK(level_ok(H, 0));
    if (!r || !e || r == e) return fail(MG_ERR_ARG, "null or aliased vectors");
    const cudaStream_t s = (cudaStream_t)stream;
    if (prec == MG_PREC_FP64)
        return ns_vcycle_level<double>(H, 0, transpose != 0, (const double *)r, (double *)e, s);
    if (prec != MG_PREC_FP32) return fail(MG_ERR_ARG, "prec %d unknown", prec);
    if (!H->p.mixed) return fail(MG_ERR_ARG, "handle built without the FP32 hierarchy (mixed=0)");
    return ns_vcycle_level<float>(H, 0, transpose != 0, (const float *)r, (float *)e, s);
}

static void ns_stats(mg_stats *st, const std::vector<double> &hist, int its, int inner,
                     double rel)
{
    if (!st) return;
    st->iterations = its;
    st->inner_iterations = inner;
    st->rel_res = rel;
    st->history_len = 0;
    if (st->history && st->history_cap > 0) {
        const int m = std::min<int>(st->history_cap, (int)hist.size());
        std::copy(hist.begin(), hist.begin() + m, st->history);
        st->history_len = m;
    }
}

extern "C" int mg_ns_solve(mg_ns_handle *H, int transpose, const double *b, double *x,
                           double tol, mg_stats *st, void *stream)
{
    CHK(level_ok(H, 0));
    if (!b || !x || b == x) return fail(MG_ERR_ARG, "null or aliased vectors");
    if (!(tol > 0.0)) return fail(MG_ERR_ARG, "tol must be > 0");
    const cudaStream_t s = (cudaStream_t)stream;
    double bb = 0;
    CHK(ns_dot<double>(H, b, b, &bb, s));
    if (bad(bb)) return fail(MG_ERR_NONFINITE, "non-finite right-hand side");
    std::vector<double> hist;
    int its = 0;
    double rel = 0;
    const Record rec{&hist, std::sqrt(bb), &its, &rel};
    const int rc = ns_solve_impl<double>(H, transpose != 0, b, x, tol, H->p.maxit, rec, bb, s,
                                         false);
    ns_stats(st, hist, its, 0, rel);
    return rc;
}

// FP32 multigrid (the configured method, on the FP32 hierarchy of H or H^T)
// inside FP64 iterative refinement: r = b - A x in FP64, the inner solve of
// (c A) e = r / sc from zero (c = scale32, sc a power of two near ||r||) to
// the inner tolerance, x += c sc e; as mg_solve_mixed for the symmetric
// operator.
extern "C" int mg_ns_solve_mixed(mg_ns_handle *H, int transpose, const double *b, double *x,
                                 double tol, mg_stats *st, void *stream)
{
    CHK(level_ok(H, 0));
    if (!b || !x || b == x) return fail(MG_ERR_ARG, "null or aliased vectors");
    if (!(tol > 0.0)) return fail(MG_ERR_ARG, "tol must be > 0");
    if (!H->p.mixed) return fail(MG_ERR_ARG, "handle built without the FP32 hierarchy (mixed=0)");
    const cudaStream_t s = (cudaStream_t)stream;
    const bool tr = transpose != 0;
    NsLevel &f = H->lev[0];
    const size_t n = f.n;
    double bb = 0;
    CHK(ns_dot<double>(H, b, b, &bb, s));
    if (bad(bb)) return fail(MG_ERR_NONFINITE, "non-finite right-hand side");
    const double bn = std::sqrt(bb);
    std::vector<double> hist;
    int outer = 0, inner = 0;
    double rel = 0, rr0 = -1;
    int rc = MG_OK;
    while (true) {
        NRUN(launch_ns_stencil<double>(view<double>(f, tr), 1, b, x, H->k64.r, s));
        double rr = 0;
        CHK(ns_dot<double>(H, H->k64.r, H->k64.r, &rr, s));
        if (bad(rr)) {
            rc = fail(MG_ERR_NONFINITE, "non-finite residual");
            break;
        }
        if (rr0 < 0) rr0 = rr;
        rel = bn > 0 ? std::sqrt(rr) / bn : 0.0;
        hist.push_back(rel);
        if (std::sqrt(rr) <= tol * bn) break;
        if (outer >= H->p.maxit) {
            rc = fail(MG_ERR_NOT_CONVERGED, "not converged after %d refinement steps", outer);
            break;
        }
        if (rr > 1e6 * rr0) {
            rc = fail(MG_ERR_DIVERGED, "residual grew to %.3e", rel);
            break;
        }
        int ex = 0;
        std::frexp(std::sqrt(rr), &ex);
        const double sc = std::ldexp(1.0, ex);
        NRUN(launch_cast_scaled(H->k64.r, f.f.b, 1.0 / sc, n, s));
        CU(cudaMemsetAsync(H->k32.x, 0, n * sizeof(float), s));
        // the inner rhs r / sc has norm in [1/2, 1): its relative tolerance
        // is the solve's own
        double bb32 = 0;
        CHK(ns_dot<float>(H, f.f.b, f.f.b, &bb32, s));
        int its_in = 0;
        double rel_in = 0;
        const Record rin{nullptr, std::sqrt(bb32), &its_in, &rel_in};
        const double itol = inner_tolerance(H->p.inner_tol, tol, rel);
        const int ri = ns_solve_impl<float>(H, tr, f.f.b, H->k32.x, itol, H->p.inner_maxit, rin,
                                            bb32, s, true);
        if (ri != MG_OK && ri != MG_ERR_NOT_CONVERGED && ri != MG_ERR_DIVERGED) {
            rc = ri;
            break;
        }
        inner += its_in;
        NRUN(launch_update_mixed(x, H->k32.x, H->scale32 * sc, n, s));
        ++outer;
    }
    ns_stats(st, hist, outer, inner, rel);
    return rc;
}

extern "C" double mg_ns_fp32_scale(const mg_ns_handle *H) { return H ? H->scale32 : 0.0; }

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
    NsLevel &v = H->lev[level];
    const NsView<double> V = view<double>(v, transpose != 0);
    const cudaStream_t s = (cudaStream_t)stream;
    const double *src[7] = {V.h, V.e, V.n, V.u, V.w, V.s, V.d};
    double *dst[7] = {h_out, tx, ty, tz, txr, tyr, tzr};
    for (int a = 0; a < 7; ++a)
        if (dst[a])
            CU(cudaMemcpyAsync(dst[a], src[a], v.n * sizeof(double), cudaMemcpyDeviceToDevice,
                               s));
    return MG_OK;
}

extern "C" int mg_ns_level_smooth(mg_ns_handle *H, int level, int transpose, int prec,
                                  const void *b, const void *u_in, void *u_out, void *stream)
{
    CHK(level_ok(H, level));
    if (!b || !u_out || u_out == u_in || u_out == b)
        return fail(MG_ERR_ARG, "null or aliased vectors");
    const cudaStream_t s = (cudaStream_t)stream;
    NsLevel &v = H->lev[level];
    if (prec == MG_PREC_FP64) {
        NRUN(launch_ns_smooth<double>(view<double>(v, transpose != 0), (const double *)b,
                                      (const double *)u_in, (double *)u_out, H->p.omega, s));
        return MG_OK;
    }
    if (prec != MG_PREC_FP32) return fail(MG_ERR_ARG, "prec %d unknown", prec);
    if (!H->p.mixed) return fail(MG_ERR_ARG, "handle built without the FP32 hierarchy (mixed=0)");
    NRUN(launch_ns_smooth<float>(view<float>(v, transpose != 0), (const float *)b,
                                 (const float *)u_in, (float *)u_out, H->p.omega, s));
    return MG_OK;
}
