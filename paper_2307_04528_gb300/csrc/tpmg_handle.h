// Host-side state of a multigrid handle, shared by the single-system driver
// (tpmg_api.cpp) and the batched ensemble driver (tpmg_batch_api.cpp).
// Internal; not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tpmg.h"
#include "tpmg_internal.h"

namespace tpmg {

// Set the thread-local error message (printf-style) and return `code`.
int fail(int code, const char *fmt, ...);

// Kernel launches issued by the library (all handles).
extern std::atomic<unsigned long long> g_launches;

// rc, or MG_ERR_TIMEOUT when a staged kernel gave up waiting on its copies
// since the last check (synchronises s).
int check_timeouts(int rc, cudaStream_t s);

struct LinkHost {
    int nlat_c = 0;
    std::vector<int> cfirst, ccnt, j0, j1, rptr, rrow;
    std::vector<double> w0, w1, rw, sy;
};

}  // namespace tpmg

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return tpmg::fail(MG_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                              __FILE__, __LINE__);                                        \
    } while (0)

#define CHK(expr)                     \
    do {                              \
        int st_ = (expr);             \
        if (st_ != MG_OK) return st_; \
    } while (0)

using tpmg::LinkHost;
using tpmg::LevelDev;
using tpmg::LinkDev;
using tpmg::CgScalars;
using tpmg::BicgScalars;

// ------------------------------------------------------------------ handle
struct LevelHost {
    int nlon = 0, nlat = 0, nz = 0;
    size_t n = 0;
    double *tx = nullptr, *ty = nullptr, *tz = nullptr, *h = nullptr, *m = nullptr, *dq = nullptr;
    float *tx32 = nullptr, *ty32 = nullptr, *tz32 = nullptr, *h32 = nullptr, *m32 = nullptr,
          *dq32 = nullptr;
    // V-cycle vectors: rhs, result, ping-pong scratch, residual
    double *b = nullptr, *u = nullptr, *w = nullptr, *r = nullptr;
    float *b32 = nullptr, *u32 = nullptr, *w32 = nullptr, *r32 = nullptr;
    // coarsest level with the PCG coarse solve: direction and its image
    double *cd = nullptr, *cq = nullptr;
    // finest level, mixed precision: h + the horizontal couplings
    double *dh = nullptr;
    float *cd32 = nullptr, *cq32 = nullptr;
    LinkHost link;
    LinkDev linkdev{};
};

// Fine-level vectors of the outer iterations.  Conjugate gradients use r, z,
// d0, d1, Ad (x: the FP32 inner solution of the mixed solve).  BiCGStab
// (carved only for its methods) uses r, rh = Ad, p = d0, ph = z, v = d1 and
// s, sh, t.
template <typename T>
struct CgVecs {
    T *r = nullptr, *z = nullptr, *d0 = nullptr, *d1 = nullptr, *Ad = nullptr, *x = nullptr;
    T *s = nullptr, *sh = nullptr, *t = nullptr;
};

struct ProfRec {
    int key;
    cudaEvent_t a, b;
};

struct Profiler {
    bool on = false;
    bool all_levels = false;
    std::vector<cudaEvent_t> pool;
    size_t next = 0;
    std::vector<ProfRec> recs;
};

// A V-cycle captured once as a CUDA graph (fixed input/output vectors of
// the solver), replayed on the caller's stream.
struct VGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned long long kernels = 0;  // kernel nodes, for the launch count
    int dot_blocks = 0;              // partial sums of the fused <r, z> it leaves
};

struct mg_handle {
    Profiler prof;
    // right-hand side / solution of the current batched solve (batch driver)
    const void *batch_b = nullptr;
    void *batch_x = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
    bool capturing = false;
    VGraph *cap_graph = nullptr;        // the graph being captured
    bool use_graphs = true;
    // V-cycles captured per precision [MG_PREC_FP64], [MG_PREC_FP32] and
    // vector pair: 0 r -> z (conjugate gradients, stationary), 1 p -> ph and
    // 2 s -> sh (BiCGStab)
    VGraph vg[2][3];
    mg_grid grid{};
    mg_params p{};
    int L = 0;
    std::vector<LevelHost> lev;
    CgVecs<double> cg64;
    CgVecs<float> cg32;
    double *partial = nullptr;
    CgScalars *sc = nullptr;
    CgScalars *sc_coarse = nullptr;  // scalars of the PCG coarse solve
    BicgScalars *bsc = nullptr;      // scalars of BiCGStab
    int *flag = nullptr;
    double scale32 = 0.0;
    double cheb_mu = 0.0;  // Chebyshev coarse solve: lower end of the spectrum of H_z^{-1} H
};

template <typename T>
LevelDev<T> dev(const LevelHost &l);
template <>
inline LevelDev<double> dev<double>(const LevelHost &l)
{
    return {l.nlon, l.nlat, l.nz, l.tx, l.ty, l.tz, l.h, l.m, l.dq};
}
template <>
inline LevelDev<float> dev<float>(const LevelHost &l)
{
    return {l.nlon, l.nlat, l.nz, l.tx32, l.ty32, l.tz32, l.h32, l.m32, l.dq32};
}
template <typename T>
struct Vec;
template <>
struct Vec<double> {
    static double *cd(LevelHost &l) { return l.cd; }
    static double *cq(LevelHost &l) { return l.cq; }
    static double *b(LevelHost &l) { return l.b; }
    static double *u(LevelHost &l) { return l.u; }
    static double *w(LevelHost &l) { return l.w; }
    static double *r(LevelHost &l) { return l.r; }
    static CgVecs<double> &cg(mg_handle *h) { return h->cg64; }
};
template <>
struct Vec<float> {
    static float *cd(LevelHost &l) { return l.cd32; }
    static float *cq(LevelHost &l) { return l.cq32; }
    static float *b(LevelHost &l) { return l.b32; }
    static float *u(LevelHost &l) { return l.u32; }
    static float *w(LevelHost &l) { return l.w32; }
    static float *r(LevelHost &l) { return l.r32; }
    static CgVecs<float> &cg(mg_handle *h) { return h->cg32; }
};


enum { K_SMOOTH = 0, K_SMOOTH0 = 1, K_RESID = 2, K_APPLY = 3, K_RESTRICT = 4, K_PROLONG = 5,
       K_VEC = 6 };

inline int prof_key(int kind, int level, int prec) { return (kind * 64 + level) * 2 + prec; }

// Run one launcher (which may issue one kernel); count it and, when
// profiling is on, bracket it with events on its stream.
template <typename F>
inline int run_k(mg_handle *H, int kind, int level, int prec, cudaStream_t s, F &&f)
{
    Profiler &P = H->prof;
    const bool rec = P.on && (P.all_levels || level == 0) && P.next + 2 <= P.pool.size();
    cudaEvent_t a = nullptr, b = nullptr;
    if (rec) {
        a = P.pool[P.next++];
        b = P.pool[P.next++];
        CU(cudaEventRecord(a, s));
    }
    const cudaError_t e = f();
    if (H->capturing) ++H->cap_graph->kernels;
    else tpmg::g_launches.fetch_add(1, std::memory_order_relaxed);
    if (e != cudaSuccess)
        return tpmg::fail(MG_ERR_CUDA, "kernel launch (kind %d, level %d): %s", kind, level,
                    cudaGetErrorString(e));
    if (rec) {
        CU(cudaEventRecord(b, s));
        P.recs.push_back({prof_key(kind, level, prec), a, b});
    }
    return MG_OK;
}

inline cudaError_t to_err(cudaError_t e) { return e != cudaSuccess ? e : cudaGetLastError(); }
inline cudaError_t to_err(int) { return cudaGetLastError(); }

#define KRUN(kind, level, prec, expr) \
    CHK(run_k(H, kind, level, prec, s, [&]() -> cudaError_t { return to_err(expr); }))

template <typename T>
constexpr int prec_of() { return sizeof(T) == 8 ? MG_PREC_FP64 : MG_PREC_FP32; }


enum { S_RZ = 0, S_RZNEW = 1, S_DAD = 2, S_RR = 3, S_ALPHA = 4, S_BETA = 5, S_MAX = 6 };

namespace tpmg {
// Build the host hierarchy and lay out the device arrays of one system in
// `ws` (nullptr: sizes only); *bytes receives the workspace size.
int handle_plan(const mg_grid *g, const mg_params *p, void *ws, size_t *bytes, mg_handle **out);
// Device setup of a planned handle (coefficient copy and validation,
// hierarchy, factors, FP32 copies).
int handle_setup(mg_handle *H, const mg_coeffs *co, void *ws, size_t ws_bytes, cudaStream_t s);
int read_scalars(mg_handle *H, int which, double *out, cudaStream_t s);
double inner_tolerance(double inner_tol, double tol, double rel);
}  // namespace tpmg
