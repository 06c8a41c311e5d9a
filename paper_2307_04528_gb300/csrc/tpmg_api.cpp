// Host driver and C ABI of the tensor-product multigrid (see include/tpmg.h).
//
// The host side builds the hierarchy's integer structure (conditional
// semi-coarsening, Section 2.2), carves every device array out of the
// caller's workspace, and sequences the kernels of tpmg_kernels.cu into
// V-cycles (Section 2, Fig. 1) and solvers.  It allocates no device memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tpmg.h"
#include "tpmg_handle.h"
#include "tpmg_internal.h"

using namespace tpmg;

static_assert(kMaxLayers == MG_MAX_NZ, "device layer bound must match the C ABI");

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

int tpmg::fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

void tpmg::set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }

std::atomic<unsigned long long> tpmg::g_launches{0};

// ------------------------------------------------------------------ hierarchy (host)
namespace {

struct LevelShape {
    int nlon, nlat;
    std::vector<double> south, north;  // row edges (latitude)
    double centre(int j) const { return 0.5 * (south[j] + north[j]); }
};

// Conditional semi-coarsening (Section 2.2): longitude halves; in each
// hemisphere rows are merged in pairs from the equator poleward while the
// merged cell keeps alpha = cos(theta_c) dlambda_c / dtheta >= alpha_c, and
// stay single from the first failure on.  The south mirrors the north.
void coarsen_rows(const LevelShape &f, int nlon_c, double alpha_c, LevelShape &c, LinkHost &K)
{
    const int n = f.nlat, half = n / 2;
    const double dlon_c = 2.0 * M_PI / nlon_c;
    std::vector<std::pair<int, int>> north;  // (first row, count)
    int q = half;
    bool merging = true;
    while (q < n) {
        if (merging && q + 1 < n) {
            const double ths = f.south[q], thn = f.north[q + 1];
            const double alpha = std::cos(0.5 * (ths + thn)) * dlon_c / (thn - ths);
            if (alpha >= alpha_c) {
                north.push_back({q, 2});
                q += 2;
                continue;
            }
            merging = false;
        }
        north.push_back({q, 1});
        q += 1;
    }
    std::vector<std::pair<int, int>> groups;
    for (auto it = north.rbegin(); it != north.rend(); ++it)
        groups.push_back({n - 1 - (it->first + it->second - 1), it->second});
    groups.insert(groups.end(), north.begin(), north.end());

    const int nc = (int)groups.size();
    c.nlon = nlon_c;
    c.nlat = nc;
    c.south.resize(nc);
    c.north.resize(nc);
    K.nlat_c = nc;
    K.cfirst.resize(nc);
    K.ccnt.resize(nc);
    std::vector<int> row_of(n);
    for (int J = 0; J < nc; ++J) {
        const int g = groups[J].first, cnt = groups[J].second;
        for (int j = g; j < g + cnt; ++j) row_of[j] = J;
        c.south[J] = f.south[g];
        c.north[J] = f.north[g + cnt - 1];
        K.cfirst[J] = g;
        K.ccnt[J] = cnt;
    }
    // prolongation weights in latitude (linear between coarse row centres)
    K.j0.assign(n, 0);
    K.j1.assign(n, -1);
    K.w0.assign(n, 1.0);
    K.w1.assign(n, 0.0);
    for (int j = 0; j < n; ++j) {
        const int J = row_of[j];
        K.j0[j] = J;
        const double d = f.centre(j) - c.centre(J);
        if (d == 0.0) continue;
        const int Jn = d > 0 ? J + 1 : J - 1;
        if (Jn < 0 || Jn >= nc) continue;
        const double w = d / (c.centre(Jn) - c.centre(J));
        K.j1[j] = Jn;
        K.w1[j] = w;
        K.w0[j] = 1.0 - w;
    }
    // restriction = transpose, as a per-coarse-row gather list
    K.rptr.assign(nc + 1, 0);
    std::vector<std::vector<std::pair<int, double>>> lists(nc);
    for (int j = 0; j < n; ++j) {
        lists[K.j0[j]].push_back({j, K.w0[j]});
        if (K.j1[j] >= 0) lists[K.j1[j]].push_back({j, K.w1[j]});
    }
    K.rrow.clear();
    K.rw.clear();
    for (int J = 0; J < nc; ++J) {
        std::sort(lists[J].begin(), lists[J].end());
        for (auto &pr : lists[J]) {
            K.rrow.push_back(pr.first);
            K.rw.push_back(pr.second);
        }
        K.rptr[J + 1] = (int)K.rrow.size();
    }
    // coarse north-face distance ratio
    K.sy.assign(nc, 0.0);
    for (int J = 0; J + 1 < nc; ++J) {
        const int top = K.cfirst[J] + K.ccnt[J] - 1;
        K.sy[J] = (f.centre(top + 1) - f.centre(top)) / (c.centre(J + 1) - c.centre(J));
    }
}

int auto_levels(int nlon)
{
    int L = 1, n = nlon;
    while (n % 2 == 0 && n / 2 >= 4) {
        n /= 2;
        ++L;
    }
    return L;
}

// Bump allocator over the caller's workspace (dry run when base == nullptr).
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base((char *)b) {}
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

}  // namespace

static bool is_bicgstab(int method)
{
    return method == MG_METHOD_BICGSTAB || method == MG_METHOD_BICGSTAB_LINE;
}

static int check_grid(const mg_grid *g, const mg_params *p, int *L_out)
{
    if (!g || !p) return fail(MG_ERR_ARG, "null grid or params");
    if (g->nz < 1 || g->nz > MG_MAX_NZ)
        return fail(MG_ERR_ARG, "nz=%d outside [1, %d]", g->nz, MG_MAX_NZ);
    if (g->nlat < 2 || g->nlat % 2)
        return fail(MG_ERR_ARG, "nlat=%d must be even and >= 2", g->nlat);
    if (g->nlon < 4) return fail(MG_ERR_ARG, "nlon=%d must be >= 4", g->nlon);
    const int L = p->levels > 0 ? p->levels : auto_levels(g->nlon);
    if (L > 1 && (g->nlon % (1 << (L - 1)) || (g->nlon >> (L - 1)) < 2))
        return fail(MG_ERR_ARG, "nlon=%d not divisible by 2^(levels-1) = %d", g->nlon,
                    1 << (L - 1));
    if (p->coarse_method != MG_COARSE_JACOBI && p->coarse_method != MG_COARSE_PCG &&
        p->coarse_method != MG_COARSE_CHEBYSHEV)
        return fail(MG_ERR_ARG, "coarse_method %d unknown", p->coarse_method);
    if (p->nu1 < 1 || p->nu2 < 0 || p->coarse_iters < 1 || p->maxit < 0 ||
        !(p->omega > 0.0 && p->omega < 2.0) ||
        (p->method != MG_METHOD_CG && p->method != MG_METHOD_STATIONARY &&
         !is_bicgstab(p->method)) ||
        (p->method == MG_METHOD_BICGSTAB_LINE && (p->line_sweeps < 1 || p->line_sweeps > 100)) ||
        p->levels < -1 || (p->levels == -1 && !(p->iso_ratio > 0.0)))
        return fail(MG_ERR_ARG, "invalid multigrid parameters");
    if ((size_t)g->nlon * g->nlat > (size_t)kReduceSlots * kBlock)
        return fail(MG_ERR_ARG, "nlon*nlat=%zu exceeds %zu columns", (size_t)g->nlon * g->nlat,
                    (size_t)kReduceSlots * kBlock);
    *L_out = L;
    return MG_OK;
}

static void build_shapes(const mg_grid *g, const mg_params *p, int L, std::vector<LevelHost> &lev)
{
    lev.assign(L, LevelHost{});
    LevelShape cur;
    cur.nlon = g->nlon;
    cur.nlat = g->nlat;
    cur.south.resize(g->nlat);
    cur.north.resize(g->nlat);
    const double dth = M_PI / g->nlat;
    for (int j = 0; j < g->nlat; ++j) {
        cur.south[j] = -0.5 * M_PI + j * dth;
        cur.north[j] = -0.5 * M_PI + (j + 1) * dth;
    }
    cur.south[0] = -0.5 * M_PI;
    cur.north[g->nlat - 1] = 0.5 * M_PI;
    for (int l = 0; l < L; ++l) {
        lev[l].nlon = cur.nlon;
        lev[l].nlat = cur.nlat;
        lev[l].nz = g->nz;
        lev[l].n = (size_t)cur.nlon * cur.nlat * g->nz;
        if (l + 1 < L) {
            LevelShape next;
            coarsen_rows(cur, cur.nlon / 2, p->alpha_c, next, lev[l].link);
            cur = next;
        }
    }
}

// Lay out every device array; with base == nullptr only sizes are computed.
static size_t carve(mg_handle *H, void *base)
{
    Carver cv(base);
    const bool mixed = H->p.mixed != 0;
    for (int l = 0; l < H->L; ++l) {
        LevelHost &v = H->lev[l];
        const size_t n = v.n;
        v.tx = cv.take<double>(n);
        v.ty = cv.take<double>(n);
        v.tz = cv.take<double>(n);
        v.h = cv.take<double>(n);
        v.m = cv.take<double>(n);
        v.dq = cv.take<double>(n);
        v.u = cv.take<double>(n);
        v.w = cv.take<double>(n);
        v.r = cv.take<double>(n);
        if (l > 0) v.b = cv.take<double>(n);
        // the coarsest level's extra vectors (PCG: direction and its image;
        // Chebyshev: step and residual ping-pong); with the isotropy rule any
        // level below the finest may end up the coarsest
        const bool pcg = (l == H->L - 1 || (H->p.levels < 0 && l > 0)) &&
                         (H->p.coarse_method == MG_COARSE_PCG ||
                          H->p.coarse_method == MG_COARSE_CHEBYSHEV);
        if (pcg) {
            v.cd = cv.take<double>(n);
            v.cq = cv.take<double>(n);
        }
        if (mixed && l == 0) v.dh = cv.take<double>(n);
        if (mixed) {
            v.tx32 = cv.take<float>(n);
            v.ty32 = cv.take<float>(n);
            v.tz32 = cv.take<float>(n);
            v.h32 = cv.take<float>(n);
            v.m32 = cv.take<float>(n);
            v.dq32 = cv.take<float>(n);
            v.u32 = cv.take<float>(n);
            v.w32 = cv.take<float>(n);
            v.r32 = cv.take<float>(n);
            v.b32 = cv.take<float>(n);  // level 0: right-hand side of the inner solve
            if (pcg) {
                v.cd32 = cv.take<float>(n);
                v.cq32 = cv.take<float>(n);
            }
        }
        if (l + 1 < H->L) {
            LinkHost &K = v.link;
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
    const bool bicg = is_bicgstab(H->p.method);
    H->cg64.r = cv.take<double>(n0);
    H->cg64.z = cv.take<double>(n0);
    H->cg64.d0 = cv.take<double>(n0);
    H->cg64.d1 = cv.take<double>(n0);
    H->cg64.Ad = cv.take<double>(n0);
    if (bicg) {
        H->cg64.s = cv.take<double>(n0);
        H->cg64.sh = cv.take<double>(n0);
        H->cg64.t = cv.take<double>(n0);
    }
    if (mixed) {
        H->cg32.r = cv.take<float>(n0);
        H->cg32.z = cv.take<float>(n0);
        H->cg32.d0 = cv.take<float>(n0);
        H->cg32.d1 = cv.take<float>(n0);
        H->cg32.Ad = cv.take<float>(n0);
        H->cg32.x = cv.take<float>(n0);
        if (bicg) {
            H->cg32.s = cv.take<float>(n0);
            H->cg32.sh = cv.take<float>(n0);
            H->cg32.t = cv.take<float>(n0);
        }
    }
    H->partial = cv.take<double>(kReduceSlots);
    H->sc = cv.take<CgScalars>(1);
    H->sc_coarse = cv.take<CgScalars>(1);
    H->bsc = cv.take<BicgScalars>(1);
    H->flag = cv.take<int>(4);
    return cv.off + 256;
}

// ------------------------------------------------------------------ C ABI: setup
extern "C" void mg_default_params(mg_params *p)
{
    if (!p) return;
    p->levels = 0;
    p->nu1 = 1;
    p->nu2 = 1;
    p->coarse_iters = 12;
    p->method = MG_METHOD_CG;
    p->mixed = 0;
    p->maxit = 200;
    p->inner_maxit = 12;
    p->omega = 0.85;
    p->alpha_c = 0.6;
    p->inner_tol = 5e-4;
    p->coarse_method = MG_COARSE_JACOBI;
    p->line_sweeps = 1;
    p->iso_ratio = 6.25;
}

extern "C" const char *mg_last_error(void) { return g_last_error.c_str(); }

extern "C" int mg_workspace_bytes(const mg_grid *grid, const mg_params *params, size_t *bytes)
{
    int L = 0;
    CHK(check_grid(grid, params, &L));
    if (!bytes) return fail(MG_ERR_ARG, "null bytes");
    mg_handle tmp;
    tmp.grid = *grid;
    tmp.p = *params;
    tmp.L = L;
    build_shapes(grid, params, L, tmp.lev);
    *bytes = carve(&tmp, nullptr);
    return MG_OK;
}

template <typename V>
static int upload(const V &host, const void *dst, cudaStream_t s)
{
    if (host.empty()) return MG_OK;
    CU(cudaMemcpyAsync(const_cast<void *>(dst), host.data(), host.size() * sizeof(host[0]),
                       cudaMemcpyHostToDevice, s));
    return MG_OK;
}

static int read_scalar(mg_handle *H, int which, double *out, cudaStream_t s)
{
    CU(cudaMemcpyAsync(out, reinterpret_cast<double *>(H->sc) + which, sizeof(double),
                       cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return MG_OK;
}


static int device_max(mg_handle *H, const double *a, size_t n, double *out, cudaStream_t s)
{
    int nb = 0;
    KRUN(K_VEC, 0, 0, nb = launch_maxabs<double>(a, n, H->partial, s));
    KRUN(K_VEC, 0, 0, launch_finalize(H->partial, nb, H->sc, S_MAX, 3, s));
    return read_scalar(H, S_MAX, out, s);
}

static int setup_impl(mg_handle *H, const mg_coeffs *co, void *ws, size_t ws_bytes, cudaStream_t s)
{
    // A coarse row gathers its own one or two fine rows and at most the
    // nearer child of each neighbouring pair: the restriction kernels hold
    // kMaxRestrictRows rows per coarse row.
    for (int l = 0; l + 1 < H->L; ++l) {
        const std::vector<int> &rp = H->lev[l].link.rptr;
        for (size_t J = 0; J + 1 < rp.size(); ++J)
            if (rp[J + 1] - rp[J] > kMaxRestrictRows)
                return fail(MG_ERR_ARG, "level %d: coarse row %zu gathers %d fine rows (> %d)", l,
                            J, rp[J + 1] - rp[J], kMaxRestrictRows);
    }
    size_t need = carve(H, nullptr);
    if (!ws) return fail(MG_ERR_WORKSPACE, "null workspace");
    if ((uintptr_t)ws % 256) return fail(MG_ERR_WORKSPACE, "workspace not 256-byte aligned");
    if (ws_bytes < need)
        return fail(MG_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, need);
    carve(H, ws);
    CU(smooth_prepare());
    CU(tma_prepare());
    {
        int dev = 0, lim = 0;
        CU(cudaGetDevice(&dev));
        CU(cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        // 256 bytes: static shared memory of the block reductions
        if (smooth_smem_bytes(H->grid.nz, sizeof(double)) + 256 > (size_t)lim)
            return fail(MG_ERR_ARG, "nz = %d needs more shared memory per block than the device has",
                        H->grid.nz);
    }
    CU(cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
    LevelHost &f = H->lev[0];
    const size_t bytes0 = f.n * sizeof(double);
    CU(cudaMemcpyAsync(f.tx, co->tx, bytes0, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(f.ty, co->ty, bytes0, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(f.tz, co->tz, bytes0, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(f.h, co->h, bytes0, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemsetAsync(H->flag, 0, 4 * sizeof(int), s));
    KRUN(K_VEC, 0, 0, launch_validate(dev<double>(f), H->flag, s));
    int flag = 0;
    CU(cudaMemcpyAsync(&flag, H->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (flag)
        return fail(MG_ERR_COEFF, "invalid coefficients (bits %d: 1 h<=0/non-finite, 2 T<0/"
                                  "non-finite, 4 non-zero pole or top face)", flag);
    for (int l = 0; l < H->L; ++l) {
        LevelHost &v = H->lev[l];
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
            LevelHost &c = H->lev[l + 1];
            KRUN(K_VEC, l, 0, launch_coarsen(dev<double>(v), D, 0.5, c.tx, c.ty, c.tz, c.h, s));
            if (H->p.levels < 0) {  // coarsen until the couplings are within iso_ratio
                int nb = 0;
                KRUN(K_VEC, l + 1, 0, nb = launch_hz_ratio(dev<double>(c), H->partial, s));
                KRUN(K_VEC, l + 1, 0, launch_finalize(H->partial, nb, H->sc, S_MAX, 3, s));
                double ratio = 0;
                CHK(read_scalar(H, S_MAX, &ratio, s));
                if (!std::isfinite(ratio)) return fail(MG_ERR_COEFF, "bad coarse coefficients");
                if (ratio - 1.0 <= H->p.iso_ratio) H->L = l + 2;  // level l+1 is the coarsest
            }
        }
        KRUN(K_VEC, l, 0, launch_column_lu(dev<double>(v), v.m, v.dq, s));
        // the uploads above read pageable host vectors: finish before they go away
        CU(cudaStreamSynchronize(s));
    }
    if (H->p.coarse_method == MG_COARSE_CHEBYSHEV) {
        // spectrum of H_z^{-1} H on the coarsest level in [mu, 2]:
        // mu = 1 / max over cells of (h + horizontal couplings) / h
        const LevelHost &c = H->lev[H->L - 1];
        int nb = 0;
        KRUN(K_VEC, H->L - 1, 0, nb = launch_hz_ratio(dev<double>(c), H->partial, s));
        KRUN(K_VEC, H->L - 1, 0, launch_finalize(H->partial, nb, H->sc, S_MAX, 3, s));
        double ratio = 0;
        CHK(read_scalar(H, S_MAX, &ratio, s));
        if (!(ratio >= 1.0) || !std::isfinite(ratio))
            return fail(MG_ERR_COEFF, "coarsest level: bad Helmholtz ratio %g", ratio);
        H->cheb_mu = 1.0 / ratio;
    }
    if (H->p.mixed) {
        double big = 0;
        for (int l = 0; l < H->L; ++l) {
            const LevelHost &v = H->lev[l];
            for (const double *a : {v.tx, v.ty, v.tz, v.h}) {
                double m = 0;
                CHK(device_max(H, a, v.n, &m, s));
                big = std::max(big, m);
            }
        }
        if (!(big > 0) || !std::isfinite(big)) return fail(MG_ERR_COEFF, "bad coefficient range");
        int ex = 0;
        std::frexp(big, &ex);
        H->scale32 = std::ldexp(1.0, -ex);
        KRUN(K_VEC, 0, 0, launch_hdiag(dev<double>(H->lev[0]), H->lev[0].dh, s));
        for (int l = 0; l < H->L; ++l) {
            LevelHost &v = H->lev[l];
            KRUN(K_VEC, l, 1, launch_to_float(v.tx, v.tx32, H->scale32, v.n, s));
            KRUN(K_VEC, l, 1, launch_to_float(v.ty, v.ty32, H->scale32, v.n, s));
            KRUN(K_VEC, l, 1, launch_to_float(v.tz, v.tz32, H->scale32, v.n, s));
            KRUN(K_VEC, l, 1, launch_to_float(v.h, v.h32, H->scale32, v.n, s));
            KRUN(K_VEC, l, 1, launch_to_float(v.m, v.m32, 1.0 / H->scale32, v.n, s));
            KRUN(K_VEC, l, 1, launch_to_float(v.dq, v.dq32, 1.0, v.n, s));
        }
    }
    CU(cudaStreamSynchronize(s));
    return MG_OK;
}

int tpmg::handle_plan(const mg_grid *g, const mg_params *p, void *ws, size_t *bytes, mg_handle **out)
{
    int L = 0;
    CHK(check_grid(g, p, &L));
    mg_handle *H = new mg_handle;
    H->grid = *g;
    H->p = *p;
    H->L = L;
    build_shapes(g, p, L, H->lev);
    *bytes = carve(H, nullptr);
    if (ws) carve(H, ws);
    *out = H;
    return MG_OK;
}

int tpmg::handle_setup(mg_handle *H, const mg_coeffs *co, void *ws, size_t ws_bytes, cudaStream_t s)
{
    return setup_impl(H, co, ws, ws_bytes, s);
}

int tpmg::read_scalars(mg_handle *H, int which, double *out, cudaStream_t s)
{
    return read_scalar(H, which, out, s);
}

extern "C" int mg_setup(const mg_grid *grid, const mg_coeffs *coeffs, const mg_params *params,
                        void *workspace, size_t ws_bytes, void *stream, mg_handle **out)
{
    if (!out) return fail(MG_ERR_ARG, "null out");
    *out = nullptr;
    int L = 0;
    CHK(check_grid(grid, params, &L));
    if (!coeffs || !coeffs->tx || !coeffs->ty || !coeffs->tz || !coeffs->h)
        return fail(MG_ERR_ARG, "null coefficient pointer");
    mg_handle *H = new mg_handle;
    H->grid = *grid;
    H->p = *params;
    H->L = L;
    build_shapes(grid, params, L, H->lev);
    const int st = setup_impl(H, coeffs, workspace, ws_bytes, (cudaStream_t)stream);
    if (st != MG_OK) {
        delete H;
        return st;
    }
    *out = H;
    return MG_OK;
}

static void prof_release(mg_handle *H)
{
    for (cudaEvent_t e : H->prof.pool) cudaEventDestroy(e);
    H->prof.pool.clear();
    H->prof.recs.clear();
    H->prof.next = 0;
    H->prof.on = false;
}

static void graphs_release(mg_handle *H)
{
    for (auto &per_prec : H->vg)
        for (VGraph &g : per_prec) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.graph) cudaGraphDestroy(g.graph);
            g = VGraph{};
        }
}

extern "C" void mg_destroy(mg_handle *h)
{
    if (!h) return;
    prof_release(h);
    graphs_release(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    delete h;
}

extern "C" int mg_profile_enable(mg_handle *H, int on)
{
    if (!H) return fail(MG_ERR_ARG, "null handle");
    prof_release(H);
    if (!on) return MG_OK;
    const int n = 2 * 16384;
    H->prof.pool.reserve(n);
    for (int i = 0; i < n; ++i) {
        cudaEvent_t e;
        CU(cudaEventCreate(&e));
        H->prof.pool.push_back(e);
    }
    H->prof.on = true;
    H->prof.all_levels = on >= 2;
    return MG_OK;
}

extern "C" int mg_profile_read(mg_handle *H, int kind, int level, int prec, int *launches, double *ms)
{
    if (!H) return fail(MG_ERR_ARG, "null handle");
    const int key = prof_key(kind, level, prec);
    int cnt = 0;
    double tot = 0;
    for (const ProfRec &r : H->prof.recs) {
        if (r.key != key) continue;
        CU(cudaEventSynchronize(r.b));
        float t = 0;
        CU(cudaEventElapsedTime(&t, r.a, r.b));
        tot += t;
        ++cnt;
    }
    if (launches) *launches = cnt;
    if (ms) *ms = tot;
    return MG_OK;
}

extern "C" unsigned long long mg_launch_count(void) { return g_launches.load(); }

static int level_check(mg_handle *H, int level, int prec, bool need_coarser);

// A staged kernel that gave up waiting on its copies (tpmg_tma.cu) turns the
// solve's status into MG_ERR_TIMEOUT.
int tpmg::check_timeouts(int rc, cudaStream_t s)
{
    const int n = tma_timeouts(s, true);
    if (n > 0) return fail(MG_ERR_TIMEOUT, "%d blocks gave up waiting on their copies", n);
    if (n < 0) return fail(MG_ERR_CUDA, "reading the copy-timeout flag failed");
    return rc;
}

// ------------------------------------------------------------------ V-cycle
// Smoother sweeps from a zero guess, alternating between two buffers so that
// the last sweep writes `out`.
template <typename T>
static int smooth_from_zero(mg_handle *H, int l, const LevelDev<T> &D, const T *b, T *out,
                            T *scratch, int sweeps, double omega, cudaStream_t s)
{
    if (coarse_solve_fits(D.nlon, D.nlat, sizeof(T))) {  // all sweeps in one launch
        KRUN(K_SMOOTH0, l, prec_of<T>(),
             launch_coarse_solve<T>(D, b, out, scratch, omega, sweeps, s));
        return MG_OK;
    }
    T *cur = (sweeps % 2 == 1) ? out : scratch;
    T *oth = (cur == out) ? scratch : out;
    KRUN(K_SMOOTH0, l, prec_of<T>(), launch_smooth<T>(D, b, nullptr, cur, omega, s));
    for (int it = 1; it < sweeps; ++it) {
        KRUN(K_SMOOTH, l, prec_of<T>(), launch_smooth<T>(D, b, cur, oth, omega, s));
        std::swap(cur, oth);
    }
    return MG_OK;
}

// The coarsest-level solve as coarse_iters iterations of conjugate
// gradients from zero, preconditioned by the column solves (z = H_z^{-1} r:
// the zero-guess sweep with omega = 1), every scalar on the device (its own
// CgScalars), so the whole solve is captured in the V-cycle's graph.
// Vectors: out = x, the level's r, w = z, cd = d, cq = H d.
template <typename T>
static int coarse_pcg(mg_handle *H, int l, const LevelDev<T> &D, const T *b, T *out, cudaStream_t s)
{
    LevelHost &v = H->lev[l];
    const size_t n = v.n;
    constexpr int P = prec_of<T>();
    T *r = Vec<T>::r(v), *z = Vec<T>::w(v), *d = Vec<T>::cd(v), *q = Vec<T>::cq(v);
    CgScalars *sc = H->sc_coarse;
    if (!d || !q) return fail(MG_ERR_ARG, "PCG coarse solve without its vectors");
    CU(cudaMemsetAsync(out, 0, n * sizeof(T), s));
    KRUN(K_VEC, l, P, launch_cg_direction<T>(b, nullptr, r, n, sc, true, s));  // r = b
    KRUN(K_SMOOTH0, l, P, launch_smooth<T>(D, r, nullptr, z, 1.0, s));
    int nb = 0;
    KRUN(K_VEC, l, P, nb = launch_dot<T>(r, z, n, H->partial, s));
    KRUN(K_VEC, l, P, launch_finalize(H->partial, nb, sc, S_RZ, 0, s));
    KRUN(K_VEC, l, P, launch_cg_direction<T>(z, nullptr, d, n, sc, true, s));  // d = z
    for (int it = 0; it < H->p.coarse_iters; ++it) {
        KRUN(K_APPLY, l, P, nb = launch_stencil<T>(D, 0, nullptr, d, q, H->partial, s));
        KRUN(K_VEC, l, P, launch_finalize(H->partial, nb, sc, S_DAD, 1, s));
        KRUN(K_VEC, l, P, launch_cg_update<T>(out, r, d, q, n, sc, H->partial, s));
        if (it + 1 == H->p.coarse_iters) break;
        KRUN(K_SMOOTH0, l, P, launch_smooth<T>(D, r, nullptr, z, 1.0, s));
        KRUN(K_VEC, l, P, nb = launch_dot<T>(r, z, n, H->partial, s));
        KRUN(K_VEC, l, P, launch_finalize(H->partial, nb, sc, S_RZNEW, 2, s));
        KRUN(K_VEC, l, P, launch_cg_direction<T>(z, d, d, n, sc, false, s));
    }
    return MG_OK;
}

// The coarsest-level solve as coarse_iters Chebyshev steps from zero on the
// column-solve preconditioner (M = H_z, z = M^{-1} r the sweep from zero with
// omega = 1), on the interval [mu, 2] holding the spectrum of H_z^{-1} H (mu
// from setup): a fixed polynomial, so the V-cycle stays a fixed linear
// operator.  theta = (2 + mu) / 2, delta = (2 - mu) / 2, sigma = theta /
// delta; d_0 = z_0 / theta, rho_0 = 1 / sigma; step k: x += d_k,
// r_{k+1} = r_k - H d_k, d_{k+1} = rho_{k+1} rho_k d_k + 2 rho_{k+1} / delta
// z_{k+1}, rho_{k+1} = 1 / (2 sigma - rho_k) (scalars on the host, passed to
// the kernels).  Vectors: out = x, the level's r and cq alternate as the
// residual, w = z, cd = d.
template <typename T>
static int coarse_chebyshev(mg_handle *H, int l, const LevelDev<T> &D, const T *b, T *out,
                            cudaStream_t s)
{
    LevelHost &v = H->lev[l];
    const size_t n = v.n;
    constexpr int P = prec_of<T>();
    T *r = Vec<T>::r(v), *r2 = Vec<T>::cq(v), *z = Vec<T>::w(v), *d = Vec<T>::cd(v);
    if (!d || !r2) return fail(MG_ERR_ARG, "Chebyshev coarse solve without its vectors");
    const double mu = H->cheb_mu, lam = 2.0;
    const double theta = 0.5 * (lam + mu), delta = 0.5 * (lam - mu), sigma = theta / delta;
    const int m = H->p.coarse_iters;
    CU(cudaMemsetAsync(out, 0, n * sizeof(T), s));
    KRUN(K_SMOOTH0, l, P, launch_smooth<T>(D, b, nullptr, z, 1.0, s));  // z_0 = M^{-1} b
    KRUN(K_VEC, l, P, launch_cheb_step<T>(out, d, z, 0.0, 1.0 / theta, n, true, s));
    const T *rk = b;
    double rho = 1.0 / sigma;
    for (int k = 0; k + 1 < m; ++k) {
        T *rn = (rk == r) ? r2 : r;
        KRUN(K_RESID, l, P, launch_stencil<T>(D, 1, rk, d, rn, nullptr, s));  // r - H d
        rk = rn;
        KRUN(K_SMOOTH0, l, P, launch_smooth<T>(D, rk, nullptr, z, 1.0, s));
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        KRUN(K_VEC, l, P,
             launch_cheb_step<T>(out, d, z, rho_new * rho, 2.0 * rho_new / delta, n, false, s));
        rho = rho_new;
    }
    KRUN(K_VEC, l, P, launch_add<T>(out, d, n, s));  // the last x += d
    return MG_OK;
}

// The V-cycle's coarsest-level solve from zero (Section 2.3).
template <typename T>
static int coarse_solve(mg_handle *H, int l, const LevelDev<T> &D, const T *b, T *out, T *scratch,
                        cudaStream_t s)
{
    if (H->p.coarse_method == MG_COARSE_PCG) return coarse_pcg<T>(H, l, D, b, out, s);
    if (H->p.coarse_method == MG_COARSE_CHEBYSHEV) return coarse_chebyshev<T>(H, l, D, b, out, s);
    return smooth_from_zero<T>(H, l, D, b, out, scratch, H->p.coarse_iters, H->p.omega, s);
}

// out = V_l b (zero initial guess).  scratch, rbuf: level-l work vectors.
// dot_blocks (level 0 only, may be null): fuse <b, out> into the last sweep
// and set *dot_blocks to the number of partial sums written (0 if the cycle
// ends without a non-zero-guess sweep on this level).
template <typename T>
static int vcycle_level(mg_handle *H, int l, const T *b, T *out, T *scratch, T *rbuf, cudaStream_t s,
                        int *dot_blocks = nullptr)
{
    if (dot_blocks) *dot_blocks = 0;
    LevelHost &v = H->lev[l];
    const LevelDev<T> D = dev<T>(v);
    const double om = H->p.omega;
    if (l == H->L - 1) return coarse_solve<T>(H, l, D, b, out, scratch, s);
    const int writes = H->p.nu1 + H->p.nu2;
    T *cur = (writes % 2 == 1) ? out : scratch;
    T *oth = (cur == out) ? scratch : out;
    constexpr int P = prec_of<T>();
    KRUN(K_SMOOTH0, l, P, launch_smooth<T>(D, b, nullptr, cur, om, s));
    for (int it = 1; it < H->p.nu1; ++it) {
        KRUN(K_SMOOTH, l, P, launch_smooth<T>(D, b, cur, oth, om, s));
        std::swap(cur, oth);
    }
    LevelHost &c = H->lev[l + 1];
    // After a single sweep from zero the residual is (1 - omega) b plus the
    // horizontal couplings (both precisions); after more sweeps the full
    // stencil (FP32 fused; FP64, bound by FP64 arithmetic, in two passes).
    const bool pre = H->p.nu1 == 1;
    if (pre || sizeof(T) == 4) {
        const T *bb = b, *uu = cur;
        if (!resid_restrict_fits(b, cur, sizeof(T))) {  // a caller's unaligned vector
            if ((uintptr_t)b % (2 * sizeof(T))) {
                CU(cudaMemcpyAsync(rbuf, b, v.n * sizeof(T), cudaMemcpyDeviceToDevice, s));
                bb = rbuf;
            }
            if ((uintptr_t)cur % (2 * sizeof(T))) {  // cur is out, oth the level's scratch
                CU(cudaMemcpyAsync(oth, cur, v.n * sizeof(T), cudaMemcpyDeviceToDevice, s));
                uu = oth;
            }
        }
        KRUN(K_RESID, l, P,
             launch_resid_restrict<T>(D, v.linkdev, bb, uu, Vec<T>::b(c), s, nullptr, pre, om));
    } else {
        KRUN(K_RESID, l, P, launch_stencil<T>(D, 1, b, cur, rbuf, nullptr, s));
        KRUN(K_RESTRICT, l, P, launch_restrict<T>(D, v.linkdev, rbuf, Vec<T>::b(c), s));
    }
    CHK(vcycle_level<T>(H, l + 1, Vec<T>::b(c), Vec<T>::u(c), Vec<T>::w(c), Vec<T>::r(c), s));
    KRUN(K_PROLONG, l, P, launch_prolong_add<T>(D, v.linkdev, Vec<T>::u(c), cur, s));
    for (int it = 0; it < H->p.nu2; ++it) {
        if (dot_blocks && it + 1 == H->p.nu2) {
            int nb = 0;
            KRUN(K_SMOOTH, l, P, nb = launch_smooth_dot<T>(D, b, cur, oth, om, H->partial, s));
            *dot_blocks = nb;
        } else {
            KRUN(K_SMOOTH, l, P, launch_smooth<T>(D, b, cur, oth, om, s));
        }
        std::swap(cur, oth);
    }
    return MG_OK;
}

template <typename T>
static int vcycle_fine(mg_handle *H, const T *r, T *e, cudaStream_t s, int *dot_blocks = nullptr)
{
    LevelHost &f = H->lev[0];
    return vcycle_level<T>(H, 0, r, e, Vec<T>::w(f), Vec<T>::r(f), s, dot_blocks);
}

// out = V in for one of the solver's fixed vector pairs (slot 0: cg.r -> cg.z;
// BiCGStab: 1 p -> ph, 2 s -> sh), replayed from a CUDA graph captured on
// first use for that pair; direct launches while profiling (events around
// each kernel) or if capture is unavailable.
// dot_blocks (slot 0 only): partial sums of <in, out> left in H->partial by
// the fused last sweep (0: none, compute the inner product separately).
template <typename T>
static int vcycle_graph(mg_handle *H, int slot, const T *in, T *out, cudaStream_t s,
                        int *dot_blocks)
{
    constexpr int P = prec_of<T>();
    if (!H->use_graphs || H->prof.on) return vcycle_fine<T>(H, in, out, s, dot_blocks);
    VGraph &g = H->vg[P][slot];
    if (!g.exec) {
        g.kernels = 0;
        CU(cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeThreadLocal));
        H->capturing = true;
        H->cap_graph = &g;
        const int st = vcycle_fine<T>(H, in, out, H->cap_stream, dot_blocks ? &g.dot_blocks : nullptr);
        H->capturing = false;
        H->cap_graph = nullptr;
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(H->cap_stream, &graph);
        if (st != MG_OK || ec != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            g = VGraph{};
            H->use_graphs = false;  // run the same kernels without a graph from now on
            return vcycle_fine<T>(H, in, out, s, dot_blocks);
        }
        const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
        if (ei != cudaSuccess) {
            cudaGraphDestroy(graph);
            cudaGetLastError();
            g = VGraph{};
            H->use_graphs = false;
            return vcycle_fine<T>(H, in, out, s, dot_blocks);
        }
        g.graph = graph;
    }
    CU(cudaGraphLaunch(g.exec, s));
    if (dot_blocks) *dot_blocks = g.dot_blocks;
    g_launches.fetch_add(g.kernels, std::memory_order_relaxed);
    return MG_OK;
}

template <typename T>
static int vcycle_solver(mg_handle *H, cudaStream_t s, int *dot_blocks)
{
    CgVecs<T> &cg = Vec<T>::cg(H);
    return vcycle_graph<T>(H, 0, cg.r, cg.z, s, dot_blocks);
}

// ------------------------------------------------------------------ solvers
static bool bad(double v) { return !(v == v) || std::isinf(v); }

// rr and the breakdown flag of the BiCGStab scalars (one copy, synchronises).
static int read_bicg(mg_handle *H, double *rr, double *brk, cudaStream_t s)
{
    double v[2] = {0, 0};
    CU(cudaMemcpyAsync(v, &H->bsc->rr, sizeof v, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    *rr = v[0];
    if (brk) *brk = v[1];
    return MG_OK;
}

// The BiCGStab preconditioner, in -> out: one V-cycle (graph slot 1 or 2),
// or line_sweeps sweeps of Eq. (1) from zero on the fine level.
template <typename T>
static int bicg_precond(mg_handle *H, int slot, const T *in, T *out, cudaStream_t s)
{
    if (H->p.method == MG_METHOD_BICGSTAB) return vcycle_graph<T>(H, slot, in, out, s, nullptr);
    LevelHost &f = H->lev[0];
    return smooth_from_zero<T>(H, 0, dev<T>(f), in, out, Vec<T>::w(f), H->p.line_sweeps,
                               H->p.omega, s);
}

// BiCGStab with right preconditioning (the solver of Section 1 that the
// multigrid replaced, with the line relaxation of Eq. (1) as preconditioner,
// or with the V-cycle):
//   rho = <rh, r>;  beta = (rho / rho_old) (alpha / omega)
//   p = r + beta (p - omega v);  ph = M p;  v = H ph;  alpha = rho / <rh, v>
//   s = r - alpha v;  sh = M s;  t = H sh;  omega = <t, s> / <t, t>
//   x += alpha ph + omega sh;  r = s - omega t
// Scalars on the device; one host read per iteration (||r||, breakdown).
// Stops on the recursively updated residual and confirms with the true
// residual, restarting with a new shadow residual rh = r when they disagree
// or on a breakdown (rho or <rh, v> zero).  inner: as in solve_impl.
template <typename T>
static int solve_bicgstab(mg_handle *H, const T *b, T *x, double tol, int maxit,
                          std::vector<double> *hist, int *its_out, double *rel_out,
                          cudaStream_t s, bool inner, bool x_zero, double bb)
{
    LevelHost &f = H->lev[0];
    const LevelDev<T> D = dev<T>(f);
    const size_t n = f.n;
    CgVecs<T> &cg = Vec<T>::cg(H);
    T *r = cg.r, *rh = cg.Ad, *p = cg.d0, *ph = cg.z, *v = cg.d1;
    T *sv = cg.s, *sh = cg.sh, *t = cg.t;
    if (!sv || !sh || !t) return fail(MG_ERR_ARG, "handle built without the BiCGStab vectors");
    BicgScalars *sc = H->bsc;
    double *pa = H->partial, *pb = H->partial + kReduceSlots / 2;
    constexpr int P = prec_of<T>();
    const double bn = std::sqrt(bb);
    int its = 0;
    double rel = 0, rr0 = -1;
    auto record = [&](double rr) {
        rel = bn > 0 ? std::sqrt(rr) / bn : 0.0;
        if (hist) hist->push_back(rel);
        *its_out = its;
        *rel_out = rel;
    };
    bool first_outer = true;
    while (true) {
        double rr = 0, brk = 0;
        int nb = 0;
        if (x_zero && first_outer) {
            KRUN(K_VEC, 0, P, launch_bicg_dir<T>(r, b, nullptr, n, sc, true, s));  // r = b
        } else {
            KRUN(K_RESID, 0, P, launch_stencil<T>(D, 1, b, x, r, nullptr, s));
        }
        first_outer = false;
        KRUN(K_VEC, 0, P, nb = launch_dot<T>(r, r, n, pa, s));
        KRUN(K_VEC, 0, P, launch_bicg_finalize(pa, nullptr, nb, sc, BICG_START, s));
        CHK(read_bicg(H, &rr, nullptr, s));
        if (bad(rr)) return fail(MG_ERR_NONFINITE, "non-finite residual");
        if (rr0 < 0) rr0 = rr;
        record(rr);
        *its_out = its;
        *rel_out = rel;
        if (std::sqrt(rr) <= tol * bn) return MG_OK;
        if (its >= maxit)
            return fail(MG_ERR_NOT_CONVERGED, "not converged after %d iterations (rel %.3e)", its,
                        rel);
        if (rr > 1e6 * rr0) return fail(MG_ERR_DIVERGED, "residual grew to %.3e", rel);
        KRUN(K_VEC, 0, P, launch_bicg_dir<T>(rh, r, nullptr, n, sc, true, s));  // rh = r
        bool first = true;
        while (its < maxit) {
            ++its;
            KRUN(K_VEC, 0, P, launch_bicg_dir<T>(p, r, v, n, sc, first, s));
            first = false;
            CHK(bicg_precond<T>(H, 1, p, ph, s));
            KRUN(K_APPLY, 0, P, launch_stencil<T>(D, 0, nullptr, ph, v, nullptr, s));
            KRUN(K_VEC, 0, P, nb = launch_dot<T>(rh, v, n, pa, s));
            KRUN(K_VEC, 0, P, launch_bicg_finalize(pa, nullptr, nb, sc, BICG_ALPHA, s));
            KRUN(K_VEC, 0, P, launch_bicg_s<T>(sv, r, v, n, sc, s));
            CHK(bicg_precond<T>(H, 2, sv, sh, s));
            KRUN(K_APPLY, 0, P, launch_stencil<T>(D, 0, nullptr, sh, t, nullptr, s));
            KRUN(K_VEC, 0, P, nb = launch_dot2<T>(t, sv, n, pa, pb, s));
            KRUN(K_VEC, 0, P, launch_bicg_finalize(pa, pb, nb, sc, BICG_OMEGA, s));
            KRUN(K_VEC, 0, P,
                 nb = launch_bicg_update<T>(x, r, ph, sh, sv, t, rh, n, sc, pa, pb, s));
            KRUN(K_VEC, 0, P, launch_bicg_finalize(pa, pb, nb, sc, BICG_NEXT, s));
            CHK(read_bicg(H, &rr, &brk, s));
            if (bad(rr)) return fail(MG_ERR_NONFINITE, "non-finite residual");
            if (std::sqrt(rr) <= tol * bn || its >= maxit || brk != 0.0) {
                if (inner && brk == 0.0) {
                    record(rr);
                    *its_out = its;
                    *rel_out = rel;
                    return std::sqrt(rr) <= tol * bn ? MG_OK : MG_ERR_NOT_CONVERGED;
                }
                break;  // confirm with the true residual (restart on a breakdown)
            }
            record(rr);
            if (rr > 1e6 * rr0) return fail(MG_ERR_DIVERGED, "residual grew to %.3e", rel);
        }
    }
}

// Conjugate gradients preconditioned by one V-cycle, or the stationary
// iteration x <- x + V(b - H x) (Section 2), or BiCGStab (solve_bicgstab).
// Scalars in FP64.
// inner: the inner solve of the mixed-precision refinement: x enters as 0
// (so r = b without a stencil) and the recursively updated residual decides
// (the FP64 outer residual is the check), no confirming residual.
template <typename T>
static int solve_impl(mg_handle *H, const T *b, T *x, double tol, int maxit, int method,
                      std::vector<double> *hist, int *its_out, double *rel_out, cudaStream_t s,
                      bool inner = false, bool x_zero = false)
{
    LevelHost &f = H->lev[0];
    const LevelDev<T> D = dev<T>(f);
    const size_t n = f.n;
    CgVecs<T> &cg = Vec<T>::cg(H);
    double bb = 0;
    {
        int nb = 0;
        KRUN(K_VEC, 0, prec_of<T>(), nb = launch_dot<T>(b, b, n, H->partial, s));
        KRUN(K_VEC, 0, prec_of<T>(), launch_finalize(H->partial, nb, H->sc, S_RR, 0, s));
        CHK(read_scalar(H, S_RR, &bb, s));
    }
    if (bad(bb)) return fail(MG_ERR_NONFINITE, "non-finite right-hand side");
    if (is_bicgstab(method))
        return solve_bicgstab<T>(H, b, x, tol, maxit, hist, its_out, rel_out, s, inner,
                                 inner || x_zero, bb);
    const double bn = std::sqrt(bb);
    constexpr int P = prec_of<T>();
    int its = 0;
    double rel = 0, rr0 = -1;
    auto record = [&](double rr) {
        rel = bn > 0 ? std::sqrt(rr) / bn : 0.0;
        if (hist) hist->push_back(rel);
        *its_out = its;
        *rel_out = rel;
    };
    bool first = true;
    while (true) {
        double rr;
        if ((inner || x_zero) && first) {  // x = 0: r = b
            KRUN(K_VEC, 0, P, launch_cg_direction<T>(b, nullptr, cg.r, n, H->sc, true, s));
            rr = bb;
        } else {
            int nb = 0;
            KRUN(K_RESID, 0, P, nb = launch_stencil<T>(D, 1, b, x, cg.r, H->partial, s));
            KRUN(K_VEC, 0, P, launch_finalize(H->partial, nb, H->sc, S_RR, 0, s));
            CHK(read_scalar(H, S_RR, &rr, s));
        }
        first = false;
        if (bad(rr)) return fail(MG_ERR_NONFINITE, "non-finite residual");
        if (rr0 < 0) rr0 = rr;
        record(rr);
        *its_out = its;
        *rel_out = rel;
        if (std::sqrt(rr) <= tol * bn) return MG_OK;
        if (its >= maxit)
            return fail(MG_ERR_NOT_CONVERGED, "not converged after %d iterations (rel %.3e)", its,
                        rel);
        if (rr > 1e6 * rr0) return fail(MG_ERR_DIVERGED, "residual grew to %.3e", rel);
        int vdot = 0;
        if (method == MG_METHOD_STATIONARY) {
            CHK(vcycle_solver<T>(H, s, &vdot));
            KRUN(K_VEC, 0, P, launch_add<T>(x, cg.z, n, s));
            ++its;
            continue;
        }
        CHK(vcycle_solver<T>(H, s, &vdot));
        int nbd = vdot;
        if (!nbd) KRUN(K_VEC, 0, P, nbd = launch_dot<T>(cg.r, cg.z, n, H->partial, s));
        KRUN(K_VEC, 0, P, launch_finalize(H->partial, nbd, H->sc, S_RZ, 0, s));
        // d: current direction (none yet).  FP32: the direction update
        // d = z + beta d runs inside the apply of the next iteration (free in a
        // bandwidth-bound kernel); FP64 (ALU-bound) keeps the separate update,
        // one FMA per cell instead of five.
        constexpr bool fuse_direction = sizeof(T) == 4;
        T *d = nullptr, *dn = cg.d0;
        while (its < maxit) {
            ++its;
            int na = 0, nu = 0;
            if (fuse_direction) {
                KRUN(K_APPLY, 0, P,
                     na = launch_dir_apply<T>(D, cg.z, d, H->sc, dn, cg.Ad, H->partial, s));
            } else {
                KRUN(K_VEC, 0, P,
                     launch_cg_direction<T>(cg.z, d, dn, n, H->sc, d == nullptr, s));
                KRUN(K_APPLY, 0, P,
                     na = launch_stencil<T>(D, 0, nullptr, dn, cg.Ad, H->partial, s));
            }
            T *const fresh = dn;               // the direction just formed
            dn = (d == nullptr) ? cg.d1 : d;   // the old one's buffer takes the next
            d = fresh;
            KRUN(K_VEC, 0, P, launch_finalize(H->partial, na, H->sc, S_DAD, 1, s));
            KRUN(K_VEC, 0, P, nu = launch_cg_update<T>(x, cg.r, d, cg.Ad, n, H->sc, H->partial, s));
            KRUN(K_VEC, 0, P, launch_finalize(H->partial, nu, H->sc, S_RR, 0, s));
            CHK(read_scalar(H, S_RR, &rr, s));
            if (bad(rr)) return fail(MG_ERR_NONFINITE, "non-finite residual");
            if (std::sqrt(rr) <= tol * bn || its >= maxit) {
                if (inner) {
                    record(rr);
                    *its_out = its;
                    *rel_out = rel;
                    return std::sqrt(rr) <= tol * bn ? MG_OK : MG_ERR_NOT_CONVERGED;
                }
                break;  // confirm with the true residual
            }
            record(rr);
            if (rr > 1e6 * rr0) return fail(MG_ERR_DIVERGED, "residual grew to %.3e", rel);
            CHK(vcycle_solver<T>(H, s, &vdot));
            nbd = vdot;
            if (!nbd) KRUN(K_VEC, 0, P, nbd = launch_dot<T>(cg.r, cg.z, n, H->partial, s));
            KRUN(K_VEC, 0, P, launch_finalize(H->partial, nbd, H->sc, S_RZNEW, 2, s));
        }
    }
}

// Relative tolerance of the FP32 inner solve of a refinement step: the
// configured inner_tol, loosened to 0.3 tol / rel when that already takes the
// outer residual (now rel relative to b) below the target tol; at most 0.5.
double tpmg::inner_tolerance(double inner_tol, double tol, double rel)
{
    double t = inner_tol;
    if (rel > 0) t = std::max(t, 0.3 * tol / rel);
    return std::min(t, 0.5);
}

static void fill_stats(mg_stats *st, const std::vector<double> &hist, int its, int inner,
                       double rel)
{
    if (!st) return;
    st->iterations = its;
    st->inner_iterations = inner;
    st->rel_res = rel;
    st->history_len = 0;
    if (st->history && st->history_cap > 0) {
        const int m = std::min<int>(st->history_cap, (int)hist.size());
        std::memcpy(st->history, hist.data(), m * sizeof(double));
        st->history_len = m;
    }
}

extern "C" int mg_solve(mg_handle *H, const double *b, double *x, double tol, mg_stats *st,
                        void *stream)
{
    if (!H || !b || !x) return fail(MG_ERR_ARG, "null argument");
    if (!(tol >= 0)) return fail(MG_ERR_ARG, "tol must be >= 0");
    std::vector<double> hist;
    int its = 0;
    double rel = 0;
    double xmax = 0;
    CHK(device_max(H, x, H->lev[0].n, &xmax, (cudaStream_t)stream));
    if (bad(xmax)) return fail(MG_ERR_NONFINITE, "non-finite initial guess");
    const int rc = solve_impl<double>(H, b, x, tol, H->p.maxit, H->p.method, &hist, &its, &rel,
                                      (cudaStream_t)stream, false, xmax == 0.0);
    fill_stats(st, hist, its, 0, rel);
    return check_timeouts(rc, (cudaStream_t)stream);
}

extern "C" int mg_solve_mixed(mg_handle *H, const double *b, double *x, double tol, mg_stats *st,
                              void *stream)
{
    if (!H || !b || !x) return fail(MG_ERR_ARG, "null argument");
    if (!H->p.mixed) return fail(MG_ERR_ARG, "handle built without the FP32 hierarchy (mixed=0)");
    if (!(tol >= 0)) return fail(MG_ERR_ARG, "tol must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    LevelHost &f = H->lev[0];
    LevelDev<double> D = dev<double>(f);
    D.h = f.dh;  // the refinement residual takes the horizontal diagonal (launch_residual_cast)
    const size_t n = f.n;
    std::vector<double> hist;
    double bb = 0;
    {
        int nb = 0;
        KRUN(K_VEC, 0, 0, nb = launch_dot<double>(b, b, n, H->partial, s));
        KRUN(K_VEC, 0, 0, launch_finalize(H->partial, nb, H->sc, S_RR, 0, s));
        CHK(read_scalar(H, S_RR, &bb, s));
    }
    if (bad(bb)) return fail(MG_ERR_NONFINITE, "non-finite right-hand side");
    const double bn = std::sqrt(bb);
    // a zero initial guess makes the first residual b itself
    double xmax = 0;
    CHK(device_max(H, x, n, &xmax, s));
    if (bad(xmax)) return fail(MG_ERR_NONFINITE, "non-finite initial guess");
    const bool x_zero = xmax == 0.0;
    int outer = 0, inner = 0;
    double rel = 0, rr0 = -1;
    double pred = bn;  // expected ||b - H x|| of this step
    int rc = MG_OK;
    while (true) {
        // The FP32 right-hand side is r / sc with sc a power of two near the
        // expected ||r||: exact scaling, so the FP32 solve sees the same
        // significands for any such sc; sc is corrected when the measured
        // norm lands outside [sc 2^-10, sc 2^10].
        int ex = 0;
        std::frexp(pred > 0 ? pred : 1.0, &ex);
        double sc = std::ldexp(1.0, ex);
        double rr;
        if (x_zero && outer == 0) {
            KRUN(K_VEC, 0, 1, launch_cast_scaled(b, f.b32, 1.0 / sc, n, s));
            rr = bb;
        } else {
            int nb = 0;
            KRUN(K_RESID, 0, 0, nb = launch_residual_cast(D, b, x, f.b32, 1.0 / sc, H->partial, s));
            KRUN(K_VEC, 0, 0, launch_finalize(H->partial, nb, H->sc, S_RR, 0, s));
            CHK(read_scalar(H, S_RR, &rr, s));
            const double rn = std::sqrt(rr);
            if (!bad(rr) && rn > 0 && (rn > std::ldexp(sc, 10) || rn < std::ldexp(sc, -10))) {
                std::frexp(rn, &ex);
                sc = std::ldexp(1.0, ex);
                KRUN(K_RESID, 0, 0,
                     launch_residual_cast(D, b, x, f.b32, 1.0 / sc, H->partial, s));
            }
        }
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
        CU(cudaMemsetAsync(H->cg32.x, 0, n * sizeof(float), s));
        int its_in = 0;
        double rel_in = 0;
        // solve no further than the outer target still needs (safety 0.3)
        const double itol = inner_tolerance(H->p.inner_tol, tol, rel);
        const int rin = solve_impl<float>(H, f.b32, H->cg32.x, itol, H->p.inner_maxit,
                                          H->p.method, nullptr, &its_in, &rel_in, s, true);
        if (rin != MG_OK && rin != MG_ERR_NOT_CONVERGED && rin != MG_ERR_DIVERGED) {
            rc = rin;
            break;
        }
        inner += its_in;
        // the FP32 hierarchy holds c H: (c H) e = r / sc  =>  x += c sc e
        KRUN(K_VEC, 0, 0, launch_update_mixed(x, H->cg32.x, H->scale32 * sc, n, s));
        pred = std::sqrt(rr) * std::max(rel_in, 1e-6);
        ++outer;
    }
    fill_stats(st, hist, outer, inner, rel);
    return check_timeouts(rc, s);
}

extern "C" int mg_solve_single(mg_handle *H, const float *b, float *x, double tol, mg_stats *st,
                               void *stream)
{
    if (!H || !b || !x || b == x) return fail(MG_ERR_ARG, "bad solve buffers");
    if (!H->p.mixed) return fail(MG_ERR_ARG, "handle built without the FP32 hierarchy (mixed=0)");
    if (!(tol >= 0)) return fail(MG_ERR_ARG, "tol must be >= 0");
    LevelHost &f = H->lev[0];
    const CgVecs<float> &cg = H->cg32;
    for (const void *q : {(const void *)cg.r, (const void *)cg.z, (const void *)cg.d0,
                          (const void *)cg.d1, (const void *)cg.Ad, (const void *)cg.x,
                          (const void *)cg.s, (const void *)cg.sh, (const void *)cg.t,
                          (const void *)f.w32, (const void *)f.r32, (const void *)f.b32})
        if (q && (q == b || q == x)) return fail(MG_ERR_ARG, "buffer aliases a solver vector");
    cudaStream_t s = (cudaStream_t)stream;
    // the FP32 hierarchy holds c H: solve (c H) y = b and return x = c y
    KRUN(K_VEC, 0, 1, launch_scale<float>(x, 1.0 / H->scale32, f.n, s));
    std::vector<double> hist;
    int its = 0;
    double rel = 0;
    const int rc = solve_impl<float>(H, b, x, tol, H->p.maxit, H->p.method, &hist, &its, &rel, s);
    KRUN(K_VEC, 0, 1, launch_scale<float>(x, H->scale32, f.n, s));
    fill_stats(st, hist, its, 0, rel);
    return check_timeouts(rc, s);
}

// ------------------------------------------------------------------ C ABI: operators
extern "C" int mg_apply(mg_handle *H, const double *x, double *y, void *stream)
{
    if (!H || !x || !y) return fail(MG_ERR_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    KRUN(K_APPLY, 0, 0, launch_stencil<double>(dev<double>(H->lev[0]), 0, nullptr, x, y, nullptr, s));
    return MG_OK;
}

extern "C" int mg_vcycle(mg_handle *H, const double *r, double *e, void *stream)
{
    if (!H || !r || !e) return fail(MG_ERR_ARG, "null argument");
    return vcycle_fine<double>(H, r, e, (cudaStream_t)stream);
}

extern "C" int mg_vcycle_prec(mg_handle *H, int prec, const void *r, void *e, void *stream)
{
    CHK(level_check(H, 0, prec, false));
    if (!r || !e || r == e) return fail(MG_ERR_ARG, "bad V-cycle buffers");
    LevelHost &f = H->lev[0];
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == MG_PREC_FP64) {
        if (r == f.w || e == f.w || r == f.r || e == f.r)
            return fail(MG_ERR_ARG, "buffer aliases a level work vector");
        return vcycle_fine<double>(H, (const double *)r, (double *)e, s);
    }
    if (r == f.w32 || e == f.w32 || r == f.r32 || e == f.r32)
        return fail(MG_ERR_ARG, "buffer aliases a level work vector");
    return vcycle_fine<float>(H, (const float *)r, (float *)e, s);
}

extern "C" int mg_coeff_grad(mg_handle *H, const double *lam, const double *x, double *gh,
                             double *gtx, double *gty, double *gtz, void *stream)
{
    if (!H || !lam || !x) return fail(MG_ERR_ARG, "null argument");
    const mg_grid &g = H->grid;
    cudaStream_t s = (cudaStream_t)stream;
    KRUN(K_VEC, 0, 0, launch_coeff_grad(g.nlon, g.nlat, g.nz, lam, x, gh, gtx, gty, gtz, s));
    return MG_OK;
}

extern "C" int mg_num_levels(const mg_handle *H) { return H ? H->L : 0; }

extern "C" int mg_level_shape(const mg_handle *H, int level, int *nlon, int *nlat, int *nz)
{
    if (!H || level < 0 || level >= H->L) return fail(MG_ERR_ARG, "level out of range");
    if (nlon) *nlon = H->lev[level].nlon;
    if (nlat) *nlat = H->lev[level].nlat;
    if (nz) *nz = H->lev[level].nz;
    return MG_OK;
}

extern "C" double mg_fp32_scale(const mg_handle *H) { return H ? H->scale32 : 0.0; }

// ------------------------------------------------------------------ C ABI: precision changes
static int conv_check(const void *a, const void *b, double scale, size_t n)
{
    if (!std::isfinite(scale) || scale == 0.0) return fail(MG_ERR_ARG, "bad scale");
    if (n > 0 && (!a || !b)) return fail(MG_ERR_ARG, "null argument");
    return MG_OK;
}

static int conv_launched(cudaError_t e)
{
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return MG_OK;
}

extern "C" int mg_cast_fp32(const double *x, float *y, double scale, size_t n, void *stream)
{
    CHK(conv_check(x, y, scale, n));
    const char *xb = (const char *)x, *yb = (const char *)y;
    if (n > 0 && xb < yb + n * sizeof(float) && yb < xb + n * sizeof(double))
        return fail(MG_ERR_ARG, "x and y overlap");
    if (n == 0) return MG_OK;
    return conv_launched(launch_cast_scaled(x, y, scale, n, (cudaStream_t)stream));
}

extern "C" int mg_update_fp64(double *x, const float *e, double scale, size_t n, void *stream)
{
    CHK(conv_check(x, e, scale, n));
    if (n == 0) return MG_OK;
    return conv_launched(launch_update_mixed(x, e, scale, n, (cudaStream_t)stream));
}

extern "C" int mg_level_coeffs(mg_handle *H, int level, double *tx, double *ty, double *tz,
                               double *hh, void *stream)
{
    if (!H || level < 0 || level >= H->L) return fail(MG_ERR_ARG, "level out of range");
    cudaStream_t s = (cudaStream_t)stream;
    const LevelHost &v = H->lev[level];
    const size_t b = v.n * sizeof(double);
    if (tx) CU(cudaMemcpyAsync(tx, v.tx, b, cudaMemcpyDeviceToDevice, s));
    if (ty) CU(cudaMemcpyAsync(ty, v.ty, b, cudaMemcpyDeviceToDevice, s));
    if (tz) CU(cudaMemcpyAsync(tz, v.tz, b, cudaMemcpyDeviceToDevice, s));
    if (hh) CU(cudaMemcpyAsync(hh, v.h, b, cudaMemcpyDeviceToDevice, s));
    return MG_OK;
}

static int level_check(mg_handle *H, int level, int prec, bool need_coarser)
{
    if (!H) return fail(MG_ERR_ARG, "null handle");
    if (level < 0 || level >= H->L || (need_coarser && level + 1 >= H->L))
        return fail(MG_ERR_ARG, "level %d out of range", level);
    if (prec != MG_PREC_FP64 && prec != MG_PREC_FP32) return fail(MG_ERR_ARG, "bad precision");
    if (prec == MG_PREC_FP32 && !H->p.mixed)
        return fail(MG_ERR_ARG, "FP32 hierarchy not built (mixed=0)");
    return MG_OK;
}

template <typename T>
static int level_op(mg_handle *H, int level, int op, const void *a, const void *b, void *out,
                    cudaStream_t s)
{
    LevelHost &v = H->lev[level];
    const LevelDev<T> D = dev<T>(v);
    constexpr int P = prec_of<T>();
    switch (op) {
    case 0:
        KRUN(K_APPLY, level, P, launch_stencil<T>(D, 0, nullptr, (const T *)a, (T *)out, nullptr, s));
        return MG_OK;
    case 1:
        KRUN(K_RESID, level, P,
             launch_stencil<T>(D, 1, (const T *)a, (const T *)b, (T *)out, nullptr, s));
        return MG_OK;
    case 2:
        KRUN(b ? K_SMOOTH : K_SMOOTH0, level, P,
             launch_smooth<T>(D, (const T *)a, (const T *)b, (T *)out, H->p.omega, s));
        return MG_OK;
    case 3:
        KRUN(K_RESTRICT, level, P, launch_restrict<T>(D, v.linkdev, (const T *)a, (T *)out, s));
        return MG_OK;
    case 4:
        KRUN(K_PROLONG, level, P, launch_prolong_add<T>(D, v.linkdev, (const T *)a, (T *)out, s));
        return MG_OK;
    }
    return fail(MG_ERR_ARG, "bad op");
}

static int level_dispatch(mg_handle *H, int level, int prec, int op, const void *a, const void *b,
                          void *out, void *stream)
{
    CHK(level_check(H, level, prec, op >= 3));
    if ((op != 2 && !a) || !out || (op == 1 && !b)) return fail(MG_ERR_ARG, "null argument");
    if (op == 2 && (!a || a == out || b == out)) return fail(MG_ERR_ARG, "bad smoother buffers");
    if (prec == MG_PREC_FP64) return level_op<double>(H, level, op, a, b, out, (cudaStream_t)stream);
    return level_op<float>(H, level, op, a, b, out, (cudaStream_t)stream);
}

extern "C" int mg_level_apply(mg_handle *H, int level, int prec, const void *x, void *y,
                              void *stream)
{
    return level_dispatch(H, level, prec, 0, x, nullptr, y, stream);
}

extern "C" int mg_level_residual(mg_handle *H, int level, int prec, const void *b, const void *u,
                                 void *r, void *stream)
{
    return level_dispatch(H, level, prec, 1, b, u, r, stream);
}

extern "C" int mg_level_smooth(mg_handle *H, int level, int prec, const void *b, const void *u_in,
                               void *u_out, void *stream)
{
    return level_dispatch(H, level, prec, 2, b, u_in, u_out, stream);
}

extern "C" int mg_level_restrict(mg_handle *H, int level, int prec, const void *r, void *bc,
                                 void *stream)
{
    return level_dispatch(H, level, prec, 3, r, nullptr, bc, stream);
}

extern "C" int mg_level_prolong_add(mg_handle *H, int level, int prec, const void *ec, void *u,
                                    void *stream)
{
    return level_dispatch(H, level, prec, 4, ec, nullptr, u, stream);
}

extern "C" int mg_level_residual_restrict(mg_handle *H, int level, int prec, const void *b,
                                          const void *u, void *bc, void *stream)
{
    CHK(level_check(H, level, prec, true));
    if (!b || !u || !bc || bc == b || bc == u) return fail(MG_ERR_ARG, "bad buffers");
    cudaStream_t s = (cudaStream_t)stream;
    LevelHost &v = H->lev[level];
    const size_t vb = prec == MG_PREC_FP64 ? 8 : 4;
    if (resid_restrict_fits(b, u, vb)) {
        if (prec == MG_PREC_FP64)
            KRUN(K_RESID, level, 0,
                 launch_resid_restrict<double>(dev<double>(v), v.linkdev, (const double *)b,
                                               (const double *)u, (double *)bc, s));
        else
            KRUN(K_RESID, level, 1,
                 launch_resid_restrict<float>(dev<float>(v), v.linkdev, (const float *)b,
                                              (const float *)u, (float *)bc, s));
        return MG_OK;
    }
    // unaligned buffers: the two passes through the level's residual vector
    if (prec == MG_PREC_FP64) {
        CHK(level_op<double>(H, level, 1, b, u, Vec<double>::r(v), s));
        return level_op<double>(H, level, 3, Vec<double>::r(v), nullptr, bc, s);
    }
    CHK(level_op<float>(H, level, 1, b, u, Vec<float>::r(v), s));
    return level_op<float>(H, level, 3, Vec<float>::r(v), nullptr, bc, s);
}

template <typename T>
static int presmooth_restrict(mg_handle *H, int level, const T *b, const T *u, T *bc,
                              cudaStream_t s)
{
    LevelHost &v = H->lev[level];
    const T *bb = b, *uu = u;
    if ((uintptr_t)b % (2 * sizeof(T))) {
        CU(cudaMemcpyAsync(Vec<T>::r(v), b, v.n * sizeof(T), cudaMemcpyDeviceToDevice, s));
        bb = Vec<T>::r(v);
    }
    if ((uintptr_t)u % (2 * sizeof(T))) {
        CU(cudaMemcpyAsync(Vec<T>::w(v), u, v.n * sizeof(T), cudaMemcpyDeviceToDevice, s));
        uu = Vec<T>::w(v);
    }
    KRUN(K_RESID, level, prec_of<T>(),
         launch_resid_restrict<T>(dev<T>(v), v.linkdev, bb, uu, bc, s, nullptr, true,
                                  H->p.omega));
    return MG_OK;
}

extern "C" int mg_level_presmooth_restrict(mg_handle *H, int level, int prec, const void *b,
                                           const void *u, void *bc, void *stream)
{
    CHK(level_check(H, level, prec, true));
    if (!b || !u || !bc || bc == b || bc == u) return fail(MG_ERR_ARG, "bad buffers");
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == MG_PREC_FP64)
        return presmooth_restrict<double>(H, level, (const double *)b, (const double *)u,
                                          (double *)bc, s);
    return presmooth_restrict<float>(H, level, (const float *)b, (const float *)u, (float *)bc,
                                     s);
}

extern "C" int mg_coarse_solve(mg_handle *H, int prec, const void *b, void *out, void *stream)
{
    if (!H) return fail(MG_ERR_ARG, "null handle");
    const int l = H->L - 1;
    CHK(level_check(H, l, prec, false));
    if (!b || !out || b == out) return fail(MG_ERR_ARG, "bad coarse-solve buffers");
    cudaStream_t s = (cudaStream_t)stream;
    LevelHost &v = H->lev[l];
    if (prec == MG_PREC_FP64) {
        const void *own[] = {Vec<double>::w(v), Vec<double>::r(v), Vec<double>::cd(v),
                             Vec<double>::cq(v)};
        for (const void *p : own)
            if (p && (p == b || p == out)) return fail(MG_ERR_ARG, "buffer aliases a work vector");
        return coarse_solve<double>(H, l, dev<double>(v), (const double *)b, (double *)out,
                                    Vec<double>::w(v), s);
    }
    const void *own[] = {Vec<float>::w(v), Vec<float>::r(v), Vec<float>::cd(v), Vec<float>::cq(v)};
    for (const void *p : own)
        if (p && (p == b || p == out)) return fail(MG_ERR_ARG, "buffer aliases a work vector");
    return coarse_solve<float>(H, l, dev<float>(v), (const float *)b, (float *)out,
                               Vec<float>::w(v), s);
}

extern "C" int mg_level_relax(mg_handle *H, int level, int prec, int sweeps, const void *b,
                              void *out, void *stream)
{
    CHK(level_check(H, level, prec, false));
    if (!b || !out || b == out) return fail(MG_ERR_ARG, "bad relaxation buffers");
    if (sweeps < 1 || sweeps > 1000) return fail(MG_ERR_ARG, "sweeps outside 1..1000");
    cudaStream_t s = (cudaStream_t)stream;
    LevelHost &v = H->lev[level];
    if (prec == MG_PREC_FP64) {
        if (out == Vec<double>::w(v) || b == Vec<double>::w(v))
            return fail(MG_ERR_ARG, "buffer aliases the level scratch");
        return smooth_from_zero<double>(H, level, dev<double>(v), (const double *)b,
                                        (double *)out, Vec<double>::w(v), sweeps, H->p.omega, s);
    }
    if (out == Vec<float>::w(v) || b == Vec<float>::w(v))
        return fail(MG_ERR_ARG, "buffer aliases the level scratch");
    return smooth_from_zero<float>(H, level, dev<float>(v), (const float *)b, (float *)out,
                                   Vec<float>::w(v), sweeps, H->p.omega, s);
}

template <typename T>
static int level_dir_apply(mg_handle *H, int level, const T *z, const T *d_old, double beta,
                           T *d_new, T *q, double *dot, cudaStream_t s)
{
    LevelHost &v = H->lev[level];
    CU(cudaMemcpyAsync(&H->sc->beta, &beta, sizeof beta, cudaMemcpyHostToDevice, s));
    int nb = 0;
    KRUN(K_APPLY, level, prec_of<T>(),
         nb = launch_dir_apply<T>(dev<T>(v), z, d_old, H->sc, d_new, q, H->partial, s));
    KRUN(K_VEC, level, prec_of<T>(), launch_finalize(H->partial, nb, H->sc, S_DAD, 0, s));
    return read_scalar(H, S_DAD, dot, s);  // also keeps beta alive until its copy ran
}

extern "C" int mg_level_dir_apply(mg_handle *H, int level, int prec, const void *z,
                                  const void *d_old, double beta, void *d_new, void *q,
                                  double *dot, void *stream)
{
    CHK(level_check(H, level, prec, false));
    if (!z || !d_new || !q || !dot || d_new == z || d_new == d_old || q == z || q == d_old ||
        q == d_new)
        return fail(MG_ERR_ARG, "bad direction-update buffers");
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == MG_PREC_FP64)
        return level_dir_apply<double>(H, level, (const double *)z, (const double *)d_old, beta,
                                       (double *)d_new, (double *)q, dot, s);
    return level_dir_apply<float>(H, level, (const float *)z, (const float *)d_old, beta,
                                  (float *)d_new, (float *)q, dot, s);
}

extern "C" int mg_level_smooth_dot(mg_handle *H, int level, int prec, const void *b,
                                   const void *u_in, void *u_out, double *dot, void *stream)
{
    CHK(level_check(H, level, prec, false));
    if (!b || !u_in || !u_out || !dot || u_in == u_out || b == u_out)
        return fail(MG_ERR_ARG, "bad smoother buffers");
    cudaStream_t s = (cudaStream_t)stream;
    LevelHost &v = H->lev[level];
    int nb = 0;
    if (prec == MG_PREC_FP64) {
        KRUN(K_SMOOTH, level, 0, nb = launch_smooth_dot<double>(dev<double>(v), (const double *)b,
                                                            (const double *)u_in,
                                                            (double *)u_out, H->p.omega,
                                                            H->partial, s));
    } else {
        KRUN(K_SMOOTH, level, 1, nb = launch_smooth_dot<float>(dev<float>(v), (const float *)b,
                                                           (const float *)u_in, (float *)u_out,
                                                           H->p.omega, H->partial, s));
    }
    KRUN(K_VEC, level, prec, launch_finalize(H->partial, nb, H->sc, S_RZ, 0, s));
    return read_scalar(H, S_RZ, dot, s);
}
