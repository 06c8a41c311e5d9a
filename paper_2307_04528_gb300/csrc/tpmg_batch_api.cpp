// Batched ensemble of independent systems of uneven sizes (C ABI mg_batch_*).
//
// Each system gets an ordinary handle (its own hierarchy, carved from the
// batch workspace).  On top of them the batch builds, once at setup:
//   * a level-synchronous program of the V-cycle: the steps of every
//     system's V-cycle (Section 2, Fig. 1) grouped into phases (down level
//     0, 1, ..., the coarsest, up ..., 0); within a phase the k-th operation
//     of every participating system forms one batched step, issued as ONE
//     persistent-kernel launch over a work list of (system level, tile);
//   * work lists for the fine-level vector operations of the conjugate-
//     gradient iteration, with per-system reductions;
//   * one CUDA graph per precision replaying the whole batched V-cycle.
// An autotuner times the candidate column-tile widths and persistent grid
// sizes on the batch itself and keeps the fastest.  Systems that converge
// are switched off through device-side activity flags, so the graph never
// changes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/tpmg.h"
#include "tpmg_handle.h"
#include "tpmg_internal.h"

using namespace tpmg;

namespace {

enum { BK_SMOOTH0 = 0, BK_SMOOTH = 1, BK_RESID = 2, BK_RESTRICT = 3, BK_PROLONG = 4,
       BK_SMOOTH_DOT = 5, BK_RESID_RESTRICT = 6, BK_COARSE = 7, BK_KINDS = 8 };

template <typename T>
struct StepHost {
    int kind;
    std::vector<BOp<T>> ops;
    std::vector<BItem> items;  // work list of the small operators (tuned tile width)
    std::vector<int> big;      // operators launched on their own (large levels)
    std::vector<int> base;     // first partial sum of each big operator
    std::vector<int> off;      // per-system partial-sum ranges: begin [0, n), end [n, 2n)
    BOp<T> *ops_dev = nullptr;
    BItem *items_dev = nullptr;
    int *off_dev = nullptr;
};

template <typename T>
struct VecPlan {            // one fine-level vector operation over all systems
    std::vector<BVec<T>> v;
    std::vector<BItem> items;
    std::vector<int> off;     // per-system item ranges (n+1)
    BVec<T> *v_dev = nullptr;
    BItem *items_dev = nullptr;
    int *off_dev = nullptr;
};

template <typename T>
struct RedPlan {            // fine-level stencil with per-system reduction
    std::vector<BOp<T>> ops;
    std::vector<BItem> items;  // column tiles of the small systems
    std::vector<int> big;      // systems launched on their own (large levels)
    std::vector<int> base;     // first partial sum of each big system
    std::vector<int> off;      // per-system partial-sum ranges: begin [0, n), end [n, 2n)
    BOp<T> *ops_dev = nullptr;
    BItem *items_dev = nullptr;
    int *off_dev = nullptr;
};

template <typename T>
struct PrecPlan {
    std::vector<StepHost<T>> vsteps;   // batched V-cycle: cg.r -> cg.z of every system
    VecPlan<T> dot_rz, dot_bb, update[2], dir[2], dir0, add, rcopy, xmax;
    RedPlan<T> resid;                  // r = b - H x (+ |r|^2), fixed b and x
    RedPlan<T> apply[2];               // Ad = H d (+ d.Ad), d = d0 / d1
    RedPlan<T> dirapply0, dirapply[2]; // d = z (+ beta d_old) and Ad = H d (+ d.Ad)
    VGraph graph;
};

// FP64 residual -> scaled FP32 right-hand side, one descriptor per system.
struct ResidPlan {
    std::vector<BResid32> ops;
    std::vector<BItem> items;
    std::vector<int> off;
    BResid32 *ops_dev = nullptr;
    BItem *items_dev = nullptr;
    int *off_dev = nullptr;
};

struct Bump {
    char *base;
    size_t off = 0;
    explicit Bump(void *b) : base((char *)b) {}
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T) + 1;
        return p;
    }
};

}  // namespace

struct mg_batch {
    int n = 0;
    mg_params p{};
    std::vector<mg_grid> grids;
    std::vector<mg_handle *> h;
    std::vector<size_t> ws_off;
    int nzmax = 1;
    // tuned launch shapes
    int smooth_block = kBlock, smooth_grid = 0, cell_grid = 0, vec_grid = 0;
    int sm_count = 0;
    // device extras
    CgScalars *sc = nullptr;          // [n]
    int *active = nullptr;            // [n]
    double *partial = nullptr;        // [max items]
    double *sdata = nullptr;          // [n] per-system scale factors
    size_t partial_cap = 0;
    PrecPlan<double> p64;
    PrecPlan<float> p32;
    // FP64 <-> FP32 transfers of the mixed solve (x: the caller's, set per call)
    std::vector<BMix> mix, mixb;       // mixb: cast of the caller's b (zero initial guess)
    std::vector<BItem> mix_items;
    BMix *mix_dev = nullptr, *mixb_dev = nullptr;
    BItem *mix_items_dev = nullptr;
    ResidPlan resid32;
    cudaStream_t cap_stream = nullptr;
};

namespace {

size_t vec_chunk(const mg_batch *B)
{
    size_t total = 0;
    for (const mg_grid &g : B->grids) total += (size_t)g.nlon * g.nlat * g.nz;
    size_t c = (total + kVecItems - 1) / kVecItems;
    c = (c + kBlock - 1) / kBlock * kBlock;
    return c < (size_t)kVecChunkMin ? (size_t)kVecChunkMin : c;
}

template <typename T>
PrecPlan<T> &plan_of(mg_batch *B);
template <>
PrecPlan<double> &plan_of<double>(mg_batch *B) { return B->p64; }
template <>
PrecPlan<float> &plan_of<float>(mg_batch *B) { return B->p32; }

// ------------------------------------------------------------------ V-cycle program
// One operation of one system's V-cycle, with its concrete vectors.
template <typename T>
struct SysOp {
    int kind;
    BOp<T> op;
};

// Levels with at least this many columns run the single-system kernels, one
// launch per operator (their own grid fills the GPU, and their kernel
// parameters live in the constant bank instead of registers); the smaller
// ones share the persistent work-list launch.
constexpr long long kBigColumns = 1LL << 18;

// Layers per work item of the cell-type steps: the residual walks whole
// columns where a level has enough of them (as the single-system path), and
// the transfers take up to 16 layers per thread on large levels.
template <typename T>
int layers_per_item(int kind, const LevelDev<T> &L, const LinkDev &K)
{
    const long long ncol = (long long)L.nlon * L.nlat;
    if (kind == BK_RESID) return ncol >= 32768 ? L.nz : 1;
    if (kind != BK_RESTRICT && kind != BK_PROLONG) return L.nz;
    const long long cols = kind == BK_RESTRICT ? (long long)(L.nlon / 2) * K.nlat_c
                                               : (long long)(L.nlon / 2) * L.nlat;
    if (cols >= 65536) return std::min(L.nz, 16);
    if (cols >= 16384) return std::min(L.nz, 4);
    return 1;
}

// The V-cycle of handle H as phases: phase l (down, 0 <= l < L) and phase
// 2 Lmax - 2 - l (up), exactly in the order vcycle_level issues them.
template <typename T>
void gen_level(mg_handle *H, int sys, int l, int Lmax, const T *b, T *out, T *scratch, T *rbuf,
               std::map<int, std::vector<std::vector<SysOp<T>>>> &phases, int nsys)
{
    LevelHost &v = H->lev[l];
    const LevelDev<T> D = dev<T>(v);
    auto push = [&](int phase, int kind, const T *a, const T *x, T *y, const LevelDev<T> &L,
                    const LinkDev &K) {
        auto &per = phases[phase];
        if (per.empty()) per.resize(nsys);
        BOp<T> op{};
        op.L = L;
        op.K = K;
        op.a = a;
        op.x = x;
        op.y = y;
        op.sys = sys;
        op.kz = layers_per_item(kind, L, K);
        per[sys].push_back({kind, op});
    };
    const LinkDev nolink{};
    const int down = l, up = 2 * Lmax - 2 - l;
    if (l == H->L - 1) {
        const int sweeps = H->p.coarse_iters;
        if (sizeof(T) == 4 && coarse_sh_fits(D.nlon * D.nlat, D.nz, sizeof(T))) {
            // all sweeps in one block per system, the level in shared memory
            push(down, BK_COARSE, b, nullptr, out, D, nolink);
            return;
        }
        T *cur = (sweeps % 2 == 1) ? out : scratch;
        T *oth = (cur == out) ? scratch : out;
        push(down, BK_SMOOTH0, b, nullptr, cur, D, nolink);
        for (int it = 1; it < sweeps; ++it) {
            push(down, BK_SMOOTH, b, cur, oth, D, nolink);
            std::swap(cur, oth);
        }
        return;
    }
    const int writes = H->p.nu1 + H->p.nu2;
    T *cur = (writes % 2 == 1) ? out : scratch;
    T *oth = (cur == out) ? scratch : out;
    push(down, BK_SMOOTH0, b, nullptr, cur, D, nolink);
    for (int it = 1; it < H->p.nu1; ++it) {
        push(down, BK_SMOOTH, b, cur, oth, D, nolink);
        std::swap(cur, oth);
    }
    LevelHost &c = H->lev[l + 1];
    if ((H->p.nu1 == 1 || sizeof(T) == 4) && resid_restrict_fits(b, cur, sizeof(T))) {
        // the fused pass as in the single-system V-cycle (the single-system
        // kernel on large levels, the work list on the others)
        push(down, BK_RESID_RESTRICT, b, cur, Vec<T>::b(c), D, v.linkdev);
    } else {
        push(down, BK_RESID, b, cur, rbuf, D, nolink);
        push(down, BK_RESTRICT, rbuf, nullptr, Vec<T>::b(c), D, v.linkdev);
    }
    gen_level<T>(H, sys, l + 1, Lmax, Vec<T>::b(c), Vec<T>::u(c), Vec<T>::w(c), Vec<T>::r(c),
                 phases, nsys);
    push(up, BK_PROLONG, Vec<T>::u(c), nullptr, cur, D, v.linkdev);
    for (int it = 0; it < H->p.nu2; ++it) {
        // the last sweep of the finest level also forms <r, z> of the CG
        const int kind = (l == 0 && it + 1 == H->p.nu2) ? BK_SMOOTH_DOT : BK_SMOOTH;
        push(up, kind, b, cur, oth, D, nolink);
        std::swap(cur, oth);
    }
}

int cdiv(long long a, int b) { return (int)((a + b - 1) / b); }

// Elements per vector work item for the batch (fixed by the sizes alone).
size_t vec_chunk(const mg_batch *B);

// Tiles of a participant for its step kind (block = column tile width of smoothers).
template <typename T>
int tiles_of(int kind, const BOp<T> &op, int block, int *nblk)
{
    const int ncol = op.L.nlon * op.L.nlat;
    switch (kind) {
    case BK_SMOOTH0:
    case BK_SMOOTH:
    case BK_SMOOTH_DOT:
        *nblk = cdiv(ncol, block);
        return *nblk;
    case BK_RESID:
        *nblk = cdiv(ncol, kBlock);
        return *nblk * cdiv(op.L.nz, op.kz);
    case BK_RESTRICT:
        *nblk = cdiv((long long)(op.L.nlon / 2) * op.K.nlat_c, kBlock);
        return *nblk * cdiv(op.L.nz, op.kz);
    case BK_RESID_RESTRICT: {  // warp blocks along longitude x layers x bands
        const int warps = cdiv(op.L.nlon / 2, kRROwned);
        *nblk = cdiv((long long)warps * 32, kBlock);
        return *nblk * op.L.nz * cdiv(op.K.nlat_c, kRRBand);
    }
    case BK_COARSE:  // one block per system, launched on its own
        *nblk = 0;
        return 0;
    default:
        *nblk = cdiv((long long)(op.L.nlon / 2) * op.L.nlat, kBlock);
        return *nblk * cdiv(op.L.nz, op.kz);
    }
}


template <typename T>
bool is_big(const BOp<T> &op)
{
    return (long long)op.L.nlon * op.L.nlat >= kBigColumns;
}

// Work list of the small operators, the big ones, and the partial-sum ranges:
// items first (partial[item]), then each big operator's blocks.
template <typename T>
void build_items(StepHost<T> &st, int block, int nsys)
{
    st.items.clear();
    st.big.clear();
    st.base.clear();
    st.off.assign(2 * nsys, 0);
    for (int i = 0; i < (int)st.ops.size(); ++i) {
        int nblk = 0;
        const int nt = tiles_of<T>(st.kind, st.ops[i], block, &nblk);
        st.ops[i].nblk = nblk;
        if (is_big(st.ops[i])) {
            st.big.push_back(i);
            continue;
        }
        const int s0 = (int)st.items.size();
        for (int t = 0; t < nt; ++t) st.items.push_back({i, t});
        st.off[st.ops[i].sys] = s0;
        st.off[nsys + st.ops[i].sys] = (int)st.items.size();
    }
    int next = (int)st.items.size();
    for (int i : st.big) {
        const BOp<T> &op = st.ops[i];
        const int grid = cdiv((long long)op.L.nlon * op.L.nlat, kBlock);
        st.base.push_back(next);
        st.off[op.sys] = next;
        st.off[nsys + op.sys] = next + grid;
        next += grid;
    }
}

template <typename T>
void build_program(mg_batch *B)
{
    PrecPlan<T> &P = plan_of<T>(B);
    int Lmax = 0;
    for (auto *H : B->h) Lmax = std::max(Lmax, H->L);
    std::map<int, std::vector<std::vector<SysOp<T>>>> phases;
    for (int s = 0; s < B->n; ++s) {
        mg_handle *H = B->h[s];
        LevelHost &f = H->lev[0];
        CgVecs<T> &cg = Vec<T>::cg(H);
        gen_level<T>(H, s, 0, Lmax, cg.r, cg.z, Vec<T>::w(f), Vec<T>::r(f), phases, B->n);
    }
    P.vsteps.clear();
    for (auto &ph : phases) {
        size_t slots = 0;
        for (auto &lst : ph.second) slots = std::max(slots, lst.size());
        for (size_t q = 0; q < slots; ++q) {
            for (int kind = 0; kind < BK_KINDS; ++kind) {
                StepHost<T> st;
                st.kind = kind;
                for (auto &lst : ph.second)
                    if (q < lst.size() && lst[q].kind == kind) st.ops.push_back(lst[q].op);
                if (!st.ops.empty()) P.vsteps.push_back(std::move(st));
            }
        }
    }
    for (auto &st : P.vsteps) build_items(st, B->smooth_block, B->n);
}

// Vector plan: one descriptor per system, items = chunks, grouped by system.
template <typename T>
void vec_plan(mg_batch *B, VecPlan<T> &V, T *(*a)(mg_handle *), T *(*b)(mg_handle *),
              T *(*c)(mg_handle *), T *(*d)(mg_handle *))
{
    V.v.clear();
    V.items.clear();
    V.off.assign(1, 0);
    for (int s = 0; s < B->n; ++s) {
        mg_handle *H = B->h[s];
        BVec<T> e{};
        e.a = a ? a(H) : nullptr;
        e.b = b ? b(H) : nullptr;
        e.c = c ? c(H) : nullptr;
        e.d = d ? d(H) : nullptr;
        e.n = H->lev[0].n;
        e.chunk = vec_chunk(B);
        e.sys = s;
        e.nchunk = (int)((e.n + e.chunk - 1) / e.chunk);
        V.v.push_back(e);
        for (int t = 0; t < e.nchunk; ++t) V.items.push_back({s, t});
        V.off.push_back((int)V.items.size());
    }
}

template <typename T>
void red_plan(mg_batch *B, RedPlan<T> &R, const T *(*a)(mg_handle *), const T *(*x)(mg_handle *),
              T *(*y)(mg_handle *), T *(*w)(mg_handle *) = nullptr, bool split = false)
{
    R.ops.clear();
    R.items.clear();
    R.big.clear();
    R.base.clear();
    R.off.assign(2 * B->n, 0);
    for (int s = 0; s < B->n; ++s) {
        mg_handle *H = B->h[s];
        BOp<T> op{};
        op.L = dev<T>(H->lev[0]);
        op.a = a ? a(H) : nullptr;
        op.x = x ? x(H) : nullptr;
        op.y = y(H);
        op.w = w ? w(H) : nullptr;
        op.kz = op.L.nz;
        op.sys = s;
        op.nblk = cdiv((long long)op.L.nlon * op.L.nlat, kBlock);
        R.ops.push_back(op);
        if (split && is_big(op)) {
            R.big.push_back(s);
            continue;
        }
        R.off[s] = (int)R.items.size();
        for (int t = 0; t < op.nblk; ++t) R.items.push_back({s, t});
        R.off[B->n + s] = (int)R.items.size();
    }
    int next = (int)R.items.size();
    for (int s : R.big) {
        // split plans run the direction update + apply: its own partial sums
        const BOp<T> &op = R.ops[s];
        const int nb = dir_apply_partials<T>(op.L, op.a, op.x, op.y, op.w);
        R.base.push_back(next);
        R.off[s] = next;
        R.off[B->n + s] = next + nb;
        next += nb;
    }
}

// Right-hand side and solution of a batched solve: the caller's FP64 arrays
// (set per call), or the fixed FP32 buffers of the inner solve.
template <typename T>
T *bx_of(mg_handle *H);
template <>
double *bx_of<double>(mg_handle *H) { return (double *)H->batch_b; }
template <>
float *bx_of<float>(mg_handle *H) { return H->lev[0].b32; }
template <typename T>
T *xx_of(mg_handle *H);
template <>
double *xx_of<double>(mg_handle *H) { return (double *)H->batch_x; }
template <>
float *xx_of<float>(mg_handle *H) { return H->cg32.x; }

template <typename T>
void build_vector_plans(mg_batch *B)
{
    PrecPlan<T> &P = plan_of<T>(B);
    auto r = [](mg_handle *H) { return Vec<T>::cg(H).r; };
    auto z = [](mg_handle *H) { return Vec<T>::cg(H).z; };
    auto d0 = [](mg_handle *H) { return Vec<T>::cg(H).d0; };
    auto d1 = [](mg_handle *H) { return Vec<T>::cg(H).d1; };
    auto Ad = [](mg_handle *H) { return Vec<T>::cg(H).Ad; };
    auto bx = [](mg_handle *H) { return bx_of<T>(H); };
    auto xx = [](mg_handle *H) { return xx_of<T>(H); };
    vec_plan<T>(B, P.dot_rz, r, z, nullptr, nullptr);
    vec_plan<T>(B, P.dot_bb, bx, bx, nullptr, nullptr);
    vec_plan<T>(B, P.update[0], xx, r, d0, Ad);
    vec_plan<T>(B, P.update[1], xx, r, d1, Ad);
    vec_plan<T>(B, P.dir[0], d1, z, d0, nullptr);   // d1 = z + beta d0
    vec_plan<T>(B, P.dir[1], d0, z, d1, nullptr);   // d0 = z + beta d1
    vec_plan<T>(B, P.dir0, d0, z, nullptr, nullptr);
    vec_plan<T>(B, P.add, xx, z, nullptr, nullptr);
    red_plan<T>(B, P.resid, [](mg_handle *H) -> const T * { return bx_of<T>(H); },
                [](mg_handle *H) -> const T * { return xx_of<T>(H); }, r);
    red_plan<T>(B, P.apply[0], nullptr, [](mg_handle *H) -> const T * { return Vec<T>::cg(H).d0; },
                Ad);
    red_plan<T>(B, P.apply[1], nullptr, [](mg_handle *H) -> const T * { return Vec<T>::cg(H).d1; },
                Ad);
    vec_plan<T>(B, P.rcopy, r, bx, nullptr, nullptr);  // r = b (inner solves start at x = 0)
    vec_plan<T>(B, P.xmax, xx, nullptr, nullptr, nullptr);
    // direction update + apply: d0 = z; d1 = z + beta d0; d0 = z + beta d1
    auto zc = [](mg_handle *H) -> const T * { return Vec<T>::cg(H).z; };
    auto d0c = [](mg_handle *H) -> const T * { return Vec<T>::cg(H).d0; };
    auto d1c = [](mg_handle *H) -> const T * { return Vec<T>::cg(H).d1; };
    red_plan<T>(B, P.dirapply0, zc, nullptr, d0, Ad, true);
    red_plan<T>(B, P.dirapply[0], zc, d0c, d1, Ad, true);
    red_plan<T>(B, P.dirapply[1], zc, d1c, d0, Ad, true);
}

void resid_plan(mg_batch *B)
{
    ResidPlan &R = B->resid32;
    R.ops.clear();
    R.items.clear();
    R.off.assign(1, 0);
    for (int s = 0; s < B->n; ++s) {
        mg_handle *H = B->h[s];
        BResid32 op{};
        op.L = dev<double>(H->lev[0]);
        op.b = (const double *)H->batch_b;
        op.x = (const double *)H->batch_x;
        op.r32 = H->lev[0].b32;
        op.sys = s;
        op.nblk = cdiv((long long)op.L.nlon * op.L.nlat, kBlock);
        R.ops.push_back(op);
        for (int t = 0; t < op.nblk; ++t) R.items.push_back({s, t});
        R.off.push_back((int)R.items.size());
    }
}

}  // namespace

// ------------------------------------------------------------------ device layout
namespace {

// Device copies of the plans: carved from the batch tail of the workspace.
struct Tail {
    Bump bump;
    explicit Tail(void *base) : bump(base) {}
};

template <typename T>
void carve_step(Bump &b, StepHost<T> &st, size_t item_cap)
{
    st.ops_dev = b.take<BOp<T>>(st.ops.size());
    st.items_dev = b.take<BItem>(item_cap);
    st.off_dev = b.take<int>(st.off.size());
}

template <typename T>
void carve_vec(Bump &b, VecPlan<T> &V)
{
    V.v_dev = b.take<BVec<T>>(V.v.size());
    V.items_dev = b.take<BItem>(V.items.size());
    V.off_dev = b.take<int>(V.off.size());
}

template <typename T>
void carve_red(Bump &b, RedPlan<T> &R)
{
    R.ops_dev = b.take<BOp<T>>(R.ops.size());
    R.items_dev = b.take<BItem>(R.items.size());
    R.off_dev = b.take<int>(R.off.size());
}

// Items a step can have at the smallest tile width the tuner tries.
template <typename T>
size_t item_cap(const StepHost<T> &st)
{
    size_t n = 0;
    for (const auto &op : st.ops) {
        int nblk = 0;
        n += tiles_of<T>(st.kind, op, 64, &nblk);
    }
    return n;
}

template <typename T>
void carve_plan(Bump &b, PrecPlan<T> &P, size_t *max_items)
{
    for (auto &st : P.vsteps) {
        const size_t cap = item_cap(st);
        carve_step(b, st, cap);
        *max_items = std::max(*max_items, cap);
        for (int o : st.off) *max_items = std::max(*max_items, (size_t)o);  // big ranges
    }
    for (VecPlan<T> *V : {&P.dot_rz, &P.dot_bb, &P.update[0], &P.update[1], &P.dir[0], &P.dir[1],
                          &P.dir0, &P.add, &P.rcopy, &P.xmax}) {
        carve_vec(b, *V);
        *max_items = std::max(*max_items, V->items.size());
    }
    for (RedPlan<T> *R : {&P.resid, &P.apply[0], &P.apply[1], &P.dirapply0, &P.dirapply[0],
                          &P.dirapply[1]}) {
        carve_red(b, *R);
        *max_items = std::max(*max_items, R->items.size());
        for (int o : R->off) *max_items = std::max(*max_items, (size_t)o);  // big ranges
    }
}

template <typename V>
int up(const std::vector<V> &h, void *d, cudaStream_t s)
{
    if (h.empty()) return MG_OK;
    CU(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice, s));
    return MG_OK;
}

template <typename T>
int upload_step(StepHost<T> &st, cudaStream_t s)
{
    CHK(up(st.ops, st.ops_dev, s));
    CHK(up(st.items, st.items_dev, s));
    CHK(up(st.off, st.off_dev, s));
    return MG_OK;
}

template <typename T>
int upload_vec(VecPlan<T> &V, cudaStream_t s)
{
    CHK(up(V.v, V.v_dev, s));
    CHK(up(V.items, V.items_dev, s));
    CHK(up(V.off, V.off_dev, s));
    return MG_OK;
}

template <typename T>
int upload_red(RedPlan<T> &R, cudaStream_t s)
{
    CHK(up(R.ops, R.ops_dev, s));
    CHK(up(R.items, R.items_dev, s));
    CHK(up(R.off, R.off_dev, s));
    return MG_OK;
}

template <typename T>
int upload_plan(PrecPlan<T> &P, cudaStream_t s)
{
    for (auto &st : P.vsteps) CHK(upload_step(st, s));
    for (VecPlan<T> *V : {&P.dot_rz, &P.dot_bb, &P.update[0], &P.update[1], &P.dir[0], &P.dir[1],
                          &P.dir0, &P.add, &P.rcopy, &P.xmax})
        CHK(upload_vec(*V, s));
    for (RedPlan<T> *R : {&P.resid, &P.apply[0], &P.apply[1], &P.dirapply0, &P.dirapply[0],
                          &P.dirapply[1]})
        CHK(upload_red(*R, s));
    return MG_OK;
}

}  // namespace

// ------------------------------------------------------------------ layout / setup
// Lay out the batch in `base` (nullptr: sizes only): every system's handle,
// then the batch's scalars, flags, partial sums and plan arrays.
static int batch_layout(mg_batch *B, void *base, size_t *total)
{
    Bump b(base);
    for (int s = 0; s < B->n; ++s) {
        b.off = (b.off + 255) & ~(size_t)255;
        B->ws_off[s] = b.off;
        size_t bytes = 0;
        mg_handle *H = nullptr;
        CHK(handle_plan(&B->grids[s], &B->p, base ? (char *)base + b.off : nullptr, &bytes, &H));
        if (B->h[s]) mg_destroy(B->h[s]);
        B->h[s] = H;
        b.off += bytes;
    }
    build_program<double>(B);
    build_vector_plans<double>(B);
    if (B->p.mixed) {
        build_program<float>(B);
        build_vector_plans<float>(B);
    }
    B->sc = b.take<CgScalars>(B->n);
    B->active = b.take<int>(B->n);
    B->sdata = b.take<double>(2 * B->n);
    if (B->p.mixed) {
        B->mix.clear();
        B->mix_items.clear();
        for (int i = 0; i < B->n; ++i) {
            mg_handle *H = B->h[i];
            BMix m{};
            m.r = H->cg64.r;
            m.r32 = H->lev[0].b32;
            m.e32 = H->cg32.x;
            m.n = H->lev[0].n;
            m.chunk = vec_chunk(B);
            m.sys = i;
            m.nchunk = (int)((m.n + m.chunk - 1) / m.chunk);
            B->mix.push_back(m);
            for (int t = 0; t < m.nchunk; ++t) B->mix_items.push_back({i, t});
        }
        B->mixb = B->mix;
        B->mix_dev = b.take<BMix>(B->mix.size());
        B->mixb_dev = b.take<BMix>(B->mixb.size());
        B->mix_items_dev = b.take<BItem>(B->mix_items.size());
        resid_plan(B);
        ResidPlan &R = B->resid32;
        R.ops_dev = b.take<BResid32>(R.ops.size());
        R.items_dev = b.take<BItem>(R.items.size());
        R.off_dev = b.take<int>(R.off.size());
    }
    size_t max_items = B->p.mixed ? B->resid32.items.size() : 0;
    carve_plan<double>(b, B->p64, &max_items);
    if (B->p.mixed) carve_plan<float>(b, B->p32, &max_items);
    B->partial_cap = max_items;
    B->partial = b.take<double>(max_items);
    *total = b.off + 256;
    return MG_OK;
}

static mg_batch *batch_new(int n, const mg_grid *grids, const mg_params *params)
{
    mg_batch *B = new mg_batch;
    B->n = n;
    B->p = *params;
    B->grids.assign(grids, grids + n);
    B->h.assign(n, nullptr);
    B->ws_off.assign(n, 0);
    for (int s = 0; s < n; ++s) B->nzmax = std::max(B->nzmax, grids[s].nz);
    return B;
}

static void batch_free(mg_batch *B)
{
    if (!B) return;
    for (VGraph *g : {&B->p64.graph, &B->p32.graph}) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
    }
    for (mg_handle *H : B->h)
        if (H) mg_destroy(H);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
    delete B;
}

// ------------------------------------------------------------------ batched execution
template <typename T>
static int run_vstep(mg_batch *B, StepHost<T> &st, cudaStream_t s)
{
    const int ni = (int)st.items.size();
    cudaError_t e = cudaSuccess;
    switch (st.kind) {
    case BK_SMOOTH0:
    case BK_SMOOTH: {
        const int grid = std::min(ni, B->smooth_grid);
        e = launch_bsmooth<T>(st.ops_dev, st.items_dev, ni, st.kind == BK_SMOOTH0, B->p.omega,
                              B->active, grid, B->smooth_block, B->nzmax, s);
        break;
    }
    case BK_SMOOTH_DOT: {
        const int grid = std::min(ni, B->smooth_grid);
        e = launch_bsmooth_dot<T>(st.ops_dev, st.items_dev, ni, B->p.omega, B->active, grid,
                                  B->smooth_block, B->nzmax, B->partial, s);
        break;
    }
    case BK_RESID_RESTRICT: {
        const int grid = ni;  // the launcher clamps to occupancy
        e = launch_bcells<T>(B->p.nu1 == 1 ? 4 : 3, st.ops_dev, st.items_dev, ni, B->active,
                             grid, s, B->p.omega);
        break;
    }
    case BK_COARSE: {
        size_t smem = 0;
        for (const BOp<T> &op : st.ops)
            smem = std::max(smem, coarse_sh_bytes(op.L.nlon * op.L.nlat, op.L.nz, sizeof(T)));
        e = launch_bcoarse_solve<T>(st.ops_dev, (int)st.ops.size(), B->p.omega,
                                    B->p.coarse_iters, B->active, smem, s);
        if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
        break;
    }
    default: {
        // as many blocks as the GPU holds (the launcher clamps to occupancy)
        const int grid = ni;
        const int kind = st.kind == BK_RESID ? 0 : (st.kind == BK_RESTRICT ? 1 : 2);
        e = launch_bcells<T>(kind, st.ops_dev, st.items_dev, ni, B->active, grid, s);
    }
    }
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, "batched step: %s", cudaGetErrorString(e));
    g_launches.fetch_add(ni > 0 ? 1 : 0, std::memory_order_relaxed);
    for (size_t q = 0; q < st.big.size(); ++q) {
        const BOp<T> &op = st.ops[st.big[q]];
        const int *flag = B->active + op.sys;
        switch (st.kind) {
        case BK_SMOOTH0: e = launch_smooth<T>(op.L, op.a, nullptr, op.y, B->p.omega, s, flag); break;
        case BK_SMOOTH: e = launch_smooth<T>(op.L, op.a, op.x, op.y, B->p.omega, s, flag); break;
        case BK_SMOOTH_DOT:
            launch_smooth_dot<T>(op.L, op.a, op.x, op.y, B->p.omega, B->partial + st.base[q], s,
                                 flag);
            e = cudaGetLastError();
            break;
        case BK_RESID:
            launch_stencil<T>(op.L, 1, op.a, op.x, op.y, nullptr, s, flag);
            e = cudaGetLastError();
            break;
        case BK_RESTRICT: e = launch_restrict<T>(op.L, op.K, op.a, op.y, s, flag); break;
        case BK_RESID_RESTRICT:
            e = launch_resid_restrict<T>(op.L, op.K, op.a, op.x, op.y, s, flag, B->p.nu1 == 1,
                                         B->p.omega);
            break;
        default: e = launch_prolong_add<T>(op.L, op.K, op.a, op.y, s, flag); break;
        }
        if (e != cudaSuccess) return fail(MG_ERR_CUDA, "batched step: %s", cudaGetErrorString(e));
        g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    return MG_OK;
}

template <typename T>
static int vcycle_direct(mg_batch *B, cudaStream_t s)
{
    for (auto &st : plan_of<T>(B).vsteps) CHK(run_vstep<T>(B, st, s));
    return MG_OK;
}

// The batched V-cycle (every active system: cg.r -> cg.z), replayed from a
// CUDA graph captured on first use.
template <typename T>
static int vcycle_batch(mg_batch *B, cudaStream_t s)
{
    PrecPlan<T> &P = plan_of<T>(B);
    VGraph &g = P.graph;
    if (!g.exec) {
        CU(cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int st = vcycle_direct<T>(B, B->cap_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(B->cap_stream, &graph);
        if (st != MG_OK || ec != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return st != MG_OK ? st : fail(MG_ERR_CUDA, "graph capture failed");
        }
        CU(cudaGraphInstantiate(&g.exec, graph, 0));
        g.graph = graph;
        g.kernels = P.vsteps.size();
        g_launches.fetch_sub(g.kernels, std::memory_order_relaxed);  // captured, not launched
    }
    CU(cudaGraphLaunch(g.exec, s));
    g_launches.fetch_add(g.kernels, std::memory_order_relaxed);
    return MG_OK;
}

template <typename T>
static int vec_op(mg_batch *B, int op, VecPlan<T> &V, cudaStream_t s)
{
    const int ni = (int)V.items.size();
    CU(launch_bvec<T>(op, V.v_dev, V.items_dev, ni, B->sc, B->partial, B->active, ni, s));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return MG_OK;
}

// Per-system sums of the partials: contiguous ranges off[s] .. off[s+1], or
// with end != nullptr explicit ranges off[s] .. end[s].
static int finalize(mg_batch *B, const int *off, int which, int op, cudaStream_t s,
                    const int *end = nullptr)
{
    CU(launch_bfinalize(B->partial, off, end ? end : off + 1, B->n, B->sc, which, op, B->active,
                        s));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return MG_OK;
}

template <typename T>
static int red_op(mg_batch *B, int mode, RedPlan<T> &R, cudaStream_t s)
{
    const int ni = (int)R.items.size();
    CU(launch_bstencil_red<T>(mode, R.ops_dev, R.items_dev, ni, B->partial, B->active, ni, s));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return MG_OK;
}

static int set_active(mg_batch *B, const std::vector<int> &act, cudaStream_t s)
{
    CU(cudaMemcpyAsync(B->active, act.data(), act.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    return MG_OK;
}

static int read_slot(mg_batch *B, int which, std::vector<double> &out, cudaStream_t s)
{
    std::vector<CgScalars> h(B->n);
    CU(cudaMemcpyAsync(h.data(), B->sc, B->n * sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    out.resize(B->n);
    for (int i = 0; i < B->n; ++i) out[i] = reinterpret_cast<const double *>(&h[i])[which];
    return MG_OK;
}

static bool bad(double v) { return !(v == v) || std::isinf(v); }

template <typename T>
static int dir_apply_op(mg_batch *B, bool first, RedPlan<T> &R, cudaStream_t s)
{
    const int ni = (int)R.items.size();
    if (ni > 0) {
        CU(launch_bdir_apply<T>(first, R.ops_dev, R.items_dev, ni, B->sc, B->partial, B->active,
                                ni, s));
        g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    for (size_t q = 0; q < R.big.size(); ++q) {
        const BOp<T> &op = R.ops[R.big[q]];
        launch_dir_apply<T>(op.L, op.a, first ? nullptr : op.x, B->sc + op.sys, op.y, op.w,
                            B->partial + R.base[q], s, B->active + op.sys);
        CU(cudaGetLastError());
        g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    return MG_OK;
}

// The CG iterations proper for the systems flagged in cgact (r holds their
// residual): z = V r, then direction, apply, update until each system's
// recursive residual meets tol, reaches maxit or grows by 1e6.  FP32 forms
// the direction inside the apply (bandwidth-bound); FP64 (ALU-bound) keeps
// the separate direction update.
template <typename T>
static int cg_iterations(mg_batch *B, std::vector<int> &cgact, const std::vector<double> &bb,
                         const std::vector<double> &rr0, const std::vector<double> &tol,
                         int maxit, std::vector<int> &its, std::vector<double> &rr,
                         cudaStream_t s)
{
    PrecPlan<T> &P = plan_of<T>(B);
    const int n = B->n;
    constexpr bool fuse_direction = sizeof(T) == 4;
    // <r, z> comes from the last sweep of the batched V-cycle when it has one
    const StepHost<T> *dotstep = nullptr;
    for (const auto &st : P.vsteps)
        if (st.kind == BK_SMOOTH_DOT) dotstep = &st;
    auto rz = [&](int which, int op) -> int {
        if (dotstep) return finalize(B, dotstep->off_dev, which, op, s, dotstep->off_dev + n);
        CHK(vec_op<T>(B, BV_DOT, P.dot_rz, s));
        return finalize(B, P.dot_rz.off_dev, which, op, s);
    };
    CHK(set_active(B, cgact, s));
    CHK(vcycle_batch<T>(B, s));
    CHK(rz(S_RZ, 0));
    int par = -1;  // current direction: none yet, d0 (0) or d1 (1)
    while (true) {
        if (fuse_direction) {
            RedPlan<T> &R = par < 0 ? P.dirapply0 : P.dirapply[par];
            CHK(dir_apply_op<T>(B, par < 0, R, s));
            CHK(finalize(B, R.off_dev, S_DAD, 1, s, R.off_dev + n));
        } else {
            if (par < 0) CHK(vec_op<T>(B, BV_DIR0, P.dir0, s));
            else CHK(vec_op<T>(B, BV_DIR, P.dir[par], s));
            RedPlan<T> &R = P.apply[par < 0 ? 0 : par ^ 1];
            CHK(red_op<T>(B, 0, R, s));
            CHK(finalize(B, R.off_dev, S_DAD, 1, s, R.off_dev + n));
        }
        par = par < 0 ? 0 : par ^ 1;
        CHK(vec_op<T>(B, BV_UPDATE, P.update[par], s));
        CHK(finalize(B, P.update[par].off_dev, S_RR, 0, s));
        CHK(read_slot(B, S_RR, rr, s));
        int running = 0;
        for (int i = 0; i < n; ++i) {
            if (!cgact[i]) continue;
            ++its[i];
            const double bn = std::sqrt(bb[i]);
            if (bad(rr[i]) || std::sqrt(rr[i]) <= tol[i] * bn || its[i] >= maxit ||
                rr[i] > 1e6 * rr0[i])
                cgact[i] = 0;
            else
                ++running;
        }
        if (!running) return MG_OK;
        CHK(set_active(B, cgact, s));
        CHK(vcycle_batch<T>(B, s));
        CHK(rz(S_RZNEW, 2));
    }
}

// V-cycle-preconditioned CG for every system in `want` (1 = solve), in lock
// step; each system stops on its own tolerance.  b/x: bx_of / xx_of.
// status[s], its[s], rel[s] per system.  inner: x = 0 on entry, so r = b, and
// the recursive residual decides (the FP32 solve of a refinement step);
// otherwise every exit is confirmed on the true residual (restarting CG).
template <typename T>
static int batch_cg(mg_batch *B, const std::vector<int> &want, const std::vector<double> &tol,
                    int maxit, std::vector<int> &status, std::vector<int> &its,
                    std::vector<double> &rel, cudaStream_t s, bool inner = false)
{
    PrecPlan<T> &P = plan_of<T>(B);
    const int n = B->n;
    std::vector<int> act = want;
    status.assign(n, MG_OK);
    its.assign(n, 0);
    rel.assign(n, 0.0);
    std::vector<double> bb, rr, rr0(n, -1.0);
    CHK(set_active(B, act, s));
    CHK(vec_op<T>(B, BV_DOT, P.dot_bb, s));
    CHK(finalize(B, P.dot_bb.off_dev, S_RR, 0, s));
    CHK(read_slot(B, S_RR, bb, s));
    for (int i = 0; i < n; ++i)
        if (act[i] && bad(bb[i])) {
            status[i] = MG_ERR_NONFINITE;
            act[i] = 0;
        }
    if (inner) {
        CHK(set_active(B, act, s));
        CHK(vec_op<T>(B, BV_DIR0, P.rcopy, s));
        int left = 0;
        for (int i = 0; i < n; ++i) {
            if (!act[i]) continue;
            rr0[i] = bb[i];
            if (bb[i] == 0.0) act[i] = 0;  // x = 0 solves it
            else ++left;
        }
        std::vector<int> cgact = act;
        if (left) CHK(cg_iterations<T>(B, cgact, bb, rr0, tol, maxit, its, rr, s));
        for (int i = 0; i < n; ++i) {
            if (!act[i]) continue;
            const double bn = std::sqrt(bb[i]);
            rel[i] = std::sqrt(rr[i]) / bn;
            status[i] = bad(rr[i]) ? MG_ERR_NONFINITE
                                   : (std::sqrt(rr[i]) <= tol[i] * bn ? MG_OK
                                                                      : MG_ERR_NOT_CONVERGED);
        }
        return MG_OK;
    }
    for (int restart = 0; restart < 4; ++restart) {
        // true residual of every system still wanted
        CHK(set_active(B, act, s));
        CHK(red_op<T>(B, 1, P.resid, s));
        CHK(finalize(B, P.resid.off_dev, S_RR, 0, s, P.resid.off_dev + n));
        CHK(read_slot(B, S_RR, rr, s));
        int left = 0;
        for (int i = 0; i < n; ++i) {
            if (!act[i]) continue;
            const double bn = std::sqrt(bb[i]);
            rel[i] = bn > 0 ? std::sqrt(rr[i]) / bn : 0.0;
            if (bad(rr[i])) {
                status[i] = MG_ERR_NONFINITE;
                act[i] = 0;
            } else if (std::sqrt(rr[i]) <= tol[i] * bn) {
                status[i] = MG_OK;
                act[i] = 0;
            } else if (its[i] >= maxit) {
                status[i] = MG_ERR_NOT_CONVERGED;
                act[i] = 0;
            } else {
                if (rr0[i] < 0) rr0[i] = rr[i];
                ++left;
            }
        }
        if (!left) break;
        std::vector<int> cgact = act;
        CHK(cg_iterations<T>(B, cgact, bb, rr0, tol, maxit, its, rr, s));
    }
    for (int i = 0; i < n; ++i)
        if (act[i]) status[i] = MG_ERR_NOT_CONVERGED;
    return MG_OK;
}

template <typename T>
static int refresh_bx_plans(mg_batch *B, cudaStream_t s)
{
    PrecPlan<T> &P = plan_of<T>(B);
    build_vector_plans<T>(B);
    for (VecPlan<T> *V : {&P.dot_bb, &P.update[0], &P.update[1], &P.add, &P.rcopy, &P.xmax})
        CHK(up(V->v, V->v_dev, s));
    CHK(up(P.resid.ops, P.resid.ops_dev, s));
    return MG_OK;
}

// ------------------------------------------------------------------ autotuner
// Times the fine-level batched smoother for each column-tile width and
// persistent grid size, and the cell-parallel steps for each grid size, on
// the batch's own data; keeps the fastest.
template <typename T>
static int autotune(mg_batch *B, cudaStream_t s)
{
    PrecPlan<T> &P = plan_of<T>(B);
    int devi = 0;
    CU(cudaGetDevice(&devi));
    CU(cudaDeviceGetAttribute(&B->sm_count, cudaDevAttrMultiProcessorCount, devi));
    const int sms = B->sm_count;
    B->vec_grid = sms * 8;
    std::vector<int> all(B->n, 1);
    CHK(set_active(B, all, s));
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    auto time_it = [&](auto &&fn) -> double {
        fn();
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r) fn();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    // the fine-level non-zero-guess smoother step (the largest one)
    StepHost<T> *sm = nullptr;
    for (auto &st : P.vsteps)
        if ((st.kind == BK_SMOOTH || st.kind == BK_SMOOTH_DOT) &&
            (!sm || st.items.size() > sm->items.size()))
            sm = &st;
    double best = 1e30;
    int best_b = kBlock, best_g = sms * 4;
    for (int block : {64, 128}) {
        if (sm) {
            build_items(*sm, block, B->n);
            CHK(upload_step(*sm, s));
        }
        for (int per_sm : {2, 4, 6, 8, 12}) {
            if ((size_t)block * per_sm > 1024) continue;
            B->smooth_block = block;
            B->smooth_grid = sms * per_sm;
            if (!sm) break;
            const double ms = time_it([&] { run_vstep<T>(B, *sm, s); });
            if (ms < best) {
                best = ms;
                best_b = block;
                best_g = B->smooth_grid;
            }
        }
    }
    B->smooth_block = best_b;
    B->smooth_grid = best_g;
    // cell-type steps and vector operations run on resident persistent grids
    // (sized by occupancy in their launchers); reported for reference
    B->cell_grid = sms * 8;

    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CU(cudaGetLastError());
    return MG_OK;
}

template <typename T>
static int rebuild_items(mg_batch *B, cudaStream_t s)
{
    PrecPlan<T> &P = plan_of<T>(B);
    for (auto &st : P.vsteps) {
        build_items(st, B->smooth_block, B->n);
        CHK(upload_step(st, s));
    }
    return MG_OK;
}

// ------------------------------------------------------------------ C ABI
extern "C" int mg_batch_workspace_bytes(int n, const mg_grid *grids, const mg_params *params,
                                        size_t *bytes)
{
    if (n < 1 || !grids || !params || !bytes) return fail(MG_ERR_ARG, "bad batch arguments");
    if (params->levels < 0)
        return fail(MG_ERR_ARG, "batched solves take a fixed number of levels");
    if (params->coarse_method != MG_COARSE_JACOBI)
        return fail(MG_ERR_ARG, "batched solves take the block-Jacobi coarsest-level solve");
    if (params->method != MG_METHOD_CG && params->method != MG_METHOD_STATIONARY)
        return fail(MG_ERR_ARG, "batched solves take conjugate gradients or the stationary "
                                "iteration");
    mg_batch *B = batch_new(n, grids, params);
    size_t total = 0;
    const int st = batch_layout(B, nullptr, &total);
    batch_free(B);
    if (st == MG_OK) *bytes = total;
    return st;
}

extern "C" int mg_batch_setup(int n, const mg_grid *grids, const mg_coeffs *coeffs,
                              const mg_params *params, void *workspace, size_t ws_bytes,
                              void *stream, mg_batch **out)
{
    if (!out) return fail(MG_ERR_ARG, "null out");
    *out = nullptr;
    if (n < 1 || !grids || !coeffs || !params) return fail(MG_ERR_ARG, "bad batch arguments");
    if (params->levels < 0)
        return fail(MG_ERR_ARG, "batched solves take a fixed number of levels");
    if (params->coarse_method != MG_COARSE_JACOBI)
        return fail(MG_ERR_ARG, "batched solves take the block-Jacobi coarsest-level solve");
    if (params->method != MG_METHOD_CG && params->method != MG_METHOD_STATIONARY)
        return fail(MG_ERR_ARG, "batched solves take conjugate gradients or the stationary "
                                "iteration");
    if (!workspace || (uintptr_t)workspace % 256)
        return fail(MG_ERR_WORKSPACE, "workspace null or not 256-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    mg_batch *B = batch_new(n, grids, params);
    auto bail = [&](int st) {
        batch_free(B);
        return st;
    };
    size_t total = 0;
    int st = batch_layout(B, nullptr, &total);
    if (st != MG_OK) return bail(st);
    if (ws_bytes < total)
        return bail(fail(MG_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, total));
    st = batch_layout(B, workspace, &total);
    if (st != MG_OK) return bail(st);
    for (int i = 0; i < n; ++i) {
        size_t bytes = 0;
        mg_handle *tmp = nullptr;
        st = handle_plan(&grids[i], params, nullptr, &bytes, &tmp);
        if (tmp) mg_destroy(tmp);
        if (st == MG_OK)
            st = handle_setup(B->h[i], &coeffs[i], (char *)workspace + B->ws_off[i], bytes, s);
        if (st != MG_OK) return bail(st);
    }
    cudaError_t e = bsmooth_prepare();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(fail(MG_ERR_CUDA, "%s", cudaGetErrorString(e)));
    CgScalars zero{};
    std::vector<CgScalars> zs(n, zero);
    if ((st = up(zs, B->sc, s)) != MG_OK) return bail(st);
    // the FP64 plans reference the caller's b and x per solve; start from the
    // handles' own residual vectors so every descriptor is valid
    for (mg_handle *H : B->h) {
        H->batch_b = H->cg64.r;
        H->batch_x = H->cg64.z;
    }
    build_vector_plans<double>(B);
    if ((st = upload_plan<double>(B->p64, s)) != MG_OK) return bail(st);
    if (B->p.mixed && (st = upload_plan<float>(B->p32, s)) != MG_OK) return bail(st);
    if (B->p.mixed) st = autotune<float>(B, s);
    else st = autotune<double>(B, s);
    if (st != MG_OK) return bail(st);
    if ((st = rebuild_items<double>(B, s)) != MG_OK) return bail(st);
    if (B->p.mixed && (st = rebuild_items<float>(B, s)) != MG_OK) return bail(st);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bail(fail(MG_ERR_CUDA, "%s", cudaGetErrorString(e)));
    *out = B;
    return MG_OK;
}

extern "C" void mg_batch_destroy(mg_batch *B) { batch_free(B); }

extern "C" int mg_batch_handle(mg_batch *B, int i, mg_handle **out)
{
    if (!B || !out || i < 0 || i >= B->n) return fail(MG_ERR_ARG, "bad system index");
    *out = B->h[i];
    return MG_OK;
}

extern "C" int mg_batch_tuning(const mg_batch *B, int *smooth_block, int *smooth_grid,
                               int *cell_grid, int *vec_grid)
{
    if (!B) return fail(MG_ERR_ARG, "null batch");
    if (smooth_block) *smooth_block = B->smooth_block;
    if (smooth_grid) *smooth_grid = B->smooth_grid;
    if (cell_grid) *cell_grid = B->cell_grid;
    if (vec_grid) *vec_grid = B->vec_grid;
    return MG_OK;
}

static void batch_stats(mg_stats *st, int i, int its, int inner, double rel)
{
    if (!st) return;
    st[i].iterations = its;
    st[i].inner_iterations = inner;
    st[i].rel_res = rel;
    st[i].history_len = 0;
}

extern "C" int mg_batch_solve(mg_batch *B, const double *const *b, double *const *x, double tol,
                              int mixed, mg_stats *stats, int *status, void *stream)
{
    if (!B || !b || !x || !(tol >= 0)) return fail(MG_ERR_ARG, "bad batch solve arguments");
    for (int i = 0; i < B->n; ++i)
        if (!b[i] || !x[i]) return fail(MG_ERR_ARG, "null field of system %d", i);
    if (mixed && !B->p.mixed) return fail(MG_ERR_ARG, "batch built without the FP32 hierarchy");
    cudaStream_t s = (cudaStream_t)stream;
    const int n = B->n;
    for (int i = 0; i < n; ++i) {
        B->h[i]->batch_b = b[i];
        B->h[i]->batch_x = x[i];
    }
    CHK(refresh_bx_plans<double>(B, s));
    std::vector<int> st(n, MG_OK), its, its_in(n, 0);
    std::vector<double> rel;
    if (!mixed) {
        std::vector<int> want(n, 1);
        CHK(batch_cg<double>(B, want, std::vector<double>(n, tol), B->p.maxit, st, its, rel, s));
        for (int i = 0; i < n; ++i) batch_stats(stats, i, its[i], 0, rel[i]);
    } else {
        // FP64 refinement in lock step; the inner FP32 solves run batched.
        // Each step writes the FP64 residual directly as the FP32 right-hand
        // side r / s_i with s_i a power of two near the expected ||r_i||
        // (exact scaling), corrected when the measured norm is outside
        // [s_i 2^-10, s_i 2^10]; a zero initial guess makes the first
        // residual b itself.
        PrecPlan<double> &P = B->p64;
        ResidPlan &R = B->resid32;
        std::vector<int> act(n, 1), outer(n, 0), xzero(n, 0);
        std::vector<double> bb, rr, xm, relv(n, 0.0), rr0(n, -1.0), sd(2 * n, 0.0), pred(n);
        for (int i = 0; i < n; ++i) {
            B->mix[i].x = x[i];
            B->mixb[i].r = b[i];
        }
        CHK(up(B->mix, B->mix_dev, s));
        CHK(up(B->mixb, B->mixb_dev, s));
        CHK(up(B->mix_items, B->mix_items_dev, s));
        resid_plan(B);
        CHK(up(R.ops, R.ops_dev, s));
        CHK(up(R.items, R.items_dev, s));
        CHK(up(R.off, R.off_dev, s));
        const int nmix = (int)B->mix_items.size();
        const int nres = (int)R.items.size();
        CHK(set_active(B, act, s));
        CHK(vec_op<double>(B, BV_DOT, P.dot_bb, s));
        CHK(finalize(B, P.dot_bb.off_dev, S_RR, 0, s));
        CHK(read_slot(B, S_RR, bb, s));
        CHK(vec_op<double>(B, BV_MAXABS, P.xmax, s));
        CHK(finalize(B, P.xmax.off_dev, S_MAX, 3, s));
        CHK(read_slot(B, S_MAX, xm, s));
        for (int i = 0; i < n; ++i) {
            pred[i] = std::sqrt(bb[i]);
            xzero[i] = xm[i] == 0.0;
            if (bad(bb[i]) || bad(xm[i])) {
                st[i] = MG_ERR_NONFINITE;
                act[i] = 0;
            }
        }
        auto scale_of = [](double v) {
            int ex = 0;
            std::frexp(v > 0 ? v : 1.0, &ex);
            return std::ldexp(1.0, ex);
        };
        // FP64 residual -> FP32 right-hand side of the systems in `which`
        auto residual_cast = [&](const std::vector<int> &which) -> int {
            bool narrow = true;
            for (int i = 0; i < n; ++i)
                if (which[i] && !(sd[i] >= 0x1p-100 && sd[i] <= 0x1p60)) narrow = false;
            CHK(set_active(B, which, s));
            CU(launch_bresid_cast(narrow, R.ops_dev, R.items_dev, nres, B->sdata, B->partial,
                                  B->active, nres, s));
            g_launches.fetch_add(1, std::memory_order_relaxed);
            return MG_OK;
        };
        while (true) {
            std::vector<int> from_b(n, 0), stencil(n, 0);
            int nb = 0, ns = 0;
            for (int i = 0; i < n; ++i) {
                if (!act[i]) continue;
                const double sc = scale_of(pred[i]);
                sd[i] = 1.0 / sc;                    // cast factor
                sd[n + i] = B->h[i]->scale32 * sc;   // update factor
                if (xzero[i] && outer[i] == 0) from_b[i] = 1, ++nb;
                else stencil[i] = 1, ++ns;
            }
            CHK(up(sd, B->sdata, s));
            rr.assign(n, 0.0);
            if (nb) {
                CHK(set_active(B, from_b, s));
                CU(launch_bmix(0, B->mixb_dev, B->mix_items_dev, nmix, B->sdata, B->active, nmix,
                               s));
                g_launches.fetch_add(1, std::memory_order_relaxed);
                for (int i = 0; i < n; ++i)
                    if (from_b[i]) rr[i] = bb[i];
            }
            if (ns) {
                CHK(residual_cast(stencil));
                CHK(finalize(B, R.off_dev, S_RR, 0, s));
                std::vector<double> rs;
                CHK(read_slot(B, S_RR, rs, s));
                std::vector<int> redo(n, 0);
                int nredo = 0;
                for (int i = 0; i < n; ++i) {
                    if (!stencil[i]) continue;
                    rr[i] = rs[i];
                    const double rn = std::sqrt(rs[i]), sc = 1.0 / sd[i];
                    if (!bad(rs[i]) && rn > 0 &&
                        (rn > std::ldexp(sc, 10) || rn < std::ldexp(sc, -10))) {
                        const double sc2 = scale_of(rn);
                        sd[i] = 1.0 / sc2;
                        sd[n + i] = B->h[i]->scale32 * sc2;
                        redo[i] = 1;
                        ++nredo;
                    }
                }
                if (nredo) {
                    CHK(up(sd, B->sdata, s));
                    CHK(residual_cast(redo));
                }
            }
            int left = 0;
            for (int i = 0; i < n; ++i) {
                if (!act[i]) continue;
                const double bn = std::sqrt(bb[i]);
                relv[i] = bn > 0 ? std::sqrt(rr[i]) / bn : 0.0;
                if (rr0[i] < 0) rr0[i] = rr[i];
                if (bad(rr[i])) { st[i] = MG_ERR_NONFINITE; act[i] = 0; }
                else if (std::sqrt(rr[i]) <= tol * bn) { st[i] = MG_OK; act[i] = 0; }
                else if (outer[i] >= B->p.maxit) { st[i] = MG_ERR_NOT_CONVERGED; act[i] = 0; }
                else if (rr[i] > 1e6 * rr0[i]) { st[i] = MG_ERR_DIVERGED; act[i] = 0; }
                else ++left;
            }
            if (!left) break;
            for (int i = 0; i < n; ++i)
                if (act[i])
                    CU(cudaMemsetAsync(B->h[i]->cg32.x, 0, B->h[i]->lev[0].n * sizeof(float), s));
            std::vector<int> ist, iits;
            std::vector<double> irel;
            // each system's inner tolerance (the rule of the single-system solve)
            std::vector<double> itol(n, 0.5);
            for (int i = 0; i < n; ++i)
                if (act[i]) itol[i] = inner_tolerance(B->p.inner_tol, tol, relv[i]);
            CHK(batch_cg<float>(B, act, itol, B->p.inner_maxit, ist, iits, irel, s, true));
            for (int i = 0; i < n; ++i) {
                if (!act[i]) continue;
                if (ist[i] == MG_ERR_NONFINITE) { st[i] = MG_ERR_NONFINITE; act[i] = 0; continue; }
                its_in[i] += iits[i];
                ++outer[i];
                pred[i] = std::sqrt(rr[i]) * std::max(irel[i], 1e-6);
            }
            CHK(set_active(B, act, s));
            CU(launch_bmix(1, B->mix_dev, B->mix_items_dev, nmix, B->sdata + n, B->active, nmix,
                           s));
            g_launches.fetch_add(1, std::memory_order_relaxed);
        }
        for (int i = 0; i < n; ++i) batch_stats(stats, i, outer[i], its_in[i], relv[i]);
    }
    int first = MG_OK;
    for (int i = 0; i < n; ++i) {
        if (status) status[i] = st[i];
        if (first == MG_OK && st[i] != MG_OK) first = st[i];
    }
    if (first != MG_OK) return fail(first, "%d system(s) did not converge", (int)std::count_if(st.begin(), st.end(), [](int v) { return v != MG_OK; }));
    return check_timeouts(MG_OK, s);
}
