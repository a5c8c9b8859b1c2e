// capi.cu -- the C ABI of include/gb3fmm.h: the context, its device workspace, and
// the order of the phases of one evaluation (the call stack of Sec. 2.2.2 and the
// phases of Table 2: tree, estimate, up, walk, down).
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "kernels.cuh"
#include "serve.cuh"

namespace gb3 {
extern thread_local char g_cuda_msg[256];
}
using namespace gb3;

namespace {

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

int ensure(Buf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return 0;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    size_t want = bytes + bytes / 4 + 256;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&b.p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            snprintf(g_cuda_msg, sizeof g_cuda_msg, "cudaMalloc of %zu bytes failed", bytes);
            return FMM_E_OOM;
        }
        want = bytes;
    }
    b.bytes = want;
    return 0;
}
void release(Buf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}
template <class T>
T* P(Buf& b) {
    return (T*)b.p;
}

enum { EV_START, EV_TREE, EV_EST, EV_UP, EV_WALK, EV_M2L, EV_P2P, EV_DOWN, EV_END, EV_M2LK0, EV_M2LK1, EV_P2PK0, EV_P2PK1,
       EV_JOINED, EV_N };

}  // namespace

struct fmm_ctx {
    fmm_params prm;
    int device = 0;
    char err[512] = {0};
    fmm_stats last;
    // host-API staging
    Buf hx, hmu, hpsi, hacc;
    // particles and sort
    Buf bounds, status, counters, coin, dtotal;
    Buf keys, keys_alt, idx, idx_alt, rtmp, xm, perm, xp;
    // cells
    Buf first, count, child, nchild, parent, level, sr, cr, mass, minscale;
    Buf split_nchild, split_oct, split_offs, scan_tmp, leaves, leaf_flag, leaf_pos, rad_tmp, owner;
    // expansions
    Buf M, F, Pw, binom, pascal, M1, F1, Ff;
    // walk
    Buf walkf;  // single-precision view of the cells for the walk's acceptance test
    Buf units;  // int[2]: the working units of the tree in use (launch_work_units)
    Buf front0, front1, m2l, p2p, sort_tmp, sort_tmp2, m2l_tmp, p2p_tmp, seg_start, seg_end, est_m2l, est_p2p,
        m2l_seg_start, m2l_seg_end;
    long long front_cap = 0, m2l_cap = 0, p2p_cap = 0, est_m2l_cap = 0, est_p2p_cap = 0;
    // per particle results (sorted order)
    Buf psi_far, acc_far, psi_near, acc_near, scale_sorted;
    unsigned long long* h_counters = nullptr;  // pinned, 16 words: the walk [0, 8), the P2P plan [8, 14)
    int* h_int = nullptr;                      // pinned
    cudaEvent_t ev[EV_N];
    bool ev_ok = false;
    // three streams of the context: s2 (lowest priority) and s_hi, s3 (highest).  The upward
    // pass runs on s2 beside the scale estimate on s_hi (which waits on the host between its
    // kernels), whose M2L branch (list sort, M2L) runs on s3 beside its P2P branch; later the
    // P2P runs on s2 beside the M2L and the downward pass on s_hi.  Events fork them from and
    // join them to the caller's stream.
    cudaStream_t s2 = nullptr, s_hi = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join_est = nullptr;
    cudaStream_t s3 = nullptr;
    cudaEvent_t ev_est_fork = nullptr, ev_est_m2l = nullptr, ev_join3 = nullptr;
    bool timed = false;  // the events of the last evaluation were recorded
    bool marked_m2l = false, marked_p2p = false;  // ... and those around its main kernels
    gb3::Serve* serve = nullptr;  // the serving loop (serve.cu), created on first use
    // ensemble of the current evaluation (nsys = 0: one system): system offsets and G
    // on the device, roots (first, count) of the non-empty systems
    Buf sys_off, sys_G, sys_roots, skey, skey_alt, spos, spos_alt;
    int nsys = 0, nroots = 1;
    // force evaluation for a subset (Sec. 7.1): per sorted particle and per cell activity
    Buf pact, act, act_i, act_scan;
    bool active_mode = false;
    Buf tid_far, tid_near;  // tidal tensor parts (Sec. 7.4), sorted order
    // the tree of the last evaluation can be reused (Sec. 7.1) when it was a single system
    // of tree_n particles that completed
    int tree_n = -1;
    std::vector<Buf*> bufs() {
        return {&hx, &hmu, &hpsi, &hacc, &bounds, &status, &counters, &coin, &dtotal, &keys, &keys_alt, &idx,
                &idx_alt, &rtmp, &xm, &perm, &xp, &first, &count, &child, &nchild, &parent, &level, &sr,
                &cr, &mass, &minscale, &split_nchild, &split_oct, &split_offs, &scan_tmp, &leaves, &leaf_flag,
                &leaf_pos, &rad_tmp, &M, &F, &Pw, &binom, &pascal, &M1, &F1, &Ff, &front0, &front1, &m2l, &p2p,
                &sort_tmp, &sort_tmp2, &m2l_tmp, &p2p_tmp, &seg_start, &seg_end, &est_m2l, &est_p2p, &m2l_seg_start,
                &m2l_seg_end, &psi_far, &acc_far, &psi_near, &acc_near, &scale_sorted, &sys_off, &sys_G,
                &sys_roots, &skey, &skey_alt, &spos, &spos_alt, &pact, &act, &act_i, &act_scan, &tid_far, &tid_near, &walkf, &owner, &units};
    }
    // tree shape of the last evaluation
    std::vector<int> lev_start;
    int n = 0, ncells = 0, nleaves = 0;
    long long n_m2l = 0, n_p2p = 0, n_est_m2l = 0, n_est_p2p = 0;
};

static int fail(fmm_ctx* ctx, int code, const char* msg) {
    if (ctx) snprintf(ctx->err, sizeof ctx->err, "%s", msg);
    return code;
}
static int fail_cuda(fmm_ctx* ctx, int code) {
    if (ctx) snprintf(ctx->err, sizeof ctx->err, "%s", g_cuda_msg);
    return code;
}

namespace gb3 {
Serve*& ctx_serve(fmm_ctx* ctx) { return ctx->serve; }
const fmm_params* ctx_params(fmm_ctx* ctx) { return &ctx->prm; }
int ctx_device(fmm_ctx* ctx) { return ctx->device; }
int ctx_fail(fmm_ctx* ctx, int code, const char* msg) { return fail(ctx, code, msg); }
}  // namespace gb3

// a failing step keeps its own message; otherwise the CUDA error text is recorded
#define TRY(expr)                                                  \
    do {                                                           \
        int _rc = (expr);                                          \
        if (_rc) return ctx->err[0] ? _rc : fail_cuda(ctx, _rc);   \
    } while (0)
#define CU(expr) TRY(([&]() -> int { GB3_CUDA_TRY(expr); return 0; })())

static Cells cells_of(fmm_ctx* ctx) {
    Cells c;
    c.first = P<int>(ctx->first);
    c.count = P<int>(ctx->count);
    c.child = P<int>(ctx->child);
    c.nchild = P<int>(ctx->nchild);
    c.parent = P<int>(ctx->parent);
    c.level = P<int>(ctx->level);
    c.sr = P<d4>(ctx->sr);
    c.cr = P<d4>(ctx->cr);
    c.mass = P<double>(ctx->mass);
    c.minscale = P<double>(ctx->minscale);
    if (ctx->active_mode) {
        c.act = P<unsigned char>(ctx->act);
        c.pact = P<unsigned char>(ctx->pact);
    }
    return c;
}

static int check_params(const fmm_params* p) {
    if (p->p < 1 || p->p > kMaxP) return FMM_E_INVALID;
    if (p->mac != FMM_MAC_A && p->mac != FMM_MAC_F && p->mac != FMM_MAC_THETA) return FMM_E_INVALID;
    if (p->mac != FMM_MAC_THETA && !(p->eps > 0)) return FMM_E_INVALID;
    if (p->mac == FMM_MAC_THETA && !(p->theta_crit > 0 && p->theta_crit < 1)) return FMM_E_INVALID;
    if (p->leaf_size < 1 || p->leaf_size > 4096) return FMM_E_INVALID;
    if (!(p->p2p_c >= 0)) return FMM_E_INVALID;
    if (p->precision != FMM_PREC_FP64 && p->precision != FMM_PREC_MIXED) return FMM_E_INVALID;
    if (p->scale_src != FMM_SCALE_ESTIMATE && p->scale_src != FMM_SCALE_CALLER) return FMM_E_INVALID;
    if (p->m2l_rot != 0 && p->m2l_rot != 1) return FMM_E_INVALID;
    if (p->adaptive_p != 0 && p->adaptive_p != 1) return FMM_E_INVALID;
    if (p->p2p_two_float < 0 || p->p2p_two_float > 3) return FMM_E_INVALID;
    return 0;
}

// ------------------------------------------------------------------ tree (A1-A4)
__global__ void k_root(Cells c, int n) {
    c.first[0] = 0;
    c.count[0] = n;
    c.level[0] = 0;
    c.parent[0] = -1;
    c.child[0] = -1;
    c.nchild[0] = 0;
}
// one root per non-empty system of an ensemble (roots[r] = first, count)
__global__ void k_roots(Cells c, const int2* __restrict__ roots, int nroots) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nroots; r += gridDim.x * blockDim.x) {
        c.first[r] = roots[r].x;
        c.count[r] = roots[r].y;
        c.level[r] = 0;
        c.parent[r] = -1;
        c.child[r] = -1;
        c.nchild[r] = 0;
    }
}
__global__ void k_leaf_flags(const int* __restrict__ nchild, int nc, int* __restrict__ flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) flag[i] = nchild[i] == 0;
}
__global__ void k_leaf_compact(const int* __restrict__ flag, const int* __restrict__ pos, int nc, int* __restrict__ leaves) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
        if (flag[i]) leaves[pos[i]] = i;
}

// the two-float records of the sorted positions and masses (the internal radii's
// single-precision bounds, the mixed-mode kernels)
static int split_positions(fmm_ctx* ctx, int n, cudaStream_t s) {
    TRY(ensure(ctx->xp, 2 * sizeof(float4) * (size_t)n));
    launch_split_positions(P<d4>(ctx->xm), n, P<float4>(ctx->xp), s);
    return 0;
}

// Sec. 7.1's re-cycled tree: the previous evaluation's particle order, cells and centres
// stay; positions and masses are gathered in that order and the radii, masses and
// centres of mass are recomputed, so the MAC sees the true extent of every cell
static int refresh_tree(fmm_ctx* ctx, int n, const double* x, const double* mu, cudaStream_t s) {
    launch_bounds(x, mu, n, P<unsigned long long>(ctx->bounds), P<unsigned>(ctx->status), s);
    // the tree's centres are in the working units it was built in: keep them
    launch_gather(x, mu, P<int>(ctx->perm), n, P<d4>(ctx->xm), P<int>(ctx->perm), s, P<int>(ctx->units));
    unsigned st = 0;
    CU(cudaMemcpyAsync(&ctx->h_int[0], ctx->status.p, sizeof st, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    memcpy(&st, &ctx->h_int[0], sizeof st);
    if (st & kStatInvalid) return fail(ctx, FMM_E_INVALID, "non-finite position or mass, or negative mass");
    Cells c = cells_of(ctx);
    const int nlev = (int)ctx->lev_start.size() - 1;
    TRY(split_positions(ctx, n, s));
    TRY(ensure(ctx->owner, sizeof(int) * (size_t)n));
    launch_leaf_geometry(P<d4>(ctx->xm), c, P<int>(ctx->leaves), ctx->nleaves, P<unsigned>(ctx->status), s, true);
    launch_leaf_owner(c, P<int>(ctx->leaves), ctx->nleaves, P<int>(ctx->owner), s);
    for (int L = nlev - 1; L >= 0; --L)
        launch_internal_geometry(P<d4>(ctx->xm), P<float4>(ctx->xp), c, ctx->lev_start[L],
                                 ctx->lev_start[L + 1], n, P<int>(ctx->owner), P<unsigned long long>(ctx->rad_tmp),
                                 P<unsigned>(ctx->status), s, true);
    return 0;
}

static int build_tree(fmm_ctx* ctx, int n, const double* x, const double* mu, cudaStream_t s) {
    const int leaf = ctx->prm.leaf_size;
    TRY(ensure(ctx->keys, sizeof(uint64_t) * n));
    TRY(ensure(ctx->keys_alt, sizeof(uint64_t) * n));
    TRY(ensure(ctx->idx, sizeof(int) * n));
    TRY(ensure(ctx->idx_alt, sizeof(int) * n));
    TRY(ensure(ctx->rtmp, sizeof(int) * radix_tmp_ints(n)));
    TRY(ensure(ctx->xm, sizeof(d4) * n));
    TRY(ensure(ctx->perm, sizeof(int) * n));
    const int nsys = ctx->nsys;
    if (nsys == 0) {
        launch_bounds(x, mu, n, P<unsigned long long>(ctx->bounds), P<unsigned>(ctx->status), s);
        launch_keys(x, n, P<unsigned long long>(ctx->bounds), P<uint64_t>(ctx->keys), P<int>(ctx->idx), s);
        radix_sort_pairs(P<uint64_t>(ctx->keys), P<int>(ctx->idx), P<uint64_t>(ctx->keys_alt), P<int>(ctx->idx_alt),
                         n, P<int>(ctx->rtmp), s);
    } else {
        // forest: per-system bounds and keys, sort by key, then (stably) by system
        TRY(ensure(ctx->bounds, sizeof(unsigned long long) * (6 * (size_t)nsys + 1)));
        TRY(ensure(ctx->skey, sizeof(uint64_t) * n));
        TRY(ensure(ctx->skey_alt, sizeof(uint64_t) * n));
        TRY(ensure(ctx->spos, sizeof(int) * n));
        TRY(ensure(ctx->spos_alt, sizeof(int) * n));
        const int* off = P<int>(ctx->sys_off);
        launch_bounds_sys(x, mu, n, off, nsys, P<unsigned long long>(ctx->bounds), P<unsigned>(ctx->status), s);
        launch_keys_sys(x, n, off, nsys, P<unsigned long long>(ctx->bounds), P<uint64_t>(ctx->keys), P<int>(ctx->idx), s);
        radix_sort_pairs(P<uint64_t>(ctx->keys), P<int>(ctx->idx), P<uint64_t>(ctx->keys_alt), P<int>(ctx->idx_alt),
                         n, P<int>(ctx->rtmp), s);
        sort_by_system(P<uint64_t>(ctx->keys), P<int>(ctx->idx), n, off, nsys, P<uint64_t>(ctx->skey),
                       P<uint64_t>(ctx->skey_alt), P<int>(ctx->spos), P<int>(ctx->spos_alt), P<int>(ctx->rtmp),
                       P<uint64_t>(ctx->keys_alt), P<int>(ctx->idx_alt), s);
        std::swap(ctx->keys, ctx->keys_alt);
        std::swap(ctx->idx, ctx->idx_alt);
    }
    // working units: mixed precision rescales positions and masses by powers of two (exact)
    TRY(ensure(ctx->units, 2 * sizeof(int)));
    if (ctx->prm.precision == FMM_PREC_MIXED) launch_work_units(P<unsigned long long>(ctx->bounds), nsys, P<int>(ctx->units), s);
    else CU(cudaMemsetAsync(ctx->units.p, 0, 2 * sizeof(int), s));
    launch_gather(x, mu, P<int>(ctx->idx), n, P<d4>(ctx->xm), P<int>(ctx->perm), s, P<int>(ctx->units));

    // cell capacity: leaves <= n, internal cells hold > leaf particles, <= 21 levels
    const int nroots = ctx->nroots;
    long long cap = (long long)n + 21LL * (n / (leaf + 1)) + nroots + 64;
    Buf* ib[] = {&ctx->first, &ctx->count, &ctx->child, &ctx->nchild, &ctx->parent, &ctx->level};
    for (Buf* b : ib) TRY(ensure(*b, sizeof(int) * cap));
    TRY(ensure(ctx->sr, sizeof(d4) * cap));
    TRY(ensure(ctx->cr, sizeof(d4) * cap));
    TRY(ensure(ctx->mass, sizeof(double) * cap));
    TRY(ensure(ctx->minscale, sizeof(double) * cap));
    Cells c = cells_of(ctx);
    if (nsys == 0) {
        k_root<<<1, 1, 0, s>>>(c, n); note_launch();
    } else {
        k_roots<<<grid_for(nroots, 256), 256, 0, s>>>(c, P<int2>(ctx->sys_roots), nroots); note_launch();
    }
    ctx->lev_start.assign({0, nroots});
    for (int L = 0;; ++L) {
        int b = ctx->lev_start[L], e = ctx->lev_start[L + 1];
        int ncl = e - b;
        if (ncl <= 0) break;
        TRY(ensure(ctx->split_nchild, sizeof(int) * ncl));
        TRY(ensure(ctx->split_oct, sizeof(int) * 9 * (size_t)ncl));
        TRY(ensure(ctx->split_offs, sizeof(int) * ncl));
        TRY(ensure(ctx->scan_tmp, sizeof(int) * scan_tmp_ints(std::max<long long>(ncl, cap))));
        launch_split_level(P<uint64_t>(ctx->keys), c, b, e, L, leaf, P<int>(ctx->split_nchild), P<int>(ctx->split_oct),
                           P<int>(ctx->split_offs), P<int>(ctx->scan_tmp), P<int>(ctx->dtotal), s);
        CU(cudaMemcpyAsync(ctx->h_int, ctx->dtotal.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        int tot = ctx->h_int[0];
        if (tot <= 0) break;
        if ((long long)e + tot > cap) return fail(ctx, FMM_E_OVERFLOW, "cell capacity exceeded");
        ctx->lev_start.push_back(e + tot);
    }
    int nc = ctx->lev_start.back();
    ctx->ncells = nc;
    // leaves
    TRY(ensure(ctx->leaf_flag, sizeof(int) * nc));
    TRY(ensure(ctx->leaf_pos, sizeof(int) * nc));
    TRY(ensure(ctx->leaves, sizeof(int) * nc));
    TRY(ensure(ctx->scan_tmp, sizeof(int) * scan_tmp_ints(nc)));
    k_leaf_flags<<<grid_for(nc, 256), 256, 0, s>>>(c.nchild, nc, P<int>(ctx->leaf_flag)); note_launch();
    scan_exclusive_i32(P<int>(ctx->leaf_flag), P<int>(ctx->leaf_pos), nc, P<int>(ctx->dtotal), P<int>(ctx->scan_tmp), s);
    k_leaf_compact<<<grid_for(nc, 256), 256, 0, s>>>(P<int>(ctx->leaf_flag), P<int>(ctx->leaf_pos), nc, P<int>(ctx->leaves)); note_launch();
    CU(cudaMemcpyAsync(ctx->h_int, ctx->dtotal.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    ctx->nleaves = ctx->h_int[0];
    unsigned st = 0;
    CU(cudaMemcpy(&st, ctx->status.p, sizeof st, cudaMemcpyDeviceToHost));
    if (st & kStatInvalid) return fail(ctx, FMM_E_INVALID, "non-finite position or mass, or negative mass");

    // geometry: leaves, then internal cells bottom-up
    int nlev = (int)ctx->lev_start.size() - 1;
    int maxlev_cells = 0;
    for (int L = 0; L < nlev; ++L) maxlev_cells = std::max(maxlev_cells, ctx->lev_start[L + 1] - ctx->lev_start[L]);
    TRY(ensure(ctx->rad_tmp, sizeof(unsigned long long) * rad_tmp_u64_per_cell() * (size_t)maxlev_cells));
    TRY(split_positions(ctx, n, s));
    TRY(ensure(ctx->owner, sizeof(int) * (size_t)n));
    launch_leaf_geometry(P<d4>(ctx->xm), c, P<int>(ctx->leaves), ctx->nleaves, P<unsigned>(ctx->status), s);
    launch_leaf_owner(c, P<int>(ctx->leaves), ctx->nleaves, P<int>(ctx->owner), s);
    for (int L = nlev - 1; L >= 0; --L)
        launch_internal_geometry(P<d4>(ctx->xm), P<float4>(ctx->xp), c, ctx->lev_start[L],
                                 ctx->lev_start[L + 1], n, P<int>(ctx->owner), P<unsigned long long>(ctx->rad_tmp),
                                 P<unsigned>(ctx->status), s);
    return 0;
}

// ------------------------------------------------------------------ walk driver (A8)
static int run_walk(fmm_ctx* ctx, WalkParams wp, Buf& m2l, long long& m2l_cap, Buf& p2p, long long& p2p_cap,
                    long long* n_m2l, long long* n_p2p, cudaStream_t s) {
    Cells c = cells_of(ctx);
    const int nc = ctx->ncells;
    // starting capacities scale with this tree (a previous, smaller evaluation may have
    // left smaller ones); an overflow grows what overflowed and the walk is redone
    ctx->front_cap = std::max<long long>(ctx->front_cap, std::max<long long>(1 << 16, 32LL * nc));
    m2l_cap = std::max<long long>(m2l_cap, std::max<long long>(1 << 16, 64LL * nc));
    p2p_cap = std::max<long long>(p2p_cap, std::max<long long>(1 << 16, 32LL * nc));
    for (int attempt = 0; attempt < 24; ++attempt) {
        TRY(ensure(ctx->front0, sizeof(int2) * ctx->front_cap));
        TRY(ensure(ctx->front1, sizeof(int2) * ctx->front_cap));
        TRY(ensure(m2l, sizeof(int2) * m2l_cap));
        TRY(ensure(p2p, sizeof(int2) * p2p_cap));
        WalkBuffers wb;
        wb.front[0] = P<int2>(ctx->front0);
        wb.front[1] = P<int2>(ctx->front1);
        wb.front_cap = ctx->front_cap;
        wb.m2l = P<int2>(m2l);
        wb.m2l_cap = m2l_cap;
        wb.p2p = P<int2>(p2p);
        wb.p2p_cap = p2p_cap;
        wb.counters = P<unsigned long long>(ctx->counters);
        // counters: [0], [4] the frontier lengths (ping-pong), [1] M2L, [2] P2P, [3] overflow,
        // [5] the largest frontier demand.  Every step of a pair descends one cell level on
        // at least one side, so 2 * levels steps end the walk; the steps read their frontier
        // lengths on the device and the host waits once, after the last one.
        CU(cudaMemsetAsync(wb.counters, 0, 8 * sizeof(unsigned long long), s));
        launch_walk_roots(wb.front[0], ctx->nroots, s, wb.counters);
        const int nlev = (int)ctx->lev_start.size() - 1;
        const int steps = 2 * nlev + 1;
        int cur = 0;
        for (int k = 0; k < steps; ++k) {
            unsigned long long* in_cnt = wb.counters + (k & 1 ? 4 : 0);
            unsigned long long* out_cnt = wb.counters + (k & 1 ? 0 : 4);
            CU(cudaMemsetAsync(out_cnt, 0, sizeof(unsigned long long), s));
            launch_walk_step_dev(c, wp, wb.front[cur], in_cnt, wb.front[cur ^ 1], wb, out_cnt, s);
            cur ^= 1;
        }
        CU(cudaMemcpyAsync(ctx->h_counters, wb.counters, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        const long long left = (long long)ctx->h_counters[(steps - 1) & 1 ? 0 : 4];
        const long long need_front = std::max<long long>((long long)ctx->h_counters[5], left);
        const bool overflow = ctx->h_counters[3] != 0;
        if (!overflow && left != 0) return fail(ctx, FMM_E_CUDA, "the tree walk did not end within 2 x levels steps");
        if (!overflow) {
            *n_m2l = (long long)ctx->h_counters[1];
            *n_p2p = (long long)ctx->h_counters[2];
            return 0;
        }
        // grow what overflowed (the counters hold at least the demand seen so far) and redo the walk
        if (need_front > ctx->front_cap)
            ctx->front_cap = std::max<long long>(2 * ctx->front_cap, 2 * need_front);
        if ((long long)ctx->h_counters[1] > m2l_cap) m2l_cap = std::max<long long>(2 * m2l_cap, 2 * (long long)ctx->h_counters[1]);
        if ((long long)ctx->h_counters[2] > p2p_cap) p2p_cap = std::max<long long>(2 * p2p_cap, 2 * (long long)ctx->h_counters[2]);
    }
    char msg[200];
    snprintf(msg, sizeof msg, "walk lists could not be grown enough (caps: front %lld, m2l %lld, p2p %lld)",
             ctx->front_cap, m2l_cap, p2p_cap);
    return fail(ctx, FMM_E_OVERFLOW, msg);
}

static int sort_and_segment(fmm_ctx* ctx, Buf& list, long long npairs, Buf& seg_start, Buf& seg_end,
                            cudaStream_t s, bool wide = false, Buf* tmp = nullptr) {
    Buf& st = tmp ? *tmp : ctx->sort_tmp;
    TRY(ensure(st, list_sort_tmp_bytes(npairs, ctx->ncells)));
    TRY(ensure(seg_start, sizeof(int) * ctx->ncells));
    TRY(ensure(seg_end, sizeof(int) * ctx->ncells));
    sort_pairs_by_sink(P<int2>(list), npairs, ctx->ncells, st.p, s, wide);
    launch_segments(P<int2>(list), npairs, ctx->ncells, P<int>(seg_start), P<int>(seg_end), s);
    return 0;
}

// mixed P2P over the segments in seg_start/seg_end of list: the work plan grows its scratch
// once if the plan needs more than the context holds
static int run_p2p_mixed(fmm_ctx* ctx, const int2* list, int mode, cudaStream_t s) {
    Cells c = cells_of(ctx);
    TRY(ensure(ctx->p2p_tmp, p2p_plan_fixed_bytes(ctx->nleaves)));
    for (int attempt = 0; attempt < 2; ++attempt) {
        const size_t need = launch_p2p_mixed(P<float4>(ctx->xp), ctx->n, c, list,
                                             P<int>(ctx->seg_start), P<int>(ctx->seg_end), P<int>(ctx->leaves),
                                             ctx->nleaves, P<double>(ctx->psi_near), P<double>(ctx->acc_near), mode,
                                             ctx->p2p_tmp.p, ctx->p2p_tmp.bytes, ctx->h_counters + 8, s);
        if (need == ~(size_t)0) return fail(ctx, FMM_E_OVERFLOW, "P2P plan beyond 2^31 source ranges or n >= 2^29");
        if (need <= ctx->p2p_tmp.bytes) return 0;
        TRY(ensure(ctx->p2p_tmp, need));
    }
    return fail(ctx, FMM_E_CUDA, "P2P plan did not fit after growing its scratch");
}

// ------------------------------------------------------------------ the low-order scale (A7)
static int estimate_scale(fmm_ctx* ctx, cudaStream_t s) {
    const int nc = ctx->ncells;
    Cells c = cells_of(ctx);
    const bool want_f = ctx->prm.mac == FMM_MAC_F;
    const int nlev = (int)ctx->lev_start.size() - 1;
    WalkParams wp;
    memset(&wp, 0, sizeof wp);
    wp.p = want_f ? 0 : 1;
    wp.mac = kMacEstimate;
    wp.p2p_thresh = ctx->prm.p2p_c * (double)wp.p * wp.p * wp.p;  // the estimate's own order (reading R-p2p)
    wp.use_com = 1;
    TRY(ensure(ctx->walkf, sizeof(float4) * 2 * (size_t)nc));
    wp.fc = P<float4>(ctx->walkf);
    launch_walk_prep(c, c.cr, nullptr, 0, 0.0, nc, P<float4>(ctx->walkf), nullptr, s);
    TRY(run_walk(ctx, wp, ctx->est_m2l, ctx->est_m2l_cap, ctx->est_p2p, ctx->est_p2p_cap, &ctx->n_est_m2l,
                 &ctx->n_est_p2p, s));
    // the M2L branch (list sort, M2L) on the third stream beside the P2P branch on s; both
    // meet before the scale
    const int pe = 1, nco = ncoef(pe);
    if (!want_f) TRY(ensure(ctx->F1, sizeof(double) * nco * (size_t)nc));
    const bool mixed = ctx->prm.precision == FMM_PREC_MIXED;
    cudaStream_t sm = want_f ? s : ctx->s3;
    if (!want_f) {
        CU(cudaEventRecord(ctx->ev_est_fork, s));
        CU(cudaStreamWaitEvent(sm, ctx->ev_est_fork, 0));
    }
    TRY(sort_and_segment(ctx, ctx->est_m2l, ctx->n_est_m2l, ctx->m2l_seg_start, ctx->m2l_seg_end, sm, false,
                         &ctx->sort_tmp2));
    if (!want_f) {
        // multipoles about the centres of mass: the masses and centres of the geometry pass
        launch_est_m2l(P<int2>(ctx->est_m2l), P<int>(ctx->m2l_seg_start), P<int>(ctx->m2l_seg_end), nc, c,
                       P<double>(ctx->F1), sm, mixed ? P<float4>(ctx->walkf) : nullptr);
        CU(cudaEventRecord(ctx->ev_est_m2l, sm));
    }
    // P2P segments of the estimate reuse seg_start/seg_end of the main lists (written later)
    TRY(ensure(ctx->seg_start, sizeof(int) * nc));
    TRY(ensure(ctx->seg_end, sizeof(int) * nc));
    TRY(ensure(ctx->sort_tmp, list_sort_tmp_bytes(ctx->n_est_p2p, nc)));
    sort_pairs_by_sink(P<int2>(ctx->est_p2p), ctx->n_est_p2p, nc, ctx->sort_tmp.p, s);
    launch_segments(P<int2>(ctx->est_p2p), ctx->n_est_p2p, nc, P<int>(ctx->seg_start), P<int>(ctx->seg_end), s);
    double* scale = P<double>(ctx->scale_sorted);
    if (want_f) {
        TRY(ensure(ctx->Ff, sizeof(double) * nc));
        launch_f_m2l(P<int2>(ctx->est_m2l), P<int>(ctx->m2l_seg_start), P<int>(ctx->m2l_seg_end), nc, c,
                     P<double>(ctx->Ff), s);
        for (int L = 1; L < nlev; ++L) launch_f_down_level(c, ctx->lev_start[L], ctx->lev_start[L + 1], P<double>(ctx->Ff), s);
        launch_f_p2p(P<d4>(ctx->xm), c, P<int2>(ctx->est_p2p), P<int>(ctx->seg_start), P<int>(ctx->seg_end),
                     P<int>(ctx->leaves), ctx->nleaves, P<double>(ctx->Ff), scale, s);
        return 0;
    }
    // (the p = 1 L2L is folded into launch_est_scale)
    if (mixed)
        TRY(run_p2p_mixed(ctx, P<int2>(ctx->est_p2p), 0, s));
    else
        launch_p2p_fp64(P<d4>(ctx->xm), c, P<int2>(ctx->est_p2p), P<int>(ctx->seg_start), P<int>(ctx->seg_end),
                        P<int>(ctx->leaves), ctx->nleaves, P<double>(ctx->psi_near), P<double>(ctx->acc_near), s);
    CU(cudaStreamWaitEvent(s, ctx->ev_est_m2l, 0));
    launch_est_scale(c, P<int>(ctx->leaves), ctx->nleaves, P<double>(ctx->F1), P<double>(ctx->acc_near), scale, s);
    return 0;
}

// phase times of the last evaluation from its events (waits for the last event)
static int phase_times(fmm_ctx* ctx) {
    if (!ctx->timed) return 0;
    CU(cudaEventSynchronize(ctx->ev[EV_END]));
    float t;
    auto el = [&](int a, int b) {
        cudaEventElapsedTime(&t, ctx->ev[a], ctx->ev[b]);
        return t;
    };
    ctx->last.t_tree = el(EV_START, EV_TREE);
    ctx->last.t_estimate = el(EV_TREE, EV_EST);
    ctx->last.t_up = el(EV_TREE, EV_UP);  // beside the estimate, on the second stream
    ctx->last.t_walk = el(EV_JOINED, EV_WALK);
    ctx->last.t_m2l = el(EV_WALK, EV_M2L);   // M2L, then the downward pass, on one stream
    ctx->last.t_p2p = el(EV_WALK, EV_P2P);   // beside them on the other
    ctx->last.t_down = el(EV_M2L, EV_DOWN);
    ctx->last.t_total = el(EV_START, EV_END);
    // the main kernels' own times; 0 when the kernel did not run (no marks recorded)
    auto kel = [&](int a, int b) {
        float k = 0.f;
        if (cudaEventElapsedTime(&k, ctx->ev[a], ctx->ev[b]) != cudaSuccess) {
            cudaGetLastError();
            k = 0.f;
        }
        return k;
    };
    ctx->last.t_m2l_kernel = ctx->marked_m2l ? kel(EV_M2LK0, EV_M2LK1) : 0.f;
    ctx->last.t_p2p_kernel = ctx->marked_p2p ? kel(EV_P2PK0, EV_P2PK1) : 0.f;
    return 0;
}

// ------------------------------------------------------------------ one evaluation
static int evaluate_device(fmm_ctx* ctx, int n, const double* x, const double* mu, double G, const double* scale,
                           double* psi, double* acc, cudaStream_t s, fmm_stats* stats,
                           const unsigned char* active = nullptr, bool reuse_tree = false,
                           const double* eps_b = nullptr, double* tidal = nullptr) {
    const fmm_params& prm = ctx->prm;
    ctx->active_mode = false;
    if (reuse_tree && (ctx->tree_n != n || ctx->nsys != 0 || n == 0))
        return fail(ctx, FMM_E_INVALID, "no tree of this system to reuse (the last evaluation on this context "
                                        "was not a completed single system of n particles)");
    const int tree_n = ctx->tree_n, tree_nc = ctx->ncells, tree_nl = ctx->nleaves;
    ctx->tree_n = -1;  // valid again once this evaluation has completed
    if (check_params(&prm)) return fail(ctx, FMM_E_INVALID, "invalid parameters");
    memset(&ctx->last, 0, sizeof ctx->last);
    ctx->last.n = n;
    ctx->last.p = prm.p;
    ctx->last.eps = prm.eps;
    ctx->last.leaf_size = prm.leaf_size;
    ctx->n = n;
    ctx->ncells = ctx->nleaves = 0;
    ctx->n_m2l = ctx->n_p2p = ctx->n_est_m2l = ctx->n_est_p2p = 0;
    if (n == 0) {
        if (stats) *stats = ctx->last;
        return 0;
    }
    if (prm.scale_src == FMM_SCALE_CALLER && prm.mac != FMM_MAC_THETA && !scale)
        return fail(ctx, FMM_E_INVALID, "scale_src = caller but scale == NULL");
    const bool timing = ctx->ev_ok;
    const long long launches0 = launches_so_far();
    ctx->timed = false;
    ctx->marked_m2l = ctx->marked_p2p = false;
    if (timing) CU(cudaEventRecord(ctx->ev[EV_START], s));
    CU(cudaMemsetAsync(ctx->status.p, 0, sizeof(unsigned), s));
    CU(cudaMemsetAsync(ctx->coin.p, 0, sizeof(unsigned long long), s));
    if (reuse_tree) {
        if (tree_nc <= 0 || tree_n != n) return fail(ctx, FMM_E_INVALID, "no tree to reuse");
        ctx->ncells = tree_nc;
        ctx->nleaves = tree_nl;
        TRY(refresh_tree(ctx, n, x, mu, s));
    } else {
        TRY(build_tree(ctx, n, x, mu, s));
    }
    if (active) {  // Sec. 7.1: only sink cells holding an active particle are evaluated
        TRY(ensure(ctx->pact, (size_t)n));
        TRY(ensure(ctx->act, (size_t)ctx->ncells));
        TRY(ensure(ctx->act_i, sizeof(int) * ((size_t)n + 1)));
        TRY(ensure(ctx->act_scan, sizeof(int) * ((size_t)n + scan_tmp_ints(n))));
        launch_active_flags(active, P<int>(ctx->perm), n, P<int>(ctx->first), P<int>(ctx->count), ctx->ncells,
                            P<unsigned char>(ctx->pact), P<unsigned char>(ctx->act), P<int>(ctx->act_i),
                            P<int>(ctx->act_scan), P<int>(ctx->act_scan) + n, s);
        ctx->active_mode = true;
    }
    if (timing) CU(cudaEventRecord(ctx->ev[EV_TREE], s));
    const int nc = ctx->ncells, nco = ncoef(prm.p);
    const int nlev = (int)ctx->lev_start.size() - 1;
    Cells c = cells_of(ctx);
    TRY(ensure(ctx->psi_far, sizeof(double) * n));
    TRY(ensure(ctx->acc_far, sizeof(double) * 3 * (size_t)n));
    TRY(ensure(ctx->psi_near, sizeof(double) * n));
    TRY(ensure(ctx->acc_near, sizeof(double) * 3 * (size_t)n));
    TRY(ensure(ctx->scale_sorted, sizeof(double) * n));
    // (the two-float positions were made with the tree)

    // A5-A6 (upward pass) and A7 (scale estimate) are independent: the upward pass is
    // queued on s2, then the estimate, which waits on the host for its list sizes, runs on
    // s_hi (and s3); s waits for both before the walk
    TRY(ensure(ctx->M, sizeof(double) * nco * (size_t)nc));
    TRY(ensure(ctx->F, sizeof(double) * nco * (size_t)nc));
    TRY(ensure(ctx->Pw, sizeof(double) * (prm.p + 1) * (size_t)nc));
    TRY(ensure(ctx->binom, sizeof(double) * (kMaxP + 1)));
    {
        double bn[kMaxP + 1];
        bn[0] = 1;
        for (int k = 1; k <= prm.p; ++k) bn[k] = bn[k - 1] * (prm.p - k + 1) / k;
        CU(cudaMemcpyAsync(ctx->binom.p, bn, sizeof(double) * (prm.p + 1), cudaMemcpyHostToDevice, s));
    }
    const bool split = prm.precision == FMM_PREC_MIXED && prm.m2l_split;
    {
        cudaStream_t u = ctx->s2;
        CU(cudaEventRecord(ctx->ev_fork, s));
        CU(cudaStreamWaitEvent(u, ctx->ev_fork, 0));
        if (split) launch_p2m_split(P<d4>(ctx->xm), c, c.sr, P<int>(ctx->leaves), ctx->nleaves, prm.p, P<double>(ctx->M), u);
        else launch_p2m(P<d4>(ctx->xm), c, c.sr, P<int>(ctx->leaves), ctx->nleaves, prm.p, P<double>(ctx->M), u);
        for (int L = nlev - 1; L >= 0; --L) {
            if (split) launch_m2m_split(c, c.sr, ctx->lev_start[L], ctx->lev_start[L + 1], prm.p, P<double>(ctx->M), u);
            else launch_m2m_level(c, c.sr, ctx->lev_start[L], ctx->lev_start[L + 1], prm.p, P<double>(ctx->M), u);
        }
        launch_power(P<double>(ctx->M), nc, prm.p, P<double>(ctx->Pw), u);
        if (timing) CU(cudaEventRecord(ctx->ev[EV_UP], u));
        CU(cudaEventRecord(ctx->ev_join, u));
    }
    // every exit from here on (errors included) leaves s behind all the work of both streams
    struct Join {
        cudaStream_t s, s2, se, s3;
        cudaEvent_t e, ee, e3;
        ~Join() {
            cudaEventRecord(e, s2);
            cudaEventRecord(ee, se);
            cudaEventRecord(e3, s3);
            cudaStreamWaitEvent(s, e, 0);
            cudaStreamWaitEvent(s, ee, 0);
            cudaStreamWaitEvent(s, e3, 0);
        }
    } join{s, ctx->s2, ctx->s_hi, ctx->s3, ctx->ev_join, ctx->ev_join_est, ctx->ev_join3};

    // A7: acceleration scale for the MAC and its per-cell minimum, on its own stream
    {
    cudaStream_t s0 = s;  // the caller's stream; s is the estimate's in this block
    CU(cudaStreamWaitEvent(ctx->s_hi, ctx->ev_fork, 0));
    s = ctx->s_hi;
    if (prm.mac != FMM_MAC_THETA) {
        if (prm.scale_src == FMM_SCALE_CALLER)
            launch_scale_from_caller(scale, P<int>(ctx->perm), n, P<double>(ctx->scale_sorted), s, P<int>(ctx->units));
        else
            TRY(estimate_scale(ctx, s));
        if (eps_b) {  // Sec. 7, opening: min over the sinks of eps_b a_b in place of eps min a_b
            launch_scale_eps(eps_b, P<int>(ctx->perm), n, prm.eps, P<double>(ctx->scale_sorted),
                             P<unsigned>(ctx->status), s);
            unsigned st = 0;
            CU(cudaMemcpyAsync(&ctx->h_int[0], ctx->status.p, sizeof st, cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            memcpy(&st, &ctx->h_int[0], sizeof st);
            if (st & kStatInvalid) return fail(ctx, FMM_E_INVALID, "eps_b must be positive and finite");
        }
        launch_minscale_leaves(P<double>(ctx->scale_sorted), c, P<int>(ctx->leaves), ctx->nleaves, s);
        for (int L = nlev - 1; L >= 0; --L) launch_minscale_level(c, ctx->lev_start[L], ctx->lev_start[L + 1], s);
    }
    if (timing) CU(cudaEventRecord(ctx->ev[EV_EST], s));
    CU(cudaEventRecord(ctx->ev_join_est, s));
    s = s0;
    }
    CU(cudaStreamWaitEvent(s, ctx->ev_join_est, 0));
    CU(cudaStreamWaitEvent(s, ctx->ev_join, 0));
    if (timing) CU(cudaEventRecord(ctx->ev[EV_JOINED], s));

    // A8: dual tree walk
    WalkParams wp;
    memset(&wp, 0, sizeof wp);
    wp.p = prm.p;
    wp.mac = prm.mac;
    wp.eps = prm.eps;
    wp.theta_crit = prm.theta_crit;
    wp.p2p_thresh = prm.p2p_c * (double)prm.p * prm.p * prm.p;
    wp.P = P<double>(ctx->Pw);
    wp.binom = P<double>(ctx->binom);
    wp.use_com = 0;
    wp.adaptive = prm.adaptive_p && prm.mac != FMM_MAC_THETA;
    wp.p_lo = prm.p < 3 ? prm.p : 3;
    wp.pascal = nullptr;
    if (wp.adaptive) {
        TRY(ensure(ctx->pascal, sizeof(double) * (kMaxP + 1) * (kMaxP + 1)));
        double pt[(kMaxP + 1) * (kMaxP + 1)] = {};
        for (int q = 0; q <= kMaxP; ++q) {
            pt[q * (kMaxP + 1)] = 1.0;
            for (int k = 1; k <= q; ++k) pt[q * (kMaxP + 1) + k] = pt[q * (kMaxP + 1) + k - 1] * (q - k + 1) / k;
        }
        CU(cudaMemcpyAsync(ctx->pascal.p, pt, sizeof pt, cudaMemcpyHostToDevice, s));
        CU(cudaStreamSynchronize(s));  // pt lives on this stack frame
        wp.pascal = P<double>(ctx->pascal);
    }
    if (prm.mac != FMM_MAC_THETA && !wp.adaptive) {
        const int fs = walk_fstride(prm.p);
        TRY(ensure(ctx->walkf, sizeof(float) * (8 + (size_t)fs) * nc));
        wp.fc = P<float4>(ctx->walkf);
        wp.fP = (float*)(wp.fc + 2 * (size_t)nc);
        wp.fstride = fs;
        launch_walk_prep(c, c.sr, wp.P, prm.p, prm.eps, nc, P<float4>(ctx->walkf), P<float>(ctx->walkf) + 8 * (size_t)nc, s);
    }
    TRY(run_walk(ctx, wp, ctx->m2l, ctx->m2l_cap, ctx->p2p, ctx->p2p_cap, &ctx->n_m2l, &ctx->n_p2p, s));
    TRY(sort_and_segment(ctx, ctx->m2l, ctx->n_m2l, ctx->m2l_seg_start, ctx->m2l_seg_end, s, wp.adaptive != 0));
    if (timing) CU(cudaEventRecord(ctx->ev[EV_WALK], s));

    // A9 M2L with A11 L2L and L2P (on the high-priority stream) and A10 P2P (on the low-priority
    // stream; it waits on the host for its work plan, which runs beside the M2L kernel) are
    // independent; s waits for both
    CU(cudaEventRecord(ctx->ev_fork, s));
    {
    cudaStream_t s0 = s;
    s = ctx->s_hi;
    CU(cudaStreamWaitEvent(s, ctx->ev_fork, 0));
    // A9: M2L
    CU(cudaMemsetAsync(ctx->F.p, 0, sizeof(double) * nco * (size_t)nc, s));
    if (split) {
        TRY(ensure(ctx->m2l_tmp, m2l_split_tmp_bytes(nc, prm.p, ctx->n_m2l)));
        kernel_marks(timing ? &ctx->ev[EV_M2LK0] : nullptr);
        launch_m2l_split(P<int2>(ctx->m2l), P<int>(ctx->m2l_seg_start), P<int>(ctx->m2l_seg_end), ctx->m2l_tmp.p, nc,
                         c.sr, P<double>(ctx->M), prm.p, P<double>(ctx->F), prm.m2l_rot != 0, s, wp.adaptive != 0,
                         ctx->n_m2l);
    } else {
        TRY(ensure(ctx->m2l_tmp, m2l_tmp_bytes(nc, prm.p)));
        launch_m2l(P<int2>(ctx->m2l), P<int>(ctx->m2l_seg_start), P<int>(ctx->m2l_seg_end), ctx->m2l_tmp.p, nc, c.sr,
                   P<double>(ctx->M), prm.p, P<double>(ctx->F), s);
    }
    ctx->marked_m2l = marks_recorded();
    kernel_marks(nullptr);
    if (timing) CU(cudaEventRecord(ctx->ev[EV_M2L], s));
    // A11-A12: L2L, L2P
    for (int L = 1; L < nlev; ++L) {
        if (split) launch_l2l_split(c, c.sr, ctx->lev_start[L], ctx->lev_start[L + 1], prm.p, P<double>(ctx->F), s);
        else launch_l2l_level(c, c.sr, ctx->lev_start[L], ctx->lev_start[L + 1], prm.p, P<double>(ctx->F), s);
    }
    if (split)
        launch_l2p_split(P<d4>(ctx->xm), c, c.sr, P<int>(ctx->leaves), ctx->nleaves, prm.p, P<double>(ctx->F),
                         P<double>(ctx->psi_far), P<double>(ctx->acc_far), s);
    else
        launch_l2p(P<d4>(ctx->xm), c, c.sr, P<int>(ctx->leaves), ctx->nleaves, prm.p, P<double>(ctx->F),
                   P<double>(ctx->psi_far), P<double>(ctx->acc_far), s);
    if (timing) CU(cudaEventRecord(ctx->ev[EV_DOWN], s));
    CU(cudaEventRecord(ctx->ev_join, s));

    // A10: P2P
    s = ctx->s2;
    CU(cudaStreamWaitEvent(s, ctx->ev_fork, 0));
    TRY(sort_and_segment(ctx, ctx->p2p, ctx->n_p2p, ctx->seg_start, ctx->seg_end, s));
    if (prm.precision == FMM_PREC_MIXED) {
        kernel_marks(timing ? &ctx->ev[EV_P2PK0] : nullptr);
        const int rc = run_p2p_mixed(ctx, P<int2>(ctx->p2p), prm.p2p_two_float, s);
        ctx->marked_p2p = marks_recorded();
        kernel_marks(nullptr);
        TRY(rc);
    } else
        launch_p2p_fp64(P<d4>(ctx->xm), c, P<int2>(ctx->p2p), P<int>(ctx->seg_start), P<int>(ctx->seg_end),
                        P<int>(ctx->leaves), ctx->nleaves, P<double>(ctx->psi_near), P<double>(ctx->acc_near), s);
    launch_coincident(P<d4>(ctx->xm), P<uint64_t>(ctx->keys), n, P<unsigned long long>(ctx->coin), s,
                      ctx->nsys ? P<int>(ctx->sys_off) : nullptr, ctx->nsys);
    if (tidal) {  // Sec. 7.4: the near part over the same sources as the P2P
        TRY(ensure(ctx->tid_near, sizeof(double) * 6 * (size_t)n));
        launch_p2p_tidal(P<d4>(ctx->xm), P<float4>(ctx->xp), n, prm.precision == FMM_PREC_MIXED,
                         c, P<int2>(ctx->p2p), P<int>(ctx->seg_start), P<int>(ctx->seg_end), P<int>(ctx->leaves),
                         ctx->nleaves, P<double>(ctx->tid_near), s);
    }
    if (timing) CU(cudaEventRecord(ctx->ev[EV_P2P], s));
    CU(cudaEventRecord(ctx->ev_join_est, s));
    s = s0;
    }
    CU(cudaStreamWaitEvent(s, ctx->ev_join, 0));
    CU(cudaStreamWaitEvent(s, ctx->ev_join_est, 0));
    const int* sys_off = ctx->nsys ? P<int>(ctx->sys_off) : nullptr;
    launch_finish(P<double>(ctx->psi_far), P<double>(ctx->acc_far), P<double>(ctx->psi_near), P<double>(ctx->acc_near),
                  P<int>(ctx->perm), n, G, psi, acc, s, sys_off, ctx->nsys ? P<double>(ctx->sys_G) : nullptr,
                  ctx->nsys, ctx->active_mode ? P<unsigned char>(ctx->pact) : nullptr, P<int>(ctx->units));
    if (tidal) {  // Sec. 7.4: the far part from Psi_2^m of the local expansions
        TRY(ensure(ctx->tid_far, sizeof(double) * 6 * (size_t)n));
        launch_l2p_tidal(P<d4>(ctx->xm), c, c.sr, P<int>(ctx->leaves), ctx->nleaves, prm.p, P<double>(ctx->F),
                         P<double>(ctx->tid_far), s);
        launch_finish_tidal(P<double>(ctx->tid_far), P<double>(ctx->tid_near), P<int>(ctx->perm), n, G,
                            ctx->active_mode ? P<unsigned char>(ctx->pact) : nullptr, tidal, s, P<int>(ctx->units));
    }
    if (timing) CU(cudaEventRecord(ctx->ev[EV_END], s));
    CU(cudaGetLastError());

    ctx->last.ncells = nc;
    ctx->last.nleaves = ctx->nleaves;
    ctx->last.n_m2l = ctx->n_m2l;
    ctx->last.n_p2p = ctx->n_p2p;
    ctx->last.est_m2l = ctx->n_est_m2l;
    ctx->last.est_p2p = ctx->n_est_p2p;
    ctx->last.depth = nlev - 1;
    ctx->last.launches = launches_so_far() - launches0;
    ctx->timed = timing;
    ctx->tree_n = ctx->nsys == 0 ? n : -1;
    if (stats) {
        CU(cudaStreamSynchronize(s));
        unsigned long long coin = 0;
        CU(cudaMemcpy(&coin, ctx->coin.p, sizeof coin, cudaMemcpyDeviceToHost));
        ctx->last.coincident = (long long)coin;
        // p2p particle interactions from the list
        std::vector<int2> pl(ctx->n_p2p);
        std::vector<int> cnt(nc);
        if (ctx->n_p2p) CU(cudaMemcpy(pl.data(), ctx->p2p.p, sizeof(int2) * ctx->n_p2p, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(cnt.data(), ctx->count.p, sizeof(int) * nc, cudaMemcpyDeviceToHost));
        long long inter = 0;
        for (auto& e : pl) inter += (long long)cnt[e.x] * cnt[e.y] - (e.x == e.y ? cnt[e.x] : 0);
        ctx->last.p2p_interactions = inter;
        TRY(phase_times(ctx));
        *stats = ctx->last;
    }
    return 0;
}

// ================================================================== C ABI
extern "C" {

void fmm_default_params(fmm_params* out) {
    if (!out) return;
    out->p = 8;
    out->eps = 1e-7;
    out->mac = FMM_MAC_A;
    out->theta_crit = 0.5;
    out->leaf_size = 64;
    out->p2p_c = 8.0;
    out->precision = FMM_PREC_MIXED;
    out->scale_src = FMM_SCALE_ESTIMATE;
    out->p2p_two_float = 1;
    out->m2l_split = 1;
    out->m2l_rot = 1;
    out->adaptive_p = 0;
}

int fmm_create(fmm_ctx** out, const fmm_params* params, int device) {
    if (!out) return FMM_E_INVALID;
    *out = nullptr;
    fmm_params prm;
    if (params) prm = *params;
    else fmm_default_params(&prm);
    if (check_params(&prm)) return FMM_E_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return FMM_E_CUDA;
    }
    fmm_ctx* ctx = new (std::nothrow) fmm_ctx();
    if (!ctx) return FMM_E_OOM;
    ctx->prm = prm;
    ctx->device = device;
    memset(&ctx->last, 0, sizeof ctx->last);
    int rc = 0;
    if (!rc) rc = ensure(ctx->bounds, 8 * sizeof(unsigned long long));
    if (!rc) rc = ensure(ctx->status, 16);
    if (!rc) rc = ensure(ctx->counters, 8 * sizeof(unsigned long long));
    if (!rc) rc = ensure(ctx->coin, 16);
    if (!rc) rc = ensure(ctx->dtotal, 16);
    if (!rc && cudaMallocHost((void**)&ctx->h_counters, 16 * sizeof(unsigned long long)) != cudaSuccess) rc = FMM_E_OOM;
    if (!rc && cudaMallocHost((void**)&ctx->h_int, 16 * sizeof(int)) != cudaSuccess) rc = FMM_E_OOM;
    if (!rc) {
        ctx->ev_ok = true;
        for (int i = 0; i < EV_N; ++i)
            if (cudaEventCreate(&ctx->ev[i]) != cudaSuccess) ctx->ev_ok = false;
    }
    int prio_least = 0, prio_greatest = 0;
    if (!rc && cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) rc = FMM_E_CUDA;
    if (!rc && (cudaStreamCreateWithPriority(&ctx->s2, cudaStreamNonBlocking, prio_least) != cudaSuccess ||
                cudaStreamCreateWithPriority(&ctx->s_hi, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
                cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ctx->ev_join_est, cudaEventDisableTiming) != cudaSuccess ||
                cudaStreamCreateWithPriority(&ctx->s3, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
                cudaEventCreateWithFlags(&ctx->ev_est_fork, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ctx->ev_est_m2l, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&ctx->ev_join3, cudaEventDisableTiming) != cudaSuccess))
        rc = FMM_E_CUDA;
    if (rc) {
        cudaGetLastError();
        fmm_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return 0;
}

int fmm_set_params(fmm_ctx* ctx, const fmm_params* params) {
    if (!ctx || !params) return FMM_E_INVALID;
    if (check_params(params)) return fail(ctx, FMM_E_INVALID, "invalid parameters");
    ctx->prm = *params;
    return 0;
}

int fmm_evaluate(fmm_ctx* ctx, int64_t n, const double* x, const double* mu, double G, const double* scale,
                 double* psi, double* acc, void* stream, fmm_stats* stats) {
    if (!ctx) return FMM_E_INVALID;
    ctx->err[0] = 0;
    if (n < 0 || n > 0x7fffffffLL) return fail(ctx, FMM_E_INVALID, "n out of range");
    if (n > 0 && (!x || !mu || !psi || !acc)) return fail(ctx, FMM_E_INVALID, "NULL buffer");
    if (!std::isfinite(G)) return fail(ctx, FMM_E_INVALID, "G is not finite");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, FMM_E_CUDA, "cudaSetDevice failed");
    return evaluate_device(ctx, (int)n, x, mu, G, scale, psi, acc, (cudaStream_t)stream, stats);
}

int fmm_evaluate_active(fmm_ctx* ctx, int64_t n, const double* x, const double* mu, double G, const double* scale,
                        const unsigned char* active, const double* eps_b, int reuse_tree, double* psi, double* acc,
                        double* tidal, void* stream, fmm_stats* stats) {
    if (!ctx) return FMM_E_INVALID;
    ctx->err[0] = 0;
    if (n < 0 || n > 0x7fffffffLL) return fail(ctx, FMM_E_INVALID, "n out of range");
    if (n > 0 && (!x || !mu || !psi || !acc)) return fail(ctx, FMM_E_INVALID, "NULL buffer");
    if (!std::isfinite(G)) return fail(ctx, FMM_E_INVALID, "G is not finite");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, FMM_E_CUDA, "cudaSetDevice failed");
    if (reuse_tree != 0 && reuse_tree != 1) return fail(ctx, FMM_E_INVALID, "reuse_tree must be 0 or 1");
    return evaluate_device(ctx, (int)n, x, mu, G, scale, psi, acc, (cudaStream_t)stream, stats, active,
                           reuse_tree != 0, eps_b, tidal);
}

int fmm_evaluate_host(fmm_ctx* ctx, int64_t n, const double* x, const double* mu, double G, double* psi, double* acc,
                      void* stream, fmm_stats* stats) {
    if (!ctx) return FMM_E_INVALID;
    ctx->err[0] = 0;
    if (n < 0 || n > 0x7fffffffLL) return fail(ctx, FMM_E_INVALID, "n out of range");
    if (n == 0) return 0;
    if (!x || !mu || !psi || !acc) return fail(ctx, FMM_E_INVALID, "NULL buffer");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, FMM_E_CUDA, "cudaSetDevice failed");
    cudaStream_t s = (cudaStream_t)stream;
    TRY(ensure(ctx->hx, sizeof(double) * 3 * (size_t)n));
    TRY(ensure(ctx->hmu, sizeof(double) * (size_t)n));
    TRY(ensure(ctx->hpsi, sizeof(double) * (size_t)n));
    TRY(ensure(ctx->hacc, sizeof(double) * 3 * (size_t)n));
    CU(cudaMemcpyAsync(ctx->hx.p, x, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(ctx->hmu.p, mu, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, s));
    int rc = evaluate_device(ctx, (int)n, P<double>(ctx->hx), P<double>(ctx->hmu), G, nullptr, P<double>(ctx->hpsi),
                             P<double>(ctx->hacc), s, stats);
    if (rc) return rc;
    CU(cudaMemcpyAsync(psi, ctx->hpsi.p, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(acc, ctx->hacc.p, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return 0;
}

int fmm_direct(fmm_ctx* ctx, int64_t n, const double* x, const double* mu, double G, int64_t nsinks,
               const int64_t* sinks, double* psi, double* acc, double* f, void* stream) {
    if (!ctx) return FMM_E_INVALID;
    ctx->err[0] = 0;
    if (n < 0 || n > 0x7fffffffLL) return fail(ctx, FMM_E_INVALID, "n out of range");
    if (!sinks) nsinks = n;
    if (nsinks < 0 || nsinks > 0x7fffffffLL) return fail(ctx, FMM_E_INVALID, "nsinks out of range");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, FMM_E_CUDA, "cudaSetDevice failed");
    launch_direct(x, mu, (int)n, G, sinks, (int)nsinks, psi, acc, f, (cudaStream_t)stream);
    CU(cudaGetLastError());
    return 0;
}

int fmm_evaluate_batch(fmm_ctx* ctx, int nsys, const int64_t* offsets, const double* x, const double* mu,
                       const double* G, double* psi, double* acc, void* stream, fmm_stats* stats) {
    if (!ctx || nsys < 0 || (nsys > 0 && (!offsets || !G))) return FMM_E_INVALID;
    if (nsys == 0) {
        if (stats) memset(stats, 0, sizeof *stats);
        return 0;
    }
    ctx->err[0] = 0;
    if (offsets[0] != 0) return fail(ctx, FMM_E_INVALID, "offsets[0] must be 0");
    for (int k = 0; k < nsys; ++k)
        if (!std::isfinite(G[k])) return fail(ctx, FMM_E_INVALID, "G is not finite");
    std::vector<int> off(nsys + 1);
    std::vector<int2> roots;
    for (int k = 0; k < nsys; ++k) {
        if (offsets[k + 1] < offsets[k]) return fail(ctx, FMM_E_INVALID, "offsets not increasing");
        if (offsets[k + 1] > (int64_t)INT32_MAX) return fail(ctx, FMM_E_INVALID, "more than 2^31-1 particles in all");
        off[k] = (int)offsets[k];
        if (offsets[k + 1] > offsets[k]) roots.push_back(make_int2((int)offsets[k], (int)(offsets[k + 1] - offsets[k])));
    }
    off[nsys] = (int)offsets[nsys];
    const int n = off[nsys];
    if (nsys == 1) return fmm_evaluate(ctx, n, x, mu, G[0], nullptr, psi, acc, stream, stats);
    if (n > 0 && (!x || !mu || !psi || !acc)) return fail(ctx, FMM_E_INVALID, "null array");
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, FMM_E_CUDA, "cudaSetDevice failed");
    TRY(ensure(ctx->sys_off, sizeof(int) * (nsys + 1)));
    TRY(ensure(ctx->sys_G, sizeof(double) * nsys));
    TRY(ensure(ctx->sys_roots, sizeof(int2) * std::max<size_t>(1, roots.size())));
    CU(cudaMemcpyAsync(ctx->sys_off.p, off.data(), sizeof(int) * (nsys + 1), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(ctx->sys_G.p, G, sizeof(double) * nsys, cudaMemcpyHostToDevice, s));
    if (!roots.empty())
        CU(cudaMemcpyAsync(ctx->sys_roots.p, roots.data(), sizeof(int2) * roots.size(), cudaMemcpyHostToDevice, s));
    // the host arrays above are pageable and local: wait for the copies before returning
    ctx->nsys = nsys;
    ctx->nroots = (int)roots.size();
    int rc = evaluate_device(ctx, n, x, mu, 1.0, nullptr, psi, acc, s, stats);
    cudaError_t e = cudaStreamSynchronize(s);
    ctx->nsys = 0;
    ctx->nroots = 1;
    if (rc) return rc;
    if (e != cudaSuccess) return fail(ctx, FMM_E_CUDA, cudaGetErrorString(e));
    return 0;
}

int fmm_debug_m2l_orders(fmm_ctx* ctx, int32_t* q) {
    if (!ctx || !q) return FMM_E_INVALID;
    const long long cnt = ctx->n_m2l;
    if (cnt <= 0) return 0;
    CU(cudaDeviceSynchronize());
    std::vector<int2> v(cnt);
    CU(cudaMemcpy(v.data(), ctx->m2l.p, sizeof(int2) * cnt, cudaMemcpyDeviceToHost));
    for (long long i = 0; i < cnt; ++i) q[i] = m2l_order(v[i].x, ctx->prm.p);
    return 0;
}

int fmm_debug_dump(fmm_ctx* ctx, int64_t* cells_int, double* cells_dbl, int64_t* m2l, int64_t* p2p, int64_t* perm,
                   double* scale_sorted) {
    if (!ctx) return FMM_E_INVALID;
    const int nc = ctx->ncells, n = ctx->n;
    CU(cudaDeviceSynchronize());
    // the caller's units: lengths 2^e0, masses 2^e1, scales (accelerations) 2^(e1 - 2 e0)
    int e[2] = {0, 0};
    if (ctx->units.p) CU(cudaMemcpy(e, ctx->units.p, sizeof e, cudaMemcpyDeviceToHost));
    if (cells_int || cells_dbl) {
        std::vector<int> lv(nc), fi(nc), co(nc), nch(nc);
        std::vector<d4> sr(nc);
        std::vector<double> ms(nc), mn(nc);
        if (nc) {
            CU(cudaMemcpy(lv.data(), ctx->level.p, sizeof(int) * nc, cudaMemcpyDeviceToHost));
            CU(cudaMemcpy(fi.data(), ctx->first.p, sizeof(int) * nc, cudaMemcpyDeviceToHost));
            CU(cudaMemcpy(co.data(), ctx->count.p, sizeof(int) * nc, cudaMemcpyDeviceToHost));
            CU(cudaMemcpy(nch.data(), ctx->nchild.p, sizeof(int) * nc, cudaMemcpyDeviceToHost));
            CU(cudaMemcpy(sr.data(), ctx->sr.p, sizeof(d4) * nc, cudaMemcpyDeviceToHost));
            CU(cudaMemcpy(ms.data(), ctx->mass.p, sizeof(double) * nc, cudaMemcpyDeviceToHost));
            CU(cudaMemcpy(mn.data(), ctx->minscale.p, sizeof(double) * nc, cudaMemcpyDeviceToHost));
        }
        for (int i = 0; i < nc; ++i) {
            if (cells_int) {
                cells_int[5 * i] = lv[i];
                cells_int[5 * i + 1] = nch[i] == 0;
                cells_int[5 * i + 2] = fi[i];
                cells_int[5 * i + 3] = co[i];
                cells_int[5 * i + 4] = nch[i];
            }
            if (cells_dbl) {
                cells_dbl[6 * i] = std::ldexp(sr[i].x, e[0]);
                cells_dbl[6 * i + 1] = std::ldexp(sr[i].y, e[0]);
                cells_dbl[6 * i + 2] = std::ldexp(sr[i].z, e[0]);
                cells_dbl[6 * i + 3] = std::ldexp(sr[i].w, e[0]);
                cells_dbl[6 * i + 4] = std::ldexp(ms[i], e[1]);
                cells_dbl[6 * i + 5] = std::ldexp(mn[i], e[1] - 2 * e[0]);
            }
        }
    }
    auto dump_list = [&](Buf& b, long long cnt, int64_t* out) -> int {
        if (!out || cnt <= 0) return 0;
        std::vector<int2> v(cnt);
        GB3_CUDA_TRY(cudaMemcpy(v.data(), b.p, sizeof(int2) * cnt, cudaMemcpyDeviceToHost));
        for (long long i = 0; i < cnt; ++i) {
            out[2 * i] = m2l_src(v[i].x);
            out[2 * i + 1] = v[i].y;
        }
        return 0;
    };
    TRY(dump_list(ctx->m2l, ctx->n_m2l, m2l));
    TRY(dump_list(ctx->p2p, ctx->n_p2p, p2p));
    if (perm && n) {
        std::vector<int> pv(n);
        CU(cudaMemcpy(pv.data(), ctx->perm.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
        for (int i = 0; i < n; ++i) perm[i] = pv[i];
    }
    if (scale_sorted && n && ctx->scale_sorted.p) {
        CU(cudaMemcpy(scale_sorted, ctx->scale_sorted.p, sizeof(double) * n, cudaMemcpyDeviceToHost));
        for (int i = 0; i < n; ++i) scale_sorted[i] = std::ldexp(scale_sorted[i], e[1] - 2 * e[0]);
    }
    return 0;
}

int fmm_last_stats(fmm_ctx* ctx, fmm_stats* out) {
    if (!ctx || !out) return FMM_E_INVALID;
    TRY(phase_times(ctx));
    *out = ctx->last;
    return 0;
}

int fmm_alu_peaks(double* fp64_tflops, double* fp32_tflops) {
    if (!fp64_tflops || !fp32_tflops) return FMM_E_INVALID;
    return alu_peaks(fp64_tflops, fp32_tflops);
}

int fmm_pair_peak(int warps_per_sm, double* gpairs_s) { return pair_peak(warps_per_sm, gpairs_s); }

int fmm_swap_probe(int npairs, int reps, double* ms, double* maxdiff) {
    return swap_probe(npairs, reps, ms, maxdiff);
}

uint64_t fmm_workspace_bytes(fmm_ctx* ctx) {
    if (!ctx) return 0;
    uint64_t b = 0;
    for (Buf* x : ctx->bufs()) b += x->bytes;
    return b + serve_workspace_bytes(ctx->serve);
}

// Workspace bound for n particles.  The particle and cell arrays follow from the
// allocation sizes (with the 25 % growth of every buffer); the interaction lists,
// their sort scratch and the M2L partial sums depend on the input and on (p, eps,
// leaf), so they are bounded per cell with allowances measured on truncated Plummer
// spheres and gamma = 1.5 cusps from 2e3 to 1e6 particles over p = 4..16,
// eps = 1e-4..1e-9, leaf = 8..64 (cells <= 4.7 n / leaf; per cell at most ~160 M2L,
// ~490 P2P, ~13 estimate-M2L and ~41 estimate-P2P pairs), with a margin.
constexpr double kCellsPerLeafN = 4.7;      // cells built <= this * n / leaf + 64
constexpr double kM2LPerCell = 200.0;       // main M2L pairs per cell
constexpr double kP2PPerCell = 600.0;       // main P2P pairs per cell
constexpr double kEstPerCell = 64.0;        // estimate M2L + P2P pairs per cell
constexpr double kPairBytes = 50.0;         // list entry with growth slack + sort scratch

int64_t fmm_footprint_bytes(const fmm_params* prm, int64_t n) {
    fmm_params d;
    if (!prm) {
        fmm_default_params(&d);
        prm = &d;
    }
    if (n < 0 || check_params(prm)) return -1;
    const double leaf = prm->leaf_size, P = (prm->p + 1.0) * (prm->p + 1.0), nd = (double)n;
    // particle arrays (sorted copies, keys, two-float positions, near/far results,
    // ensemble sort keys, owning cells of the radii pass, a serving slot's staging)
    const double particles = 1.25 * 268.0 * nd;
    // cell arrays sized by the cell capacity n + 21 n / (leaf + 1)
    const double cap = nd + 21.0 * std::floor(nd / (leaf + 1.0)) + 64.0;
    const double cellcap = 1.25 * 104.0 * cap;
    // per cell built: M, F, their FP32/FP64 split copies and M2L scratch, power,
    // the low-order estimate, the walk's single-precision view (<= 128 B), the radii
    // scratch (72 B) and per-cell scratch; then the lists
    const double cells = kCellsPerLeafN * nd / leaf + 64.0;
    const double per_cell = 1.25 * 48.0 * P + 2200.0 + kM2LPerCell * (kPairBytes + 1.25 * 8.0 * P / 32.0) +
                            (kP2PPerCell + kEstPerCell) * kPairBytes;
    return (int64_t)(particles + cellcap + per_cell * cells) + (int64_t)(16 << 20);
}

int fmm_destroy(fmm_ctx* ctx) {
    if (!ctx) return 0;
    cudaSetDevice(ctx->device);
    if (ctx->serve) serve_destroy(ctx->serve);
    for (Buf* b : ctx->bufs()) release(*b);
    if (ctx->h_counters) cudaFreeHost(ctx->h_counters);
    if (ctx->h_int) cudaFreeHost(ctx->h_int);
    if (ctx->ev_ok)
        for (int i = 0; i < EV_N; ++i) cudaEventDestroy(ctx->ev[i]);
    if (ctx->s2) cudaStreamSynchronize(ctx->s2);
    if (ctx->s_hi) cudaStreamSynchronize(ctx->s_hi);
    if (ctx->s3) cudaStreamSynchronize(ctx->s3);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_join_est) cudaEventDestroy(ctx->ev_join_est);
    if (ctx->ev_est_fork) cudaEventDestroy(ctx->ev_est_fork);
    if (ctx->ev_est_m2l) cudaEventDestroy(ctx->ev_est_m2l);
    if (ctx->ev_join3) cudaEventDestroy(ctx->ev_join3);
    if (ctx->s2) cudaStreamDestroy(ctx->s2);
    if (ctx->s_hi) cudaStreamDestroy(ctx->s_hi);
    if (ctx->s3) cudaStreamDestroy(ctx->s3);
    delete ctx;
    return 0;
}

const char* fmm_strerror(int code) {
    switch (code) {
        case FMM_OK: return "ok";
        case FMM_E_INVALID: return "invalid argument or input";
        case FMM_E_OOM: return "device allocation failed";
        case FMM_E_ADMISSION: return "footprint above the memory budget";
        case FMM_E_CUDA: return "CUDA runtime error";
        case FMM_E_TIMEOUT: return "bounded wait ran out";
        case FMM_E_OVERFLOW: return "internal capacity exceeded";
        case FMM_E_NOTFOUND: return "unknown system or ticket";
        case FMM_E_BUSY: return "not finished";
        default: return "unknown error";
    }
}

const char* fmm_last_error(fmm_ctx* ctx) { return ctx ? ctx->err : ""; }

const char* fmm_version(void) { return "gb3fmm 0.1 (sm_103a)"; }

}  // extern "C"
