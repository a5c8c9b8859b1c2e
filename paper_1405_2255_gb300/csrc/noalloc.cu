// noalloc.cu -- fmm_evaluate_noalloc: the force evaluation of fmm_evaluate for
// small systems, with every piece of scratch memory taken from one fixed array
// in device global memory instead of from cudaMalloc.
//
// Some callers cannot allocate device memory: simulation codes whose memory is
// owned by their own pool allocator, and plugins that are not allowed to grow the
// process's device footprint.  This entry point lets them evaluate systems of up
// to kNoAllocMaxN particles.  It waits for its stream several times (level sizes
// and frontier lengths are read on the host), like fmm_evaluate.
//
// The scratch array is a file-scope __device__ variable: every GPU that loads
// the library holds it (kNoAllocBytes) until the process exits.  Host code cannot
// pass the variable itself to a kernel (in host code its name is only a host-side
// stand-in); its device address is looked up once per device with
// cudaGetSymbolAddress, while that device is current, on the first call made on
// that device.  That first call should therefore come before any stream capture.
// All calls share the one array and it keeps the previous call's contents, so
// everything that must start at zero is cleared here; two calls whose work
// overlaps on the GPU (different streams, or different host threads) race on it
// and give wrong results: serialise them.
#include <cmath>
#include <mutex>
#include <stdio.h>
#include <string.h>

#include "kernels.cuh"

namespace gb3 {
extern thread_local char g_cuda_msg[256];
}
using namespace gb3;

namespace {

constexpr int kNoAllocMaxN = 8192;
constexpr size_t kNoAllocBytes = 32u << 20;  // 32 MiB
constexpr int kMaxDevices = 64;
constexpr int kMaxLevels = 24;
constexpr long long kFrontCap = 192 * 1024, kListCap = 192 * 1024, kEstCap = 96 * 1024;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// bump allocation inside the static array
struct Arena {
    unsigned char* base;
    size_t used = 0;
    bool ok = true;
    template <class T>
    T* take(size_t count) {
        size_t off = (used + 255) & ~(size_t)255;
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        if (off + bytes > kNoAllocBytes) {
            ok = false;
            return nullptr;
        }
        used = off + bytes;
        return (T*)(base + off);
    }
};

int scratch_for_current_device(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FMM_E_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return FMM_E_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return 0;
}

__global__ void k_root_na(Cells c, int n) {
    c.first[0] = 0;
    c.count[0] = n;
    c.level[0] = 0;
    c.parent[0] = -1;
    c.child[0] = -1;
    c.nchild[0] = 0;
}
__global__ void k_leaf_flags_na(const int* __restrict__ nchild, int nc, int* __restrict__ flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) flag[i] = nchild[i] == 0;
}
__global__ void k_leaf_compact_na(const int* __restrict__ flag, const int* __restrict__ pos, int nc,
                                  int* __restrict__ leaves) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
        if (flag[i]) leaves[pos[i]] = i;
}

struct Run {
    Arena a;
    cudaStream_t s;
    const char* err = "";
    int n = 0, nc = 0, nleaves = 0, nlev = 0;
    int lev[kMaxLevels + 2];
    Cells c;
    d4* xm = nullptr;
    int* perm = nullptr;
    uint64_t* keys = nullptr;
    int* leaves = nullptr;
    unsigned long long* counters = nullptr;
    unsigned* status = nullptr;
    int* dtotal = nullptr;
    int2 *front0 = nullptr, *front1 = nullptr;
    void* sort_tmp = nullptr;
    void* p2p_tmp = nullptr;
    size_t p2p_tmp_bytes = 0;
};

int fail_na(Run& r, int code, const char* msg) {
    r.err = msg;
    return code;
}

#define NA_CU(expr)                                         \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) {                            \
            cudaGetLastError();                             \
            return fail_na(r, FMM_E_CUDA, #expr " failed"); \
        }                                                   \
    } while (0)

// one breadth-first walk into fixed-capacity lists
int walk_na(Run& r, WalkParams wp, int2* m2l, long long m2l_cap, int2* p2p, long long p2p_cap, long long* nm,
            long long* np) {
    WalkBuffers wb;
    wb.front[0] = r.front0;
    wb.front[1] = r.front1;
    wb.front_cap = kFrontCap;
    wb.m2l = m2l;
    wb.m2l_cap = m2l_cap;
    wb.p2p = p2p;
    wb.p2p_cap = p2p_cap;
    wb.counters = r.counters;
    int2 root = make_int2(0, 0);
    NA_CU(cudaMemcpyAsync(wb.front[0], &root, sizeof root, cudaMemcpyHostToDevice, r.s));
    NA_CU(cudaMemsetAsync(wb.counters, 0, 4 * sizeof(unsigned long long), r.s));
    long long nfront = 1;
    int cur = 0;
    unsigned long long h[4];
    while (nfront > 0) {
        NA_CU(cudaMemsetAsync(wb.counters, 0, sizeof(unsigned long long), r.s));
        launch_walk_step(r.c, wp, wb.front[cur], nfront, wb.front[cur ^ 1], wb, r.s);
        NA_CU(cudaMemcpyAsync(h, wb.counters, sizeof h, cudaMemcpyDeviceToHost, r.s));
        NA_CU(cudaStreamSynchronize(r.s));
        if (h[3]) return fail_na(r, FMM_E_OVERFLOW, "interaction lists exceed the static scratch capacity");
        nfront = (long long)h[0];
        cur ^= 1;
    }
    *nm = (long long)h[1];
    *np = (long long)h[2];
    return 0;
}

// mixed P2P with its work plan in the rest of the static array (shared with the list sorts)
int p2p_na(Run& r, const float4* xp, const int2* list, const int* seg_start, const int* seg_end,
           double* psi, double* acc, int mode) {
    unsigned long long h_tot[6] = {0, 0, 0, 0, 0, 0};
    const size_t have = r.p2p_tmp_bytes;
    const size_t need = launch_p2p_mixed(xp, r.n, r.c, list, seg_start, seg_end, r.leaves, r.nleaves, psi, acc,
                                         mode, r.p2p_tmp, have, h_tot, r.s);
    if (need > have) return fail_na(r, FMM_E_OVERFLOW, "the P2P work plan exceeds the static scratch capacity");
    return 0;
}

int evaluate_na(Run& r, const fmm_params& prm, const double* x, const double* mu, double G, double* psi, double* acc) {
    const int n = r.n;
    Arena& A = r.a;
    cudaStream_t s = r.s;
    // particles and sort
    r.keys = A.take<uint64_t>(n);
    uint64_t* keys_alt = A.take<uint64_t>(n);
    int* idx = A.take<int>(n);
    int* idx_alt = A.take<int>(n);
    int* rtmp = A.take<int>(radix_tmp_ints(n));
    r.xm = A.take<d4>(n);
    r.perm = A.take<int>(n);
    unsigned long long* bounds = A.take<unsigned long long>(8);
    r.status = A.take<unsigned>(4);
    r.counters = A.take<unsigned long long>(8);
    r.dtotal = A.take<int>(4);
    const long long cap = (long long)n + 21LL * (n / (prm.leaf_size + 1)) + 64;
    int* ib[6];
    for (int k = 0; k < 6; ++k) ib[k] = A.take<int>(cap);
    r.c.first = ib[0]; r.c.count = ib[1]; r.c.child = ib[2]; r.c.nchild = ib[3]; r.c.parent = ib[4]; r.c.level = ib[5];
    r.c.sr = A.take<d4>(cap);
    r.c.cr = A.take<d4>(cap);
    r.c.mass = A.take<double>(cap);
    r.c.minscale = A.take<double>(cap);
    int* split_nchild = A.take<int>(cap);
    int* split_oct = A.take<int>(9 * cap);
    int* split_offs = A.take<int>(cap);
    int* scan_tmp = A.take<int>(scan_tmp_ints(cap));
    if (!A.ok) return fail_na(r, FMM_E_OVERFLOW, "static scratch too small for the particle arrays");
    NA_CU(cudaMemsetAsync(r.status, 0, sizeof(unsigned), s));
    // working units of the mixed path (positions and masses scaled by powers of two)
    int* units = A.take<int>(2);
    if (!A.ok) return fail_na(r, FMM_E_OVERFLOW, "static scratch too small for the particle arrays");
    launch_bounds(x, mu, n, bounds, r.status, s);
    if (prm.precision == FMM_PREC_MIXED) launch_work_units(bounds, 0, units, s);
    else NA_CU(cudaMemsetAsync(units, 0, 2 * sizeof(int), s));
    launch_keys(x, n, bounds, r.keys, idx, s);
    radix_sort_pairs(r.keys, idx, keys_alt, idx_alt, n, rtmp, s);
    launch_gather(x, mu, idx, n, r.xm, r.perm, s, units);
    k_root_na<<<1, 1, 0, s>>>(r.c, n);
    note_launch();
    // top-down levels
    r.lev[0] = 0;
    r.lev[1] = 1;
    int nl = 1;
    for (int L = 0;; ++L) {
        int b = r.lev[L], e = r.lev[L + 1];
        if (e - b <= 0) break;
        launch_split_level(r.keys, r.c, b, e, L, prm.leaf_size, split_nchild, split_oct, split_offs, scan_tmp,
                           r.dtotal, s);
        int tot = 0;
        NA_CU(cudaMemcpyAsync(&tot, r.dtotal, sizeof tot, cudaMemcpyDeviceToHost, s));
        NA_CU(cudaStreamSynchronize(s));
        if (tot <= 0) break;
        if ((long long)e + tot > cap || nl + 1 > kMaxLevels) return fail_na(r, FMM_E_OVERFLOW, "cell capacity exceeded");
        r.lev[++nl] = e + tot;
    }
    r.nlev = nl;
    r.nc = r.lev[nl];
    const int nc = r.nc;
    int* leaf_flag = A.take<int>(nc);
    int* leaf_pos = A.take<int>(nc);
    r.leaves = A.take<int>(nc);
    unsigned long long* rad_tmp = A.take<unsigned long long>(rad_tmp_u64_per_cell() * (size_t)nc);
    if (!A.ok) return fail_na(r, FMM_E_OVERFLOW, "static scratch too small for the tree");
    k_leaf_flags_na<<<grid_for(nc, 256), 256, 0, s>>>(r.c.nchild, nc, leaf_flag);
    note_launch();
    scan_exclusive_i32(leaf_flag, leaf_pos, nc, r.dtotal, scan_tmp, s);
    k_leaf_compact_na<<<grid_for(nc, 256), 256, 0, s>>>(leaf_flag, leaf_pos, nc, r.leaves);
    note_launch();
    unsigned st = 0;
    NA_CU(cudaMemcpyAsync(&r.nleaves, r.dtotal, sizeof(int), cudaMemcpyDeviceToHost, s));
    NA_CU(cudaMemcpyAsync(&st, r.status, sizeof st, cudaMemcpyDeviceToHost, s));
    NA_CU(cudaStreamSynchronize(s));
    if (st & kStatInvalid) return fail_na(r, FMM_E_INVALID, "non-finite position or mass, or negative mass");
    // two-float positions: the internal radii's single-precision bounds and the mixed P2P
    float4* xp = A.take<float4>(2 * (size_t)n);  // two records per particle: hi and mass, lo
    if (!A.ok) return fail_na(r, FMM_E_OVERFLOW, "static scratch too small for the tree");
    int* owner = A.take<int>(n);
    if (!A.ok) return fail_na(r, FMM_E_OVERFLOW, "static scratch too small for the tree");
    launch_split_positions(r.xm, n, xp, s);
    launch_leaf_geometry(r.xm, r.c, r.leaves, r.nleaves, r.status, s);
    launch_leaf_owner(r.c, r.leaves, r.nleaves, owner, s);
    for (int L = nl - 1; L >= 0; --L)
        launch_internal_geometry(r.xm, xp, r.c, r.lev[L], r.lev[L + 1], n, owner, rad_tmp, r.status, s);

    // per-particle results and lists
    double* psi_far = A.take<double>(n);
    double* acc_far = A.take<double>(3 * (size_t)n);
    double* psi_near = A.take<double>(n);
    double* acc_near = A.take<double>(3 * (size_t)n);
    double* scale = A.take<double>(n);
    r.front0 = A.take<int2>(kFrontCap);
    r.front1 = A.take<int2>(kFrontCap);
    int2* m2l = A.take<int2>(kListCap);
    int2* p2p = A.take<int2>(kListCap);
    int2* est_m2l = A.take<int2>(kEstCap);
    int2* est_p2p = A.take<int2>(kEstCap);
    int* m2l_seg_start = A.take<int>(nc);
    int* m2l_seg_end = A.take<int>(nc);
    int* seg_start = A.take<int>(nc);
    int* seg_end = A.take<int>(nc);
    const int p = prm.p, nco = ncoef(p);
    double* M = A.take<double>((size_t)nco * nc);
    double* F = A.take<double>((size_t)nco * nc);
    double* Pw = A.take<double>((size_t)(p + 1) * nc);
    double* binom = A.take<double>(kMaxP + 1);
    double* F1 = A.take<double>(4 * (size_t)nc);
    double* Ff = A.take<double>(nc);
    float4* walkf = A.take<float4>((size_t)(2 + walk_fstride(p) / 4) * nc);
    void* m2l_tmp = A.take<unsigned char>(m2l_split_tmp_bytes(nc, p > 1 ? p : 1, kListCap));
    if (!A.ok) return fail_na(r, FMM_E_OVERFLOW, "static scratch too small for the expansions and lists");
    // the rest of the array serves the list sorts and, once a list is sorted, the mixed P2P's
    // work plan (the two never overlap on the stream)
    const size_t used = (A.used + 255) & ~(size_t)255;
    r.p2p_tmp_bytes = used < kNoAllocBytes ? kNoAllocBytes - used : 0;
    if (r.p2p_tmp_bytes < list_sort_tmp_bytes(kListCap, (int)cap))
        return fail_na(r, FMM_E_OVERFLOW, "static scratch too small for the list sorts");
    r.p2p_tmp = A.take<unsigned char>(r.p2p_tmp_bytes);
    r.sort_tmp = r.p2p_tmp;

    // A7: scale estimate and its per-cell minimum
    if (prm.mac != FMM_MAC_THETA) {
        const bool want_f = prm.mac == FMM_MAC_F;
        WalkParams ew;
        memset(&ew, 0, sizeof ew);
        ew.p = want_f ? 0 : 1;
        ew.mac = kMacEstimate;
        ew.p2p_thresh = prm.p2p_c * (double)ew.p * ew.p * ew.p;  // the estimate's own order
        ew.use_com = 1;
        ew.fc = walkf;
        launch_walk_prep(r.c, r.c.cr, nullptr, 0, 0.0, nc, walkf, nullptr, s);
        long long nm = 0, np = 0;
        int rc = walk_na(r, ew, est_m2l, kEstCap, est_p2p, kEstCap, &nm, &np);
        if (rc) return rc;
        sort_pairs_by_sink(est_m2l, nm, nc, r.sort_tmp, s);
        launch_segments(est_m2l, nm, nc, m2l_seg_start, m2l_seg_end, s);
        sort_pairs_by_sink(est_p2p, np, nc, r.sort_tmp, s);
        launch_segments(est_p2p, np, nc, seg_start, seg_end, s);
        if (want_f) {
            launch_f_m2l(est_m2l, m2l_seg_start, m2l_seg_end, nc, r.c, Ff, s);
            for (int L = 1; L < nl; ++L) launch_f_down_level(r.c, r.lev[L], r.lev[L + 1], Ff, s);
            launch_f_p2p(r.xm, r.c, est_p2p, seg_start, seg_end, r.leaves, r.nleaves, Ff, scale, s);
        } else {
            // the estimate's monopole M2L about the centres of mass, as fmm_evaluate takes it
            // (FP32 from the walk's single-precision view in mixed mode)
            launch_est_m2l(est_m2l, m2l_seg_start, m2l_seg_end, nc, r.c, F1, s,
                           prm.precision == FMM_PREC_MIXED ? walkf : nullptr);
            // (the p = 1 L2L is folded into launch_est_scale)
            if (prm.precision == FMM_PREC_MIXED) {
                rc = p2p_na(r, xp, est_p2p, seg_start, seg_end, psi_near, acc_near, 0);
                if (rc) return rc;
            } else
                launch_p2p_fp64(r.xm, r.c, est_p2p, seg_start, seg_end, r.leaves, r.nleaves, psi_near, acc_near, s);
            launch_est_scale(r.c, r.leaves, r.nleaves, F1, acc_near, scale, s);
        }
        launch_minscale_leaves(scale, r.c, r.leaves, r.nleaves, s);
        for (int L = nl - 1; L >= 0; --L) launch_minscale_level(r.c, r.lev[L], r.lev[L + 1], s);
    }

    // A5-A6: upward pass
    double bn[kMaxP + 1];
    bn[0] = 1;
    for (int k = 1; k <= p; ++k) bn[k] = bn[k - 1] * (p - k + 1) / k;
    NA_CU(cudaMemcpyAsync(binom, bn, sizeof(double) * (p + 1), cudaMemcpyHostToDevice, s));
    const bool split = prm.precision == FMM_PREC_MIXED && prm.m2l_split;
    if (split) launch_p2m_split(r.xm, r.c, r.c.sr, r.leaves, r.nleaves, p, M, s);
    else launch_p2m(r.xm, r.c, r.c.sr, r.leaves, r.nleaves, p, M, s);
    for (int L = nl - 1; L >= 0; --L) {
        if (split) launch_m2m_split(r.c, r.c.sr, r.lev[L], r.lev[L + 1], p, M, s);
        else launch_m2m_level(r.c, r.c.sr, r.lev[L], r.lev[L + 1], p, M, s);
    }
    launch_power(M, nc, p, Pw, s);

    // A8: dual tree walk
    WalkParams wp;
    memset(&wp, 0, sizeof wp);
    wp.p = p;
    wp.mac = prm.mac;
    wp.eps = prm.eps;
    wp.theta_crit = prm.theta_crit;
    wp.p2p_thresh = prm.p2p_c * (double)p * p * p;
    wp.P = Pw;
    wp.binom = binom;
    wp.use_com = 0;
    wp.adaptive = 0;  // this path keeps every interaction at p
    wp.p_lo = p;
    wp.pascal = nullptr;
    if (prm.mac != FMM_MAC_THETA) {
        wp.fc = walkf;
        wp.fP = (const float*)(walkf + 2 * (size_t)nc);
        wp.fstride = walk_fstride(p);
        launch_walk_prep(r.c, r.c.sr, Pw, p, prm.eps, nc, walkf, (float*)(walkf + 2 * (size_t)nc), s);
    }
    long long nm = 0, np = 0;
    int rc = walk_na(r, wp, m2l, kListCap, p2p, kListCap, &nm, &np);
    if (rc) return rc;
    sort_pairs_by_sink(m2l, nm, nc, r.sort_tmp, s);
    launch_segments(m2l, nm, nc, m2l_seg_start, m2l_seg_end, s);

    // A9-A12
    NA_CU(cudaMemsetAsync(F, 0, sizeof(double) * nco * (size_t)nc, s));
    if (split)
        launch_m2l_split(m2l, m2l_seg_start, m2l_seg_end, m2l_tmp, nc, r.c.sr, M, p, F, prm.m2l_rot != 0, s, false, nm);
    else
        launch_m2l(m2l, m2l_seg_start, m2l_seg_end, m2l_tmp, nc, r.c.sr, M, p, F, s);
    sort_pairs_by_sink(p2p, np, nc, r.sort_tmp, s);
    launch_segments(p2p, np, nc, seg_start, seg_end, s);
    if (prm.precision == FMM_PREC_MIXED) {
        rc = p2p_na(r, xp, p2p, seg_start, seg_end, psi_near, acc_near, prm.p2p_two_float);
        if (rc) return rc;
    } else
        launch_p2p_fp64(r.xm, r.c, p2p, seg_start, seg_end, r.leaves, r.nleaves, psi_near, acc_near, s);
    for (int L = 1; L < nl; ++L) {
        if (split) launch_l2l_split(r.c, r.c.sr, r.lev[L], r.lev[L + 1], p, F, s);
        else launch_l2l_level(r.c, r.c.sr, r.lev[L], r.lev[L + 1], p, F, s);
    }
    if (split) launch_l2p_split(r.xm, r.c, r.c.sr, r.leaves, r.nleaves, p, F, psi_far, acc_far, s);
    else launch_l2p(r.xm, r.c, r.c.sr, r.leaves, r.nleaves, p, F, psi_far, acc_far, s);
    launch_finish(psi_far, acc_far, psi_near, acc_near, r.perm, n, G, psi, acc, s, nullptr, nullptr, 0, nullptr,
                  units);
    NA_CU(cudaGetLastError());
    return 0;
}

}  // namespace

extern "C" int fmm_evaluate_noalloc(int64_t n, const double* x, const double* mu, double G, const fmm_params* params,
                                    double* psi, double* acc, void* stream, char* errbuf, int errlen) {
    Run r;
    int rc = 0;
    auto report = [&](int code) {
        if (errbuf && errlen > 0) snprintf(errbuf, (size_t)errlen, "%s", code ? r.err : "");
        return code;
    };
    if (!params) return report(fail_na(r, FMM_E_INVALID, "params == NULL"));
    const fmm_params& prm = *params;
    if (prm.p < 1 || prm.p > 10) return report(fail_na(r, FMM_E_INVALID, "p must be in [1, 10] here"));
    if (prm.mac != FMM_MAC_A && prm.mac != FMM_MAC_F && prm.mac != FMM_MAC_THETA)
        return report(fail_na(r, FMM_E_INVALID, "unknown mac"));
    if (prm.mac != FMM_MAC_THETA && !(prm.eps > 0)) return report(fail_na(r, FMM_E_INVALID, "eps must be > 0"));
    if (prm.mac == FMM_MAC_THETA && !(prm.theta_crit > 0 && prm.theta_crit < 1))
        return report(fail_na(r, FMM_E_INVALID, "theta_crit must be in (0,1)"));
    if (prm.leaf_size < 24 || prm.leaf_size > 4096)
        return report(fail_na(r, FMM_E_INVALID, "leaf_size must be in [24, 4096] here"));
    if (prm.precision != FMM_PREC_FP64 && prm.precision != FMM_PREC_MIXED)
        return report(fail_na(r, FMM_E_INVALID, "unknown precision"));
    if (prm.scale_src != FMM_SCALE_ESTIMATE)
        return report(fail_na(r, FMM_E_INVALID, "only the low-order scale estimate is supported here"));
    if (!(prm.p2p_c >= 0)) return report(fail_na(r, FMM_E_INVALID, "p2p_c must be >= 0"));
    if (n < 0 || n > kNoAllocMaxN)
        return report(fail_na(r, FMM_E_INVALID, "n exceeds the static-scratch maximum of 8192 particles"));
    if (n == 0) return report(0);
    if (!x || !mu || !psi || !acc) return report(fail_na(r, FMM_E_INVALID, "NULL buffer"));
    if (!std::isfinite(G)) return report(fail_na(r, FMM_E_INVALID, "G is not finite"));
    void* base = nullptr;
    rc = scratch_for_current_device(&base);
    if (rc) return report(fail_na(r, rc, "cudaGetSymbolAddress of the static scratch failed"));
    r.a.base = (unsigned char*)base;
    r.s = (cudaStream_t)stream;
    r.n = (int)n;
    rc = evaluate_na(r, prm, x, mu, G, psi, acc);
    return report(rc);
}
