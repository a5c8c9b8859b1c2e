// kernels.cuh -- device data layout and the launchers of every phase of the path.
//
// Layout in HBM (all arrays owned by the context's workspace):
//   particles, sorted by Morton key:  xm[n] d4 (x, y, z, mu), perm[n] int
//   (sorted -> caller index), keys[n] uint64.
//   cells in breadth-first order (level by level, each level in key order):
//   first/count (particle range), child/nchild (daughters are contiguous),
//   parent, level; sr[c] d4 (s = z, rho), cr[c] d4 (centre of mass,
//   rho about it), mass[c], minscale[c]; expansions M[c][(p+1)^2] and
//   F[c][(p+1)^2] in the real storage of App. A.3.2; power P[c][p+1].
//   interaction lists: int2 (source cell, sink cell), sorted by (sink, source).
#pragma once
#include "common.cuh"

namespace gb3 {

struct Cells {
    int* first;
    int* count;
    int* child;
    int* nchild;
    int* parent;
    int* level;
    d4* sr;      // expansion centre s = z and radius rho (Sec. 4, Sec. 5.1.1)
    d4* cr;      // centre of mass and radius about it (low-order estimate)
    double* mass;
    double* minscale; // min over the cell's sinks of the MAC scale (eqs. 18a,b)
    // force evaluation for a subset of the particles (Sec. 7.1): act[cell] != 0 when the
    // cell holds an active particle, pact[i] != 0 for an active sorted particle i; both
    // nullptr when every particle is active
    const unsigned char* act = nullptr;
    const unsigned char* pact = nullptr;
};
__device__ __forceinline__ bool cell_active(const Cells& c, int cell) { return !c.act || c.act[cell]; }

// ---------------------------------------------------------------- tree (tree.cu)
// A1: bounding box + validation; bounds[6] = dbl_key of (min x,y,z, max x,y,z)
void launch_bounds(const double* x, const double* mu, int n, unsigned long long* bounds,
                   unsigned* status, cudaStream_t s);
// A2: Morton keys and the (key, index) radix sort; returns the buffers holding the result
void launch_keys(const double* x, int n, const unsigned long long* bounds, uint64_t* keys, int* idx,
                 cudaStream_t s);
size_t radix_tmp_ints(long long n);
// LSD passes over key bits [begin_bit, end_bit); returns 1 if the result is in the _alt buffers
int radix_sort_pairs_bits(uint64_t* keys, int* idx, uint64_t* keys_alt, int* idx_alt, long long n, int* tmp,
                          int begin_bit, int end_bit, cudaStream_t s);
void radix_sort_pairs(uint64_t* keys, int* idx, uint64_t* keys_alt, int* idx_alt, int n, int* tmp,
                      cudaStream_t s);
// e (nullable, device): positions enter scaled by 2^-e[0], masses by 2^-e[1] (launch_work_units)
void launch_gather(const double* x, const double* mu, const int* idx, int n, d4* xm, int* perm,
                   cudaStream_t s, const int* e = nullptr);
// working units of the mixed-precision path: e[0] = floor(log2 extent), e[1] = floor(log2 max mass)
// from the bounds of launch_bounds (nsys = 0; the largest mass in bounds[6]) or
// launch_bounds_sys (the largest mass in bounds[6 nsys])
void launch_work_units(const unsigned long long* bounds, int nsys, int* e, cudaStream_t s);
// A1-A2 for an ensemble of nsys systems, system k = caller particles [off[k], off[k+1])
// (off on the device): per-system bounds (bounds[6k..6k+5]) and keys in the system's
// own root cube; then a stable sort of the key-sorted (keys, idx) by system into
// (keys_out, idx_out), so that each system keeps its block and its key order.
void launch_bounds_sys(const double* x, const double* mu, int n, const int* off, int nsys,
                       unsigned long long* bounds, unsigned* status, cudaStream_t s);
void launch_keys_sys(const double* x, int n, const int* off, int nsys, const unsigned long long* bounds,
                     uint64_t* keys, int* idx, cudaStream_t s);
int sort_by_system(const uint64_t* keys, const int* idx, int n, const int* off, int nsys, uint64_t* skey,
                   uint64_t* skey_alt, int* pos, int* pos_alt, int* tmp, uint64_t* keys_out, int* idx_out,
                   cudaStream_t s);
// A3: one level of the top-down build.  Cells [lev_begin, lev_end) are split;
// nchild_tmp/oct_tmp are scratch of the level's size.  Daughters are appended at
// lev_end; *d_total receives their number.
void launch_split_level(const uint64_t* keys, Cells c, int lev_begin, int lev_end, int level, int leaf_size,
                        int* nchild_tmp, int* oct_tmp, int* offs_tmp, int* scan_tmp, int* d_total,
                        cudaStream_t s);
// A4: geometry.  Leaves: smallest enclosing ball of the particles, rho, mass,
// centre of mass.  Internal cells of one level: smallest ball of the daughter balls,
// mass and centre of mass from the daughters, then the exact radii over particles.
// keep_centre: a reused tree (Sec. 7.1) keeps the cells' centres s and recomputes the
// radii, masses and centres of mass for the particles' new positions
void launch_leaf_geometry(const d4* xm, Cells c, const int* leaves, int nleaves, unsigned* status,
                          cudaStream_t s, bool keep_centre = false);
// xp: the two-float position records (launch_split_positions); owner: per particle, set by
// launch_leaf_owner before the deepest level and moved up as the levels are processed
// bottom-up; rad_tmp: rad_tmp_u64_per_cell() words per cell of the largest level
void launch_internal_geometry(const d4* xm, const float4* xp, Cells c, int lev_begin, int lev_end,
                              int n, int* owner, unsigned long long* rad_tmp, unsigned* status, cudaStream_t s,
                              bool keep_centre = false);
void launch_leaf_owner(Cells c, const int* leaves, int nleaves, int* owner, cudaStream_t s);
size_t rad_tmp_u64_per_cell();

// ---------------------------------------------------------------- upward (upward.cu)
// P2M (eq. 3c) at leaves about centre cen (sr or cr), M2M (eq. 4) for the internal
// cells of one level, multipole power (eq. 14).
void launch_p2m(const d4* xm, Cells c, const d4* cen, const int* leaves, int nleaves, int p,
                double* M, cudaStream_t s);
void launch_m2m_level(Cells c, const d4* cen, int lev_begin, int lev_end, int p, double* M,
                      cudaStream_t s);
void launch_power(const double* M, int ncells, int p, double* P, cudaStream_t s);
// minimum of a per-particle scale over leaves, then over the daughters of one level
void launch_minscale_leaves(const double* scale_sorted, Cells c, const int* leaves, int nleaves,
                            cudaStream_t s);
void launch_minscale_level(Cells c, int lev_begin, int lev_end, cudaStream_t s);
void launch_scale_from_caller(const double* scale, const int* perm, int n, double* scale_sorted,
                              cudaStream_t s, const int* e = nullptr);

// ---------------------------------------------------------------- walk (walk.cu)
struct WalkParams {
    int p;              // expansion order used in E_{A->B}
    int mac;            // FMM_MAC_* or kMacEstimate
    double eps, theta_crit, p2p_thresh;
    const double* P;    // multipole power [nc][p+1]
    const double* binom;// device C(p,k)
    int use_com;        // radii/centres from cr (estimator) instead of sr
    // per-interaction order (Sec. 7, opening): an accepted pair takes the lowest q in
    // [p_lo, p] for which the criterion holds with E~ of order q; pascal[q * (kMaxP + 1) + k]
    // = C(q, k)
    int adaptive, p_lo;
    const double* pascal;
    // single-precision view of the cells for the acceptance test (nullable, then every
    // decision is taken in FP64): fc[2 c] = centre high parts and rho, fc[2 c + 1] = centre
    // low parts and P_0; fP[c * fstride + k] = P_k / (P_0 rho^k) for k <= p and, at k = p + 1,
    // eps * minscale.  A decision within a margin of its threshold is taken in FP64.
    const float4* fc;
    const float* fP;
    int fstride;
};
// row stride of fP for order p (P_0..P_p, eps * minscale, padded to float4)
inline int walk_fstride(int p) { return (p + 2 + 3) & ~3; }
// fill the single-precision view: centres from cen (sr, or cr for the estimator); with P
// (nullable) also the normalised powers and eps * minscale, without it the masses
void launch_walk_prep(Cells c, const d4* cen, const double* P, int p, double eps, int nc, float4* fc, float* fP,
                      cudaStream_t s);
// M2L list entries of an adaptive-order walk carry the pair's order q in the top bits of
// the source index: x = source | (q << kM2LOrderShift); q = 0 stands for the global p
constexpr int kM2LOrderShift = 27;
constexpr int kM2LSrcMask = (1 << kM2LOrderShift) - 1;
__host__ __device__ inline int m2l_src(int x) { return x & kM2LSrcMask; }
__host__ __device__ inline int m2l_order(int x, int p) {
    const int q = (int)((unsigned)x >> kM2LOrderShift);
    return q ? q : p;
}
constexpr int kMacEstimate = 3;  // theta < 1 only (low-order estimate, Sec. 5.3.2)

struct WalkBuffers {
    int2* front[2];
    long long front_cap;
    int2* m2l;
    long long m2l_cap;
    int2* p2p;
    long long p2p_cap;
    unsigned long long* counters;  // [0] next frontier, [1] m2l, [2] p2p, [3] overflow flag
};
// the first frontier: (r, r) for the roots r = 0 .. nroots-1
// count (nullable): receives nroots, the first frontier's length on the device
void launch_walk_roots(int2* front, int nroots, cudaStream_t s, unsigned long long* count = nullptr);
// one breadth-first step over a frontier of nfront pairs (host value); the next frontier is
// counted in wb.counters[0]
void launch_walk_step(Cells c, WalkParams wp, const int2* front_in, long long nfront, int2* front_out,
                      WalkBuffers wb, cudaStream_t s);
// the same with the frontier's length read on the device from *nfront_dev (no host round
// trip between steps); the next frontier is counted in *out_cnt and wb.counters[5] keeps
// the largest frontier demand seen
void launch_walk_step_dev(Cells c, WalkParams wp, const int2* front_in, const unsigned long long* nfront_dev,
                          int2* front_out, WalkBuffers wb, unsigned long long* out_cnt, cudaStream_t s);
// sort a pair list by (sink, first entry) -- the first entry taken as unsigned, so an adaptive
// walk's M2L entries (wide: order bits above the source index) sort by (sink, order, source) --
// then mark per-sink segments [seg_start, seg_end); tmp: list_sort_tmp_bytes(npairs, ncells)
size_t list_sort_tmp_bytes(long long npairs, int ncells);
void sort_pairs_by_sink(int2* list, long long npairs, int ncells, void* tmp, cudaStream_t s, bool wide = false);
void launch_segments(const int2* list, long long npairs, int ncells, int* seg_start, int* seg_end,
                     cudaStream_t s);

// ---------------------------------------------------------------- interactions (interact.cu)
size_t m2l_tmp_bytes(int ncells, int p);
void launch_m2l(const int2* list, const int* seg_start, const int* seg_end, void* tmp, int ncells,
                const d4* cen, const double* M, int p, double* F, cudaStream_t s);
// mixed mode: orders <= 2 of Theta in FP64, the rest in FP32 on scaled harmonics, either
// directly (eq. 3b) or, when rot is set and m2l_rot_supported(p), through rotations into
// the interaction's z frame (App. A.5, m2l_rot.cu)
size_t m2l_split_tmp_bytes(int ncells, int p, long long npairs);
// adaptive: the list comes from an adaptive-order walk (pairs carry their orders);
// npairs: the list's length (bounds the work items)
void launch_m2l_split(const int2* list, const int* seg_start, const int* seg_end, void* tmp, int ncells,
                      const d4* cen, const double* M, int p, double* F, bool rot, cudaStream_t s,
                      bool adaptive = false, long long npairs = 0);
// M2L pairs per work item of the mixed-mode M2L: each sink's list is cut into chunks of
// this many pairs from its start, summed separately and then added in chunk order
constexpr int kM2LChunk = 32;
// items per piece of a long sink in the rotated M2L without the adaptive order: a sink of more
// items is cut into pieces of this many, summed separately and then added in piece order (a
// constant, so that a sink is summed the same way whatever else is in the list)
constexpr int kM2LPieceItems = 8;
constexpr int kRotMaxP = 16;  // largest order with a rotation-accelerated M2L
bool m2l_rot_supported(int p);
// sinks in `order` (work[1] of them, cnt[i] items of sink position i from item_start[i]);
// Mt (ncells x (p+1)^2 floats) and M64 (ncells x 9) are scratch.  Without adaptive, every
// warp takes whole sinks, or pieces of kM2LPieceItems items of the longer sinks (work[3] the
// counter of these units, work[4] their number, work[5] the number of cut sinks; the unit
// list in gtmp), and writes a whole sink's F once; a piece writes its partial expansion to the
// part slot of its first item, and the pieces of each cut sink are then added into F in piece
// order.  adaptive: the items are grouped by the largest order of their pairs and
// each group runs the kernel of that order (gtmp: m2l_rot_group_bytes(items_cap) bytes; work[0]
// the item counter, work[2] the number of items); part receives one expansion per item, except
// that a sink whose list is a single item has its expansion written to F (zeroed beforehand)
// directly; returns the per-item orders (device) for the reduction
const int* launch_m2l_rot(const int2* list, const int* seg_start, const int* seg_end, const int* order,
                          const int* item_start, const int* cnt, unsigned* work, const d4* cen, const double* M,
                          int ncells, int p, float* Mt, cd* M64, double* part, double* F, bool adaptive, void* gtmp,
                          long long items_cap, cudaStream_t s);
size_t m2l_rot_group_bytes(long long items_cap);
void launch_l2l_level(Cells c, const d4* cen, int lev_begin, int lev_end, int p, double* F,
                      cudaStream_t s);
// L2P (eqs. 3a, 7) for every particle of every leaf: psi_far, acc_far (sorted order)
void launch_l2p(const d4* xm, Cells c, const d4* cen, const int* leaves, int nleaves, int p,
                const double* F, double* psi, double* acc, cudaStream_t s);
// mixed mode: P2M and L2P with orders <= 2 in FP64 and higher orders in FP32 (split.cu)
void launch_p2m_split(const d4* xm, Cells c, const d4* cen, const int* leaves, int nleaves, int p, double* M,
                      cudaStream_t s);
void launch_l2p_split(const d4* xm, Cells c, const d4* cen, const int* leaves, int nleaves, int p, const double* F,
                      double* psi, double* acc, cudaStream_t s);
void launch_m2m_split(Cells c, const d4* cen, int lev_begin, int lev_end, int p, double* M, cudaStream_t s);
void launch_l2l_split(Cells c, const d4* cen, int lev_begin, int lev_end, int p, double* F, cudaStream_t s);
// P2P (eq. 1) into psi_near/acc_near (sorted order): every leaf takes the sources of
// its own P2P segment and those of its ancestors' segments.
void launch_p2p_fp64(const d4* xm, Cells c, const int2* list, const int* seg_start,
                     const int* seg_end, const int* leaves, int nleaves, double* psi, double* acc, cudaStream_t s);
// Mixed P2P (p2p.cu).  mode (fmm_params.p2p_two_float): 0 dx from the FP32 high parts (the
// low-order estimate), 1 two-float dx for near source cells and FP32 offsets from the sink
// leaf's centre for the others, 2 offsets for all, 3 two-float for all.  tmp holds the work
// plan: at least p2p_plan_fixed_bytes(nleaves); the call plans, reads the plan's size on the
// host (h_tot: 6 host words; the stream is synchronised once) and runs the P2P if tmp_bytes
// holds it.  Returns the bytes the call needs: a value above tmp_bytes means nothing was
// computed (call again with that much), ~0 a plan beyond 2^31 ranges or items or n >= 2^29.
size_t p2p_plan_fixed_bytes(int nleaves);
size_t launch_p2p_mixed(const float4* xp, int n, Cells c, const int2* list, const int* seg_start,
                        const int* seg_end, const int* leaves, int nleaves, double* psi, double* acc, int mode,
                        void* tmp, size_t tmp_bytes, unsigned long long* h_tot, cudaStream_t s);
// ordered pairs of distinct particles at distance 0 (sorted keys and positions); with
// an ensemble (off != nullptr) only pairs inside one system count
void launch_coincident(const d4* xm, const uint64_t* keys, int n, unsigned long long* coincident, cudaStream_t s,
                       const int* off = nullptr, int nsys = 0);
// two-float position records, 32 bytes per particle: xp[2i] = (hi x, hi y, hi z, mass),
// xp[2i + 1] = (lo x, lo y, lo z, 0) with hi = fl32(x) and lo = fl32(x - hi)
void launch_split_positions(const d4* xm, int n, float4* xp, cudaStream_t s);
// low-order f estimate (p = 0, 1/r^2 kernel): M2L, pass-down, P2P, evaluation
void launch_f_m2l(const int2* list, const int* seg_start, const int* seg_end, int ncells, Cells c, double* Ff,
                  cudaStream_t s);
void launch_f_down_level(Cells c, int lev_begin, int lev_end, double* Ff, cudaStream_t s);
void launch_f_p2p(const d4* xm, Cells c, const int2* list, const int* seg_start, const int* seg_end,
                  const int* leaves, int nleaves, const double* Ff, double* f_sorted, cudaStream_t s);
// p = 1 M2L of the acceleration estimate from the monopoles about the centres of mass
// (the dipole vanishes there) into F1[nc][4]
void launch_est_m2l(const int2* list, const int* seg_start, const int* seg_end, int ncells, Cells c, double* F1,
                    cudaStream_t s, const float4* fc = nullptr);
// the estimate's far field at p = 1 plus its near field, as the scale |a| per sorted particle
void launch_est_scale(Cells c, const int* leaves, int nleaves, const double* F1, const double* acc_near,
                      double* scale, cudaStream_t s);
// combine far + near, multiply by G and scatter to the caller's order (A12)
// (ensemble: Gsys[k] for the caller particles [off[k], off[k+1]) instead of G)
// e (nullable): the working units (launch_work_units); psi is scaled back by 2^(e1 - e0), a by
// 2^(e1 - 2 e0)
void launch_finish(const double* psi_far, const double* acc_far, const double* psi_near,
                   const double* acc_near, const int* perm, int n, double G, double* psi, double* acc,
                   cudaStream_t s, const int* off = nullptr, const double* Gsys = nullptr, int nsys = 0,
                   const unsigned char* pact = nullptr, const int* e = nullptr);
// Sec. 7.1: pact[i] = active[perm[i]] != 0 (sorted order) and act[cell] = the cell holds an
// active particle (from a prefix sum of pact over the cells' particle ranges); ai holds
// n + 1 ints, scan n ints, scan_tmp scan_tmp_ints(n) ints
// tidal tensor (Sec. 7.4, tidal.cu): far part from Psi_2^m at the particles (sorted order,
// [n][6]), near part over the P2P lists (fp32: the two-float position records xp), and the
// combination G (far + near) scattered to the caller's order (active particles only)
void launch_l2p_tidal(const d4* xm, Cells c, const d4* cen, const int* leaves, int nleaves, int p, const double* F,
                      double* T, cudaStream_t s);
void launch_p2p_tidal(const d4* xm, const float4* xp, int n, bool fp32, Cells c, const int2* list,
                      const int* seg_start, const int* seg_end, const int* leaves, int nleaves, double* T,
                      cudaStream_t s);
void launch_finish_tidal(const double* Tf, const double* Tn, const int* perm, int n, double G,
                         const unsigned char* pact, double* T, cudaStream_t s, const int* e = nullptr);
// individual accuracy parameters (Sec. 7, opening): scale_sorted[i] *= eps_b[perm[i]] / eps
void launch_scale_eps(const double* eps_b, const int* perm, int n, double eps, double* scale_sorted, unsigned* status,
                      cudaStream_t s);
void launch_active_flags(const unsigned char* active, const int* perm, int n, const int* first, const int* count,
                         int ncells, unsigned char* pact, unsigned char* act, int* ai, int* scan, int* scan_tmp,
                         cudaStream_t s);

// ---------------------------------------------------------------- peaks (peaks.cu)
int alu_peaks(double* fp64_tflops, double* fp32_tflops);
// the mixed P2P's pair arithmetic alone (peaks.cu), in 10^9 pairs per second
int pair_peak(int warps_per_sm, double* gpairs_s);
// the swap stage of the rotated M2L at p = 14 as FMA immediates and as 3xTF32 mma.sync
// (swap_probe.cu); ms[0], ms[1] their kernel times, *maxdiff the largest difference
int swap_probe(int npairs, int reps, double* ms, double* maxdiff);

// ---------------------------------------------------------------- direct (direct.cu)
void launch_direct(const double* x, const double* mu, int n, double G, const int64_t* sinks, int nsinks,
                   double* psi, double* acc, double* f, cudaStream_t s);

}  // namespace gb3
