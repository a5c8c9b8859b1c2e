// p2p.cu -- the mixed-precision P2P of eq. (1): for every sink leaf B, Psi_b += mu_a / r and
// a_b += mu_a (x_a - x_b) / r^3 over the particles a of its source cells (its own P2P segment
// and those of its ancestors), a != b and r > 0 (coincident pairs skipped).
//
// Pair terms are FP32; each lane's FP32 sums over one tile (at most 128 pairs) are added to
// two-float accumulators (TwoSum), so the sum over a sink's thousands of sources is compensated.
// What a pair needs in FP32 is an accurate difference dx = x_a - x_b.  Two forms:
//   near: dx = (h_a - h_b) + (l_a - l_b) from the two-float positions (hi = fl32(x),
//         lo = fl32(x - hi)), one FP32 rounding relative to |dx| itself however close the pair;
//   far:  every source of a tile is turned once into its FP32 offset from the sink leaf's centre
//         c, o_a = (h_a - c_h) + (l_a - c_l), the sink likewise, and dx = o_a - o_b: one FP32
//         operation per coordinate and pair instead of three.  o_a and o_b carry absolute errors
//         of about 2^-24 |o|, so dx is relatively accurate to about 2^-24 (1 + 2 rho_B / |dx|).
// A source cell A is near when some pair of A x B could be closer than rho_B (the sink leaf's
// radius): |s_A - s_B| < rho_A + 2 rho_B.  Far pairs are then at least rho_B apart and their dx
// is good to about 3 x 2^-24, the same order as the rsqrt.approx of every pair.
//
// Work plan, built once per evaluation (k_p2p_count, k_p2p_emit): per leaf, its sources as
// particle ranges with their class (consecutive source cells of one class whose particles are
// contiguous are merged), in a region sized by its number of source cells, near ranges from the
// front and far ones from the back; and the work items (leaf, sink chunk).  Every lane holds two
// sinks, so that each source read from shared memory serves two pairs: a leaf of c sinks is cut
// into k items of at most 2 S sinks (slot s of an item holds its sinks s and S + s), each item
// replicated R <= 8 times across a warp (lane = replica * S + slot; replica r takes every R-th
// group of four sources of a tile), with (k, R) the cheapest by a cost per item of the lanes'
// pair work (2 / R per source) and the staging of its sources.  Every item streams its leaf's
// ranges as tiles of up to 128 sources: 32-byte position records copied asynchronously into a
// raw tile while the previous tile is computed, then converted into the structure-of-arrays
// tile the pairs read (offsets from the leaf centre for far tiles); a tile holds one class.
// Items run in decreasing order of their length (source particles / R) from an atomic counter.
#include <climits>

#include "kernels.cuh"

namespace gb3 {

constexpr int kP2PWarpsM = 4;        // warps per block
constexpr int kP2PTileM = 128;       // sources per staged tile at the largest replica count (4 x 32)
constexpr int kRangeCountBits = 29;  // a range record holds count | near << 30 | guard << 29
constexpr int kRangeMax = (1 << kRangeCountBits) - 1;

typedef unsigned long long f2;  // two packed floats
__device__ __forceinline__ f2 f2_pack(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// the sink of a lane, its coordinates duplicated in both halves
struct SinkPk {
    f2 hx, hy, hz, lx, ly, lz;
};
struct AccPk {
    f2 ps, ax, ay, az;
};

// two sources against the sink; TWO_FLOAT: dx from the two-float parts, else from X, Y, Z alone
// (FP32 offsets, or the high parts for the low-order estimate); GUARD: skip r = 0
template <bool TWO_FLOAT, bool GUARD>
__device__ __forceinline__ void pair2(f2 X, f2 Y, f2 Z, f2 W, f2 XL, f2 YL, f2 ZL, const SinkPk& b, AccPk& a) {
    f2 dx = f2_sub(X, b.hx), dy = f2_sub(Y, b.hy), dz = f2_sub(Z, b.hz);
    if (TWO_FLOAT) {
        dx = f2_add(dx, f2_sub(XL, b.lx));
        dy = f2_add(dy, f2_sub(YL, b.ly));
        dz = f2_add(dz, f2_sub(ZL, b.lz));
    }
    const f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
    float r2a, r2b;
    f2_unpack(r2, r2a, r2b);
    float ia = rsqrt_ftz(r2a), ib = rsqrt_ftz(r2b);
    if (GUARD) {
        ia = r2a > 0.f ? ia : 0.f;
        ib = r2b > 0.f ? ib : 0.f;
    }
    const f2 rinv = f2_pack(ia, ib);
    const f2 qm = f2_mul(W, rinv);
    const f2 q3 = f2_mul(qm, f2_mul(rinv, rinv));
    a.ps = f2_add(a.ps, qm);
    a.ax = f2_fma(q3, dx, a.ax);
    a.ay = f2_fma(q3, dy, a.ay);
    a.az = f2_fma(q3, dz, a.az);
}

// one group of four sources of the tile (index g) against the lane's two sinks
template <bool TWO_FLOAT, bool GUARD>
__device__ __forceinline__ void group4(const float* __restrict__ T, int g, const SinkPk& b0, const SinkPk& b1,
                                       AccPk& a0, AccPk& a1) {
    // 16-byte loads straight into packed pairs (sources 0, 1 and 2, 3 of the group)
    const ulonglong2 X = ((const ulonglong2*)(T + 0 * kP2PTileM))[g], Y = ((const ulonglong2*)(T + 1 * kP2PTileM))[g],
                     Z = ((const ulonglong2*)(T + 2 * kP2PTileM))[g], W = ((const ulonglong2*)(T + 3 * kP2PTileM))[g];
    ulonglong2 XL = make_ulonglong2(0ull, 0ull), YL = XL, ZL = XL;
    if (TWO_FLOAT) {
        XL = ((const ulonglong2*)(T + 4 * kP2PTileM))[g];
        YL = ((const ulonglong2*)(T + 5 * kP2PTileM))[g];
        ZL = ((const ulonglong2*)(T + 6 * kP2PTileM))[g];
    }
    const f2 x01 = X.x, y01 = Y.x, z01 = Z.x, w01 = W.x, x23 = X.y, y23 = Y.y, z23 = Z.y, w23 = W.y;
    const f2 l01 = XL.x, m01 = YL.x, n01 = ZL.x, l23 = XL.y, m23 = YL.y, n23 = ZL.y;
    pair2<TWO_FLOAT, GUARD>(x01, y01, z01, w01, l01, m01, n01, b0, a0);
    pair2<TWO_FLOAT, GUARD>(x01, y01, z01, w01, l01, m01, n01, b1, a1);
    pair2<TWO_FLOAT, GUARD>(x23, y23, z23, w23, l23, m23, n23, b0, a0);
    pair2<TWO_FLOAT, GUARD>(x23, y23, z23, w23, l23, m23, n23, b1, a1);
}

constexpr int kP2PRmax = 8;  // replicas of an item across a warp
// groups of four per replica in a full tile, and sources per full tile: 4 R (32 / R) <= 128
__host__ __device__ constexpr int p2p_groups(int R) { return 32 / R; }
__host__ __device__ constexpr int p2p_tile(int R) { return 4 * R * (32 / R); }

// replica r0 of R takes groups r0, r0 + R, ... of a tile of ng groups (one loop for every R,
// so that the four forms of the pair code stay small enough for the instruction cache)
template <bool TWO_FLOAT, bool GUARD>
__device__ __forceinline__ void tile_any(const float* __restrict__ T, int ng, int r0, int R, const SinkPk& b0,
                                         const SinkPk& b1, AccPk& a0, AccPk& a1) {
#pragma unroll 2
    for (int g = r0; g < ng; g += R) group4<TWO_FLOAT, GUARD>(T, g, b0, b1, a0, a1);
}

// s.hi += v with the rounding error of that addition (TwoSum) kept in s.lo; s.lo is not
// renormalised against s.hi (its own rounding, u |s.lo|, stays far below u |s.hi|)
__device__ __forceinline__ void acc2(ff& s, float v) {
    const ff t = two_sum(s.hi, v);
    s.hi = t.hi;
    s.lo = __fadd_rn(s.lo, t.lo);
}

// the FP32 partials of one sink folded into its two-float sums (4 per sink)
__device__ __forceinline__ void fold(AccPk& a, ff* sum) {
    float u0, u1;
    f2_unpack(a.ps, u0, u1);
    acc2(sum[0], u0 + u1);
    f2_unpack(a.ax, u0, u1);
    acc2(sum[1], u0 + u1);
    f2_unpack(a.ay, u0, u1);
    acc2(sum[2], u0 + u1);
    f2_unpack(a.az, u0, u1);
    acc2(sum[3], u0 + u1);
    const f2 zero = f2_pack(0.f, 0.f);
    a = AccPk{zero, zero, zero, zero};
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// (k items, R replicas, S slots) for a leaf of c sinks, two sinks per slot: the least cost
// k (2 / R + 0.6) per source over k >= ceil(c / 64) (the lanes' pair work and the staging of
// the sources, in units of a lane's pair), then k = ceil(c / (2 S)) so that no item is empty
__host__ __device__ inline void p2p_chunking(int c, int& k, int& R, int& S) {
    k = R = S = 1;
    if (c <= 0) return;
    const int kmin = (c + 63) / 64;
    float best = 3.0e38f;
    for (int kk = kmin; kk < kmin + 12; ++kk) {
        const int SS = (c + 2 * kk - 1) / (2 * kk);
        const int RR = 32 / SS < kP2PRmax ? 32 / SS : kP2PRmax;
        const float cost = (float)kk * (2.0f / (float)RR + 0.6f);
        if (cost < best) {
            best = cost;
            k = kk;
            R = RR;
            S = SS;
        }
    }
    k = (c + 2 * S - 1) / (2 * S);
}

// class of source cell A for sink leaf B (see the file comment); mode 1 only
__device__ inline bool p2p_near(const d4& a, const d4& b) {
    const double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    const double lim = a.w + 2.0 * b.w;
    return dx * dx + dy * dy + dz * dz < lim * lim;
}

// Long items are split: a leaf whose item would take a lane more than kP2PPieceSteps pair steps
// (2 sources / R) has its stream of source cells cut into P = ceil(steps / kP2PPieceSteps) <=
// kP2PMaxPieces pieces of about equal numbers of source cells, each with its own ranges, items
// and FP64 partial sums, which k_p2p_reduce adds in piece order.  The split depends on the leaf
// alone, so a system gives the same result in an ensemble as alone.
constexpr int kP2PMaxPieces = 64;
constexpr unsigned kP2PPieceSteps = 8192;

// per leaf index t (one warp each): the number of its source cells nb[t] (the ranges it can need
// at most: its own and its ancestors' segment lengths) and the length of its items (a lane's
// pair steps, 2 source particles / R; 0 for a leaf without active particles); tot[0] += nb
__global__ void k_p2p_count(Cells c, const int2* __restrict__ list, const int* __restrict__ seg_start,
                            const int* __restrict__ seg_end, const int* __restrict__ leaves, int nleaves,
                            int* __restrict__ nb, unsigned* __restrict__ len, unsigned long long* __restrict__ tot) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    unsigned long long my = 0;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nleaves; t += nw) {
        const int leaf = leaves[t];
        long long e = 0, src = 0;
        for (int cell = leaf; cell >= 0; cell = c.parent[cell]) {
            const int s0 = seg_start[cell], s1 = seg_end[cell];
            e += s1 - s0;
            for (int i = s0 + lane; i < s1; i += 32) src += c.count[list[i].x];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) src += __shfl_xor_sync(0xffffffffu, src, o);
        if (lane == 0) {
            nb[t] = (int)e;
            my += (unsigned long long)e;
            int k, R, S;
            p2p_chunking(c.count[leaf], k, R, S);
            const unsigned long long l = 2ull * (unsigned long long)src / (unsigned long long)R + 1;
            const unsigned w32 = !cell_active(c, leaf) ? 0u : (l > 0xfffffffeull ? 0xfffffffeu : (unsigned)l);
            len[t] = w32;
        }
    }
    if (lane == 0 && my) atomicAdd(&tot[0], my);
}

// per leaf index t: its pieces np[t] and its sort key, descending in the length of a piece's items
__global__ void k_p2p_pieces(const unsigned* __restrict__ len, const int* __restrict__ nb, int nleaves,
                             int* __restrict__ np, uint64_t* __restrict__ keys) {
    const unsigned long long lmax = kP2PPieceSteps;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nleaves; t += gridDim.x * blockDim.x) {
        const unsigned l = len[t];
        int P = (int)(((unsigned long long)l + lmax - 1) / lmax);
        const int cap = nb[t] < kP2PMaxPieces ? nb[t] : kP2PMaxPieces;
        P = P < 1 ? 1 : (P > cap ? (cap > 0 ? cap : 1) : P);
        np[t] = P;
        const unsigned w32 = l ? (unsigned)(((unsigned long long)l + P - 1) / P) : 0u;
        keys[t] = ((uint64_t)(255u - qlen8(w32)) << 32) | (unsigned)t;
    }
}

// per position q of the sorted order: items nit[q] (pieces x items per piece; 0 for a leaf
// without active particles) and pieces npc[q]; tot[1] += items, tot[3] += pieces, tot[4] += the
// partial sums of split leaves (pieces x sinks), tot[5] += split leaves
__global__ void k_p2p_nitems(const uint64_t* __restrict__ keys, const int* __restrict__ leaves, int nleaves, Cells c,
                             const int* __restrict__ np, int* __restrict__ order, int* __restrict__ nit,
                             int* __restrict__ npc, unsigned long long* __restrict__ tot) {
    unsigned long long my = 0, mp = 0, mpart = 0, msplit = 0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nleaves; q += gridDim.x * blockDim.x) {
        const int t = (int)(keys[q] & 0xffffffffu);
        order[q] = t;
        const int leaf = leaves[t];
        int k = 0, R, S, P = 0;
        if (cell_active(c, leaf)) {
            p2p_chunking(c.count[leaf], k, R, S);
            P = np[t];
        }
        nit[q] = k * P;
        npc[q] = P;
        my += (unsigned long long)(k * P);
        mp += (unsigned long long)P;
        if (P > 1) {
            mpart += (unsigned long long)P * (unsigned long long)c.count[leaf];
            ++msplit;
        }
    }
    if (my) atomicAdd(&tot[1], my);
    if (mp) atomicAdd(&tot[3], mp);
    if (mpart) atomicAdd(&tot[4], mpart);
    if (msplit) atomicAdd(&tot[5], msplit);
}

// per piece v: its leaf index, its region of ranges [r0, r1) (near ranges from the front, far
// ones from the back), their numbers, and the first of its partial sums (-1: the piece is the
// whole leaf and writes psi and acc directly)
struct Pieces {
    int *leaf, *r0, *r1, *nnear, *nfar, *part;
};

// ranges of the pieces of leaf index t (sorted position q); items (piece, chunk).  One warp per
// position.  Piece j takes the source cells j e / P .. (j + 1) e / P - 1 of the leaf's stream
// (its own segment, then each ancestor's; e cells in all) and owns that part of the leaf's region
// [roff[t], roff[t] + e).  Within a piece the sources are merged per class in stream order: an
// entry joins the open range of its class when its particles follow that range's directly.  The
// lanes take up to 32 entries at a time; each finds its class predecessor (the closest lower
// lane of its class, else the open range carried from the earlier entries), the entries that do
// not join start a run, a run's count and guard flag are summed in shared memory, and every run
// but the last of its class is written out; the last stays open until the piece ends.  This is
// the result of the sequential pass.  A split leaf takes its partial-sum slots (P x sinks) and
// an entry of the split list (t, first slot) from the counters tot[6], tot[7].
constexpr int kEmitWarps = 4;
__global__ void __launch_bounds__(kEmitWarps * 32)
    k_p2p_emit(Cells c, const int2* __restrict__ list, const int* __restrict__ seg_start,
               const int* __restrict__ seg_end, const int* __restrict__ leaves, int nleaves, int mode,
               const int* __restrict__ order, const int* __restrict__ roff, const int* __restrict__ nb,
               const int* __restrict__ ioff, const int* __restrict__ nit, const int* __restrict__ voff,
               const int* __restrict__ npc, Pieces pc, int2* __restrict__ ranges, int2* __restrict__ items,
               int2* __restrict__ split, unsigned long long* __restrict__ tot) {
    __shared__ int rsum_all[kEmitWarps][33], rg_all[kEmitWarps][33];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int* rsum = rsum_all[wid];  // [0]: the open range carried in; [1 + L]: the run starting at lane L
    int* rg = rg_all[wid];
    const unsigned below = (1u << lane) - 1u, upto = below | (1u << lane);
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nleaves; q += nw) {
        const int P = npc[q];
        if (P == 0) continue;  // no active particle: no items, no ranges
        const int t = order[q];
        const int kper = nit[q] / P;  // items per piece
        const int leaf = leaves[t];
        const int count = c.count[leaf];
        int pbase = -1;
        if (P > 1 && lane == 0) {
            pbase = (int)atomicAdd(&tot[6], (unsigned long long)P * (unsigned long long)count);
            const int si = (int)atomicAdd(&tot[7], 1ull);
            split[si] = make_int2(t, pbase);
        }
        pbase = __shfl_sync(0xffffffffu, pbase, 0);
        for (int j = lane; j < nit[q]; j += 32) items[ioff[q] + j] = make_int2(voff[q] + j / kper, j % kper);
        const d4 sb = c.sr[leaf];
        const long long b0 = c.first[leaf], b1 = b0 + count;
        const long long e = nb[t];
        // the cursor over the leaf's stream of source cells: cell, its list segment, position
        int cell = leaf, s1 = seg_end[leaf], at = seg_start[leaf];
        for (int pj = 0; pj < P; ++pj) {
            const int v = voff[q] + pj;
            const long long f0 = e * pj / P, f1 = e * (pj + 1) / P;
            const int r0 = roff[t] + (int)f0, r1 = roff[t] + (int)f1;
            int cf[2] = {0, 0}, cn[2] = {0, 0}, cnt[2] = {0, 0};  // open range and records written per class
            bool cg[2] = {false, false};
            auto put = [&](int k, int idx, int f, int n, bool g) {
                ranges[k ? r0 + idx : r1 - 1 - idx] =
                    make_int2(f, n | (k << 30) | ((g ? 1 : 0) << kRangeCountBits));
            };
            for (long long fi = f0; fi < f1;) {
                while (at >= s1) {  // on to the next ancestor's segment
                    cell = c.parent[cell];
                    at = seg_start[cell];
                    s1 = seg_end[cell];
                }
                const int m = (int)min((long long)min(32, s1 - at), f1 - fi);
                int f = 0, n = 0, kk = -1;
                if (lane < m) {
                    const int A = list[at + lane].x;
                    f = c.first[A];
                    n = c.count[A];
                    kk = mode == 1 ? (p2p_near(c.sr[A], sb) ? 1 : 0) : (mode == 3 ? 1 : 0);
                    if (n <= 0) kk = -1;
                }
                at += m;
                fi += m;
                const bool g = kk >= 0 && f < b1 && b0 < (long long)f + n;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const unsigned M = __ballot_sync(0xffffffffu, kk == k);
                    if (!M) continue;
                    const unsigned pm = M & below;
                    const int pl = pm ? 31 - __clz(pm) : lane;
                    const int pf = __shfl_sync(0xffffffffu, f, pl), pn = __shfl_sync(0xffffffffu, n, pl);
                    const long long pe = pm ? (long long)pf + pn : (cn[k] > 0 ? (long long)cf[k] + cn[k] : -1);
                    const bool mine = kk == k;
                    const unsigned S = __ballot_sync(0xffffffffu, mine && pe != f);
                    const unsigned sm = S & upto;
                    const int rs = sm ? 31 - __clz(sm) : -1;  // the run this lane belongs to
                    rsum[lane] = 0;
                    rg[lane] = 0;
                    if (lane == 0) rsum[32] = rg[32] = 0;
                    __syncwarp();
                    if (mine) {
                        atomicAdd(&rsum[rs + 1], n);
                        if (g) atomicOr(&rg[rs + 1], 1);
                    }
                    __syncwarp();
                    if (!S) {  // every entry joins the open range
                        cn[k] += rsum[0];
                        cg[k] = cg[k] || rg[0];
                    } else {
                        int base = cnt[k];
                        if (cn[k] > 0) {  // the open range closes at the first start
                            if (lane == 0) put(k, base, cf[k], cn[k] + rsum[0], cg[k] || rg[0]);
                            ++base;
                        }
                        const int last = 31 - __clz(S);
                        if (((S >> lane) & 1) && lane != last)
                            put(k, base + __popc(S & below), f, rsum[lane + 1], rg[lane + 1] != 0);
                        cnt[k] = base + __popc(S) - 1;
                        cf[k] = __shfl_sync(0xffffffffu, f, last);
                        cn[k] = rsum[last + 1];
                        cg[k] = rg[last + 1] != 0;
                    }
                    __syncwarp();
                }
            }
            if (lane == 0) {
                for (int k = 1; k >= 0; --k)
                    if (cn[k] > 0) put(k, cnt[k]++, cf[k], cn[k], cg[k]);
                pc.leaf[v] = t;
                pc.r0[v] = r0;
                pc.r1[v] = r1;
                pc.nnear[v] = cnt[1];
                pc.nfar[v] = cnt[0];
                pc.part[v] = P > 1 ? pbase + pj * count : -1;
            }
            __syncwarp();
        }
    }
}

// the FP64 partial sums of the split leaves added in piece order into psi and acc: one warp per
// entry (t, first slot) of the split list, lanes over the leaf's sinks
__global__ void k_p2p_reduce(Cells c, const int* __restrict__ leaves, const int* __restrict__ np,
                             const int2* __restrict__ split, int nsplit, const double* __restrict__ part,
                             double* __restrict__ psi, double* __restrict__ acc) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nsplit; w += nw) {
        const int2 sp = split[w];
        const int leaf = leaves[sp.x], P = np[sp.x];
        const int first = c.first[leaf], count = c.count[leaf];
        for (int sk = lane; sk < count; sk += 32) {
            double v[4] = {0.0, 0.0, 0.0, 0.0};
            for (int j = 0; j < P; ++j) {
                const double* pp = part + 4 * ((size_t)sp.y + (size_t)j * count + sk);
#pragma unroll
                for (int d = 0; d < 4; ++d) v[d] += pp[d];
            }
            const size_t i = (size_t)first + sk;
            psi[i] = v[0];
            acc[3 * i] = v[1];
            acc[3 * i + 1] = v[2];
            acc[3 * i + 2] = v[3];
        }
    }
}

// The ranges of one item as a stream of tiles.  The item's records (its near segment, then
// its far segment) are read 32 at a time into a register window, lane j holding record
// w0 + j, and the next window is loaded as soon as the current one is taken.  A tile takes
// sources from consecutive ranges of one class; fill() copies their position records (two
// float4 each, one with LOADLO false) into the raw tile and returns their number (0 when the
// stream is exhausted) with the tile's class and guard flag.
struct RangeStream {
    int a0, na, b0, total;  // flattened record i: i < na ? a0 + i : b0 + i - na; total records
    int pos, w0;            // next record, first record of the window
    int2 win, nwin;         // the window and the one after it
    int af, an, off;        // the current range and the position in it
    bool near, guard;       // its class and guard flag
    __device__ int2 load(const int2* __restrict__ ranges, int w, int lane) const {
        const int i = w + lane;
        return i < total ? ranges[i < na ? a0 + i : b0 + (i - na)] : make_int2(0, 0);
    }
    __device__ void start(const int2* __restrict__ ranges, int lane, int r0, int r1, int s0, int s1) {
        a0 = r0;
        na = r1 - r0;
        b0 = s0;
        total = na + (s1 - s0);
        pos = w0 = 0;
        win = load(ranges, 0, lane);
        nwin = load(ranges, 32, lane);
        af = an = off = 0;
        near = guard = false;
    }
    template <bool LOADLO>
    __device__ int fill(const int2* __restrict__ ranges, const float4* __restrict__ xp, int lane, int T,
                        float4* raw, bool& tile_near, bool& tile_guard) {
        int m = 0;
        tile_guard = false;
        tile_near = near;
        while (m < T) {
            if (off == an) {  // next range
                if (pos >= total) break;
                if (pos - w0 >= 32) {  // on to the prefetched window
                    win = nwin;
                    w0 += 32;
                    nwin = load(ranges, w0 + 32, lane);
                }
                const int rx = __shfl_sync(0xffffffffu, win.x, pos - w0);
                const int ry = __shfl_sync(0xffffffffu, win.y, pos - w0);
                const bool nr = (ry >> 30) & 1;
                if (m > 0 && nr != tile_near) break;  // a tile holds one class
                ++pos;
                af = rx;
                an = ry & kRangeMax;
                off = 0;
                near = nr;
                guard = (ry >> kRangeCountBits) & 1;
                tile_near = nr;
                continue;
            }
            const int k = min(T - m, an - off);
            for (int q = lane; q < k; q += 32) {
                const float4* g = xp + 2 * ((size_t)af + off + q);
                float4* t = raw + 2 * (m + q);
                cp_async16(t, g);
                if (LOADLO) cp_async16(t + 1, g + 1);
            }
            tile_guard = tile_guard || guard;
            m += k;
            off += k;
        }
        return m;
    }
};

// MODE 0: dx from the FP32 high parts (the low-order estimate); 1: near ranges two-float,
// far ranges FP32 offsets from the leaf centre; 2: offsets for every range; 3: two-float for
// every range
template <int MODE>
__global__ void __launch_bounds__(kP2PWarpsM * 32, 4)
    k_p2p_mixed(const float4* __restrict__ xp, Cells c, const int* __restrict__ leaves,
                const int2* __restrict__ ranges, const Pieces pc, const int2* __restrict__ items, int nitems,
                unsigned* __restrict__ counter, double* __restrict__ psi, double* __restrict__ acc,
                double* __restrict__ part) {
    constexpr bool LOADLO = MODE >= 1;  // the tiles carry the low parts
    constexpr bool CENTRE = MODE == 1 || MODE == 2;
    constexpr int NA = LOADLO ? 7 : 4;  // arrays of the computed tile
    // per warp: the raw position records of the tile in flight, and the tile being computed
    // (structure of arrays X | Y | Z | W [| XL | YL | ZL], high parts or offsets)
    __shared__ __align__(16) float4 raws[kP2PWarpsM][2 * kP2PTileM];
    __shared__ __align__(16) float tiles[kP2PWarpsM][NA * kP2PTileM];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float4* raw = raws[wid];
    float* tile = tiles[wid];
    const f2 zero = f2_pack(0.f, 0.f);
    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(counter, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= (unsigned)nitems) break;
        const int2 it = items[w];
        const int v = it.x, t = pc.leaf[v], leaf = leaves[t];
        const int first = c.first[leaf], count = c.count[leaf];
        int k, R, S;
        p2p_chunking(count, k, R, S);
        const int s0 = it.y * 2 * S, chunk = min(2 * S, count - s0);
        // lanes past S * R repeat replica 0's work; their sums are not used.  The lane's sinks
        // are s0 + slot and s0 + S + slot; a missing one repeats the item's first sink
        const int slot = lane % S, rep = lane / S < R ? lane / S : 0;
        const bool okA = lane < S * R && slot < chunk, okB = lane < S * R && S + slot < chunk;
        const int iA = first + s0 + (slot < chunk ? slot : 0);
        const int iB = first + s0 + (S + slot < chunk ? S + slot : 0);
        // the leaf centre as two floats; the sinks as FP32 offsets from it (CENTRE) or their
        // high parts
        float chx = 0.f, chy = 0.f, chz = 0.f, clx = 0.f, cly = 0.f, clz = 0.f;
        if (CENTRE) {
            const d4 sc = c.sr[leaf];
            chx = (float)sc.x;
            chy = (float)sc.y;
            chz = (float)sc.z;
            clx = (float)(sc.x - (double)chx);
            cly = (float)(sc.y - (double)chy);
            clz = (float)(sc.z - (double)chz);
        }
        auto far_sink = [&](int i) {
            const float4 h = xp[2 * (size_t)i];
            float ox = h.x, oy = h.y, oz = h.z;
            if (CENTRE) {
                const float4 l = xp[2 * (size_t)i + 1];
                ox = __fadd_rn(__fsub_rn(h.x, chx), __fsub_rn(l.x, clx));
                oy = __fadd_rn(__fsub_rn(h.y, chy), __fsub_rn(l.y, cly));
                oz = __fadd_rn(__fsub_rn(h.z, chz), __fsub_rn(l.z, clz));
            }
            return SinkPk{f2_pack(ox, ox), f2_pack(oy, oy), f2_pack(oz, oz), zero, zero, zero};
        };
        auto near_sink = [&](int i) {
            const float4 h = xp[2 * (size_t)i], l = xp[2 * (size_t)i + 1];
            return SinkPk{f2_pack(h.x, h.x), f2_pack(h.y, h.y), f2_pack(h.z, h.z),
                          f2_pack(l.x, l.x), f2_pack(l.y, l.y), f2_pack(l.z, l.z)};
        };
        const SinkPk fA = far_sink(iA), fB = far_sink(iB);
        AccPk aA{zero, zero, zero, zero}, aB{zero, zero, zero, zero};
        ff sA[4], sB[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) sA[q] = sB[q] = ff{0.f, 0.f};
        RangeStream cur;
        {
            const int r0 = pc.r0[v], r1 = pc.r1[v];
            cur.start(ranges, lane, r0, r0 + pc.nnear[v], r1 - pc.nfar[v], r1);
        }
        const int T = p2p_tile(R);  // sources per tile, shared by the replicas
        bool near = false, guard = false, near_next = false, guard_next = false;
        int nt = cur.fill<LOADLO>(ranges, xp, lane, T, raw, near, guard);
        cp_async_commit();
        while (nt > 0) {
            cp_async_wait0();
            __syncwarp();  // the raw tile has arrived; every lane is done with the previous tile
            const int ng = (nt + 3) >> 2;
            const bool two = MODE == 3 || (MODE == 1 && near);
            // the computed tile: offsets from the leaf centre (far, CENTRE) or the parts as they
            // are; padded to whole groups with massless sources far away
            for (int j = lane; j < 4 * ng; j += 32) {
                float x = 1e15f, y = 1e15f, z = 1e15f, wm = 0.f, xl = 0.f, yl = 0.f, zl = 0.f;
                if (j < nt) {
                    const float4 h = raw[2 * j];
                    wm = h.w;
                    if (LOADLO) {
                        const float4 l = raw[2 * j + 1];
                        if (CENTRE && !two) {
                            x = __fadd_rn(__fsub_rn(h.x, chx), __fsub_rn(l.x, clx));
                            y = __fadd_rn(__fsub_rn(h.y, chy), __fsub_rn(l.y, cly));
                            z = __fadd_rn(__fsub_rn(h.z, chz), __fsub_rn(l.z, clz));
                        } else {
                            x = h.x;
                            y = h.y;
                            z = h.z;
                            xl = l.x;
                            yl = l.y;
                            zl = l.z;
                        }
                    } else {
                        x = h.x;
                        y = h.y;
                        z = h.z;
                    }
                }
                tile[j] = x;
                tile[kP2PTileM + j] = y;
                tile[2 * kP2PTileM + j] = z;
                tile[3 * kP2PTileM + j] = wm;
                if (LOADLO && two) {
                    tile[4 * kP2PTileM + j] = xl;
                    tile[5 * kP2PTileM + j] = yl;
                    tile[6 * kP2PTileM + j] = zl;
                }
            }
            __syncwarp();  // the computed tile is complete and the raw tile free
            // the next tile's copies run while this one is computed
            const int nx = cur.fill<LOADLO>(ranges, xp, lane, T, raw, near_next, guard_next);
            cp_async_commit();
            if (two) {  // the sinks' two-float parts, read again for this tile
                const SinkPk nA = near_sink(iA), nB = near_sink(iB);
                if (guard) tile_any<true, true>(tile, ng, rep, R, nA, nB, aA, aB);
                else tile_any<true, false>(tile, ng, rep, R, nA, nB, aA, aB);
            } else {
                if (guard) tile_any<false, true>(tile, ng, rep, R, fA, fB, aA, aB);
                else tile_any<false, false>(tile, ng, rep, R, fA, fB, aA, aB);
            }
            // fold the FP32 partials (<= 128 pairs per sink) into the two-float sums
            fold(aA, sA);
            fold(aB, sB);
            nt = nx;
            near = near_next;
            guard = guard_next;
        }
        // add the replicas' partial sums into the lanes of replica 0 (a tree over the replicas:
        // at step h, replica r takes replica r + h when r is a multiple of 2 h)
        for (int h = 1; h < R; h *= 2) {
            const int src = min(lane + h * S, 31);
            const bool take = rep % (2 * h) == 0 && rep + h < R && lane < S * R;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ff ta = sA[q], tb = sB[q];
                ff_add_lane(ta, src);
                ff_add_lane(tb, src);
                if (take) {
                    sA[q] = ta;
                    sB[q] = tb;
                }
            }
        }
        // a whole leaf writes psi and acc; a piece of a split leaf its partial-sum slots
        const int pslot = pc.part[v];
        auto out = [&](int i, const ff* sm) {
            double* o4 = pslot >= 0 ? part + 4 * ((size_t)pslot + (size_t)(i - first)) : nullptr;
            const double vv[4] = {(double)sm[0].hi + (double)sm[0].lo, (double)sm[1].hi + (double)sm[1].lo,
                                  (double)sm[2].hi + (double)sm[2].lo, (double)sm[3].hi + (double)sm[3].lo};
            if (o4) {
#pragma unroll
                for (int d = 0; d < 4; ++d) o4[d] = vv[d];
            } else {
                psi[i] = vv[0];
                acc[3 * (size_t)i] = vv[1];
                acc[3 * (size_t)i + 1] = vv[2];
                acc[3 * (size_t)i + 2] = vv[3];
            }
        };
        if (lane < S) {
            if (okA) out(iA, sA);
            if (okB) out(iB, sB);
        }
    }
}

namespace {
// layout of the fixed part of the scratch (depends on the number of leaves only)
struct PlanLayout {
    uint64_t *k0, *k1;
    unsigned* len;
    int *order, *nb, *roff, *np, *npc, *voff, *nit, *ioff, *stmp, *rtmp;
    unsigned long long* tot;  // [0] ranges, [1] items, [3] pieces, [4] partial slots, [5] split
                              // leaves, [6] [7] allocators of the emit ([2] unused)
    unsigned* counter;
    size_t bytes;
};
PlanLayout plan_layout(void* base, int nleaves) {
    PlanLayout L;
    const size_t nl = (size_t)(nleaves > 0 ? nleaves : 1);
    unsigned char* p = (unsigned char*)base;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        unsigned char* r = p ? p + off : nullptr;
        off += bytes;
        return r;
    };
    L.k0 = (uint64_t*)take(nl * 8);
    L.k1 = (uint64_t*)take(nl * 8);
    L.len = (unsigned*)take(nl * 4);
    L.order = (int*)take(nl * 4);
    L.nb = (int*)take(nl * 4);
    L.roff = (int*)take((nl + 1) * 4);
    L.np = (int*)take(nl * 4);
    L.npc = (int*)take(nl * 4);
    L.voff = (int*)take((nl + 1) * 4);
    L.nit = (int*)take(nl * 4);
    L.ioff = (int*)take((nl + 1) * 4);
    L.stmp = (int*)take(scan_tmp_ints((long long)nl + 1) * 4);
    L.rtmp = (int*)take(radix_tmp_ints((long long)nl) * 4);
    L.tot = (unsigned long long*)take(8 * 8);
    L.counter = (unsigned*)take(4 * 4);
    L.bytes = (off + 255) & ~(size_t)255;
    return L;
}
}  // namespace

size_t p2p_plan_fixed_bytes(int nleaves) { return plan_layout(nullptr, nleaves).bytes; }

size_t launch_p2p_mixed(const float4* xp, int n, Cells c, const int2* list, const int* seg_start,
                        const int* seg_end, const int* leaves, int nleaves, double* psi, double* acc, int mode,
                        void* tmp, size_t tmp_bytes, unsigned long long* h_tot, cudaStream_t s) {
    if (nleaves <= 0) return 0;
    if (n > kRangeMax) return ~(size_t)0;  // no range is ever cut: a leaf's region holds its source cells
    PlanLayout L = plan_layout(tmp, nleaves);
    if (tmp_bytes < L.bytes) return L.bytes;
    int bps = 1;
    auto kern_of = [&]() {
        return mode == 1 ? k_p2p_mixed<1> : mode == 2 ? k_p2p_mixed<2> : mode == 3 ? k_p2p_mixed<3> : k_p2p_mixed<0>;
    };
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern_of(), kP2PWarpsM * 32, 0);
    if (bps < 1) bps = 1;
    const int nblocks = sm_count() * bps;
    cudaMemsetAsync(L.tot, 0, 8 * sizeof(unsigned long long), s);
    cudaMemsetAsync(L.counter, 0, 4 * sizeof(unsigned), s);
    k_p2p_count<<<grid_for((long long)nleaves * 32, 128, 16), 128, 0, s>>>(c, list, seg_start, seg_end, leaves,
                                                                           nleaves, L.nb, L.len, L.tot);
    note_launch();
    scan_exclusive_i32(L.nb, L.roff, nleaves, L.roff + nleaves, L.stmp, s);
    k_p2p_pieces<<<grid_for(nleaves, 256), 256, 0, s>>>(L.len, L.nb, nleaves, L.np, L.k0);
    note_launch();
    // the low 32 bits are the leaf index, already in order: sort the 8 length bits only
    const int flip = radix_sort_pairs_bits(L.k0, nullptr, L.k1, nullptr, nleaves, L.rtmp, 32, 40, s);
    k_p2p_nitems<<<grid_for(nleaves, 256), 256, 0, s>>>(flip ? L.k1 : L.k0, leaves, nleaves, c, L.np, L.order,
                                                         L.nit, L.npc, L.tot);
    note_launch();
    scan_exclusive_i32(L.nit, L.ioff, nleaves, L.ioff + nleaves, L.stmp, s);
    scan_exclusive_i32(L.npc, L.voff, nleaves, L.voff + nleaves, L.stmp, s);
    cudaMemcpyAsync(h_tot, L.tot, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    const unsigned long long nranges = h_tot[0], nitems = h_tot[1], npieces = h_tot[3], nslots = h_tot[4],
                             nsplit = h_tot[5];
    if (nranges > (unsigned long long)INT_MAX || nitems > (unsigned long long)INT_MAX ||
        nslots > (unsigned long long)INT_MAX)
        return ~(size_t)0;
    auto a256 = [](unsigned long long b) { return (size_t)((b + 255) & ~255ull); };
    const size_t o_ranges = L.bytes, o_items = o_ranges + a256(nranges * sizeof(int2)),
                 o_pieces = o_items + a256(nitems * sizeof(int2)), o_split = o_pieces + a256(npieces * 6 * sizeof(int)),
                 o_part = o_split + a256(nsplit * sizeof(int2)), need = o_part + a256(nslots * 4 * sizeof(double)) + 256;
    if (tmp_bytes < need) return need;
    unsigned char* b = (unsigned char*)tmp;
    int2* ranges = (int2*)(b + o_ranges);
    int2* items = (int2*)(b + o_items);
    int* pv = (int*)(b + o_pieces);
    const size_t npv = (size_t)npieces;
    const Pieces pc{pv, pv + npv, pv + 2 * npv, pv + 3 * npv, pv + 4 * npv, pv + 5 * npv};
    int2* split = (int2*)(b + o_split);
    double* part = (double*)(b + o_part);
    const unsigned g = grid_for((long long)nleaves * 32, kEmitWarps * 32, 16);  // one warp per leaf
    k_p2p_emit<<<g, kEmitWarps * 32, 0, s>>>(c, list, seg_start, seg_end, leaves, nleaves, mode, L.order, L.roff,
                                             L.nb, L.ioff, L.nit, L.voff, L.npc, pc, ranges, items, split, L.tot);
    note_launch();
    if (nitems == 0) return need;
    auto go = [&](auto kern) {
        kern<<<nblocks, kP2PWarpsM * 32, 0, s>>>(xp, c, leaves, ranges, pc, items, (int)nitems, L.counter, psi, acc,
                                                 part);
    };
    mark_begin(s);
    if (mode == 1) go(k_p2p_mixed<1>);
    else if (mode == 2) go(k_p2p_mixed<2>);
    else if (mode == 3) go(k_p2p_mixed<3>);
    else go(k_p2p_mixed<0>);
    mark_end(s);
    note_launch();
    if (nsplit > 0) {
        k_p2p_reduce<<<grid_for((long long)nsplit * 32, 128, 16), 128, 0, s>>>(c, leaves, L.np, split, (int)nsplit,
                                                                              part, psi, acc);
        note_launch();
    }
    return need;
}

}  // namespace gb3
