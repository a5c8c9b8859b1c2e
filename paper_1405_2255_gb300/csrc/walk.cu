// walk.cu -- A8 of the path: the one-sided dual tree walk (Sec. 2.2.2) with the
// acceptance criteria of eqs. (9), (15)-(18), run breadth-first: every step takes
// the current frontier of cell pairs and writes M2L pairs, P2P pairs and the next
// frontier.  Afterwards the lists are sorted by (sink, source), which fixes the
// order in which every sink accumulates its interactions.
#include "kernels.cuh"

namespace gb3 {

// exclusive warp prefix of v; returns the warp total in *tot
__device__ inline unsigned warp_excl(unsigned v, unsigned* tot) {
    const int lane = threadIdx.x & 31;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    *tot = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// reserve `mine` slots in a list for each lane; returns the lane's first slot or -1 on overflow
__device__ inline long long warp_reserve(unsigned mine, unsigned long long* counter, long long cap,
                                         unsigned long long* overflow) {
    unsigned tot;
    unsigned ex = warp_excl(mine, &tot);
    unsigned long long base = 0;
    if ((threadIdx.x & 31) == 31 && tot) base = atomicAdd(counter, (unsigned long long)tot);
    base = __shfl_sync(0xffffffffu, base, 31);
    if (tot && (long long)(base + tot) > cap) {
        if ((threadIdx.x & 31) == 31) atomicOr(overflow, 1ull);
        return -1;
    }
    return (long long)(base + ex);
}

enum : int { kActNone = 0, kActM2L, kActP2P, kActSelf, kActSplitA, kActSplitB };

// ---------------------------------------------------------------- single-precision pre-test
// The decisions theta < 1 (eq. 9) and E~_{A->B} M_A / r^2 < eps minscale_B (eqs. 15-18)
// are first taken in FP32 with bounds on the rounding error; a value within a margin of
// its threshold, or outside the range in which the bounds hold, leaves the decision to
// the FP64 form below, so every decision is the one FP64 takes.
//  r: each centre difference is formed from two-float centres (high parts, then low
//     parts) with an error of at most 2^-23 |d| + 2^-46 (|a| + |b|); requiring
//     2^-24 sum|coordinates| < r keeps the relative error of r below 2^-19
//  theta = (rho_A + rho_B) / r: relative error below 3e-6 (rsqrt.approx within 2^-22);
//     margin 1e-5
//  E~ M_A / r^2 = fac P_0 h / r^2 with h = sum_k C(p,k) Pn_k u_A^k u_B^(p-k), u = rho / r < 1
//     and Pn_k = P_k / (P_0 rho_A^k) in [0, 1]: every factor of a term carries at most
//     3e-6, so h is within (p + 3) 3e-6 < 6e-5 for p <= 16; margin 2e-4; an h below
//     2^-90 (underflowed terms) is left to FP64
constexpr float kThetaMargin = 1e-5f, kMacMargin = 2e-4f;

struct PascalF {
    float c[kMaxP + 1][kMaxP + 1];
    constexpr PascalF() : c{} {
        for (int q = 0; q <= kMaxP; ++q) {
            c[q][0] = 1.f;
            for (int k = 1; k <= q; ++k) c[q][k] = c[q - 1][k - 1] + (k < q ? c[q - 1][k] : 0.f);
        }
    }
};
// C(q, k) for q <= 20: integers below 2^24, exact in FP32
static __constant__ PascalF c_pascalf = PascalF();

__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 1: accepted, 0: not accepted, -1: left to FP64
__device__ __forceinline__ int accept_fp32(const WalkParams& wp, int A, int B) {
    const float4 ah = wp.fc[2 * A], al = wp.fc[2 * A + 1];
    const float4 bh = wp.fc[2 * B], bl = wp.fc[2 * B + 1];
    const float dx = (bh.x - ah.x) + (bl.x - al.x);
    const float dy = (bh.y - ah.y) + (bl.y - al.y);
    const float dz = (bh.z - ah.z) + (bl.z - al.z);
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float e = (fabsf(ah.x) + fabsf(ah.y) + fabsf(ah.z) + fabsf(bh.x) + fabsf(bh.y) + fabsf(bh.z)) * 0x1p-24f;
    if (!(r2 >= 0x1p-100f) || !(e * e < r2)) return -1;
    const float rinv = rsqrt_approx(r2);
    const float ra = ah.w, rb = bh.w;
    const float th = (ra + rb) * rinv;
    if (th >= 1.0f + kThetaMargin) return 0;
    if (!(th < 1.0f - kThetaMargin)) return -1;
    if (wp.mac == kMacEstimate) return 1;
    const float* Pn = wp.fP + (size_t)A * wp.fstride;
    const float rhs = wp.fP[(size_t)B * wp.fstride + wp.p + 1];
    const float ua = ra * rinv, ub = rb * rinv;
    const float* C = c_pascalf.c[wp.p];
    float h = 0.f, uak = 1.f;
    for (int k = 0; k <= wp.p; ++k) {
        h = h * ub + C[k] * (Pn[k] * uak);
        uak *= ua;
    }
    if (!(h >= 0x1p-90f)) return -1;
    const float mx = ra > rb ? ra : rb;
    const float fac = (ra + rb > 0.f) ? 8.0f * mx / (ra + rb) : 8.0f;
    const float lhs = fac * h * al.w * (rinv * rinv);
    if (lhs < rhs * (1.0f - kMacMargin)) return 1;
    if (lhs > rhs * (1.0f + kMacMargin)) return 0;
    return -1;
}

// the single-precision view of one cell; a cell out of the bounds' range gets NaN radius
// and P_0, which sends its pairs to FP64.  Without P (the estimator's walk) the P_0 slot
// holds the cell's mass instead
__global__ void k_walk_prep(Cells c, const d4* __restrict__ cen, const double* __restrict__ P, int p, double eps,
                            int nc, float4* __restrict__ fc, float* __restrict__ fP, int fstride) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= nc) return;
    const d4 v = cen[cell];
    const double lim = 0x1p100;
    bool ok = fabs(v.x) <= lim && fabs(v.y) <= lim && fabs(v.z) <= lim && v.w >= 0.0 && v.w <= lim;
    const float hx = (float)v.x, hy = (float)v.y, hz = (float)v.z;
    const float lx = (float)(v.x - (double)hx), ly = (float)(v.y - (double)hy), lz = (float)(v.z - (double)hz);
    float p0 = 0.f;
    if (P) {
        const double* Pc = P + (size_t)cell * (p + 1);
        float* row = fP + (size_t)cell * fstride;
        const double P0 = Pc[0];
        bool okp = P0 >= 0x1p-100 && P0 <= lim;
        const double rinv = v.w > 0.0 ? 1.0 / v.w : 0.0;
        double sc = okp ? 1.0 / P0 : 0.0;
        row[0] = 1.f;
        for (int k = 1; k <= p; ++k) {
            if (v.w > 0.0) {
                sc *= rinv;
                const double t = Pc[k] * sc;
                okp = okp && t >= 0.0 && t <= 2.0;
                row[k] = (float)t;
            } else {
                okp = okp && Pc[k] == 0.0;
                row[k] = 0.f;
            }
        }
        const double rhs = eps * c.minscale[cell];
        row[p + 1] = (rhs >= 0x1p-100 && rhs <= lim) ? (float)rhs : __int_as_float(0x7fc00000);
        p0 = okp ? (float)P0 : __int_as_float(0x7fc00000);
    }
    else {  // the estimator's view: the cell's mass in the P_0 slot
        const double m = c.mass[cell];
        ok = ok && (m == 0.0 || (m >= 0x1p-100 && m <= lim));
        p0 = (float)m;
    }
    const float rho = ok ? (float)v.w : __int_as_float(0x7fc00000);
    if (!ok) p0 = __int_as_float(0x7fc00000);
    fc[2 * cell] = make_float4(hx, hy, hz, rho);
    fc[2 * cell + 1] = make_float4(lx, ly, lz, p0);
}

void launch_walk_prep(Cells c, const d4* cen, const double* P, int p, double eps, int nc, float4* fc, float* fP,
                      cudaStream_t s) {
    if (nc <= 0) return;
    k_walk_prep<<<(nc + 127) / 128, 128, 0, s>>>(c, cen, P, p, eps, nc, fc, fP, walk_fstride(p));
    note_launch();
}

// nfront_dev (nullable): the frontier's length on the device (read here, capped at the
// buffer's capacity), else nfront; the next frontier is counted in *out_cnt
// 32 registers (a few spills) so that the launch of 8 blocks per SM is one wave: the steps are
// bound by the latency of the cell gathers
__global__ void __launch_bounds__(256, 8) k_walk(Cells c, WalkParams wp, const int2* __restrict__ front_in, long long nfront,
                       const unsigned long long* __restrict__ nfront_dev, int2* __restrict__ front_out, WalkBuffers wb,
                       unsigned long long* __restrict__ out_cnt) {
    if (nfront_dev) {
        const unsigned long long nd = *nfront_dev;
        if (blockIdx.x == 0 && threadIdx.x == 0 && nd) atomicMax(&wb.counters[5], nd);  // demand seen
        // after an overflow the frontier may have holes: no further steps (the walk is redone)
        if (*(volatile const unsigned long long*)&wb.counters[3]) return;
        nfront = (long long)nd < wb.front_cap ? (long long)nd : wb.front_cap;
    }
    // cnt_A cnt_B < p2p_thresh as integers: the product of two counts is exact in FP64
    // below 2^53 and far above any threshold beyond it
    const double tc = ceil(wp.p2p_thresh);
    const long long thr = tc <= 0.0 ? 0LL : (tc >= 0x1p62 ? (1LL << 62) : (long long)tc);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < nfront; base += stride) {
        long long i = base + threadIdx.x;
        int act = kActNone, A = -1, B = -1, nchA = 0, nchB = 0, chA = 0, chB = 0;
        if (i < nfront && cell_active(c, front_in[i].y)) {  // a sink without active particles has no work
            int2 pr = front_in[i];
            A = pr.x;
            B = pr.y;
            const long long cntA = c.count[A], cntB = c.count[B];
            nchA = c.nchild[A];
            nchB = c.nchild[B];
            chA = c.child[A];
            chB = c.child[B];
            if (cntA * cntB < thr) {
                act = kActP2P;  // reading R-p2p: direct summation is preferable
            } else if (A == B) {
                act = nchA ? kActSelf : kActP2P;
            } else {
                const d4* cen = wp.use_com ? c.cr : c.sr;
                const int dec = (wp.fc && !wp.adaptive && wp.mac != FMM_MAC_THETA) ? accept_fp32(wp, A, B) : -1;
                bool accept = dec == 1;
                if (dec < 0) {
                    const d4 za = cen[A], sb = cen[B];
                    double ra = za.w, rb = sb.w;
                    double dx = sb.x - za.x, dy = sb.y - za.y, dz = sb.z - za.z;
                    double r = sqrt(dx * dx + dy * dy + dz * dz);
                    double theta = (ra + rb) / r;  // eq. (9)
                    if (wp.mac == FMM_MAC_THETA) accept = theta < wp.theta_crit;
                    else if (!(theta < 1.0)) accept = false;
                    else if (wp.mac == kMacEstimate) accept = true;
                    else {
                        // E~_{A->B} M_A / r^2 (eqs. 15-17) without dividing by M_A:
                        // 8 max/(rhoA+rhoB) * sum_k C(p,k) P_k rhoB^{p-k} / r^{p+2}
                        const double* P = wp.P + (size_t)A * (wp.p + 1);
                        double rinv = 1.0 / r, u = rb * rinv, rk = 1.0, h = 0.0;
                        for (int k = 0; k <= wp.p; ++k) {
                            h = h * u + wp.binom[k] * (P[k] * rk);
                            rk *= rinv;
                        }
                        double mx = ra > rb ? ra : rb;
                        double fac = (ra + rb > 0) ? 8.0 * mx / (ra + rb) : 8.0;
                        double lhs = fac * h / (r * r);
                        const double rhs = wp.eps * c.minscale[B];
                        accept = lhs < rhs;  // eqs. (18a,b)
                        if (accept && wp.adaptive) {
                            // the lowest order q whose E~ (eq. 17 with q for p) passes as well
                            for (int q = wp.p_lo; q < wp.p; ++q) {
                                const double* C = wp.pascal + q * (kMaxP + 1);
                                double hq = 0.0, rq = 1.0;
                                for (int k = 0; k <= q; ++k) {
                                    hq = hq * u + C[k] * (P[k] * rq);
                                    rq *= rinv;
                                }
                                if (fac * hq / (r * r) < rhs) {
                                    A |= q << kM2LOrderShift;
                                    break;
                                }
                            }
                        }
                    }
                }
                if (accept) act = kActM2L;
                else if (!nchA && !nchB) act = kActP2P;
                else {
                    // rounding to FP32 keeps the order of distinct radii except for ties
                    bool split_a;
                    const float fa = dec >= 0 ? wp.fc[2 * A].w : 0.f, fb = dec >= 0 ? wp.fc[2 * B].w : 0.f;
                    if (dec >= 0 && fa != fb) split_a = fa > fb;
                    else split_a = cen[A].w >= cen[B].w;
                    if (!nchA) split_a = false;
                    if (!nchB) split_a = true;
                    act = split_a ? kActSplitA : kActSplitB;
                }
            }
        }
        unsigned nm = act == kActM2L, np = act == kActP2P;
        unsigned nf = act == kActSelf ? nchA * nchA : act == kActSplitA ? nchA : act == kActSplitB ? nchB : 0;
        long long om = warp_reserve(nm, &wb.counters[1], wb.m2l_cap, &wb.counters[3]);
        long long op = warp_reserve(np, &wb.counters[2], wb.p2p_cap, &wb.counters[3]);
        long long of = warp_reserve(nf, out_cnt, wb.front_cap, &wb.counters[3]);
        if (nm && om >= 0) wb.m2l[om] = make_int2(A, B);
        if (np && op >= 0) wb.p2p[op] = make_int2(A, B);
        if (nf && of >= 0) {
            if (act == kActSelf) {
                for (int a = 0; a < nchA; ++a)
                    for (int b = 0; b < nchA; ++b) front_out[of + a * nchA + b] = make_int2(chA + a, chA + b);
            } else if (act == kActSplitA) {
                for (int a = 0; a < nchA; ++a) front_out[of + a] = make_int2(chA + a, B);
            } else {
                for (int b = 0; b < nchB; ++b) front_out[of + b] = make_int2(A, chB + b);
            }
        }
    }
}

__global__ void k_walk_roots(int2* front, int nroots, unsigned long long* count) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nroots; r += gridDim.x * blockDim.x) front[r] = make_int2(r, r);
    if (count && blockIdx.x == 0 && threadIdx.x == 0) *count = (unsigned long long)nroots;
}
void launch_walk_roots(int2* front, int nroots, cudaStream_t s, unsigned long long* count) {
    if (nroots > 0) k_walk_roots<<<grid_for(nroots, 256), 256, 0, s>>>(front, nroots, count); note_launch();
}

void launch_walk_step(Cells c, WalkParams wp, const int2* front_in, long long nfront, int2* front_out,
                      WalkBuffers wb, cudaStream_t s) {
    if (nfront <= 0) return;
    k_walk<<<grid_for(nfront, 256, 16), 256, 0, s>>>(c, wp, front_in, nfront, nullptr, front_out, wb,
                                                             &wb.counters[0]);
    note_launch();
}
void launch_walk_step_dev(Cells c, WalkParams wp, const int2* front_in, const unsigned long long* nfront_dev,
                          int2* front_out, WalkBuffers wb, unsigned long long* out_cnt, cudaStream_t s) {
    k_walk<<<sm_count() * 8, 256, 0, s>>>(c, wp, front_in, 0, nfront_dev, front_out, wb, out_cnt);
    note_launch();
}

// ---------------------------------------------------------------- list sort
static int bits_for(long long v) {
    int b = 1;
    while ((1LL << b) < v) ++b;
    return b;
}

// key = (sink << xb) | first entry: the first entry (taken as unsigned) in the low xb bits
__global__ void k_pack_pairs(const int2* __restrict__ list, long long n, int xb, uint64_t* __restrict__ keys) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int2 v = list[i];
        keys[i] = ((uint64_t)(unsigned)v.y << xb) | (uint64_t)(unsigned)v.x;
    }
}
__global__ void k_unpack_pairs(const uint64_t* __restrict__ keys, long long n, int xb, int2* __restrict__ list) {
    const uint64_t mask = xb >= 32 ? 0xffffffffull : (1ull << xb) - 1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        list[i] = make_int2((int)(unsigned)(k & mask), (int)(k >> xb));
    }
}

size_t list_sort_tmp_bytes(long long npairs, int /*ncells*/) {
    const size_t n = (size_t)(npairs > 0 ? npairs : 1);
    return n * 2 * sizeof(uint64_t) + radix_tmp_ints((long long)n) * sizeof(int) + 256;
}

// LSD radix passes over the keys alone (8 bits per pass over the xb + sb bits in use)
void sort_pairs_by_sink(int2* list, long long npairs, int ncells, void* tmp, cudaStream_t s, bool wide) {
    if (npairs <= 1) return;
    const int sb = bits_for(ncells);
    const int xb = wide ? 32 : sb;
    uint64_t* k0 = (uint64_t*)tmp;
    uint64_t* k1 = k0 + npairs;
    int* rtmp = (int*)(k1 + npairs);
    const unsigned g = grid_for(npairs, 256);
    k_pack_pairs<<<g, 256, 0, s>>>(list, npairs, xb, k0);
    note_launch();
    const int flip = radix_sort_pairs_bits(k0, nullptr, k1, nullptr, npairs, rtmp, 0, xb + sb, s);
    k_unpack_pairs<<<g, 256, 0, s>>>(flip ? k1 : k0, npairs, xb, list);
    note_launch();
}

__global__ void k_segments(const int2* __restrict__ list, long long n, int* __restrict__ seg_start,
                           int* __restrict__ seg_end) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int b = list[i].y;
        if (i == 0 || list[i - 1].y != b) seg_start[b] = (int)i;
        if (i == n - 1 || list[i + 1].y != b) seg_end[b] = (int)(i + 1);
    }
}

void launch_segments(const int2* list, long long npairs, int ncells, int* seg_start, int* seg_end, cudaStream_t s) {
    cudaMemsetAsync(seg_start, 0, sizeof(int) * (size_t)ncells, s);
    cudaMemsetAsync(seg_end, 0, sizeof(int) * (size_t)ncells, s);
    if (npairs > 0) k_segments<<<grid_for(npairs, 256), 256, 0, s>>>(list, npairs, seg_start, seg_end); note_launch();
}

}  // namespace gb3
