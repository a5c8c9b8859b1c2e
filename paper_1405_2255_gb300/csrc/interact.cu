// interact.cu -- A9-A12 of the path: M2L (eq. 3b), L2L (eq. 5), L2P (eqs. 3a, 7),
// P2P (eq. 1) in FP64 and in mixed precision, the p = 0 kernels of the low-order
// f estimate (Sec. 5.3.2), and the final scatter to the caller's order.
#include "harmonics.cuh"
#include "kernels.cuh"

namespace gb3 {

// ---------------------------------------------------------------- M2L
// conj(M_A) of every cell as a full complex array (all m), once per evaluation, so
// that M2L reads it instead of re-expanding the real storage for every pair
__global__ void k_expand_conj(const double* __restrict__ M, int ncells, int p, cd* __restrict__ Mc) {
    const int nco = ncoef(p);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)ncells * nco;
         t += (long long)gridDim.x * blockDim.x) {
        const int cell = (int)(t / nco), i = (int)(t % nco);
        int n = (int)sqrtf((float)i);
        while (n * n > i) --n;
        while ((n + 1) * (n + 1) <= i) ++n;
        const cd v = load_real_storage(M + (size_t)cell * nco, n, i - n * n - n);
        Mc[t] = conjc(v);
    }
}

// One warp per sink cell B.  Its sources (a segment of the sorted M2L list) are
// taken NB at a time: the warp copies conj(M_A) of the NB sources to shared
// memory and builds Theta(s_B - z_A) for all NB pairs at once (32/NB lanes per
// pair, each lane a few m-columns), so that the serial recurrences of one pair
// do not leave the other lanes idle; then each lane accumulates its scheduled
// outputs F_n^m(s_B) over the NB pairs in registers.  Warps take sinks from an
// atomic counter over the sinks ordered by decreasing list length.
template <int MAXQ, int NB>
__global__ void __launch_bounds__(64) k_m2l(const int2* __restrict__ list, const int* __restrict__ seg_start,
                                            const int* __restrict__ seg_end, const int* __restrict__ order,
                                            int nsinks, unsigned* __restrict__ work, const d4* __restrict__ cen,
                                            const cd* __restrict__ Mc, int p, double* __restrict__ F,
                                            LaneSched sched) {
    extern __shared__ cd csm[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nco = ncoef(p);
    cd* T = csm + (size_t)wid * 2 * NB * nco;  // [NB][nco]
    cd* Mb = T + NB * nco;                     // [NB][nco]
    constexpr int LPP = 32 / NB;               // lanes per pair while building Theta
    const int cnt = sched.cnt[lane];
    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(work, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= (unsigned)nsinks) break;
        const int B = order[w];
        const int e0 = seg_start[B], e1 = seg_end[B];
        if (e1 <= e0) continue;
        const d4 sB = cen[B];
        cd acc[MAXQ];
#pragma unroll
        for (int q = 0; q < MAXQ; ++q) acc[q] = mkc(0.0, 0.0);
        for (int eb = e0; eb < e1; eb += NB) {
            const int nb = min(NB, e1 - eb);
            // conj(M) of the batch
            for (int b = 0; b < nb; ++b) {
                const cd* src = Mc + (size_t)m2l_src(list[eb + b].x) * nco;
                for (int i = lane; i < nco; i += 32) Mb[b * nco + i] = src[i];
            }
            // Theta of the batch
            {
                const int b = lane / LPP, sub = lane % LPP;
                if (b < nb) {
                    const d4 zA = cen[m2l_src(list[eb + b].x)];
                    const double x = sB.x - zA.x, y = sB.y - zA.y, z = sB.z - zA.z;
                    for (int m = sub; m <= p; m += LPP) theta_column(p, m, x, y, z, T + b * nco);
                }
            }
            __syncwarp();
            for (int b = 0; b < nb; ++b) {
                const int pb = m2l_order(list[eb + b].x, p);  // the pair's order (adaptive walk) or p
#pragma unroll
                for (int q = 0; q < MAXQ; ++q)
                    if (q < cnt && sched.n[lane][q] <= pb)
                        acc[q] = acc[q] + contract(pb, sched.n[lane][q], sched.m[lane][q], Mb + b * nco, T + b * nco);
            }
            __syncwarp();
        }
        double* out = F + (size_t)B * nco;
#pragma unroll
        for (int q = 0; q < MAXQ; ++q) {
            if (q < cnt) {
                int n = sched.n[lane][q], m = sched.m[lane][q];
                out[cix(n, m)] = acc[q].re;
                if (m) out[cix(n, -m)] = acc[q].im;
            }
        }
    }
}

// sinks with a non-empty M2L segment, ordered by decreasing segment length (eight steps per
// octave, qlen8)
__global__ void k_sink_keys(const int* __restrict__ seg_start, const int* __restrict__ seg_end, int ncells,
                            uint64_t* __restrict__ keys, int* __restrict__ vals) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncells; i += gridDim.x * blockDim.x) {
        unsigned len = (unsigned)(seg_end[i] - seg_start[i]);
        keys[i] = ((uint64_t)(255u - qlen8(len)) << 32) | (unsigned)i;
        vals[i] = len ? 1 : 0;
    }
}
__global__ void k_sink_order(const uint64_t* __restrict__ keys, int ncells, int* __restrict__ order,
                             unsigned* __restrict__ nsinks) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncells; i += gridDim.x * blockDim.x) {
        uint64_t k = keys[i];
        unsigned q = 255u - (unsigned)(k >> 32);  // 0: an empty list (sorted last)
        order[i] = (int)(k & 0xffffffffu);
        if (q && (i == ncells - 1 || (255u - (unsigned)(keys[i + 1] >> 32)) == 0)) *nsinks = (unsigned)(i + 1);
    }
}

size_t m2l_tmp_bytes(int ncells, int p) {
    size_t n = (size_t)(ncells > 0 ? ncells : 1);
    return n * (2 * sizeof(uint64_t) + 3 * sizeof(int)) + radix_tmp_ints(n) * sizeof(int) + 256 +
           n * (size_t)ncoef(p) * sizeof(cd);
}

template <int MAXQ, int NB>
static void m2l_launch(const int2* list, const int* seg_start, const int* seg_end, const int* order, int ncells,
                       unsigned* work, const d4* cen, const cd* Mc, int p, double* F, const LaneSched& sched,
                       cudaStream_t s) {
    const int wpb = 2;
    size_t sm = (size_t)wpb * 2 * NB * ncoef(p) * sizeof(cd);
    cudaFuncSetAttribute(k_m2l<MAXQ, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int dev = 0, nsm = 152, bps = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_m2l<MAXQ, NB>, wpb * 32, sm);
    unsigned g = (unsigned)(nsm * (bps > 0 ? bps : 1));
    k_m2l<MAXQ, NB><<<g, wpb * 32, sm, s>>>(list, seg_start, seg_end, order, ncells, work, cen, Mc, p, F, sched);
    note_launch();
}

void launch_m2l(const int2* list, const int* seg_start, const int* seg_end, void* tmp, int ncells, const d4* cen,
                const double* M, int p, double* F, cudaStream_t s) {
    if (ncells <= 0) return;
    init_rec_tables();
    // order the sinks by decreasing work
    uint64_t* k0 = (uint64_t*)tmp;
    uint64_t* k1 = k0 + ncells;
    int* v0 = (int*)(k1 + ncells);
    int* v1 = v0 + ncells;
    int* order = v1 + ncells;
    unsigned* work = (unsigned*)(order + ncells);  // [0] counter, [1] number of sinks
    int* rtmp = (int*)(work + 4);
    cd* Mc = (cd*)(((uintptr_t)(rtmp + radix_tmp_ints(ncells)) + 255) & ~(uintptr_t)255);
    cudaMemsetAsync(work, 0, 4 * sizeof(unsigned), s);
    k_sink_keys<<<grid_for(ncells, 256), 256, 0, s>>>(seg_start, seg_end, ncells, k0, v0); note_launch();
    // the low 32 bits are the sink's index, already in order: the stable pass over the 8
    // length bits alone keeps ties in index order
    int flip = radix_sort_pairs_bits(k0, v0, k1, v1, ncells, rtmp, 32, 40, s);
    k_sink_order<<<grid_for(ncells, 256), 256, 0, s>>>(flip ? k1 : k0, ncells, order, work + 1); note_launch();
    k_expand_conj<<<grid_for((long long)ncells * ncoef(p), 256), 256, 0, s>>>(M, ncells, p, Mc); note_launch();
    LaneSched sched = make_lane_sched(p, kSchedDown);
    int maxq = 0;
    for (int l = 0; l < 32; ++l) maxq = sched.cnt[l] > maxq ? sched.cnt[l] : maxq;
    // every cell is visited (empty segments cost one counter step); the order puts them last
    if (p <= 12) {
        if (maxq <= 4) m2l_launch<4, 8>(list, seg_start, seg_end, order, ncells, work, cen, Mc, p, F, sched, s);
        else m2l_launch<8, 8>(list, seg_start, seg_end, order, ncells, work, cen, Mc, p, F, sched, s);
    } else if (p <= 16) {
        if (maxq <= 8) m2l_launch<8, 4>(list, seg_start, seg_end, order, ncells, work, cen, Mc, p, F, sched, s);
        else m2l_launch<12, 4>(list, seg_start, seg_end, order, ncells, work, cen, Mc, p, F, sched, s);
    } else {
        m2l_launch<24, 2>(list, seg_start, seg_end, order, ncells, work, cen, Mc, p, F, sched, s);
    }
}

// ---------------------------------------------------------------- M2L, precision-split (mixed mode)
// F_n^m = sum_{k,l} M_k^{l*} Theta_{n+k}^{m+l} split by the order j = n + k of Theta.
// Terms with j <= kJ64 (monopole, dipole, quadrupole of the source seen by the
// sink's lowest orders) are summed in FP64.  All other terms are summed in FP32:
// the acceptance criterion keeps theta of an accepted pair near eps^(1/p), so a
// term of order j carries a fraction <~ theta^(j-1) of the interaction and its
// FP32 rounding (6e-8 relative) is far below the targeted force error.  To keep
// FP32 in range the FP32 part is evaluated on scaled quantities:
//   Mt_k = M_k / rho_A^k (per source cell),  That_j = Theta_j(r/|r|) (unit vector),
//   Mhat_k = Mt_k (rho_A/|r|)^k,  G_n = sum Mhat* That = |r|^{n+1} F_n(pair),
//   H_n = sum_pairs G_n (sigma_B/|r|)^{n+1} = sigma_B^{n+1} F_n(FP32 part),
// with sigma_B = rho_B (or half the closest pair distance when rho_B = 0); the sink
// converts H_n / sigma_B^{n+1} to FP64 once.
constexpr int kJ64 = 2;
constexpr int kN64 = (kJ64 + 1) * (kJ64 + 1);  // FP64 coefficients per expansion (orders <= kJ64)
constexpr int kT64 = 20;                       // FP64 complex terms per pair for kJ64 = 2

struct TermTab {
    unsigned char n[kT64], m[kT64], k[kT64];
    signed char l[kT64];
    unsigned char out[kT64];  // output index n(n+1)/2 + m
};
static __constant__ TermTab c_terms;
static __constant__ unsigned char c_idx_n[(kMaxP + 1) * (kMaxP + 1)];

static void init_split_tables() {
    static DeviceOnce once;
    once_per_device(once, [] {
        TermTab t;
        int q = 0;
        for (int n = 0; n <= kJ64; ++n)
            for (int m = 0; m <= n; ++m)
                for (int k = 0; k + n <= kJ64; ++k)
                    for (int l = -k; l <= k; ++l) {
                        t.n[q] = (unsigned char)n; t.m[q] = (unsigned char)m; t.k[q] = (unsigned char)k;
                        t.l[q] = (signed char)l; t.out[q] = (unsigned char)(n * (n + 1) / 2 + m);
                        ++q;
                    }
        cudaMemcpyToSymbol(c_terms, &t, sizeof t);
        unsigned char idx[(kMaxP + 1) * (kMaxP + 1)];
        for (int n = 0; n <= kMaxP; ++n)
            for (int m = -n; m <= n; ++m) idx[cix(n, m)] = (unsigned char)n;
        cudaMemcpyToSymbol(c_idx_n, idx, sizeof idx);
    });
}


// Theta_j^m(r), j <= 2, m >= 0, in closed form (consistent with the recurrences)
__device__ inline cd theta_low(int j, int m, double x, double y, double z, double rinv) {
    const double r2i = rinv * rinv, r3 = rinv * r2i, r5 = r3 * r2i;
    if (j == 0) return mkc(rinv, 0.0);
    if (j == 1) return m == 0 ? mkc(z * r3, 0.0) : mkc(x * r3, y * r3);
    if (m == 0) return mkc((3.0 * z * z - (x * x + y * y + z * z)) * r5, 0.0);
    if (m == 1) return mkc(3.0 * z * x * r5, 3.0 * z * y * r5);
    return mkc(3.0 * (x * x - y * y) * r5, 6.0 * x * y * r5);
}

// per cell: conj(M_k / rho^k) in FP32 (all orders) and conj(M_k) in FP64 (orders <= kJ64);
// one warp per cell, lane n holding rho^-n
__global__ void k_prep_split(const double* __restrict__ M, const d4* __restrict__ cen, int ncells, int p,
                             float2* __restrict__ Mf, cd* __restrict__ M64) {
    const int nco = ncoef(p), lane = threadIdx.x & 31;
    for (long long cell = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; cell < ncells;
         cell += ((long long)gridDim.x * blockDim.x) >> 5) {
        const double rho = cen[cell].w;
        double pw = lane == 0 ? 1.0 : 0.0;  // a source of radius 0 has no moments above the monopole
        if (rho > 0 && lane > 0 && lane <= p) {
            const double rinv = 1.0 / rho;
            pw = rinv;
            for (int k = 1; k < lane; ++k) pw *= rinv;
        }
        const double* R = M + (size_t)cell * nco;
        for (int i0 = 0; i0 < nco; i0 += 32) {  // uniform trip count: the shuffle needs every lane
            const int i = i0 + lane;
            const int n = i < nco ? c_idx_n[i] : 0;
            const double sc = __shfl_sync(0xffffffffu, pw, n);
            if (i < nco) {
                const cd v = load_real_storage(R, n, i - n * n - n);
                Mf[(size_t)cell * nco + i] = make_float2((float)(v.re * sc), (float)(-v.im * sc));
                if (i < kN64) M64[(size_t)cell * kN64 + i] = conjc(v);
            }
        }
    }
}

struct PairInfo {
    double x, y, z, rinv;
};

constexpr int kChunk = kM2LChunk;

// ---------------------------------------------------------------- split M2L by rounds of equal n
// Terms of order n + k <= 2 are summed in FP64 (spread over the lanes), the others
// in FP32 on the scaled quantities above.  A batch of up to kRB pairs of one sink
// is processed order by order: for output order n every lane takes one (pair, m)
// unit, so all lanes run the same k and l loops (their lengths depend on n only),
// and the units of a round are summed over the pairs in pair order.
constexpr int kRoundsBatch = 4;  // pairs per batch (the per-warp shared memory sets the occupancy)

template <int kRB>
struct RoundsSmem {
    static constexpr int kRBLo = (kRB * kT64 + 31) / 32;  // FP64 terms per lane per batch
    int nco;
    size_t Mh, Th, pi, thA, thB, res, outs, unit, M64, T64, red, lowF, idx, terms, pws, total;
    __host__ __device__ RoundsSmem(int p) {
        nco = (p + 1) * (p + 1);
        size_t o = 0;
        auto take = [&](size_t bytes) {
            const size_t at = o;
            o = (o + bytes + 15) & ~(size_t)15;
            return at;
        };
        Mh = take((size_t)kRB * nco * sizeof(float2));
        Th = take((size_t)kRB * nco * sizeof(float2));
        pi = take(kRB * sizeof(PairInfo));
        thA = take(kRB * (kMaxP + 2) * sizeof(float));
        thB = take(kRB * (kMaxP + 2) * sizeof(float));
        res = take((size_t)kRB * (kMaxP + 1) * sizeof(float2));
        outs = take((size_t)nco * sizeof(float));
        unit = take(kRB * sizeof(float4));
        M64 = take(kRB * kN64 * sizeof(cd));
        T64 = take(kRB * kN64 * sizeof(cd));
        red = take(32 * kRBLo * sizeof(cd));
        lowF = take(8 * sizeof(cd));
        idx = take((size_t)nco);
        terms = take(sizeof(TermTab));
        pws = take((kMaxP + 2) * sizeof(double));
        total = o;
    }
};

// one column m of Theta on a unit vector into full complex storage (coefficients of
// the recurrences computed in place: no lane-dependent constant-memory reads)
__device__ inline void theta_column_unit_f2(int p, int m, float x, float y, float z, float2* out) {
    float2 d = make_float2(1.f, 0.f);
    for (int j = 1; j <= m; ++j) {
        const float s = (float)(2 * j - 1);
        d = make_float2(s * (x * d.x - y * d.y), s * (x * d.y + y * d.x));
    }
    float2 prev2 = make_float2(0.f, 0.f), prev = d;
    const float sg = (m & 1) ? -1.f : 1.f;
    for (int n = m; n <= p; ++n) {
        float2 v = d;
        if (n > m) {
            const float a = (float)(2 * n - 1) * z, b = (float)((n - 1) * (n - 1) - m * m);
            v = make_float2(a * prev.x - b * prev2.x, a * prev.y - b * prev2.y);
            prev2 = prev;
            prev = v;
        }
        out[n * n + n + m] = v;
        if (m) out[n * n + n - m] = make_float2(sg * v.x, -sg * v.y);
    }
}

// sum over l = -k..k of X_k^l Y^{m+l}: offsets 0..2k of x and y, unrolled for each k
template <int K>
__device__ __forceinline__ void m2l_row_k(const float2* __restrict__ x, const float2* __restrict__ y, float2& a0,
                                          float2& a1, float2& a2, float2& a3) {
#pragma unroll
    for (int o = 0; o <= 2 * K; o += 4) {
        cmacf(a0, x[o], y[o]);
        if (o + 1 <= 2 * K) cmacf(a1, x[o + 1], y[o + 1]);
        if (o + 2 <= 2 * K) cmacf(a2, x[o + 2], y[o + 2]);
        if (o + 3 <= 2 * K) cmacf(a3, x[o + 3], y[o + 3]);
    }
}
__device__ __forceinline__ void m2l_row(int k, const float2* __restrict__ x, const float2* __restrict__ y, float2& a0,
                                        float2& a1, float2& a2, float2& a3) {
#define GB3_ROW(K) \
    case K: m2l_row_k<K>(x, y, a0, a1, a2, a3); break;
    switch (k) {
        GB3_ROW(0) GB3_ROW(1) GB3_ROW(2) GB3_ROW(3) GB3_ROW(4) GB3_ROW(5) GB3_ROW(6) GB3_ROW(7) GB3_ROW(8)
        GB3_ROW(9) GB3_ROW(10) GB3_ROW(11) GB3_ROW(12) GB3_ROW(13) GB3_ROW(14) GB3_ROW(15) GB3_ROW(16)
        GB3_ROW(17) GB3_ROW(18) GB3_ROW(19)
        default: m2l_row_k<20>(x, y, a0, a1, a2, a3); break;
    }
#undef GB3_ROW
}

template <int kRB>
__global__ void __launch_bounds__(32, 16) k_m2l_rounds(const int2* __restrict__ list,
                                                       const int* __restrict__ seg_start,
                                                       const int* __restrict__ seg_end, const int* __restrict__ order,
                                                       const int* __restrict__ item_start,
                                                       unsigned* __restrict__ work, const d4* __restrict__ cen,
                                                       const float2* __restrict__ Mf, const cd* __restrict__ M64g,
                                                       int p, double* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const RoundsSmem<kRB> L(p);
    constexpr int kRBLo = RoundsSmem<kRB>::kRBLo;
    const int nco = L.nco, lane = threadIdx.x;
    float2* Mh = (float2*)(sm_raw + L.Mh);    // [kRB][nco]
    float2* Th = (float2*)(sm_raw + L.Th);    // [kRB][nco]
    PairInfo* pi = (PairInfo*)(sm_raw + L.pi);
    float* thA = (float*)(sm_raw + L.thA);    // [kRB][kMaxP+2]: (rho_A/r)^k
    float* thB = (float*)(sm_raw + L.thB);    // [kRB][kMaxP+2]: (sigma_B/r)^k
    float2* res = (float2*)(sm_raw + L.res);  // [kRB * (n+1)] results of one order
    float* outs = (float*)(sm_raw + L.outs);     // FP32 part of the item's outputs
    float4* unit = (float4*)(sm_raw + L.unit);   // [kRB] unit vectors of the batch's pairs
    cd* M64 = (cd*)(sm_raw + L.M64);
    cd* T64 = (cd*)(sm_raw + L.T64);
    cd* red = (cd*)(sm_raw + L.red);
    cd* lowF = (cd*)(sm_raw + L.lowF);
    unsigned char* idx_n = sm_raw + L.idx;
    TermTab* terms = (TermTab*)(sm_raw + L.terms);
    double* pws = (double*)(sm_raw + L.pws);  // sigma_B^-n
    for (int i = lane; i < nco; i += 32) idx_n[i] = c_idx_n[i];
    if (lane == 0) *terms = c_terms;
    __syncwarp();
    const unsigned nitems = work[2], nsinks = work[1];
    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(work, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= nitems) break;
        int lo_i = 0, hi_i = (int)nsinks - 1;
        while (lo_i < hi_i) {
            const int mid = (lo_i + hi_i + 1) >> 1;
            if ((unsigned)item_start[mid] <= w) lo_i = mid;
            else hi_i = mid - 1;
        }
        const int B = order[lo_i];
        const int s0 = seg_start[B], s1 = seg_end[B];
        const int e0 = s0 + (int)(w - (unsigned)item_start[lo_i]) * kChunk, e1 = min(e0 + kChunk, s1);
        const d4 sB = cen[B];
        double sigma = sB.w;
        if (!(sigma > 0)) {  // radius 0: half the closest source distance (over the whole list)
            double rmin = INFINITY;
            for (int e = s0 + lane; e < s1; e += 32) {
                const d4 zA = cen[m2l_src(list[e].x)];
                const double dx = sB.x - zA.x, dy = sB.y - zA.y, dz = sB.z - zA.z;
                rmin = fmin(rmin, sqrt(dx * dx + dy * dy + dz * dz));
            }
            sigma = 0.5 * warp_min(rmin);
        }
        for (int i = lane; i < nco; i += 32) outs[i] = 0.f;
        cd lo[kRBLo];
#pragma unroll
        for (int i = 0; i < kRBLo; ++i) lo[i] = mkc(0.0, 0.0);
        for (int eb = e0; eb < e1; eb += kRB) {
            const int nb = min(kRB, e1 - eb);
            if (lane < nb) {
                const int xe = list[eb + lane].x;
                const d4 zA = cen[m2l_src(xe)];
                const double x = sB.x - zA.x, y = sB.y - zA.y, z = sB.z - zA.z;
                const double rinv = rsqrt(x * x + y * y + z * z);
                pi[lane] = PairInfo{x, y, z, rinv};
                // .w: the pair's order (adaptive walk) or p
                unit[lane] = make_float4((float)(x * rinv), (float)(y * rinv), (float)(z * rinv), (float)m2l_order(xe, p));
                const float ta = (float)(zA.w * rinv), tb = (float)(sigma * rinv);
                float a = 1.f, b = 1.f;
                for (int k = 0; k <= p + 1; ++k) {
                    thA[lane * (kMaxP + 2) + k] = a;
                    thB[lane * (kMaxP + 2) + k] = b;
                    a *= ta;
                    b *= tb;
                }
            }
            __syncwarp();
            // scaled FP32 moments and FP64 low orders of the batch's sources
            for (int b = 0; b < nb; ++b) {
                const int A = m2l_src(list[eb + b].x);
                const float2* src = Mf + (size_t)A * nco;
                const float* ta = thA + b * (kMaxP + 2);
                for (int i = lane; i < nco; i += 32) {
                    const float2 v = src[i];
                    const float sc = ta[idx_n[i]];
                    Mh[b * nco + i] = make_float2(v.x * sc, v.y * sc);
                }
                if (lane < kN64) M64[b * kN64 + lane] = M64g[(size_t)A * kN64 + lane];
            }
            // FP64 Theta of orders <= kJ64
            for (int t = lane; t < nb * 6; t += 32) {
                const int b = t / 6, o = t % 6;
                const int j = o < 1 ? 0 : (o < 3 ? 1 : 2), m = o - j * (j + 1) / 2;
                const PairInfo q = pi[b];
                const cd v = theta_low(j, m, q.x, q.y, q.z, q.rinv);
                T64[b * kN64 + cix(j, m)] = v;
                if (m) T64[b * kN64 + cix(j, -m)] = (m & 1) ? mkc(-v.re, v.im) : mkc(v.re, -v.im);
            }
            // FP32 Theta on the unit vectors: one column (pair, m) per lane and round
            for (int t = lane; t < nb * (p + 1); t += 32) {
                const int b = t / (p + 1), m = t % (p + 1);
                const float4 q = unit[b];
                theta_column_unit_f2(p, m, q.x, q.y, q.z, Th + b * nco);
            }
            __syncwarp();
            // FP64 terms of orders n + k <= kJ64, spread over the lanes
#pragma unroll
            for (int i = 0; i < kRBLo; ++i) {
                const int t = lane + 32 * i, b = t / kT64, id = t % kT64;
                if (t < kRB * kT64 && b < nb) {
                    const int n = terms->n[id], m = terms->m[id], k = terms->k[id], l = terms->l[id];
                    cmac(lo[i], M64[b * kN64 + cix(k, l)], T64[b * kN64 + cix(n + k, m + l)]);
                }
            }
            // FP32 terms of orders n + k > kJ64: order by order, one (pair, m) unit per lane
            for (int n = 0; n <= p; ++n) {
                const int kmin = n > kJ64 ? 0 : kJ64 + 1 - n;
                if (kmin > p - n) continue;
                const int units = nb * (n + 1);
                for (int u0 = 0; u0 < units; u0 += 32) {
                    const int u = u0 + lane;
                    const bool act = u < units;
                    const int b = act ? u / (n + 1) : 0, m = act ? u % (n + 1) : 0;
                    const float2* X = Mh + b * nco;
                    const float2* Y = Th + b * nco;
                    const int kmax = (int)unit[b].w - n;  // k <= q - n for a pair of order q
                    float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
                    for (int k = kmin; k <= kmax; ++k)
                        m2l_row(k, X + k * k, Y + (n + k) * (n + k) + n + m, a0, a1, a2, a3);
                    if (act) {
                        const float sc = thB[b * (kMaxP + 2) + n + 1];
                        res[u] = make_float2((a0.x + a1.x + a2.x + a3.x) * sc, (a0.y + a1.y + a2.y + a3.y) * sc);
                    }
                }
                __syncwarp();
                for (int m = lane; m <= n; m += 32) {
                    float2 t = res[m];
                    for (int b = 1; b < nb; ++b) {
                        const float2 v = res[b * (n + 1) + m];
                        t.x += v.x;
                        t.y += v.y;
                    }
                    outs[n * n + n + m] += t.x;
                    if (m) outs[n * n + n - m] += t.y;
                }
                __syncwarp();
            }
        }
        // reduce the FP64 terms per output in a fixed order
#pragma unroll
        for (int i = 0; i < kRBLo; ++i) red[lane * kRBLo + i] = lo[i];
        __syncwarp();
        if (lane < 6) {
            cd sum = mkc(0.0, 0.0);
            for (int Ln = 0; Ln < 32; ++Ln)
                for (int i = 0; i < kRBLo; ++i) {
                    const int t = Ln + 32 * i;
                    if (t >= kRB * kT64) continue;
                    if (terms->out[t % kT64] == lane) sum = sum + red[Ln * kRBLo + i];
                }
            lowF[lane] = sum;
        }
        __syncwarp();
        double* out = part + (size_t)w * nco;
        warp_pow_table(1.0 / sigma, p + 1, lane, pws);
        __syncwarp();
        for (int i = lane; i < nco; i += 32) {
            const int n = idx_n[i], m = i - n * n - n;
            double v = (double)outs[i] * pws[n + 1];
            if (n <= kJ64) {
                const cd lv = lowF[n * (n + 1) / 2 + (m < 0 ? -m : m)];
                v += m >= 0 ? lv.re : lv.im;
            }
            out[i] = v;
        }
        __syncwarp();
    }
}

template <int kRB>
static void m2l_rounds_launch(const int2* list, const int* seg_start, const int* seg_end, const int* order,
                              const int* item_start, unsigned* work, const d4* cen, const float2* Mf, const cd* M64,
                              int p, double* part, cudaStream_t s) {
    const size_t sm = RoundsSmem<kRB>(p).total;
    cudaFuncSetAttribute(k_m2l_rounds<kRB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int dev = 0, nsm = 152, bps = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_m2l_rounds<kRB>, 32, sm);
    const unsigned g = (unsigned)(nsm * (bps > 0 ? bps : 1));
    k_m2l_rounds<kRB><<<g, 32, sm, s>>>(list, seg_start, seg_end, order, item_start, work, cen, Mf, M64, p, part);
    note_launch();
}

size_t m2l_split_tmp_bytes(int ncells, int p, long long npairs) {
    size_t n = (size_t)(ncells > 0 ? ncells : 1);
    size_t items = (size_t)(npairs / kChunk) + n + 1;
    return m2l_tmp_bytes(ncells, p) + n * (size_t)ncoef(p) * sizeof(float2) + n * kN64 * sizeof(cd) +
           2 * n * sizeof(int) + scan_tmp_ints(n) * sizeof(int) + items * (size_t)ncoef(p) * sizeof(double) +
           m2l_rot_group_bytes((long long)items) + 4096;
}

// chunks per sorted sink
__global__ void k_item_counts(const int* __restrict__ order, const int* __restrict__ seg_start,
                              const int* __restrict__ seg_end, int ncells, int* __restrict__ cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncells; i += gridDim.x * blockDim.x) {
        const int B = order[i];
        const int len = seg_end[B] - seg_start[B];
        cnt[i] = (len + kChunk - 1) / kChunk;
    }
}

// F_B = sum of its chunks' partial expansions, in chunk order
// item_q (nullable): the order of item w's partial expansion (its coefficients of higher
// order are not written and count as zero)
// single: sinks of one item were written to F by the M2L kernel itself (and sinks without an
// item hold the zeros F starts with), so only sinks of two or more items are summed here
__global__ void k_m2l_reduce(const int* __restrict__ order, const int* __restrict__ item_start,
                             const int* __restrict__ cnt, const unsigned* __restrict__ work, int ncells, int nco,
                             const double* __restrict__ part, double* __restrict__ F, const int* __restrict__ item_q,
                             bool single) {
    const unsigned nsinks = work[1];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)ncells * nco;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / nco), j = (int)(t % nco);
        if ((unsigned)i >= nsinks) continue;
        if (single && cnt[i] <= 1) continue;
        const int a = item_start[i], b = a + cnt[i];
        const int nj = (int)sqrtf((float)j);
        double v = 0.0;
        for (int w = a; w < b; ++w)
            if (!item_q || nj <= item_q[w]) v += part[(size_t)w * nco + j];
        F[(size_t)order[i] * nco + j] = v;
    }
}

void launch_m2l_split(const int2* list, const int* seg_start, const int* seg_end, void* tmp, int ncells, const d4* cen,
                      const double* M, int p, double* F, bool rot, cudaStream_t s, bool adaptive, long long npairs) {
    if (ncells <= 0) return;
    if (p <= kJ64) {  // nothing to split
        launch_m2l(list, seg_start, seg_end, tmp, ncells, cen, M, p, F, s);
        return;
    }
    init_split_tables();
    uint64_t* k0 = (uint64_t*)tmp;
    uint64_t* k1 = k0 + ncells;
    int* v0 = (int*)(k1 + ncells);
    int* v1 = v0 + ncells;
    int* order = v1 + ncells;
    // [0] item counter, [1] sinks, [2] items, [3]-[5] the rotated M2L's units (launch_m2l_rot)
    unsigned* work = (unsigned*)(order + ncells);
    int* rtmp = (int*)(work + 8);
    unsigned char* after = (unsigned char*)(rtmp + radix_tmp_ints(ncells));
    float2* Mf = (float2*)(((uintptr_t)after + 255) & ~(uintptr_t)255);
    cd* M64 = (cd*)(((uintptr_t)(Mf + (size_t)ncells * ncoef(p)) + 255) & ~(uintptr_t)255);
    int* cnt = (int*)(M64 + (size_t)ncells * kN64);
    int* item_start = cnt + ncells;
    int* stmp = item_start + ncells;
    double* part = (double*)(((uintptr_t)(stmp + scan_tmp_ints(ncells)) + 255) & ~(uintptr_t)255);
    const long long items_cap = npairs / kChunk + ncells + 1;
    void* gtmp = (void*)(((uintptr_t)(part + (size_t)items_cap * ncoef(p)) + 255) & ~(uintptr_t)255);
    const int* item_q = nullptr;
    bool single = false;
    cudaMemsetAsync(work, 0, 8 * sizeof(unsigned), s);
    k_sink_keys<<<grid_for(ncells, 256), 256, 0, s>>>(seg_start, seg_end, ncells, k0, v0); note_launch();
    // the low 32 bits are the sink's index, already in order: the stable pass over the 8
    // length bits alone keeps ties in index order
    int flip = radix_sort_pairs_bits(k0, v0, k1, v1, ncells, rtmp, 32, 40, s);
    k_sink_order<<<grid_for(ncells, 256), 256, 0, s>>>(flip ? k1 : k0, ncells, order, work + 1); note_launch();
    k_item_counts<<<grid_for(ncells, 256), 256, 0, s>>>(order, seg_start, seg_end, ncells, cnt); note_launch();
    scan_exclusive_i32(cnt, item_start, ncells, (int*)(work + 2), stmp, s);
    if (rot && m2l_rot_supported(p)) {
        item_q = launch_m2l_rot(list, seg_start, seg_end, order, item_start, cnt, work, cen, M, ncells, p, (float*)Mf,
                                M64, part, F, adaptive, gtmp, items_cap, s);
        single = true;
        if (!adaptive) return;  // every sink's F was written once by the kernel
    } else {
        k_prep_split<<<grid_for((long long)ncells * 32, 256), 256, 0, s>>>(M, cen, ncells, p, Mf, M64); note_launch();
        m2l_rounds_launch<kRoundsBatch>(list, seg_start, seg_end, order, item_start, work, cen, Mf, M64, p, part, s);
    }
    k_m2l_reduce<<<grid_for((long long)ncells * ncoef(p), 256), 256, 0, s>>>(order, item_start, cnt, work, ncells,
                                                                            ncoef(p), part, F, item_q, single);
    note_launch();
}

// ---------------------------------------------------------------- L2L
// F_n^m(s') += sum_{k<=p-n} sum_l Upsilon_k^{l*}(s - s') F_{n+k}^{m+l}(s) for every
// cell of one level (s = its parent's centre), one warp per cell.
__global__ void __launch_bounds__(128) k_l2l(Cells c, const d4* __restrict__ cen, int lev_begin, int lev_end, int p,
                                             double* __restrict__ F, LaneSched sched) {
    extern __shared__ cd csm[];
    const int wpb = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nco = ncoef(p);
    cd* X = csm + (size_t)wid * 2 * nco;
    cd* Y = X + nco;
    int cell = lev_begin + blockIdx.x * wpb + wid;
    if (cell >= lev_end || !cell_active(c, cell)) return;
    int par = c.parent[cell];
    const d4 s = cen[par], sp = cen[cell];
    if (lane <= p) upsilon_column(p, lane, s.x - sp.x, s.y - sp.y, s.z - sp.z, X, true);
    expand_real(p, F + (size_t)par * nco, Y, false, lane, 32);
    __syncwarp();
    double* out = F + (size_t)cell * nco;
    const int cnt = sched.cnt[lane];
    for (int q = 0; q < cnt; ++q) {
        int n = sched.n[lane][q], m = sched.m[lane][q];
        cd v = contract(p, n, m, X, Y);
        out[cix(n, m)] += v.re;
        if (m) out[cix(n, -m)] += v.im;
    }
}

void launch_l2l_level(Cells c, const d4* cen, int lev_begin, int lev_end, int p, double* F, cudaStream_t s) {
    int ncl = lev_end - lev_begin;
    if (ncl <= 0) return;
    const int wpb = 4;
    size_t sm = (size_t)wpb * 2 * ncoef(p) * sizeof(cd);
    LaneSched sched = make_lane_sched(p, kSchedDown);
    init_rec_tables();
    k_l2l<<<(ncl + wpb - 1) / wpb, wpb * 32, sm, s>>>(c, cen, lev_begin, lev_end, p, F, sched); note_launch();
}

// ---------------------------------------------------------------- L2P
// Psi_n^m(x_b) = sum_{k<=p-n} sum_l Upsilon_k^{l*}(s_B - x_b) F_{n+k}^{m+l}(s_B) for
// n = 0, 1; psi = Psi_0^0, a = -(Re Psi_1^1, Im Psi_1^1, Psi_1^0).  One block per
// leaf, F in shared memory, one thread per particle streaming the Upsilon columns.
constexpr int kL2PThreads = 64;
__global__ void __launch_bounds__(kL2PThreads) k_l2p(const d4* __restrict__ xm, Cells c, const d4* __restrict__ cen,
                                                     const int* __restrict__ leaves, int nleaves, int p,
                                                     const double* __restrict__ F, double* __restrict__ psi,
                                                     double* __restrict__ acc) {
    extern __shared__ cd Fc[];
    const int nco = ncoef(p);
    for (int t = blockIdx.x; t < nleaves; t += gridDim.x) {
        const int cell = leaves[t];
        if (!cell_active(c, cell)) continue;  // block-uniform
        __syncthreads();
        expand_real(p, F + (size_t)cell * nco, Fc, false, threadIdx.x, blockDim.x);
        __syncthreads();
        const d4 s = cen[cell];
        const int first = c.first[cell], count = c.count[cell];
        for (int j = threadIdx.x; j < count; j += blockDim.x) {
            const d4 xb = xm[first + j];
            const double x = s.x - xb.x, y = s.y - xb.y, z = s.z - xb.z;
            const double r2 = x * x + y * y + z * z;
            double p00 = 0.0;
            cd p10 = mkc(0.0, 0.0), p11 = mkc(0.0, 0.0);
            cd d = mkc(1.0, 0.0);
            for (int l = 0; l <= p; ++l) {
                if (l > 0) {
                    double sc = 1.0 / (2.0 * l);
                    d = cd{sc * (x * d.re - y * d.im), sc * (x * d.im + y * d.re)};
                }
                const double sg = (l & 1) ? -1.0 : 1.0;
                cd prev2 = mkc(0.0, 0.0), prev = d;
                for (int k = l; k <= p; ++k) {
                    cd Y;
                    if (k == l) Y = d;
                    else {
                        double inv = 1.0 / (double)(k * k - l * l);
                        double a = (2.0 * k - 1.0) * z;
                        Y = cd{(a * prev.re - r2 * prev2.re) * inv, (a * prev.im - r2 * prev2.im) * inv};
                        prev2 = prev;
                        prev = Y;
                    }
                    const cd Xp = conjc(Y);                 // X_k^l
                    const cd Xn = cd{sg * Y.re, sg * Y.im};  // X_k^{-l} = (-1)^l Upsilon_k^l
                    const cd* Fk = Fc + k * k + k;
                    if (l == 0) p00 += Xp.re * Fk[0].re - Xp.im * Fk[0].im;
                    else p00 += 2.0 * (Xp.re * Fk[l].re - Xp.im * Fk[l].im);
                    if (k < p) {
                        const cd* Fk1 = Fc + (k + 1) * (k + 1) + (k + 1);
                        cmac(p10, Xp, Fk1[l]);
                        cmac(p11, Xp, Fk1[1 + l]);
                        if (l > 0) {
                            cmac(p10, Xn, Fk1[-l]);
                            cmac(p11, Xn, Fk1[1 - l]);
                        }
                    }
                }
            }
            const int i = first + j;
            psi[i] = p00;
            acc[3 * (size_t)i] = -p11.re;
            acc[3 * (size_t)i + 1] = -p11.im;
            acc[3 * (size_t)i + 2] = -p10.re;
        }
    }
}

void launch_l2p(const d4* xm, Cells c, const d4* cen, const int* leaves, int nleaves, int p, const double* F,
                double* psi, double* acc, cudaStream_t s) {
    if (nleaves <= 0) return;
    size_t sm = (size_t)ncoef(p) * sizeof(cd);
    unsigned g = (unsigned)std::min<long long>(nleaves, (long long)sm_count() * 64);
    k_l2p<<<g, kL2PThreads, sm, s>>>(xm, c, cen, leaves, nleaves, p, F, psi, acc); note_launch();
}

// ---------------------------------------------------------------- P2P, FP64
// One warp per chunk of up to 32 sinks of a leaf (lane = sink).  The sources are
// the P2P segments of the leaf and of all its ancestors (a pair (A, B) with B
// internal covers every leaf below B); they pass through a warp-private tile of
// 32 in shared memory.
constexpr int kP2PWarps = 4;

__global__ void __launch_bounds__(kP2PWarps * 32) k_p2p_fp64(const d4* __restrict__ xm, Cells c,
                                                             const int2* __restrict__ list,
                                                             const int* __restrict__ seg_start,
                                                             const int* __restrict__ seg_end,
                                                             const int* __restrict__ leaves, int nleaves,
                                                             double* __restrict__ psi, double* __restrict__ acc) {
    __shared__ d4 tile_all[kP2PWarps][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    d4* tile = tile_all[wid];
    for (int t = blockIdx.x * kP2PWarps + wid; t < nleaves; t += gridDim.x * kP2PWarps) {
        const int leaf = leaves[t];
        if (!cell_active(c, leaf)) continue;
        const int first = c.first[leaf], count = c.count[leaf];
        for (int s0 = 0; s0 < count; s0 += 32) {
            const int i = first + s0 + lane;
            const bool active = s0 + lane < count;
            const d4 xb = active ? xm[i] : mk4(0, 0, 0, 0);
            double ps = 0, ax = 0, ay = 0, az = 0;
            for (int cell = leaf; cell >= 0; cell = c.parent[cell]) {
                const int e0 = seg_start[cell], e1 = seg_end[cell];
                for (int e = e0; e < e1; ++e) {
                    const int A = list[e].x;
                    const int af = c.first[A], an = c.count[A];
                    for (int j0 = 0; j0 < an; j0 += 32) {
                        __syncwarp();
                        if (j0 + lane < an) tile[lane] = xm[af + j0 + lane];
                        __syncwarp();
                        const int nt = min(32, an - j0);
                        for (int j = 0; j < nt; ++j) {
                            const d4 q = tile[j];
                            const double dx = q.x - xb.x, dy = q.y - xb.y, dz = q.z - xb.z;
                            const double r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 > 0.0) {
                                const double rinv = rsqrt(r2);
                                const double qm = q.w * rinv;
                                const double q3 = qm * rinv * rinv;
                                ps += qm;
                                ax = fma(q3, dx, ax);
                                ay = fma(q3, dy, ay);
                                az = fma(q3, dz, az);
                            }
                        }
                    }
                }
            }
            if (active) {
                psi[i] = ps;
                acc[3 * (size_t)i] = ax;
                acc[3 * (size_t)i + 1] = ay;
                acc[3 * (size_t)i + 2] = az;
            }
        }
    }
}

static unsigned p2p_grid(int nleaves) {
    long long g = ((long long)nleaves + kP2PWarps - 1) / kP2PWarps;
    return (unsigned)std::min<long long>(g, (long long)sm_count() * 48);
}

void launch_p2p_fp64(const d4* xm, Cells c, const int2* list, const int* seg_start, const int* seg_end,
                     const int* leaves, int nleaves, double* psi, double* acc, cudaStream_t s) {
    if (nleaves <= 0) return;
    k_p2p_fp64<<<p2p_grid(nleaves), kP2PWarps * 32, 0, s>>>(xm, c, list, seg_start, seg_end, leaves, nleaves, psi,
                                                            acc);
    note_launch();
}

// ---------------------------------------------------------------- P2P, mixed
// Positions as two floats (hi + lo, exact to 2^-48 relative), so that
// dx = (hi_a - hi_b) + (lo_a - lo_b) keeps its relative accuracy even for close
// pairs.  Pair terms are FP32; the FP32 sums of every ~32 pairs are added to
// two-float accumulators (TwoSum), so the sum over tiles is compensated.
// Layout: one 32-byte record per particle, xp[2i] = (high parts of the position, mass as
// FP32), xp[2i + 1] = (low parts, 0), so that a range of particles is one contiguous block.
__global__ void k_split_positions(const d4* __restrict__ xm, int n, float4* __restrict__ xp) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        d4 v = xm[i];
        const float hx = (float)v.x, hy = (float)v.y, hz = (float)v.z;
        xp[2 * (size_t)i] = make_float4(hx, hy, hz, (float)v.w);
        xp[2 * (size_t)i + 1] =
            make_float4((float)(v.x - (double)hx), (float)(v.y - (double)hy), (float)(v.z - (double)hz), 0.f);
    }
}
void launch_split_positions(const d4* xm, int n, float4* xp, cudaStream_t s) {
    if (n > 0) k_split_positions<<<grid_for(n, 256), 256, 0, s>>>(xm, n, xp); note_launch();
}

// number of ordered pairs (a != b) at distance 0: equal positions have equal keys,
// so they sit next to each other in key order inside one leaf
__global__ void k_coincident(const d4* __restrict__ xm, const uint64_t* __restrict__ keys, int n,
                             unsigned long long* coincident, const int* __restrict__ off, int nsys) {
    unsigned long long cnt = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const d4 p = xm[i];
        int j0 = 0;  // first particle of i's system (systems keep their blocks when sorted)
        if (off) {
            int lo = 0, hi = nsys - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (off[mid] <= i) lo = mid;
                else hi = mid - 1;
            }
            j0 = off[lo];
        }
        for (int j = i - 1; j >= j0 && keys[j] == keys[i]; --j) {
            const d4 q = xm[j];
            cnt += (q.x == p.x && q.y == p.y && q.z == p.z) ? 2 : 0;
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(coincident, cnt);
}

void launch_coincident(const d4* xm, const uint64_t* keys, int n, unsigned long long* coincident, cudaStream_t s,
                       const int* off, int nsys) {
    if (n > 1) {
        k_coincident<<<grid_for(n, 256), 256, 0, s>>>(xm, keys, n, coincident, off, nsys);
        note_launch();
    }
}

// ---------------------------------------------------------------- low-order f estimate
// p = 0 with the 1/r^2 kernel (Sec. 5.3.2): the "M2L" is F_B += M_A / |s_B - z_A|^2
// about the centres of mass; one thread per sink, its segment in list order.
__global__ void k_f_m2l(const int2* __restrict__ list, const int* __restrict__ seg_start, const int* __restrict__ seg_end,
                        int ncells, Cells c, double* __restrict__ Ff) {
    int B = blockIdx.x * blockDim.x + threadIdx.x;
    if (B >= ncells) return;
    const d4 sb = c.cr[B];
    double f = 0;
    for (int e = seg_start[B]; e < seg_end[B]; ++e) {
        int A = list[e].x;
        d4 za = c.cr[A];
        double dx = sb.x - za.x, dy = sb.y - za.y, dz = sb.z - za.z;
        f += c.mass[A] / (dx * dx + dy * dy + dz * dz);
    }
    Ff[B] = f;
}
// p = 1 M2L of the acceleration estimate (Sec. 5.3.2) with multipoles about the
// centres of mass: the dipole about the centre of mass vanishes, so eq. (3b) keeps
// only the monopole, F_n^m = M_A Theta_n^m(s_B - z_A) for n <= 1 (real storage:
// F_0^0, Im F_1^1, F_1^0, Re F_1^1).  One thread per sink cell, sources in list order.
__global__ void k_est_m2l(const int2* __restrict__ list, const int* __restrict__ seg_start,
                          const int* __restrict__ seg_end, int ncells, Cells c, double* __restrict__ F1) {
    const int B = blockIdx.x * blockDim.x + threadIdx.x;
    if (B >= ncells) return;
    const d4 sb = c.cr[B];
    double f0 = 0, fx = 0, fy = 0, fz = 0;
    for (int e = seg_start[B]; e < seg_end[B]; ++e) {
        const int A = list[e].x;
        const d4 za = c.cr[A];
        const double x = sb.x - za.x, y = sb.y - za.y, z = sb.z - za.z;
        const double rinv = 1.0 / sqrt(x * x + y * y + z * z);
        const double q = c.mass[A] * rinv, q3 = q * rinv * rinv;
        f0 += q;
        fx += q3 * x;
        fy += q3 * y;
        fz += q3 * z;
    }
    F1[4 * (size_t)B] = f0;
    F1[4 * (size_t)B + 1] = fy;
    F1[4 * (size_t)B + 2] = fz;
    F1[4 * (size_t)B + 3] = fx;
}
// The same sums in single precision (mixed mode, where the estimate's P2P is FP32 too):
// one warp per sink cell, lanes over its sources, two-float centre differences from the
// walk's single-precision view (fc[2 c] = high parts and rho, fc[2 c + 1] = low parts
// and M); a pair with a cell outside that view's range (NaN rho) is summed in FP64.
// Lane partial sums are added in a fixed butterfly order.
__global__ void k_est_m2l_f32(const int2* __restrict__ list, const int* __restrict__ seg_start,
                              const int* __restrict__ seg_end, int ncells, Cells c, const float4* __restrict__ fc,
                              double* __restrict__ F1) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int B = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; B < ncells; B += nw) {
        const int e0 = seg_start[B], e1 = seg_end[B];
        if (e0 >= e1) {
            if (lane < 4) F1[4 * (size_t)B + lane] = 0.0;
            continue;
        }
        const float4 bh = fc[2 * B], bl = fc[2 * B + 1];
        float f0 = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
        for (int e = e0 + lane; e < e1; e += 32) {
            const int A = list[e].x;
            const float4 ah = fc[2 * A], al = fc[2 * A + 1];
            if (ah.w == ah.w && bh.w == bh.w) {
                const float x = (bh.x - ah.x) + (bl.x - al.x);
                const float y = (bh.y - ah.y) + (bl.y - al.y);
                const float z = (bh.z - ah.z) + (bl.z - al.z);
                const float rinv = rsqrt_ftz(x * x + y * y + z * z);
                const float q = al.w * rinv, q3 = q * rinv * rinv;
                f0 += q;
                fx += q3 * x;
                fy += q3 * y;
                fz += q3 * z;
            } else {
                const d4 sb = c.cr[B], za = c.cr[A];
                const double x = sb.x - za.x, y = sb.y - za.y, z = sb.z - za.z;
                const double rinv = 1.0 / sqrt(x * x + y * y + z * z);
                const double q = c.mass[A] * rinv, q3 = q * rinv * rinv;
                f0 += (float)q;
                fx += (float)(q3 * x);
                fy += (float)(q3 * y);
                fz += (float)(q3 * z);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            f0 += __shfl_xor_sync(0xffffffffu, f0, o);
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
        }
        if (lane == 0) {
            F1[4 * (size_t)B] = f0;
            F1[4 * (size_t)B + 1] = fy;
            F1[4 * (size_t)B + 2] = fz;
            F1[4 * (size_t)B + 3] = fx;
        }
    }
}
void launch_est_m2l(const int2* list, const int* seg_start, const int* seg_end, int ncells, Cells c, double* F1,
                    cudaStream_t s, const float4* fc) {
    if (ncells <= 0) return;
    if (fc) {
        const long long warps = ncells;
        const unsigned g = (unsigned)std::min<long long>((warps + 7) / 8, (long long)sm_count() * 16);
        k_est_m2l_f32<<<g, 256, 0, s>>>(list, seg_start, seg_end, ncells, c, fc, F1);
    } else {
        k_est_m2l<<<(ncells + 127) / 128, 128, 0, s>>>(list, seg_start, seg_end, ncells, c, F1);
    }
    note_launch();
}

// The estimate's far field at p = 1.  L2L (eq. 5) at p = 1 passes F_1^m down unchanged
// (only the k = 0 term, Upsilon_0^0 = 1, reaches n = 1), so a leaf's F_1 is its own M2L
// result plus its parent's F_1, which is added here along the ancestor chain, root first,
// in the order of the level-by-level pass.  L2P (eq. 7) at p = 1 gives the same
// acceleration at every particle of the leaf, a = -(Re F_1^1, Im F_1^1, F_1^0); the scale
// is |a_far + a_near| of each particle.  One warp per leaf.
__global__ void k_est_scale(Cells c, const int* __restrict__ leaves, int nleaves, const double* __restrict__ F1,
                            const double* __restrict__ an, double* __restrict__ scale) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < nleaves; t += nw) {
        const int cell = leaves[t];
        if (!cell_active(c, cell)) continue;
        int chain[24], depth = 0;  // at most 22 levels: 21 key bits per axis below the root
        for (int a = cell; a >= 0 && depth < 24; a = c.parent[a]) chain[depth++] = a;
        double f1 = 0.0, f2 = 0.0, f3 = 0.0;
        for (int k = depth - 1; k >= 0; --k) {
            const double* f = F1 + 4 * (size_t)chain[k];
            f1 = f[1] + f1;
            f2 = f[2] + f2;
            f3 = f[3] + f3;
        }
        const double ax = -f3, ay = -f1, az = -f2;
        const int first = c.first[cell], count = c.count[cell];
        for (int j = lane; j < count; j += 32) {
            const size_t i = (size_t)first + j;
            const double x = ax + an[3 * i], y = ay + an[3 * i + 1], z = az + an[3 * i + 2];
            scale[i] = sqrt(x * x + y * y + z * z);
        }
    }
}
void launch_est_scale(Cells c, const int* leaves, int nleaves, const double* F1, const double* acc_near,
                      double* scale, cudaStream_t s) {
    if (nleaves <= 0) return;
    const unsigned g = (unsigned)std::min<long long>(((long long)nleaves + 7) / 8, (long long)sm_count() * 16);
    k_est_scale<<<g, 256, 0, s>>>(c, leaves, nleaves, F1, acc_near, scale);
    note_launch();
}
void launch_f_m2l(const int2* list, const int* seg_start, const int* seg_end, int ncells, Cells c, double* Ff,
                  cudaStream_t s) {
    if (ncells > 0) k_f_m2l<<<(ncells + 127) / 128, 128, 0, s>>>(list, seg_start, seg_end, ncells, c, Ff); note_launch();
}
__global__ void k_f_down(Cells c, int lev_begin, int lev_end, double* __restrict__ Ff) {
    int cell = lev_begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= lev_end) return;
    Ff[cell] += Ff[c.parent[cell]];
}
void launch_f_down_level(Cells c, int lev_begin, int lev_end, double* Ff, cudaStream_t s) {
    int ncl = lev_end - lev_begin;
    if (ncl > 0) k_f_down<<<(ncl + 127) / 128, 128, 0, s>>>(c, lev_begin, lev_end, Ff); note_launch();
}
__global__ void __launch_bounds__(kP2PWarps * 32) k_f_p2p(const d4* __restrict__ xm, Cells c,
                                                          const int2* __restrict__ list,
                                                          const int* __restrict__ seg_start,
                                                          const int* __restrict__ seg_end,
                                                          const int* __restrict__ leaves, int nleaves,
                                                          const double* __restrict__ Ff, double* __restrict__ fout) {
    __shared__ d4 tile_all[kP2PWarps][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    d4* tile = tile_all[wid];
    for (int t = blockIdx.x * kP2PWarps + wid; t < nleaves; t += gridDim.x * kP2PWarps) {
        const int leaf = leaves[t];
        const int first = c.first[leaf], count = c.count[leaf];
        for (int s0 = 0; s0 < count; s0 += 32) {
            const int i = first + s0 + lane;
            const bool active = s0 + lane < count;
            const d4 xb = active ? xm[i] : mk4(0, 0, 0, 0);
            double f = 0;
            for (int cell = leaf; cell >= 0; cell = c.parent[cell]) {
                for (int e = seg_start[cell]; e < seg_end[cell]; ++e) {
                    const int A = list[e].x;
                    const int af = c.first[A], an = c.count[A];
                    for (int j0 = 0; j0 < an; j0 += 32) {
                        __syncwarp();
                        if (j0 + lane < an) tile[lane] = xm[af + j0 + lane];
                        __syncwarp();
                        const int nt = min(32, an - j0);
                        for (int j = 0; j < nt; ++j) {
                            const d4 q = tile[j];
                            const double dx = q.x - xb.x, dy = q.y - xb.y, dz = q.z - xb.z;
                            const double r2 = dx * dx + dy * dy + dz * dz;
                            if (r2 > 0.0) f += q.w / r2;
                        }
                    }
                }
            }
            if (active) fout[i] = Ff[leaf] + f;
        }
    }
}
void launch_f_p2p(const d4* xm, Cells c, const int2* list, const int* seg_start, const int* seg_end,
                  const int* leaves, int nleaves, const double* Ff, double* f_sorted, cudaStream_t s) {
    if (nleaves <= 0) return;
    k_f_p2p<<<p2p_grid(nleaves), kP2PWarps * 32, 0, s>>>(xm, c, list, seg_start, seg_end, leaves, nleaves, Ff, f_sorted);
    note_launch();
}

// ---------------------------------------------------------------- finish (A12)
__global__ void k_finish(const double* __restrict__ pf, const double* __restrict__ af, const double* __restrict__ pn,
                         const double* __restrict__ an, const int* __restrict__ perm, int n, double G,
                         double* __restrict__ psi, double* __restrict__ acc, const int* __restrict__ off,
                         const double* __restrict__ Gsys, int nsys, const unsigned char* __restrict__ pact,
                         const int* __restrict__ e) {
    // back from the working units: Psi ~ mu / x, a ~ mu / x^2 (exact powers of two)
    const int kp = e ? e[1] - e[0] : 0, ka = e ? e[1] - 2 * e[0] : 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (pact && !pact[i]) continue;  // outputs of inactive particles are left as they are
        int o = perm[i];
        if (Gsys) {  // the system of sorted particle i (systems keep their blocks when sorted)
            int lo = 0, hi = nsys - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (off[mid] <= i) lo = mid;
                else hi = mid - 1;
            }
            G = Gsys[lo];
        }
        psi[o] = ldexp(G * (pf[i] + pn[i]), kp);
#pragma unroll
        for (int d = 0; d < 3; ++d)
            acc[3 * (size_t)o + d] = ldexp(G * (af[3 * (size_t)i + d] + an[3 * (size_t)i + d]), ka);
    }
}
void launch_finish(const double* psi_far, const double* acc_far, const double* psi_near, const double* acc_near,
                   const int* perm, int n, double G, double* psi, double* acc, cudaStream_t s, const int* off,
                   const double* Gsys, int nsys, const unsigned char* pact, const int* e) {
    if (n > 0)
        k_finish<<<grid_for(n, 256), 256, 0, s>>>(psi_far, acc_far, psi_near, acc_near, perm, n, G, psi, acc, off,
                                                  Gsys, nsys, pact, e);
    note_launch();
}

}  // namespace gb3
