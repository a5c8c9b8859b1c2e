// m2l_rot.cu -- host side of the rotation-accelerated M2L (App. A.5) of the mixed-precision
// path: the per-cell preparation of the scaled FP32 multipoles and the dispatch on p to
// the kernels of m2l_rot.cuh (instantiated in m2l_rot_p*.cu).
#include "m2l_rot.cuh"

namespace gb3 {
namespace {

// per cell: Mt = N_n^m M_n^m / rho^n in FP32 (real storage) and conj(M) of orders <= 2 in FP64
// (the kernel reads the orders <= kRotJ64)
__global__ void k_prep_rot(const double* __restrict__ M, const d4* __restrict__ cen, int ncells, int p,
                           float* __restrict__ Mt, cd* __restrict__ M64) {
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
            const int n = i < nco ? (int)sqrtf((float)i) : 0;
            const double sc = __shfl_sync(0xffffffffu, pw, n);
            if (i < nco) {
                Mt[(size_t)cell * nco + i] = (float)(R[i] * c_rot_norm.v[i] * sc);
                if (i < 9) M64[(size_t)cell * 9 + i] = conjc(load_real_storage(R, n, i - n * n - n));
            }
        }
    }
}

}  // namespace

extern template void rot_launch<3>(const RotArgs&, cudaStream_t);
extern template void rot_launch<4>(const RotArgs&, cudaStream_t);
extern template void rot_launch<5>(const RotArgs&, cudaStream_t);
extern template void rot_launch<6>(const RotArgs&, cudaStream_t);
extern template void rot_launch<7>(const RotArgs&, cudaStream_t);
extern template void rot_launch<8>(const RotArgs&, cudaStream_t);
extern template void rot_launch<9>(const RotArgs&, cudaStream_t);
extern template void rot_launch<10>(const RotArgs&, cudaStream_t);
extern template void rot_launch<11>(const RotArgs&, cudaStream_t);
extern template void rot_launch<12>(const RotArgs&, cudaStream_t);
extern template void rot_launch<13>(const RotArgs&, cudaStream_t);
extern template void rot_launch<14>(const RotArgs&, cudaStream_t);
extern template void rot_launch<15>(const RotArgs&, cudaStream_t);
extern template void rot_launch<16>(const RotArgs&, cudaStream_t);

bool m2l_rot_supported(int p) { return p >= 3 && p <= kRotMaxP; }

namespace {
// item w (of the sorted sinks' chunks): the largest order of its pairs; key = (q << 32) | w
__global__ void k_item_qmax(const int2* __restrict__ list, const int* __restrict__ seg_start,
                            const int* __restrict__ seg_end, const int* __restrict__ order,
                            const int* __restrict__ item_start, const unsigned* __restrict__ work, int p,
                            uint64_t* __restrict__ keys, int* __restrict__ vals, int* __restrict__ item_q,
                            unsigned* __restrict__ qcount, unsigned cap) {
    const unsigned nitems = work[2], nsinks = work[1];
    for (unsigned w = blockIdx.x * blockDim.x + threadIdx.x; w < cap; w += gridDim.x * blockDim.x) {
        if (w >= nitems) {  // unused slots sort last
            keys[w] = ~0ull;
            vals[w] = 0;
            continue;
        }
        int lo_i = 0, hi_i = (int)nsinks - 1;
        while (lo_i < hi_i) {
            const int mid = (lo_i + hi_i + 1) >> 1;
            if ((unsigned)item_start[mid] <= w) lo_i = mid;
            else hi_i = mid - 1;
        }
        const int B = order[lo_i];
        const int e0 = seg_start[B] + (int)(w - (unsigned)item_start[lo_i]) * kM2LChunk;
        const int e1 = min(e0 + kM2LChunk, seg_end[B]);
        int q = 0;
        for (int e = e0; e < e1; ++e) q = max(q, m2l_order(list[e].x, p));
        item_q[w] = q;
        keys[w] = ((uint64_t)(unsigned)q << 32) | w;
        vals[w] = 0;
        atomicAdd(&qcount[q], 1u);
    }
}
// goff[q] = number of items of order < q (q = 0 .. kMaxP + 1); ilist[k] = item of sorted key k
__global__ void k_item_groups(const unsigned* __restrict__ qcount, unsigned* __restrict__ goff,
                              const uint64_t* __restrict__ keys, const unsigned* __restrict__ work,
                              int* __restrict__ ilist) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned a = 0;
        for (int q = 0; q <= kMaxP + 1; ++q) {
            goff[q] = a;
            if (q <= kMaxP) a += qcount[q];
        }
    }
    const unsigned nitems = work[2];
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < nitems; k += gridDim.x * blockDim.x)
        ilist[k] = (int)(keys[k] & 0xffffffffu);
}

// by-sink units: the number of pieces of sorted sink i (0 past the sinks with a list)
__global__ void k_piece_counts(const int* __restrict__ cnt, const unsigned* __restrict__ nsinks, int ncells,
                               int* __restrict__ npc) {
    const int ns = (int)*nsinks;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncells; i += gridDim.x * blockDim.x)
        npc[i] = i < ns ? (cnt[i] + kM2LPieceItems - 1) / kM2LPieceItems : 0;
}
// units[pstart[i] + k] = (i, k) in sorted-sink order; the sinks of two or more pieces are
// listed in splits (in any order: each is summed on its own)
__global__ void k_units(const int* __restrict__ npc, const int* __restrict__ pstart, int ncells,
                        int2* __restrict__ units, int* __restrict__ splits, unsigned* __restrict__ nsplit) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncells; i += gridDim.x * blockDim.x) {
        const int np = npc[i];
        for (int k = 0; k < np; ++k) units[pstart[i] + k] = make_int2(i, k);
        if (np > 1) splits[atomicAdd(nsplit, 1u)] = i;
    }
}
// F of a cut sink = its pieces' partial expansions added in piece order
__global__ void k_piece_reduce(const int* __restrict__ order, const int* __restrict__ item_start,
                               const int* __restrict__ cnt, const int* __restrict__ splits,
                               const unsigned* __restrict__ nsplit, int nco, const double* __restrict__ part,
                               double* __restrict__ F) {
    const long long total = (long long)*nsplit * nco;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = splits[t / nco], j = (int)(t % nco);
        const int a = item_start[i], c = cnt[i];
        double v = 0.0;
        for (int k = 0; k < c; k += kM2LPieceItems) v += part[(size_t)(a + k) * nco + j];
        F[(size_t)order[i] * nco + j] = v;
    }
}
}  // namespace

size_t m2l_rot_group_bytes(long long items_cap) {
    const size_t n = (size_t)(items_cap > 0 ? items_cap : 1);
    return n * (2 * sizeof(uint64_t) + 4 * sizeof(int)) + radix_tmp_ints((long long)n) * sizeof(int) +
           4 * (kMaxP + 2) * sizeof(unsigned) + 1024;
}

const int* launch_m2l_rot(const int2* list, const int* seg_start, const int* seg_end, const int* order,
                          const int* item_start, const int* cnt, unsigned* work, const d4* cen, const double* M,
                          int ncells, int p, float* Mt, cd* M64, double* part, double* F, bool adaptive, void* gtmp,
                          long long items_cap, cudaStream_t s) {
    k_prep_rot<<<grid_for((long long)ncells * 32, 256), 256, 0, s>>>(M, cen, ncells, p, Mt, M64);
    note_launch();
    const int nco = ncoef(p);
#define GB3_ROT(PP)                                                                                      \
    case PP:                                                                                             \
        rot_launch<PP>(RotArgs{list, seg_start, seg_end, order, item_start, work, cen, Mt, M64, part, F, il,  \
                               go, gq, ctr, nco, adapt, by_sink ? cnt : nullptr, by_sink ? work + 3 : nullptr,  \
                               units, work + 4},                                                         \
                       s);                                                                               \
        break;
    const int2* units = nullptr;
    auto launch_p = [&](int q, const int* il, const unsigned* go, int gq, unsigned* ctr, int adapt, bool by_sink) {
        switch (q) {
            GB3_ROT(3) GB3_ROT(4) GB3_ROT(5) GB3_ROT(6) GB3_ROT(7) GB3_ROT(8) GB3_ROT(9) GB3_ROT(10) GB3_ROT(11)
            GB3_ROT(12) GB3_ROT(13) GB3_ROT(14) GB3_ROT(15) GB3_ROT(16)
            default: break;
        }
    };
#undef GB3_ROT
    if (!adaptive) {
        // every pair at p: units of whole sinks and of pieces of the longer ones (the sink
        // count is on the device, work[1]), taken through work[3]; a whole sink's F is written
        // once by the kernel, the cut sinks' pieces are added after it.  gtmp holds the units
        // (at most one per item), the piece counts and starts, the cut sinks and scan scratch.
        const size_t cap = (size_t)(items_cap > 0 ? items_cap : 1);
        int2* u = (int2*)gtmp;
        int* npc = (int*)(u + cap);
        int* pstart = npc + ncells;
        int* splits = pstart + ncells;
        int* stmp = splits + ncells;
        k_piece_counts<<<grid_for(ncells, 256), 256, 0, s>>>(cnt, work + 1, ncells, npc);
        note_launch();
        scan_exclusive_i32(npc, pstart, ncells, (int*)(work + 4), stmp, s);
        k_units<<<grid_for(ncells, 256), 256, 0, s>>>(npc, pstart, ncells, u, splits, work + 5);
        note_launch();
        units = u;
        mark_begin(s);
        launch_p(p, nullptr, nullptr, 0, work, 0, true);
        mark_end(s);
        k_piece_reduce<<<sm_count() * 8, 256, 0, s>>>(order, item_start, cnt, splits, work + 5, nco, part, F);
        note_launch();
        return nullptr;
    }
    // group the items by the largest order of their pairs; each group runs its own kernel
    const size_t cap = (size_t)(items_cap > 0 ? items_cap : 1);
    uint64_t* k0 = (uint64_t*)gtmp;
    uint64_t* k1 = k0 + cap;
    int* v0 = (int*)(k1 + cap);
    int* v1 = v0 + cap;
    int* item_q = v1 + cap;
    int* ilist = item_q + cap;
    unsigned* qcount = (unsigned*)(ilist + cap);
    unsigned* goff = qcount + (kMaxP + 2);
    unsigned* ctr = goff + (kMaxP + 2);
    int* rtmp = (int*)(ctr + (kMaxP + 2));
    cudaMemsetAsync(qcount, 0, 3 * (kMaxP + 2) * sizeof(unsigned), s);
    k_item_qmax<<<grid_for(items_cap, 256), 256, 0, s>>>(list, seg_start, seg_end, order, item_start, work, p, k0, v0,
                                                          item_q, qcount, (unsigned)cap);
    note_launch();
    // the items are at most items_cap; keys past work[2] are never read
    const int flip = radix_sort_pairs_bits(k0, v0, k1, v1, items_cap, rtmp, 32, 40, s);
    k_item_groups<<<grid_for(items_cap, 256), 256, 0, s>>>(qcount, goff, flip ? k1 : k0, work, ilist);
    note_launch();
    mark_begin(s);
    for (int q = (p < 3 ? p : 3); q <= p; ++q) launch_p(q, ilist, goff, q, ctr + q, 1, false);
    mark_end(s);
    return item_q;
}
}  // namespace gb3

extern "C" int fmm_swap_matrix(int n, double* B) {
    if (n < 0 || n > gb3::kRotMaxP || !B) return FMM_E_INVALID;
    for (int m = -n; m <= n; ++m)
        for (int l = -n; l <= n; ++l)
            B[(m + n) * (2 * n + 1) + (l + n)] = gb3::kSwap.full[n][gb3::kO + m][gb3::kO + l];
    return FMM_OK;
}
