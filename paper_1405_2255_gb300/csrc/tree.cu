// tree.cu -- A1-A4 of the path: bounds and validation, Morton keys, radix sort,
// the top-down oct-tree build, and the cell geometry (expansion centres, radii,
// masses, centres of mass).
//
// Compiled with --fmad=false: the decision quantities (keys, centres, radii) are
// plain IEEE FP64 sums and products, so that the tree and the acceptance tests do
// not depend on how a compiler contracts them.
#include "kernels.cuh"

namespace gb3 {

// ------------------------------------------------------------------ A1 bounds
__global__ void k_bounds_init(unsigned long long* b) {
    int i = threadIdx.x;
    if (i < 3) b[i] = ~0ull;
    else if (i < 7) b[i] = 0ull;  // [6]: the largest mass
}

constexpr int kBoundsThreads = 256;
__global__ void __launch_bounds__(kBoundsThreads) k_bounds(const double* __restrict__ x, const double* __restrict__ mu, int n,
                         unsigned long long* bounds, unsigned* status) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double mmax = 0.0;
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v[3] = {x[3 * (long long)i], x[3 * (long long)i + 1], x[3 * (long long)i + 2]};
        double m = mu[i];
        bad |= !(isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(m) && m >= 0.0);
        mmax = fmax(mmax, m);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            lo[d] = fmin(lo[d], v[d]);
            hi[d] = fmax(hi[d], v[d]);
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        lo[d] = warp_min(lo[d]);
        hi[d] = warp_max(hi[d]);
    }
    mmax = warp_max(mmax);
    // then over the block's warps, so that each block (not each warp) does the atomics
    __shared__ double sv[kBoundsThreads / 32][7];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool bbad = __syncthreads_or(bad);
    if (lane == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            sv[w][d] = lo[d];
            sv[w][3 + d] = hi[d];
        }
        sv[w][6] = mmax;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            lo[d] = warp_min(lane < nw ? sv[lane][d] : (double)INFINITY);
            hi[d] = warp_max(lane < nw ? sv[lane][3 + d] : -(double)INFINITY);
        }
        mmax = warp_max(lane < nw ? sv[lane][6] : 0.0);
        if (lane == 0) {
            if (bbad) atomicOr(status, kStatInvalid);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (lo[d] <= hi[d]) {
                    atomicMin(&bounds[d], dbl_key(lo[d]));
                    atomicMax(&bounds[3 + d], dbl_key(hi[d]));
                }
            }
            if (mmax > 0.0 && isfinite(mmax)) atomicMax(&bounds[6], dbl_key(mmax));
        }
    }
}

void launch_bounds(const double* x, const double* mu, int n, unsigned long long* bounds, unsigned* status,
                   cudaStream_t s) {
    k_bounds_init<<<1, 32, 0, s>>>(bounds); note_launch();
    if (n > 0) k_bounds<<<grid_for(n, kBoundsThreads, 8), kBoundsThreads, 0, s>>>(x, mu, n, bounds, status); note_launch();
}

// ------------------------------------------------------------------ A2 keys
__device__ inline uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffull;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

// Root cube: side = max extent * (1 + 2^-20), anchored at the lower corner.
__device__ inline void root_cube(const unsigned long long* bounds, double lo[3], double& side) {
    double ext = 0;
    for (int d = 0; d < 3; ++d) {
        lo[d] = key_dbl(bounds[d]);
        double e = key_dbl(bounds[3 + d]) - lo[d];
        if (e > ext) ext = e;
    }
    side = ext * (1.0 + 0x1p-20);
    if (!(side > 0)) side = 1.0;
}

// 21 bits per axis of (x - lo) / side, interleaved x-major
__device__ inline uint64_t morton_key(const double* __restrict__ xi, const double lo[3], double side) {
    uint32_t q[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double t = (xi[d] - lo[d]) / side;
        double u = t * 2097152.0;
        double f = floor(u);
        long long v = (long long)f;
        if (v < 0) v = 0;
        if (v > 2097151) v = 2097151;
        q[d] = (uint32_t)v;
    }
    return (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
}

__global__ void k_keys(const double* __restrict__ x, int n, const unsigned long long* __restrict__ bounds,
                       uint64_t* __restrict__ keys, int* __restrict__ idx) {
    double lo[3], side;
    root_cube(bounds, lo, side);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        keys[i] = morton_key(x + 3 * (long long)i, lo, side);
        idx[i] = i;
    }
}

void launch_keys(const double* x, int n, const unsigned long long* bounds, uint64_t* keys, int* idx,
                 cudaStream_t s) {
    if (n > 0) k_keys<<<grid_for(n, 256), 256, 0, s>>>(x, n, bounds, keys, idx); note_launch();
}

// ------------------------------------------------------------------ A1-A2 for an ensemble
// An ensemble of independent systems (contiguous particle ranges off[k] .. off[k+1]
// of the caller's arrays) is built as a forest: every system gets the bounding box,
// root cube and keys it would get alone, and its particles stay in their own block
// after sorting, so each tree is exactly the tree of the system alone.
__device__ inline int system_of(const int* __restrict__ off, int nsys, int i) {
    int lo = 0, hi = nsys - 1;  // last k with off[k] <= i
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_bounds_init_sys(unsigned long long* b, int nsys) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= 6 * nsys; i += gridDim.x * blockDim.x)
        b[i] = (i < 6 * nsys && (i % 6) < 3) ? ~0ull : 0ull;  // [6 nsys]: the largest mass
}

__global__ void k_bounds_sys(const double* __restrict__ x, const double* __restrict__ mu, int n,
                             const int* __restrict__ off, int nsys, unsigned long long* bounds, unsigned* status) {
    const int lane = threadIdx.x & 31;
    for (int i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
        const int i = i0 + threadIdx.x;
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        double mmax = 0.0;
        int k = -1;
        bool bad = false;
        if (i < n) {
            k = system_of(off, nsys, i);
            double v[3] = {x[3 * (long long)i], x[3 * (long long)i + 1], x[3 * (long long)i + 2]};
            double m = mu[i];
            bad = !(isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(m) && m >= 0.0);
#pragma unroll
            for (int d = 0; d < 3; ++d) lo[d] = hi[d] = v[d];
            if (m > 0.0 && isfinite(m)) mmax = m;
        }
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kStatInvalid);
        mmax = warp_max(mmax);
        if (lane == 0 && mmax > 0.0) atomicMax(&bounds[6 * nsys], dbl_key(mmax));
        const int k0 = __shfl_sync(0xffffffffu, k, 0);
        if (__all_sync(0xffffffffu, k == k0)) {  // the whole warp in one system: reduce first
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                lo[d] = warp_min(lo[d]);
                hi[d] = warp_max(hi[d]);
            }
            if (lane == 0 && k0 >= 0)
                for (int d = 0; d < 3; ++d) {
                    atomicMin(&bounds[6 * k0 + d], dbl_key(lo[d]));
                    atomicMax(&bounds[6 * k0 + 3 + d], dbl_key(hi[d]));
                }
        } else if (k >= 0) {
            for (int d = 0; d < 3; ++d) {
                atomicMin(&bounds[6 * k + d], dbl_key(lo[d]));
                atomicMax(&bounds[6 * k + 3 + d], dbl_key(hi[d]));
            }
        }
    }
}

void launch_bounds_sys(const double* x, const double* mu, int n, const int* off, int nsys,
                       unsigned long long* bounds, unsigned* status, cudaStream_t s) {
    k_bounds_init_sys<<<grid_for(6LL * nsys + 1, 256), 256, 0, s>>>(bounds, nsys); note_launch();
    if (n > 0) k_bounds_sys<<<grid_for(n, 256, 8), 256, 0, s>>>(x, mu, n, off, nsys, bounds, status); note_launch();
}

__global__ void k_keys_sys(const double* __restrict__ x, int n, const int* __restrict__ off, int nsys,
                           const unsigned long long* __restrict__ bounds, uint64_t* __restrict__ keys,
                           int* __restrict__ idx) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double lo[3], side;
        root_cube(bounds + 6 * system_of(off, nsys, i), lo, side);
        keys[i] = morton_key(x + 3 * (long long)i, lo, side);
        idx[i] = i;
    }
}

void launch_keys_sys(const double* x, int n, const int* off, int nsys, const unsigned long long* bounds,
                     uint64_t* keys, int* idx, cudaStream_t s) {
    if (n > 0) k_keys_sys<<<grid_for(n, 256), 256, 0, s>>>(x, n, off, nsys, bounds, keys, idx); note_launch();
}

// second stage of the ensemble sort: a stable sort of the key-sorted items by system
__global__ void k_system_keys(const int* __restrict__ idx, int n, const int* __restrict__ off, int nsys,
                              uint64_t* __restrict__ skey, int* __restrict__ pos) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        skey[i] = (uint64_t)system_of(off, nsys, idx[i]);
        pos[i] = i;
    }
}
__global__ void k_take(const uint64_t* __restrict__ kin, const int* __restrict__ vin, const int* __restrict__ pos,
                       int n, uint64_t* __restrict__ kout, int* __restrict__ vout) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = pos[i];
        kout[i] = kin[j];
        vout[i] = vin[j];
    }
}

int sort_by_system(const uint64_t* keys, const int* idx, int n, const int* off, int nsys, uint64_t* skey,
                   uint64_t* skey_alt, int* pos, int* pos_alt, int* tmp, uint64_t* keys_out, int* idx_out,
                   cudaStream_t s) {
    if (n <= 0) return 0;
    int bits = 8;
    while (bits < 32 && (1LL << bits) < nsys) bits += 8;
    k_system_keys<<<grid_for(n, 256), 256, 0, s>>>(idx, n, off, nsys, skey, pos); note_launch();
    const int flip = radix_sort_pairs_bits(skey, pos, skey_alt, pos_alt, n, tmp, 0, bits, s);
    k_take<<<grid_for(n, 256), 256, 0, s>>>(keys, idx, flip ? pos_alt : pos, n, keys_out, idx_out); note_launch();
    return 0;
}

// ------------------------------------------------------------------ A2 radix sort
// Stable LSD radix sort of (key, index) pairs, 8 bits per pass, 8 passes over the
// 63 key bits (index arrays nullptr: the keys alone).  Per pass: a digit histogram per tile, a device-wide exclusive scan
// in digit-major order, and a stable scatter that ranks equal digits inside the
// tile in item order with warp match masks.
constexpr int kRsThreads = 256;
constexpr int kRsRounds = 16;
constexpr int kRsTile = kRsThreads * kRsRounds;

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t* __restrict__ keys, int n, int shift,
                                                        int* __restrict__ hist, int nblocks) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    long long base = (long long)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsRounds; ++r) {
        long long i = base + r * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1);
    }
    __syncthreads();
    hist[threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t* __restrict__ kin,
                                                           const int* __restrict__ vin,
                                                           uint64_t* __restrict__ kout, int* __restrict__ vout,
                                                           int n, int shift, const int* __restrict__ offs,
                                                           int nblocks) {
    __shared__ int running[256];
    __shared__ int wc[kRsThreads / 32][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    running[threadIdx.x] = offs[threadIdx.x * nblocks + blockIdx.x];
    long long base = (long long)blockIdx.x * kRsTile;
    for (int r = 0; r < kRsRounds; ++r) {
#pragma unroll
        for (int k = 0; k < kRsThreads / 32; ++k) wc[k][threadIdx.x] = 0;
        __syncthreads();
        long long i = base + r * kRsThreads + threadIdx.x;
        bool valid = i < n;
        uint64_t key = valid ? kin[i] : 0;
        int val = (valid && vin) ? vin[i] : 0;
        int d = valid ? (int)((key >> shift) & 255) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & ((1u << lane) - 1));
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wc[w][d] = __popc(peers);
        __syncthreads();
        {   // per digit: exclusive prefix over the warps of this round
            int dg = threadIdx.x;
            int b = running[dg];
#pragma unroll
            for (int k = 0; k < kRsThreads / 32; ++k) {
                int c = wc[k][dg];
                wc[k][dg] = b;
                b += c;
            }
            running[dg] = b;
        }
        __syncthreads();
        if (valid) {
            int dst = wc[w][d] + rank;
            kout[dst] = key;
            if (vout) vout[dst] = val;
        }
        __syncthreads();
    }
}

size_t radix_tmp_ints(long long n) {
    long long nb = (n + kRsTile - 1) / kRsTile;
    if (nb < 1) nb = 1;
    return (size_t)(2 * 256 * nb) + scan_tmp_ints(256 * nb) + 8;
}

int radix_sort_pairs_bits(uint64_t* keys, int* idx, uint64_t* keys_alt, int* idx_alt, long long n, int* tmp,
                          int begin_bit, int end_bit, cudaStream_t s) {
    if (n <= 1) return 0;
    int nb = (int)((n + kRsTile - 1) / kRsTile);
    int* hist = tmp;
    int* offs = tmp + 256 * nb;
    int* stmp = tmp + 2 * 256 * nb;
    uint64_t *ka = keys, *kb = keys_alt;
    int *va = idx, *vb = idx_alt;
    int flips = 0;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        k_rs_hist<<<nb, kRsThreads, 0, s>>>(ka, (int)n, shift, hist, nb); note_launch();
        scan_exclusive_i32(hist, offs, 256LL * nb, nullptr, stmp, s);
        k_rs_scatter<<<nb, kRsThreads, 0, s>>>(ka, va, kb, vb, (int)n, shift, offs, nb); note_launch();
        uint64_t* tk = ka; ka = kb; kb = tk;
        int* tv = va; va = vb; vb = tv;
        flips ^= 1;
    }
    return flips;
}

void radix_sort_pairs(uint64_t* keys, int* idx, uint64_t* keys_alt, int* idx_alt, int n, int* tmp,
                      cudaStream_t s) {
    // 8 passes over the 63 key bits: the result is back in (keys, idx)
    radix_sort_pairs_bits(keys, idx, keys_alt, idx_alt, n, tmp, 0, 64, s);
}

// e (nullable): the working units, positions times 2^-e[0] and masses times 2^-e[1]
__global__ void k_gather(const double* __restrict__ x, const double* __restrict__ mu, const int* __restrict__ idx,
                         int n, d4* __restrict__ xm, int* __restrict__ perm, const int* __restrict__ e) {
    const double fx = e ? pow2i(-e[0]) : 1.0, fm = e ? pow2i(-e[1]) : 1.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int j = idx[i];
        xm[i] = mk4(x[3 * (long long)j] * fx, x[3 * (long long)j + 1] * fx, x[3 * (long long)j + 2] * fx, mu[j] * fm);
        perm[i] = j;
    }
}

void launch_gather(const double* x, const double* mu, const int* idx, int n, d4* xm, int* perm,
                   cudaStream_t s, const int* e) {
    if (n > 0) k_gather<<<grid_for(n, 256), 256, 0, s>>>(x, mu, idx, n, xm, perm, e); note_launch();
}

// The mixed-precision path works in units in which the system's extent and its largest mass
// lie in [1, 2): positions and masses are scaled by powers of two (exact), so the FP32
// parts (pair terms, high expansion orders, estimate) stay in range whatever the caller's
// units, and the outputs are scaled back exactly.  One thread; e[0], e[1]: the exponents.
__global__ void k_work_units(const unsigned long long* __restrict__ b, int nsys, int* __restrict__ e) {
    if (blockIdx.x || threadIdx.x) return;
    const int ns = nsys > 0 ? nsys : 1;
    double ext = 0.0;
    for (int k = 0; k < ns; ++k)
        for (int d = 0; d < 3; ++d) {
            const double lo = key_dbl(b[6 * k + d]), hi = key_dbl(b[6 * k + 3 + d]);
            if (hi >= lo) ext = fmax(ext, hi - lo);
        }
    const double mmax = key_dbl(b[6 * ns]);
    const bool use_m = b[6 * ns] != 0ull && mmax > 0.0 && isfinite(mmax);
    int el = (ext > 0.0 && isfinite(ext)) ? ilogb(ext) : 0, em = use_m ? ilogb(mmax) : 0;
    e[0] = max(-1000, min(1000, el));
    e[1] = max(-1000, min(1000, em));
}
void launch_work_units(const unsigned long long* bounds, int nsys, int* e, cudaStream_t s) {
    k_work_units<<<1, 32, 0, s>>>(bounds, nsys, e);
    note_launch();
}

// ------------------------------------------------------------------ A3 oct-tree
// A cell of level L holding more than leaf_size particles (and L < 21) is split
// into its non-empty octants, in key order.  One warp per cell; lane o < 8 finds
// the first particle whose level-(L+1) digit is >= o by binary search.
__global__ void k_split(const uint64_t* __restrict__ keys, Cells c, int lev_begin, int lev_end, int level,
                        int leaf_size, int* __restrict__ nchild_tmp, int* __restrict__ oct_tmp) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    int cell = lev_begin + warp;
    if (cell >= lev_end) return;
    int first = c.first[cell], count = c.count[cell];
    bool split = count > leaf_size && level < kMaxLevel;
    int b = first + count;
    if (split && lane < 8) {
        int shift = 3 * (kMaxLevel - (level + 1));
        int lo = first, hi = first + count;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            int dg = (int)((keys[mid] >> shift) & 7);
            if (dg < lane) lo = mid + 1;
            else hi = mid;
        }
        b = lo;
    }
    int bnext = __shfl_down_sync(0xffffffffu, b, 1);
    int size = (lane < 8) ? ((lane == 7 ? first + count : bnext) - b) : 0;
    unsigned nonempty = __ballot_sync(0xffffffffu, split && lane < 8 && size > 0);
    if (lane < 8) oct_tmp[9 * (long long)warp + lane] = b;
    if (lane == 8) oct_tmp[9 * (long long)warp + 8] = first + count;
    if (lane == 0) nchild_tmp[warp] = split ? __popc(nonempty) : 0;
}

__global__ void k_write_children(Cells c, int lev_begin, int lev_end, int level, const int* __restrict__ nchild_tmp,
                                 const int* __restrict__ oct_tmp, const int* __restrict__ offs) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    int cell = lev_begin + w;
    if (cell >= lev_end) return;
    int nc = nchild_tmp[w];
    int base = lev_end + offs[w];
    c.nchild[cell] = nc;
    c.child[cell] = nc ? base : -1;
    if (!nc) return;
    int k = 0;
    for (int o = 0; o < 8; ++o) {
        int b0 = oct_tmp[9 * (long long)w + o], b1 = oct_tmp[9 * (long long)w + o + 1];
        if (b1 > b0) {
            int d = base + k++;
            c.first[d] = b0;
            c.count[d] = b1 - b0;
            c.level[d] = level + 1;
            c.parent[d] = cell;
            c.nchild[d] = 0;
            c.child[d] = -1;
        }
    }
}

void launch_split_level(const uint64_t* keys, Cells c, int lev_begin, int lev_end, int level, int leaf_size,
                        int* nchild_tmp, int* oct_tmp, int* offs_tmp, int* scan_tmp, int* d_total,
                        cudaStream_t s) {
    int ncl = lev_end - lev_begin;
    k_split<<<(unsigned)(((long long)ncl * 32 + 255) / 256), 256, 0, s>>>(keys, c, lev_begin, lev_end, level,
                                                                         leaf_size, nchild_tmp, oct_tmp); note_launch();
    scan_exclusive_i32(nchild_tmp, offs_tmp, ncl, d_total, scan_tmp, s);
    k_write_children<<<(ncl + 255) / 256, 256, 0, s>>>(c, lev_begin, lev_end, level, nchild_tmp, oct_tmp, offs_tmp); note_launch();
}

// ------------------------------------------------------------------ A4 geometry
// Expansion centres z = s = centre of the smallest enclosing sphere (Sec. 5.1.1).
// The balls are computed in IEEE single precision in coordinates relative to a
// reference point of the cell (its first particle, or its first daughter's
// centre); the centre is converted back to FP64 and the radius rho is then
// recomputed exactly in FP64 over the cell's particles (Sec. 4).  Single
// precision keeps these small serial solves off the scarce FP64 pipe.
// support_ball: the smallest ball whose boundary touches each of k <= 4 balls
// (c_i, r_i) from inside, centre in the affine hull of the c_i: with
// u = c - c_0 = sum_j lam_j d_j, d_j = c_j - c_0, the tangency conditions give
// G lam = a + R b (G the Gram matrix of the d_j, a_j = (|d_j|^2 - r_j^2 + r_0^2)/2,
// b_j = r_j - r_0), and |u| = R - r_0 gives a quadratic in R.  With all r_i = 0 it
// is the circumsphere of the points.
constexpr float kMebSing = 1e-6f;  // singular support set (relative to the Gram scale)
constexpr float kMebIn = 1e-5f;    // inside tolerance, relative to the radius

// Gaussian elimination with partial pivoting of the K x K system A x = b0, b1 (K
// fixed at compile time so that the arrays stay in registers; the row swap is a
// select per candidate row, the arithmetic and its order as in the plain form)
template <int K>
__device__ __forceinline__ bool solve_small_k(const float (&A)[3][3], const float (&b0)[3], const float (&b1)[3],
                                              float (&x0)[3], float (&x1)[3]) {
    float M[K][K + 2];
    float scale = 0;
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (fabsf(A[i][j]) > scale) scale = fabsf(A[i][j]);
    if (scale == 0) return false;
#pragma unroll
    for (int i = 0; i < K; ++i) {
#pragma unroll
        for (int j = 0; j < K; ++j) M[i][j] = A[i][j];
        M[i][K] = b0[i];
        M[i][K + 1] = b1[i];
    }
#pragma unroll
    for (int col = 0; col < K; ++col) {
        int piv = col;
        float pv = fabsf(M[col][col]);
#pragma unroll
        for (int r = col + 1; r < K; ++r)
            if (fabsf(M[r][col]) > pv) {
                piv = r;
                pv = fabsf(M[r][col]);
            }
        if (pv <= kMebSing * scale) return false;
#pragma unroll
        for (int r = col + 1; r < K; ++r)
            if (piv == r)
#pragma unroll
                for (int j = 0; j < K + 2; ++j) {
                    const float t = M[col][j];
                    M[col][j] = M[r][j];
                    M[r][j] = t;
                }
#pragma unroll
        for (int r = col + 1; r < K; ++r) {
            const float fct = M[r][col] / M[col][col];
#pragma unroll
            for (int j = col; j < K + 2; ++j) M[r][j] -= fct * M[col][j];
        }
    }
#pragma unroll
    for (int r = K - 1; r >= 0; --r) {
        float s0 = M[r][K], s1 = M[r][K + 1];
#pragma unroll
        for (int j = r + 1; j < K; ++j) {
            s0 -= M[r][j] * x0[j];
            s1 -= M[r][j] * x1[j];
        }
        x0[r] = s0 / M[r][r];
        x1[r] = s1 / M[r][r];
    }
    return true;
}

// support_ball for a support set of NS = 1..4 balls (size fixed at compile time)
template <int NS>
__device__ __forceinline__ bool support_ball_k(const float (*c)[3], const float* r, float oc[3], float& orad) {
    if (NS == 1) {
        oc[0] = c[0][0]; oc[1] = c[0][1]; oc[2] = c[0][2];
        orad = r[0];
        return true;
    }
    constexpr int q = NS > 1 ? NS - 1 : 1;
    float D[3][3], G[3][3], a[3], b[3], la[3], lb[3];
#pragma unroll
    for (int j = 0; j < q; ++j)
#pragma unroll
        for (int d = 0; d < 3; ++d) D[j][d] = c[j + 1][d] - c[0][d];
#pragma unroll
    for (int i = 0; i < q; ++i) {
#pragma unroll
        for (int j = 0; j < q; ++j) G[i][j] = D[i][0] * D[j][0] + D[i][1] * D[j][1] + D[i][2] * D[j][2];
        a[i] = 0.5f * (G[i][i] - r[i + 1] * r[i + 1] + r[0] * r[0]);
        b[i] = r[i + 1] - r[0];
    }
    if (!solve_small_k<q>(G, a, b, la, lb)) return false;
    float A[3] = {0, 0, 0}, B[3] = {0, 0, 0};
#pragma unroll
    for (int j = 0; j < q; ++j)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            A[d] += la[j] * D[j][d];
            B[d] += lb[j] * D[j][d];
        }
    float qa = B[0] * B[0] + B[1] * B[1] + B[2] * B[2] - 1.0f;
    float qb = A[0] * B[0] + A[1] * B[1] + A[2] * B[2] + r[0];
    float qc = A[0] * A[0] + A[1] * A[1] + A[2] * A[2] - r[0] * r[0];
    float rmax = r[0];
#pragma unroll
    for (int i = 1; i < NS; ++i)
        if (r[i] > rmax) rmax = r[i];
    float R;
    if (fabsf(qa) < 1e-6f) {
        if (qb == 0) return false;
        R = -qc / (2.0f * qb);
    } else {
        float disc = qb * qb - qa * qc;
        if (disc < 0) {
            if (disc < -kMebSing * (qb * qb + fabsf(qa * qc))) return false;
            disc = 0;
        }
        float sq = sqrtf(disc);
        float r1 = (-qb - sq) / qa, r2 = (-qb + sq) / qa;
        float lo = r1 < r2 ? r1 : r2, hi = r1 < r2 ? r2 : r1;
        float tol = kMebSing * fabsf(rmax);
        if (lo >= rmax - tol) R = lo;
        else if (hi >= rmax - tol) R = hi;
        else return false;
    }
    if (!(R >= 0) || R < rmax - kMebSing * rmax) return false;
#pragma unroll
    for (int d = 0; d < 3; ++d) oc[d] = c[0][d] + A[d] + R * B[d];
    orad = R;
    return true;
}

// the smallest ball whose boundary touches each of k <= 4 balls (c_i, r_i) from
// inside (k at run time)
__device__ __noinline__ bool support_ball_dev(int k, const float (*c)[3], const float* r, float oc[3], float& orad) {
    switch (k) {
        case 1: return support_ball_k<1>(c, r, oc, orad);
        case 2: return support_ball_k<2>(c, r, oc, orad);
        case 3: return support_ball_k<3>(c, r, oc, orad);
        default: return support_ball_k<4>(c, r, oc, orad);
    }
}

__device__ inline float dist3f_dev(const float a[3], const float b[3]) {
    float dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrtf(dx * dx + dy * dy + dz * dz);
}

// Welzl's b_md(empty, R): the smallest ball with the support points on its boundary.
// When the nr points admit no ball through all of them (a degenerate set), the
// smallest ball through a subset that still contains the others
struct Pts4 {
    float p[4][3];
};
struct Ball4 {
    float c[3], r;
};
__device__ __noinline__ Ball4 trivial_ball_subsets(int nr, Pts4 R, Ball4 cur) {
    const float zr[4] = {0, 0, 0, 0};
    float best = -1;
    for (int mask = 1; mask < (1 << nr); ++mask) {
        float sub[4][3];
        int k = 0;
        for (int i = 0; i < nr; ++i)
            if (mask & (1 << i)) {
                for (int d = 0; d < 3; ++d) sub[k][d] = R.p[i][d];
                ++k;
            }
        float cc[3], rr;
        if (!support_ball_dev(k, sub, zr, cc, rr)) continue;
        bool ok = true;
        for (int i = 0; i < nr; ++i)
            if (dist3f_dev(R.p[i], cc) > rr * (1.0f + kMebIn)) {
                ok = false;
                break;
            }
        if (ok && (best < 0 || rr < best)) {
            best = rr;
            cur.c[0] = cc[0]; cur.c[1] = cc[1]; cur.c[2] = cc[2];
            cur.r = rr;
        }
    }
    return cur;
}
template <int NR>
__device__ __forceinline__ void trivial_ball_dev(const float (&R)[4][3], float (&c)[3], float& rad) {
    const float zr[4] = {0, 0, 0, 0};
    if (NR == 0) {
        c[0] = c[1] = c[2] = 0;
        rad = -1.0f;
        return;
    }
    if (support_ball_k<NR == 0 ? 1 : NR>(R, zr, c, rad)) return;
    Pts4 P;
    Ball4 cur;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int d = 0; d < 3; ++d) P.p[i][d] = R[i][d];
    cur.c[0] = c[0]; cur.c[1] = c[1]; cur.c[2] = c[2];
    cur.r = rad;
    cur = trivial_ball_subsets(NR, P, cur);
    c[0] = cur.c[0]; c[1] = cur.c[1]; c[2] = cur.c[2];
    rad = cur.r;
}

__device__ inline bool in_ball_dev(const float p[3], const float c[3], float rad) {
    if (rad < 0) return false;
    return dist3f_dev(p, c) <= rad * (1.0f + kMebIn);
}

__device__ inline void ld3(const d4* xm, int i, double p[3]) {
    d4 v = xm[i];
    p[0] = v.x; p[1] = v.y; p[2] = v.z;
}

// leaf points relative to the first one, in single precision, in the order of
// Welzl's recursion: from the warp's shared buffer (the first kMebBuf positions of
// that order) or converted on the fly
constexpr int kMebBuf = 128;
struct LeafPts {
    const float (*buf)[3];
    const d4* X;
    double o[3];
    __device__ inline void get(int i, float q[3]) const {
        if (i < kMebBuf) {
            q[0] = buf[i][0]; q[1] = buf[i][1]; q[2] = buf[i][2];
        } else {
            d4 v = X[i];
            q[0] = (float)(v.x - o[0]); q[1] = (float)(v.y - o[1]); q[2] = (float)(v.z - o[2]);
        }
    }
};

// Welzl's recursion for points (smallest ball of P with R on its boundary):
// W(i, R) scans P[0..i) in order and, at the first point outside the current
// ball, restarts one level deeper with that point added to R.  The warp form
// below scans each prefix 32 points at a time with a ballot for the first point
// outside, so the sequence of balls is exactly that of the sequential recursion.
__device__ int first_outside(const LeafPts& P, int from, int to, const float c[3], float rad, int lane) {
    for (int b = from; b < to; b += 32) {
        int i = b + lane;
        bool out = false;
        if (i < to) {
            float q[3];
            P.get(i, q);
            out = !in_ball_dev(q, c, rad);
        }
        unsigned m = __ballot_sync(0xffffffffu, out);
        if (m) return b + __ffs(m) - 1;
    }
    return -1;
}

__device__ __noinline__ void meb_points_warp(const LeafPts& P, int n, float c[3], float& rad, int lane) {
    float R[4][3];
    float c0[3], r0, c1[3], r1, c2[3], r2, c3[3], r3;
    trivial_ball_dev<0>(R, c0, r0);
    int i = first_outside(P, 0, n, c0, r0, lane);
    while (i >= 0) {
        P.get(i, R[0]);
        trivial_ball_dev<1>(R, c1, r1);
        int j = first_outside(P, 0, i, c1, r1, lane);
        while (j >= 0) {
            P.get(j, R[1]);
            trivial_ball_dev<2>(R, c2, r2);
            int k = first_outside(P, 0, j, c2, r2, lane);
            while (k >= 0) {
                P.get(k, R[2]);
                trivial_ball_dev<3>(R, c3, r3);
                int l = first_outside(P, 0, k, c3, r3, lane);
                while (l >= 0) {
                    P.get(l, R[3]);
                    trivial_ball_dev<4>(R, c3, r3);
                    l = first_outside(P, l + 1, k, c3, r3, lane);
                }
                for (int d = 0; d < 3; ++d) c2[d] = c3[d];
                r2 = r3;
                k = first_outside(P, k + 1, j, c2, r2, lane);
            }
            for (int d = 0; d < 3; ++d) c1[d] = c2[d];
            r1 = r2;
            j = first_outside(P, j + 1, i, c1, r1, lane);
        }
        for (int d = 0; d < 3; ++d) c0[d] = c1[d];
        r0 = r1;
        i = first_outside(P, i + 1, n, c0, r0, lane);
    }
    for (int d = 0; d < 3; ++d) c[d] = c0[d];
    rad = r0 < 0 ? 0 : r0;
}

// Welzl's recursion with the move-to-front rule for leaves held entirely in the
// warp's buffer (at most kMebBuf points): a point found outside is moved to the front
// of the list once the level it starts has finished, so later scans meet it first.
// The nested loops are the recursion levels 0..3 (a fourth support point ends it).
__device__ int first_outside_buf(const float (*L)[3], int from, int to, const float c[3], float rad, int lane) {
    for (int b = from; b < to; b += 32) {
        const int i = b + lane;
        const bool out = i < to && !in_ball_dev(L[i], c, rad);
        const unsigned m = __ballot_sync(0xffffffffu, out);
        if (m) return b + __ffs(m) - 1;
    }
    return -1;
}
// L[0..i] <- (L[i], L[0], ..., L[i-1])
__device__ void move_to_front(float (*L)[3], int i, int lane) {
    float v[kMebBuf / 32][3];
#pragma unroll
    for (int t = 0; t < kMebBuf / 32; ++t) {
        const int j = lane + 32 * t;
        if (j <= i) {
            v[t][0] = L[j][0];
            v[t][1] = L[j][1];
            v[t][2] = L[j][2];
        }
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < kMebBuf / 32; ++t) {
        const int j = lane + 32 * t;
        if (j <= i) {
            const int d = j == i ? 0 : j + 1;
            L[d][0] = v[t][0];
            L[d][1] = v[t][1];
            L[d][2] = v[t][2];
        }
    }
    __syncwarp();
}
__device__ inline void cp3(float d[3], const float s[3]) {
    d[0] = s[0];
    d[1] = s[1];
    d[2] = s[2];
}
__device__ void meb_points_mtf_warp(float (*L)[3], int n, float c[3], float& rad, int lane) {
    float R[4][3];
    float c0[3], r0, c1[3], r1, c2[3], r2, c3[3], r3;
    trivial_ball_dev<0>(R, c0, r0);
    for (int i0 = first_outside_buf(L, 0, n, c0, r0, lane); i0 >= 0;
         i0 = first_outside_buf(L, i0 + 1, n, c0, r0, lane)) {
        cp3(R[0], L[i0]);
        trivial_ball_dev<1>(R, c1, r1);
        for (int i1 = first_outside_buf(L, 0, i0, c1, r1, lane); i1 >= 0;
             i1 = first_outside_buf(L, i1 + 1, i0, c1, r1, lane)) {
            cp3(R[1], L[i1]);
            trivial_ball_dev<2>(R, c2, r2);
            for (int i2 = first_outside_buf(L, 0, i1, c2, r2, lane); i2 >= 0;
                 i2 = first_outside_buf(L, i2 + 1, i1, c2, r2, lane)) {
                cp3(R[2], L[i2]);
                trivial_ball_dev<3>(R, c3, r3);
                for (int i3 = first_outside_buf(L, 0, i2, c3, r3, lane); i3 >= 0;
                     i3 = first_outside_buf(L, i3 + 1, i2, c3, r3, lane)) {
                    cp3(R[3], L[i3]);
                    trivial_ball_dev<4>(R, c3, r3);
                    move_to_front(L, i3, lane);
                }
                cp3(c2, c3);
                r2 = r3;
                move_to_front(L, i2, lane);
            }
            cp3(c1, c2);
            r1 = r2;
            move_to_front(L, i1, lane);
        }
        cp3(c0, c1);
        r0 = r1;
        move_to_front(L, i0, lane);
    }
    cp3(c, c0);
    rad = r0 < 0 ? 0 : r0;
}

// one warp per leaf: smallest enclosing ball, exact radius, mass, centre of mass
constexpr int kGeoWarps = 4;
__global__ void __maxnreg__(128) k_leaf_geometry(const d4* __restrict__ xm, Cells c,
                                                                 const int* __restrict__ leaves, int nleaves,
                                                                 unsigned* status, bool keep_centre) {
    __shared__ float pbuf[kGeoWarps][kMebBuf][3];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int t = blockIdx.x * kGeoWarps + wid;
    if (t >= nleaves) return;
    const int cell = leaves[t];
    const int first = c.first[cell], count = c.count[cell];
    const d4* X = xm + first;
    double s[3];
    if (keep_centre) {  // a reused tree keeps its centres; radii, masses and centres of mass are new
        const d4 v = c.sr[cell];
        s[0] = v.x; s[1] = v.y; s[2] = v.z;
    } else {
    LeafPts P;
    P.buf = pbuf[wid];
    P.X = X;
    ld3(X, 0, P.o);
    // the buffer holds the first min(count, kMebBuf) points in the order Welzl's
    // recursion takes them: bit-reversed index order (t = 0, 1, ... over the next
    // power of two, keeping bitreverse(t) when it is below the count); points past
    // the buffer follow in index order
    {
        const int m = count < kMebBuf ? count : kMebBuf;
        int K = 1, bits = 0;
        while (K < m) {
            K <<= 1;
            ++bits;
        }
        int base = 0;
        for (int t0 = 0; t0 < K; t0 += 32) {
            const int t = t0 + lane;
            const int v = bits ? (int)(__brev((unsigned)t) >> (32 - bits)) : 0;
            const bool valid = t < K && v < m;
            const unsigned msk = __ballot_sync(0xffffffffu, valid);
            if (valid) {
                const int k = base + __popc(msk & ((1u << lane) - 1u));
                const d4 q = X[v];
                pbuf[wid][k][0] = (float)(q.x - P.o[0]);
                pbuf[wid][k][1] = (float)(q.y - P.o[1]);
                pbuf[wid][k][2] = (float)(q.z - P.o[2]);
            }
            base += __popc(msk);
        }
    }
    __syncwarp();
    float cf[3], radf;
    if (count <= kMebBuf) meb_points_mtf_warp(pbuf[wid], count, cf, radf, lane);
    else meb_points_warp(P, count, cf, radf, lane);
    s[0] = P.o[0] + (double)cf[0];
    s[1] = P.o[1] + (double)cf[1];
    s[2] = P.o[2] + (double)cf[2];
    }
    // radii as the square root of the largest squared distance (sqrt is monotonic and
    // correctly rounded, so this equals the largest distance)
    double r2max = 0, m = 0, mx[3] = {0, 0, 0};
    for (int i = lane; i < count; i += 32) {
        double p[3];
        ld3(X, i, p);
        const double dx = p[0] - s[0], dy = p[1] - s[1], dz = p[2] - s[2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 > r2max) r2max = r2;
        double w = X[i].w;
        m += w;
        for (int k = 0; k < 3; ++k) mx[k] += w * p[k];
    }
    const double rmax = sqrt(warp_max(r2max));
    m = warp_sum(m);
    for (int k = 0; k < 3; ++k) mx[k] = warp_sum(mx[k]);
    double com[3];
    for (int k = 0; k < 3; ++k) com[k] = (m > 0) ? mx[k] / m : s[k];
    double rc2 = 0;
    for (int i = lane; i < count; i += 32) {
        double p[3];
        ld3(X, i, p);
        const double dx = p[0] - com[0], dy = p[1] - com[1], dz = p[2] - com[2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 > rc2) rc2 = r2;
    }
    const double rc = sqrt(warp_max(rc2));
    if (lane == 0) {
        c.sr[cell] = mk4(s[0], s[1], s[2], rmax);
        c.cr[cell] = mk4(com[0], com[1], com[2], rc);
        c.mass[cell] = m;
    }
}

void launch_leaf_geometry(const d4* xm, Cells c, const int* leaves, int nleaves, unsigned* status,
                          cudaStream_t s, bool keep_centre) {
    if (nleaves > 0) {
        k_leaf_geometry<<<(nleaves + kGeoWarps - 1) / kGeoWarps, kGeoWarps * 32, 0, s>>>(xm, c, leaves, nleaves,
                                                                                       status, keep_centre);
        note_launch();
    }
}

// tmp layout per cell of the level (ncl cells): keys[2 ncl] (u64), lb[2 ncl] (float),
// cen[12 ncl] (float: s hi, s lo, com hi, com lo)
struct RadTmp {
    unsigned long long* key;
    float* lb;
    float* cen;
    __host__ __device__ RadTmp(unsigned long long* t, int ncl)
        : key(t), lb((float*)(t + 2 * (size_t)ncl)), cen((float*)(t + 3 * (size_t)ncl)) {}
};
size_t rad_tmp_u64_per_cell() { return 9; }

__device__ inline void write_cen_f(const RadTmp& R, int k, const double s[3], const double m[3]) {
    float* q = R.cen + 12 * (size_t)k;
    for (int d = 0; d < 3; ++d) {
        const float h = (float)s[d];
        q[d] = h;
        q[3 + d] = (float)(s[d] - (double)h);
        const float hm = (float)m[d];
        q[6 + d] = hm;
        q[9 + d] = (float)(m[d] - (double)hm);
    }
}

// Internal cells of one level: smallest ball enclosing the daughter balls (s_d, rho_d),
// as the smallest support ball (over all subsets of 1..4 daughters, enumerated by
// mask) that contains every daughter ball; single precision relative to the first
// daughter's centre.  One warp per cell, lanes take masks; ties go to the smaller mask.
// one block of kMebWarps warps per internal cell; warp w tries the support sets with
// bit masks 1 + 32 w + lane (at most 4 daughters), and the block keeps the smallest
// valid ball (ties: the smaller mask)
constexpr int kMebWarps = 8;
__global__ void __launch_bounds__(kMebWarps * 32) k_internal_meb(Cells c, int lev_begin, int lev_end,
                                                                 unsigned* status, unsigned long long* tmp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int cell = lev_begin + blockIdx.x;
    if (cell >= lev_end) return;
    const int nch = c.nchild[cell];
    if (nch == 0) return;  // leaves are done
    const int ch = c.child[cell];
    const d4 o = c.sr[ch];
    // the daughters' balls relative to the first one (registers: loops over all 8 slots)
    float cen[8][3], rad[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        cen[i][0] = cen[i][1] = cen[i][2] = rad[i] = 0.f;
        if (i < nch) {
            const d4 v = c.sr[ch + i];
            cen[i][0] = (float)(v.x - o.x);
            cen[i][1] = (float)(v.y - o.y);
            cen[i][2] = (float)(v.z - o.z);
            rad[i] = (float)v.w;
        }
    }
    float best = -1, bc[3] = {0, 0, 0};
    int bmask = 1 << 30;
    const int mask = 1 + lane + 32 * wid;
    if (mask < (1 << nch) && __popc(mask) <= 4) {
        // the k-th daughter of the mask into slot k of the support set
        float sc[4][3] = {}, sr[4] = {};
        int k = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (mask & (1 << i)) {
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (k == t) {
                        sc[t][0] = cen[i][0]; sc[t][1] = cen[i][1]; sc[t][2] = cen[i][2];
                        sr[t] = rad[i];
                    }
                ++k;
            }
        float cc[3], rr;
        bool found;
        switch (k) {
            case 1: found = support_ball_k<1>(sc, sr, cc, rr); break;
            case 2: found = support_ball_k<2>(sc, sr, cc, rr); break;
            case 3: found = support_ball_k<3>(sc, sr, cc, rr); break;
            default: found = support_ball_k<4>(sc, sr, cc, rr); break;
        }
        if (found) {
            bool ok = true;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (i < nch && dist3f_dev(cen[i], cc) + rad[i] > rr * (1.0f + kMebIn)) ok = false;
            if (ok) {
                best = rr;
                bmask = mask;
                bc[0] = cc[0]; bc[1] = cc[1]; bc[2] = cc[2];
            }
        }
    }
    // warp argmin of (radius, mask), then across the warps
    for (int off = 16; off > 0; off >>= 1) {
        float ob = __shfl_xor_sync(0xffffffffu, best, off);
        int om = __shfl_xor_sync(0xffffffffu, bmask, off);
        float o0 = __shfl_xor_sync(0xffffffffu, bc[0], off);
        float o1 = __shfl_xor_sync(0xffffffffu, bc[1], off);
        float o2 = __shfl_xor_sync(0xffffffffu, bc[2], off);
        bool take = (ob >= 0) && (best < 0 || ob < best || (ob == best && om < bmask));
        if (take) {
            best = ob; bmask = om;
            bc[0] = o0; bc[1] = o1; bc[2] = o2;
        }
    }
    __shared__ float wbest[kMebWarps], wbc[kMebWarps][3];
    __shared__ int wmask[kMebWarps];
    if (lane == 0) {
        wbest[wid] = best;
        wmask[wid] = bmask;
        wbc[wid][0] = bc[0]; wbc[wid][1] = bc[1]; wbc[wid][2] = bc[2];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kMebWarps; ++w) {
            const float ob = wbest[w];
            const int om = wmask[w];
            if ((ob >= 0) && (best < 0 || ob < best || (ob == best && om < bmask))) {
                best = ob; bmask = om;
                bc[0] = wbc[w][0]; bc[1] = wbc[w][1]; bc[2] = wbc[w][2];
            }
        }
        if (best < 0) {  // no valid support set: the first daughter's centre
            atomicOr(status, kStatMeb);
            bc[0] = bc[1] = bc[2] = 0.f;
        }
        double m = 0, mx[3] = {0, 0, 0};
        for (int i = 0; i < nch; ++i) {
            const double md = c.mass[ch + i];
            const d4 cm = c.cr[ch + i];
            m += md;
            mx[0] += md * cm.x; mx[1] += md * cm.y; mx[2] += md * cm.z;
        }
        double s[3] = {o.x + (double)bc[0], o.y + (double)bc[1], o.z + (double)bc[2]};
        double com[3];
        for (int k = 0; k < 3; ++k) com[k] = (m > 0) ? mx[k] / m : s[k];
        c.sr[cell] = mk4(s[0], s[1], s[2], 0.0);
        c.cr[cell] = mk4(com[0], com[1], com[2], 0.0);
        c.mass[cell] = m;
        write_cen_f(RadTmp(tmp, lev_end - lev_begin), cell - lev_begin, s, com);
    }
}

// Exact radii of the internal cells of one level: max over their particles of |x - s|
// and |x - com| (Sec. 4), taken in FP64, but only for the particles that can attain the
// maximum.  A first pass bounds every distance in FP32 from the two-float positions and
// the two-float centres: the difference of two-float values carries at most 2^-23 |d| +
// 2^-46 (|x| + |s|) per coordinate, so with d_f the FP32 distance
//   d_f (1 - 2^-20) - E <= d <= d_f (1 + 2^-20) + E,  E = 2^-44 sum_c (|x_c| + |s_c|)
// (the FP32 square and square root stay inside the relative margin; below the coordinate
// range 2^-18 an underflowed square would escape E and above 2^60 it would overflow, so
// there every particle is a candidate).  The per-cell maximum LB of the lower bounds is
// at most the largest distance, so the particle attaining it has an upper bound >= LB;
// the second pass takes the FP64 distance of every particle whose upper bound reaches LB,
// and the maximum over those is the maximum over all, bit for bit.
// owner[i]: the particle's ancestor at the level processed last (its leaf to begin with).
// The levels are processed bottom-up, so at level L the owner moves up one cell when it
// lies below L; the particle belongs to an internal cell of level L iff its owner is one.
__global__ void k_leaf_owner(Cells c, const int* __restrict__ leaves, int nleaves, int* __restrict__ owner) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nleaves; t += gridDim.x * blockDim.x) {
        const int leaf = leaves[t];
        for (int i = c.first[leaf], e = c.first[leaf] + c.count[leaf]; i < e; ++i) owner[i] = leaf;
    }
}
void launch_leaf_owner(Cells c, const int* leaves, int nleaves, int* owner, cudaStream_t s) {
    if (nleaves > 0) {
        k_leaf_owner<<<grid_for(nleaves, 128), 128, 0, s>>>(c, leaves, nleaves, owner);
        note_launch();
    }
}
__device__ inline int level_cell_up(const Cells& c, int L, int* __restrict__ owner, int i) {
    int a = owner[i];
    if (c.level[a] > L) {
        a = c.parent[a];
        owner[i] = a;
    }
    return (c.level[a] == L && c.nchild[a] > 0) ? a : -1;
}
__device__ inline int level_cell_now(const Cells& c, int L, const int* __restrict__ owner, int i) {
    const int a = owner[i];
    return (c.level[a] == L && c.nchild[a] > 0) ? a : -1;
}

// FP32 bounds of the distance of particle i from a two-float centre q (hi[3], lo[3])
__device__ inline void dist_bounds_f(const float4* __restrict__ xp, int i, const float* q, float& lb, float& ub) {
    const float4 h = xp[2 * (size_t)i], l = xp[2 * (size_t)i + 1];
    const float xhs[3] = {h.x, h.y, h.z}, xls[3] = {l.x, l.y, l.z};
    float d2 = 0.f, mag = 0.f;
    for (int d = 0; d < 3; ++d) {
        const float xh = xhs[d];
        const float dd = __fadd_rn(__fsub_rn(xh, q[d]), __fsub_rn(xls[d], q[3 + d]));
        d2 = __fmaf_rn(dd, dd, d2);
        mag = __fadd_rn(mag, __fadd_rn(fabsf(xh), fabsf(q[d])));
    }
    if (!(mag >= 0x1p-18f && mag <= 0x1p60f)) {
        lb = 0.f;
        ub = __int_as_float(0x7f800000);
        return;
    }
    const float df = sqrtf(d2), E = mag * 0x1p-44f;
    lb = fmaxf(0.f, df * (1.0f - 0x1p-20f) - E);
    ub = df * (1.0f + 0x1p-20f) + E;
}

constexpr int kRadThreads = 256;
__global__ void __launch_bounds__(kRadThreads) k_internal_radii_lb(const float4* __restrict__ xp, int n, Cells c,
                                    int lev_begin, int lev_end, int* __restrict__ owner,
                                    unsigned long long* __restrict__ tmp) {
    __shared__ int s_cell;
    __shared__ float s_l[kRadThreads / 32][2];
    const RadTmp R(tmp, lev_end - lev_begin);
    const int L = c.level[lev_begin];
    const int pbeg = c.first[lev_begin];
    const int pend = c.first[lev_end - 1] + c.count[lev_end - 1];
    for (int i0 = blockIdx.x * blockDim.x; i0 < pend - pbeg; i0 += gridDim.x * blockDim.x) {
        const int i = pbeg + i0 + threadIdx.x;
        int cell = -1;
        float l0 = 0.f, l1 = 0.f;
        if (i < pend) {
            cell = level_cell_up(c, L, owner, i);
            if (cell >= 0) {
                const float* q = R.cen + 12 * (size_t)(cell - lev_begin);
                float u;
                dist_bounds_f(xp, i, q, l0, u);
                dist_bounds_f(xp, i, q + 6, l1, u);
            }
        }
        // non-negative floats order as their bit patterns
        const int c0 = __shfl_sync(0xffffffffu, cell, 0);
        const bool wsame = __all_sync(0xffffffffu, cell == c0);
        if (wsame) {
            for (int o = 16; o > 0; o >>= 1) {
                l0 = fmaxf(l0, __shfl_xor_sync(0xffffffffu, l0, o));
                l1 = fmaxf(l1, __shfl_xor_sync(0xffffffffu, l1, o));
            }
        }
        // near the root every particle of a block shares its cell: one atomic per block
        // (the max does not depend on the order it is taken in)
        if (threadIdx.x == 0) s_cell = cell;
        __syncthreads();
        if (__syncthreads_and(wsame && c0 == s_cell)) {
            if ((threadIdx.x & 31) == 0) {
                s_l[threadIdx.x >> 5][0] = l0;
                s_l[threadIdx.x >> 5][1] = l1;
            }
            __syncthreads();
            if (threadIdx.x == 0 && cell >= 0) {
                for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
                    l0 = fmaxf(l0, s_l[k][0]);
                    l1 = fmaxf(l1, s_l[k][1]);
                }
                atomicMax((int*)&R.lb[2 * (cell - lev_begin)], __float_as_int(l0));
                atomicMax((int*)&R.lb[2 * (cell - lev_begin) + 1], __float_as_int(l1));
            }
            __syncthreads();
        } else if (wsame) {
            if ((threadIdx.x & 31) == 0 && c0 >= 0) {
                atomicMax((int*)&R.lb[2 * (c0 - lev_begin)], __float_as_int(l0));
                atomicMax((int*)&R.lb[2 * (c0 - lev_begin) + 1], __float_as_int(l1));
            }
        } else if (cell >= 0) {
            atomicMax((int*)&R.lb[2 * (cell - lev_begin)], __float_as_int(l0));
            atomicMax((int*)&R.lb[2 * (cell - lev_begin) + 1], __float_as_int(l1));
        }
    }
}

__global__ void k_internal_radii(const d4* __restrict__ xm, const float4* __restrict__ xp, int n, Cells c,
                                 int lev_begin, int lev_end,
                                 const int* __restrict__ owner, unsigned long long* __restrict__ tmp) {
    const RadTmp R(tmp, lev_end - lev_begin);
    const int L = c.level[lev_begin];
    const int pbeg = c.first[lev_begin];
    const int pend = c.first[lev_end - 1] + c.count[lev_end - 1];
    for (int i0 = blockIdx.x * blockDim.x; i0 < pend - pbeg; i0 += gridDim.x * blockDim.x) {
        const int i = pbeg + i0 + threadIdx.x;
        if (i >= pend) continue;
        const int cell = level_cell_now(c, L, owner, i);
        if (cell < 0) continue;
        const int k = cell - lev_begin;
        const float* q = R.cen + 12 * (size_t)k;
        float l, u0, u1;
        dist_bounds_f(xp, i, q, l, u0);
        dist_bounds_f(xp, i, q + 6, l, u1);
        const bool want0 = u0 >= R.lb[2 * k], want1 = u1 >= R.lb[2 * k + 1];
        if (!want0 && !want1) continue;
        const d4 p = xm[i];
        if (want0) {
            const d4 sc = c.sr[cell];
            const double dx = p.x - sc.x, dy = p.y - sc.y, dz = p.z - sc.z;
            atomicMax(&R.key[2 * k], dbl_key(dx * dx + dy * dy + dz * dz));
        }
        if (want1) {
            const d4 m = c.cr[cell];
            const double ex = p.x - m.x, ey = p.y - m.y, ez = p.z - m.z;
            atomicMax(&R.key[2 * k + 1], dbl_key(ex * ex + ey * ey + ez * ez));
        }
    }
}

__global__ void k_internal_radii_finish(Cells c, int lev_begin, int lev_end,
                                        const unsigned long long* __restrict__ rad_tmp) {
    int cell = lev_begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= lev_end || c.nchild[cell] == 0) return;
    double d2 = key_dbl(rad_tmp[2 * (cell - lev_begin)]);
    double e2 = key_dbl(rad_tmp[2 * (cell - lev_begin) + 1]);
    c.sr[cell].w = sqrt(d2);
    c.cr[cell].w = sqrt(e2);
}

// a reused tree: the centres stay, mass and centre of mass from the daughters
__global__ void k_internal_keep(Cells c, int lev_begin, int lev_end, unsigned long long* tmp) {
    const int cell = lev_begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= lev_end) return;
    const int nch = c.nchild[cell];
    if (nch == 0) return;
    const int ch = c.child[cell];
    double m = 0, mx[3] = {0, 0, 0};
    for (int i = 0; i < nch; ++i) {
        const double md = c.mass[ch + i];
        const d4 cm = c.cr[ch + i];
        m += md;
        mx[0] += md * cm.x; mx[1] += md * cm.y; mx[2] += md * cm.z;
    }
    const d4 s = c.sr[cell];
    const double com[3] = {m > 0 ? mx[0] / m : s.x, m > 0 ? mx[1] / m : s.y, m > 0 ? mx[2] / m : s.z};
    c.cr[cell] = mk4(com[0], com[1], com[2], 0.0);
    c.mass[cell] = m;
    const double sv[3] = {s.x, s.y, s.z};
    write_cen_f(RadTmp(tmp, lev_end - lev_begin), cell - lev_begin, sv, com);
}

void launch_internal_geometry(const d4* xm, const float4* xp, Cells c, int lev_begin, int lev_end,
                              int n, int* owner, unsigned long long* rad_tmp, unsigned* status, cudaStream_t s,
                              bool keep_centre) {
    int ncl = lev_end - lev_begin;
    if (ncl <= 0) return;
    // bounds and keys start at 0 (every distance is >= 0)
    cudaMemsetAsync(rad_tmp, 0, sizeof(unsigned long long) * 3 * (size_t)ncl, s);
    if (keep_centre) k_internal_keep<<<(ncl + 127) / 128, 128, 0, s>>>(c, lev_begin, lev_end, rad_tmp);
    else k_internal_meb<<<(unsigned)ncl, kMebWarps * 32, 0, s>>>(c, lev_begin, lev_end, status, rad_tmp);
    note_launch();
    k_internal_radii_lb<<<grid_for(n, kRadThreads, 16), kRadThreads, 0, s>>>(xp, n, c, lev_begin, lev_end, owner,
                                                                     rad_tmp);
    note_launch();
    k_internal_radii<<<grid_for(n, 256, 16), 256, 0, s>>>(xm, xp, n, c, lev_begin, lev_end, owner,
                                                                  rad_tmp);
    note_launch();
    k_internal_radii_finish<<<(ncl + 255) / 256, 256, 0, s>>>(c, lev_begin, lev_end, rad_tmp); note_launch();
}

}  // namespace gb3
