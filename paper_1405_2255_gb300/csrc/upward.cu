// upward.cu -- A5-A6 of the path (P2M eq. 3c, M2M eq. 4, multipole power eq. 14)
// and the per-cell minimum of the acceleration scale used by eqs. (18a,b).
#include <vector>
#include <algorithm>

#include "harmonics.cuh"
#include "kernels.cuh"

namespace gb3 {

LaneSched make_lane_sched(int p, SchedKind kind) {
    LaneSched s;
    memset(&s, 0, sizeof s);
    std::vector<std::pair<int, int>> outs;
    for (int n = 0; n <= p; ++n)
        for (int m = 0; m <= n; ++m) outs.push_back({n, m});
    auto cost = [p, kind](int n) -> long long {
        long long t = kind == kSchedDown ? (p - n + 1) : (n + 1);
        return t * t;
    };
    std::stable_sort(outs.begin(), outs.end(), [&](const std::pair<int, int>& a, const std::pair<int, int>& b) {
        return cost(a.first) > cost(b.first);
    });
    long long load[32] = {0};
    for (auto& o : outs) {
        int best = 0;
        for (int l = 1; l < 32; ++l)
            if (load[l] < load[best] || (load[l] == load[best] && s.cnt[l] < s.cnt[best])) best = l;
        if (s.cnt[best] >= kMaxPerLane) {  // fall back to the lane with the fewest outputs
            for (int l = 0; l < 32; ++l)
                if (s.cnt[l] < s.cnt[best]) best = l;
        }
        int k = s.cnt[best]++;
        s.n[best][k] = (unsigned char)o.first;
        s.m[best][k] = (unsigned char)o.second;
        load[best] += cost(o.first);
    }
    return s;
}

// ---------------------------------------------------------------- P2M
// One warp per leaf; lane j takes particles j, j+32, ...; for each m-column the
// Upsilon_n^m(x - z) values of the 32 particles are summed over the warp.
__global__ void k_p2m(const d4* __restrict__ xm, Cells c, const d4* __restrict__ cen, const int* __restrict__ leaves,
                      int nleaves, int p, double* __restrict__ M) {
    extern __shared__ double smem[];
    const int wpb = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nco = ncoef(p);
    double* acc = smem + (size_t)wid * nco;
    int t = blockIdx.x * wpb + wid;
    if (t >= nleaves) return;
    int cell = leaves[t];
    for (int i = lane; i < nco; i += 32) acc[i] = 0.0;
    __syncwarp();
    const d4 z = cen[cell];
    const int first = c.first[cell], count = c.count[cell];
    for (int b = 0; b < count; b += 32) {
        int i = b + lane;
        double x = 0, y = 0, zz = 0, mu = 0;
        if (i < count) {
            d4 q = xm[first + i];
            x = q.x - z.x; y = q.y - z.y; zz = q.z - z.z; mu = q.w;
        }
        const double r2 = x * x + y * y + zz * zz;
        cd d = mkc(mu, 0.0);  // mu * Upsilon_m^m
        for (int m = 0; m <= p; ++m) {
            if (m > 0) {
                double s = 1.0 / (2.0 * m);
                d = cd{s * (x * d.re - y * d.im), s * (x * d.im + y * d.re)};
            }
            cd prev2 = mkc(0.0, 0.0), prev = d;
            for (int n = m; n <= p; ++n) {
                cd v;
                if (n == m) v = d;
                else {
                    double inv = 1.0 / (double)(n * n - m * m);
                    double a = (2.0 * n - 1.0) * zz;
                    v = cd{(a * prev.re - r2 * prev2.re) * inv, (a * prev.im - r2 * prev2.im) * inv};
                    prev2 = prev;
                    prev = v;
                }
                double sr = warp_sum(v.re);
                double si = warp_sum(v.im);
                if (lane == 0) {
                    acc[cix(n, m)] += sr;
                    if (m) acc[cix(n, -m)] += si;
                }
            }
        }
    }
    __syncwarp();
    double* out = M + (size_t)cell * nco;
    for (int i = lane; i < nco; i += 32) out[i] = acc[i];
}

void launch_p2m(const d4* xm, Cells c, const d4* cen, const int* leaves, int nleaves, int p, double* M,
                cudaStream_t s) {
    if (nleaves <= 0) return;
    const int wpb = 4;
    size_t sm = (size_t)wpb * ncoef(p) * sizeof(double);
    k_p2m<<<(nleaves + wpb - 1) / wpb, wpb * 32, sm, s>>>(xm, c, cen, leaves, nleaves, p, M); note_launch();
}

// ---------------------------------------------------------------- M2M
// M_n^m(z') = sum_{k<=n} sum_l Upsilon_k^l(z - z') M_{n-k}^{m-l}(z), one warp per
// parent; daughters one after another through shared memory.
__global__ void k_m2m(Cells c, const d4* __restrict__ cen, int lev_begin, int lev_end, int p,
                      double* __restrict__ M, LaneSched sched) {
    extern __shared__ cd csm[];
    const int wpb = blockDim.x >> 5;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nco = ncoef(p);
    cd* Yw = csm + (size_t)wid * 2 * nco;
    cd* Mw = Yw + nco;
    int cell = lev_begin + blockIdx.x * wpb + wid;
    if (cell >= lev_end) return;
    int nch = c.nchild[cell];
    if (nch == 0) return;
    const d4 zp = cen[cell];
    cd acc[kMaxPerLane];
    const int cnt = sched.cnt[lane];
#pragma unroll
    for (int k = 0; k < kMaxPerLane; ++k) acc[k] = mkc(0.0, 0.0);
    for (int j = 0; j < nch; ++j) {
        int d = c.child[cell] + j;
        const d4 z = cen[d];
        if (lane <= p) upsilon_column(p, lane, z.x - zp.x, z.y - zp.y, z.z - zp.z, Yw, false);
        expand_real(p, M + (size_t)d * nco, Mw, false, lane, 32);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < kMaxPerLane; ++q) {
            if (q < cnt) {
                int n = sched.n[lane][q], m = sched.m[lane][q];
                cd s = mkc(0.0, 0.0);
                for (int k = 0; k <= n; ++k) {
                    int nn = n - k;
                    int lmin = max(-k, m - nn), lmax = min(k, m + nn);
                    for (int l = lmin; l <= lmax; ++l) cmac(s, Yw[cix(k, l)], Mw[cix(nn, m - l)]);
                }
                acc[q] = acc[q] + s;
            }
        }
        __syncwarp();
    }
    double* out = M + (size_t)cell * nco;
#pragma unroll
    for (int q = 0; q < kMaxPerLane; ++q) {
        if (q < cnt) {
            int n = sched.n[lane][q], m = sched.m[lane][q];
            out[cix(n, m)] = acc[q].re;
            if (m) out[cix(n, -m)] = acc[q].im;
        }
    }
}

void launch_m2m_level(Cells c, const d4* cen, int lev_begin, int lev_end, int p, double* M, cudaStream_t s) {
    int ncl = lev_end - lev_begin;
    if (ncl <= 0) return;
    const int wpb = 4;
    size_t sm = (size_t)wpb * 2 * ncoef(p) * sizeof(cd);
    LaneSched sched = make_lane_sched(p, kSchedUp);
    init_rec_tables();
    k_m2m<<<(ncl + wpb - 1) / wpb, wpb * 32, sm, s>>>(c, cen, lev_begin, lev_end, p, M, sched); note_launch();
}

// ---------------------------------------------------------------- power
__constant__ double c_fact[41];

__global__ void k_power(const double* __restrict__ M, int ncells, int p, double* __restrict__ P) {
    int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= ncells) return;
    const double* R = M + (size_t)cell * ncoef(p);
    for (int n = 0; n <= p; ++n) {
        double s = c_fact[n] * c_fact[n] * R[cix(n, 0)] * R[cix(n, 0)];
        for (int m = 1; m <= n; ++m) {
            double re = R[cix(n, m)], im = R[cix(n, -m)];
            s += 2.0 * c_fact[n - m] * c_fact[n + m] * (re * re + im * im);
        }
        P[(size_t)cell * (p + 1) + n] = sqrt(s);
    }
}

void launch_power(const double* M, int ncells, int p, double* P, cudaStream_t s) {
    static DeviceOnce once;
    once_per_device(once, [] {
        double f[41];
        f[0] = 1;
        for (int i = 1; i <= 40; ++i) f[i] = f[i - 1] * i;
        cudaMemcpyToSymbol(c_fact, f, sizeof f);
    });
    if (ncells > 0) k_power<<<(ncells + 127) / 128, 128, 0, s>>>(M, ncells, p, P); note_launch();
}

// ---------------------------------------------------------------- min scale
__global__ void k_minscale_leaves(const double* __restrict__ sc, Cells c, const int* __restrict__ leaves,
                                  int nleaves) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nleaves) return;
    int cell = leaves[t];
    double m = INFINITY;
    for (int i = c.first[cell], e = c.first[cell] + c.count[cell]; i < e; ++i)
        if (!c.pact || c.pact[i]) m = fmin(m, sc[i]);  // over the active sinks only (Sec. 7.1)
    c.minscale[cell] = m;
}
void launch_minscale_leaves(const double* scale_sorted, Cells c, const int* leaves, int nleaves, cudaStream_t s) {
    if (nleaves > 0) k_minscale_leaves<<<(nleaves + 127) / 128, 128, 0, s>>>(scale_sorted, c, leaves, nleaves); note_launch();
}
__global__ void k_minscale_level(Cells c, int lev_begin, int lev_end) {
    int cell = lev_begin + blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= lev_end) return;
    int nch = c.nchild[cell];
    if (!nch) return;
    double m = INFINITY;
    for (int j = 0; j < nch; ++j) m = fmin(m, c.minscale[c.child[cell] + j]);
    c.minscale[cell] = m;
}
void launch_minscale_level(Cells c, int lev_begin, int lev_end, cudaStream_t s) {
    int ncl = lev_end - lev_begin;
    if (ncl > 0) k_minscale_level<<<(ncl + 127) / 128, 128, 0, s>>>(c, lev_begin, lev_end); note_launch();
}
// the caller's scale (an acceleration, ~ mu / x^2) in the working units (e nullable)
__global__ void k_scale_from_caller(const double* __restrict__ scale, const int* __restrict__ perm, int n,
                                    double* __restrict__ out, const int* __restrict__ e) {
    const int ks = e ? 2 * e[0] - e[1] : 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = ldexp(scale[perm[i]], ks);
}
void launch_scale_from_caller(const double* scale, const int* perm, int n, double* scale_sorted, cudaStream_t s,
                              const int* e) {
    if (n > 0) k_scale_from_caller<<<grid_for(n, 256), 256, 0, s>>>(scale, perm, n, scale_sorted, e); note_launch();
}

}  // namespace gb3

namespace gb3 {
// ---------------------------------------------------------------- active subsets (Sec. 7.1)
__global__ void k_active_sorted(const unsigned char* __restrict__ active, const int* __restrict__ perm, int n,
                                unsigned char* __restrict__ pact, int* __restrict__ ai) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned char a = active[perm[i]] != 0;
        pact[i] = a;
        ai[i] = a;
    }
}
__global__ void k_active_cells(const int* __restrict__ first, const int* __restrict__ count, int ncells,
                               const int* __restrict__ scan, const int* __restrict__ total, int n,
                               unsigned char* __restrict__ act) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        const int f = first[c], e = f + count[c];
        const int hi = e < n ? scan[e] : *total;
        act[c] = hi - scan[f] > 0;
    }
}
void launch_active_flags(const unsigned char* active, const int* perm, int n, const int* first, const int* count,
                         int ncells, unsigned char* pact, unsigned char* act, int* ai, int* scan, int* scan_tmp,
                         cudaStream_t s) {
    if (n <= 0) return;
    k_active_sorted<<<grid_for(n, 256), 256, 0, s>>>(active, perm, n, pact, ai);
    note_launch();
    int* total = ai + n;  // ai holds n + 1 ints
    scan_exclusive_i32(ai, scan, n, total, scan_tmp, s);
    k_active_cells<<<grid_for(ncells, 256), 256, 0, s>>>(first, count, ncells, scan, total, n, act);
    note_launch();
}
}  // namespace gb3

namespace gb3 {
// ---------------------------------------------------------------- individual accuracy (Sec. 7, opening)
// scale_sorted[i] *= eps_b[perm[i]] / eps, so that eps * min_B(scale) = min_B(eps_b a_b);
// a non-positive or non-finite eps_b sets kStatInvalid
__global__ void k_scale_eps(const double* __restrict__ eps_b, const int* __restrict__ perm, int n, double eps,
                            double* __restrict__ scale_sorted, unsigned* __restrict__ status) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double e = eps_b[perm[i]];
        if (!(e > 0) || !isfinite(e)) atomicOr(status, kStatInvalid);
        scale_sorted[i] *= e / eps;
    }
}
void launch_scale_eps(const double* eps_b, const int* perm, int n, double eps, double* scale_sorted, unsigned* status,
                      cudaStream_t s) {
    if (n > 0) k_scale_eps<<<grid_for(n, 256), 256, 0, s>>>(eps_b, perm, n, eps, scale_sorted, status); note_launch();
}
}  // namespace gb3
