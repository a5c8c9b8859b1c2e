// split.cu -- mixed-mode P2M (eq. 3c) and L2P (eqs. 3a, 7) with the same order
// split as the M2L: the expansion orders n <= 2 are formed in FP64, the higher
// orders in FP32 on quantities scaled by the cell radius (Upsilon evaluated at
// (x - z)/rho, whose values are bounded by 1/n!), then rescaled in FP64.  The
// higher orders carry a fraction ~ theta^n of an expansion's contribution, so
// FP32 rounding there stays far below the targeted force error.
#include "harmonics.cuh"
#include "kernels.cuh"

namespace gb3 {

static __constant__ float c_inv_upf[kMaxP + 1][kMaxP + 1];  // 1 / (n^2 - m^2)
static __constant__ float c_twf2[kMaxP + 2];                // 2n - 1
static __constant__ float c_inv2jf[kMaxP + 1];              // 1 / (2j)

static void init_split_up_tables() {
    static DeviceOnce once;
    once_per_device(once, [] {
        float a[kMaxP + 1][kMaxP + 1], b[kMaxP + 2], c[kMaxP + 1];
        for (int n = 0; n <= kMaxP; ++n)
            for (int m = 0; m <= kMaxP; ++m) a[n][m] = (n * n != m * m) ? 1.0f / (float)(n * n - m * m) : 0.f;
        for (int n = 0; n <= kMaxP + 1; ++n) b[n] = (float)(2 * n - 1);
        c[0] = 0.f;
        for (int j = 1; j <= kMaxP; ++j) c[j] = 1.0f / (2.0f * j);
        cudaMemcpyToSymbol(c_inv_upf, a, sizeof a);
        cudaMemcpyToSymbol(c_twf2, b, sizeof b);
        cudaMemcpyToSymbol(c_inv2jf, c, sizeof c);
    });
}

__device__ inline float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// the nine real-storage coefficients of Upsilon_n^m(d), n <= 2 (App. A.3.1 in closed form):
// U0 = 1, U1^0 = z, U1^1 = (x+iy)/2, U2^0 = (3z^2-r^2)/4, U2^1 = z(x+iy)/2, U2^2 = (x+iy)^2/8
__device__ inline void upsilon_low(double x, double y, double z, double u[9]) {
    const double r2 = x * x + y * y + z * z;
    u[cix(0, 0)] = 1.0;
    u[cix(1, -1)] = 0.5 * y;
    u[cix(1, 0)] = z;
    u[cix(1, 1)] = 0.5 * x;
    u[cix(2, -2)] = 0.25 * x * y;
    u[cix(2, -1)] = 0.5 * z * y;
    u[cix(2, 0)] = 0.25 * (3.0 * z * z - r2);
    u[cix(2, 1)] = 0.5 * z * x;
    u[cix(2, 2)] = 0.125 * (x * x - y * y);
}

// ---------------------------------------------------------------- P2M
constexpr int kSplitWarps = 4;

__global__ void __launch_bounds__(kSplitWarps * 32) k_p2m_split(const d4* __restrict__ xm, Cells c,
                                                                const d4* __restrict__ cen,
                                                                const int* __restrict__ leaves, int nleaves, int p,
                                                                double* __restrict__ M) {
    extern __shared__ float fsm[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nco = ncoef(p);
    float* acc = fsm + (size_t)wid * nco;
    const int t = blockIdx.x * kSplitWarps + wid;
    if (t >= nleaves) return;
    const int cell = leaves[t];
    for (int i = lane; i < nco; i += 32) acc[i] = 0.f;
    __syncwarp();
    const d4 z = cen[cell];
    const double rho = z.w, rinv = rho > 0 ? 1.0 / rho : 0.0;
    const int first = c.first[cell], count = c.count[cell];
    double lo[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) lo[i] = 0.0;
    for (int b = 0; b < count; b += 32) {
        const int i = b + lane;
        double dx = 0, dy = 0, dz = 0, mu = 0;
        if (i < count) {
            const d4 q = xm[first + i];
            dx = q.x - z.x; dy = q.y - z.y; dz = q.z - z.z; mu = q.w;
        }
        double u[9];
        upsilon_low(dx, dy, dz, u);
#pragma unroll
        for (int k = 0; k < 9; ++k) lo[k] = fma(mu, u[k], lo[k]);
        if (rho > 0 && p > 2) {
            // mu * Upsilon_n^m((x - z)/rho) in FP32, n >= 3 kept
            const float x = (float)(dx * rinv), y = (float)(dy * rinv), zz = (float)(dz * rinv), w = (float)mu;
            const float r2 = x * x + y * y + zz * zz;
            float2 d = make_float2(w, 0.f);
            for (int m = 0; m <= p; ++m) {
                if (m > 0) {
                    const float s = c_inv2jf[m];
                    d = make_float2(s * (x * d.x - y * d.y), s * (x * d.y + y * d.x));
                }
                float2 prev2 = make_float2(0.f, 0.f), prev = d;
                for (int n = m; n <= p; ++n) {
                    float2 v;
                    if (n == m) v = d;
                    else {
                        const float a = c_twf2[n] * zz, iv = c_inv_upf[n][m];
                        v = make_float2((a * prev.x - r2 * prev2.x) * iv, (a * prev.y - r2 * prev2.y) * iv);
                        prev2 = prev;
                        prev = v;
                    }
                    if (n >= 3) {
                        const float sr = warp_sumf(v.x), si = warp_sumf(v.y);
                        if (lane == 0) {
                            acc[cix(n, m)] += sr;
                            if (m) acc[cix(n, -m)] += si;
                        }
                    }
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) lo[k] = warp_sum(lo[k]);
    __syncwarp();
    double* out = M + (size_t)cell * nco;
    __shared__ double pw_all[kSplitWarps][kMaxP + 1];
    double* pw = pw_all[wid];
    warp_pow_table(rho, p, lane, pw);
    __syncwarp();
    if (lane == 0)
        for (int k = 0; k < 9 && k < nco; ++k) out[k] = lo[k];
    for (int i = 9 + lane; i < nco; i += 32) {
        int n = (int)sqrtf((float)i);
        while (n * n > i) --n;
        while ((n + 1) * (n + 1) <= i) ++n;
        out[i] = (double)acc[i] * pw[n];
    }
}

void launch_p2m_split(const d4* xm, Cells c, const d4* cen, const int* leaves, int nleaves, int p, double* M,
                      cudaStream_t s) {
    if (nleaves <= 0) return;
    if (p < 2) {
        launch_p2m(xm, c, cen, leaves, nleaves, p, M, s);
        return;
    }
    init_split_up_tables();
    size_t sm = (size_t)kSplitWarps * ncoef(p) * sizeof(float);
    k_p2m_split<<<(nleaves + kSplitWarps - 1) / kSplitWarps, kSplitWarps * 32, sm, s>>>(xm, c, cen, leaves, nleaves,
                                                                                          p, M);
    note_launch();
}

// ---------------------------------------------------------------- L2P
// Psi_0^0 = sum_{k,l} Upsilon_k^{l*} F_k^l and Psi_1^m = sum_{k,l} Upsilon_k^{l*} F_{k+1}^{m+l}
// (Upsilon at s_B - x_b): terms with k <= 2 in FP64; terms with k >= 3 in FP32 as
// Uhat_k^{l*} Fhat_k^l and Uhat_k^{l*} Fhat_{k+1}^{m+l} / rho with Uhat_k = Upsilon_k((s - x)/rho),
// Fhat_n = F_n rho^n.  One warp per leaf, lane = particle.
__global__ void __launch_bounds__(kSplitWarps * 32) k_l2p_split(const d4* __restrict__ xm, Cells c,
                                                                const d4* __restrict__ cen,
                                                                const int* __restrict__ leaves, int nleaves, int p,
                                                                const double* __restrict__ F, double* __restrict__ psi,
                                                                double* __restrict__ acc) {
    extern __shared__ unsigned char sraw[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nco = ncoef(p);
    const size_t per_warp = ((size_t)nco * sizeof(float2) + 16 * sizeof(cd) + 15) & ~(size_t)15;
    float2* Fh = (float2*)(sraw + wid * per_warp);  // [nco] F_n rho^n
    cd* F64 = (cd*)(Fh + nco);                      // [16] F_n, n <= 3
    const int t = blockIdx.x * kSplitWarps + wid;
    if (t >= nleaves) return;
    const int cell = leaves[t];
    if (!cell_active(c, cell)) return;
    const d4 s = cen[cell];
    const double rho = s.w;
    const double* Fr = F + (size_t)cell * nco;
    __shared__ double pw_all[kSplitWarps][kMaxP + 1];
    double* pw = pw_all[wid];
    warp_pow_table(rho, p, lane, pw);
    __syncwarp();
    for (int i = lane; i < nco; i += 32) {
        int n = (int)sqrtf((float)i);
        while (n * n > i) --n;
        while ((n + 1) * (n + 1) <= i) ++n;
        const cd v = load_real_storage(Fr, n, i - n * n - n);
        const double sc = pw[n];
        Fh[i] = make_float2((float)(v.re * sc), (float)(v.im * sc));
        if (i < 16) F64[i] = v;
    }
    __syncwarp();
    const double rinv = rho > 0 ? 1.0 / rho : 0.0;
    const int first = c.first[cell], count = c.count[cell];
    for (int j = lane; j < count; j += 32) {
        const d4 xb = xm[first + j];
        const double vx = s.x - xb.x, vy = s.y - xb.y, vz = s.z - xb.z;
        // k <= 2 in FP64
        double u[9];
        upsilon_low(vx, vy, vz, u);
        double p00 = 0;
        cd p10 = mkc(0, 0), p11 = mkc(0, 0);
        for (int k = 0; k <= 2 && k <= p; ++k) {
            for (int l = 0; l <= k; ++l) {
                const cd Y = mkc(u[cix(k, l)], l ? u[cix(k, -l)] : 0.0);  // Upsilon_k^l
                const cd Xp = conjc(Y);
                const double sg = (l & 1) ? -1.0 : 1.0;
                const cd Xn = mkc(sg * Y.re, sg * Y.im);                 // conj(Upsilon_k^{-l})
                const cd* Fk = F64 + k * k + k;
                if (l == 0) p00 += Xp.re * Fk[0].re - Xp.im * Fk[0].im;
                else p00 += 2.0 * (Xp.re * Fk[l].re - Xp.im * Fk[l].im);
                if (k + 1 <= p) {
                    const cd* Fk1 = F64 + (k + 1) * (k + 1) + (k + 1);
                    cmac(p10, Xp, Fk1[l]);
                    cmac(p11, Xp, Fk1[1 + l]);
                    if (l > 0) {
                        cmac(p10, Xn, Fk1[-l]);
                        cmac(p11, Xn, Fk1[1 - l]);
                    }
                }
            }
        }
        // k >= 3 in FP32 on the scaled offset
        float h00 = 0.f;
        float2 h10 = make_float2(0.f, 0.f), h11 = make_float2(0.f, 0.f);
        if (rho > 0 && p >= 3) {
            const float x = (float)(vx * rinv), y = (float)(vy * rinv), z = (float)(vz * rinv);
            const float r2 = x * x + y * y + z * z;
            float2 d = make_float2(1.f, 0.f);
            for (int l = 0; l <= p; ++l) {
                if (l > 0) {
                    const float sc = c_inv2jf[l];
                    d = make_float2(sc * (x * d.x - y * d.y), sc * (x * d.y + y * d.x));
                }
                const float sg = (l & 1) ? -1.f : 1.f;
                float2 prev2 = make_float2(0.f, 0.f), prev = d;
                for (int k = l; k <= p; ++k) {
                    float2 Y;
                    if (k == l) Y = d;
                    else {
                        const float a = c_twf2[k] * z, iv = c_inv_upf[k][l];
                        Y = make_float2((a * prev.x - r2 * prev2.x) * iv, (a * prev.y - r2 * prev2.y) * iv);
                        prev2 = prev;
                        prev = Y;
                    }
                    if (k < 3) continue;
                    const float2 Xp = make_float2(Y.x, -Y.y);
                    const float2 Xn = make_float2(sg * Y.x, sg * Y.y);
                    const float2* Fk = Fh + k * k + k;
                    if (l == 0) h00 += Xp.x * Fk[0].x - Xp.y * Fk[0].y;
                    else h00 += 2.f * (Xp.x * Fk[l].x - Xp.y * Fk[l].y);
                    if (k < p) {
                        const float2* Fk1 = Fh + (k + 1) * (k + 1) + (k + 1);
                        cmacf(h10, Xp, Fk1[l]);
                        cmacf(h11, Xp, Fk1[1 + l]);
                        if (l > 0) {
                            cmacf(h10, Xn, Fk1[-l]);
                            cmacf(h11, Xn, Fk1[1 - l]);
                        }
                    }
                }
            }
        }
        const int i = first + j;
        psi[i] = p00 + (double)h00;
        acc[3 * (size_t)i] = -(p11.re + (double)h11.x * rinv);
        acc[3 * (size_t)i + 1] = -(p11.im + (double)h11.y * rinv);
        acc[3 * (size_t)i + 2] = -(p10.re + (double)h10.x * rinv);
    }
}

void launch_l2p_split(const d4* xm, Cells c, const d4* cen, const int* leaves, int nleaves, int p, const double* F,
                      double* psi, double* acc, cudaStream_t s) {
    if (nleaves <= 0) return;
    if (p < 3) {
        launch_l2p(xm, c, cen, leaves, nleaves, p, F, psi, acc, s);
        return;
    }
    init_split_up_tables();
    const size_t per_warp = ((size_t)ncoef(p) * sizeof(float2) + 16 * sizeof(cd) + 15) & ~(size_t)15;
    k_l2p_split<<<(nleaves + kSplitWarps - 1) / kSplitWarps, kSplitWarps * 32, kSplitWarps * per_warp, s>>>(
        xm, c, cen, leaves, nleaves, p, F, psi, acc);
    note_launch();
}

// full complex Upsilon_k^l(v), k <= 2, from the closed forms (conj_out: conjugates)
__device__ inline void upsilon_low_full(double x, double y, double z, cd out[9], bool conj_out) {
    double u[9];
    upsilon_low(x, y, z, u);
    for (int k = 0; k <= 2; ++k)
        for (int l = 0; l <= k; ++l) {
            cd v = mkc(u[cix(k, l)], l ? u[cix(k, -l)] : 0.0);
            if (conj_out) v = conjc(v);
            out[cix(k, l)] = v;
            if (l) {
                const double sg = (l & 1) ? -1.0 : 1.0;
                // X^{-l} = (-1)^l conj(X^l) for both Upsilon and its conjugate
                out[cix(k, -l)] = mkc(sg * v.re, -sg * v.im);
            }
        }
}

// FP32 column m of Upsilon at a scaled offset (|v| <= 1), optionally conjugated
__device__ inline void upsilon_column_f(int p, int m, float x, float y, float z, float2* out, bool conj_out) {
    const float r2 = x * x + y * y + z * z;
    float2 d = make_float2(1.f, 0.f);
    for (int j = 1; j <= m; ++j) {
        const float s = c_inv2jf[j];
        d = make_float2(s * (x * d.x - y * d.y), s * (x * d.y + y * d.x));
    }
    float2 prev2 = make_float2(0.f, 0.f), prev = d;
    const float sg = (m & 1) ? -1.f : 1.f;
    for (int n = m; n <= p; ++n) {
        float2 v;
        if (n == m) v = d;
        else {
            const float a = c_twf2[n] * z, iv = c_inv_upf[n][m];
            v = make_float2((a * prev.x - r2 * prev2.x) * iv, (a * prev.y - r2 * prev2.y) * iv);
            prev2 = prev;
            prev = v;
        }
        if (conj_out) v.y = -v.y;
        out[cix(n, m)] = v;
        if (m) out[cix(n, -m)] = make_float2(sg * v.x, -sg * v.y);
    }
}

__device__ inline int n_of(int i) {
    int n = (int)sqrtf((float)i);
    while (n * n > i) --n;
    while ((n + 1) * (n + 1) <= i) ++n;
    return n;
}

// ---------------------------------------------------------------- M2M
// M_n^m(z') = sum_{k<=n} sum_l Upsilon_k^l(z - z') M_{n-k}^{m-l}(z): outputs n <= 2 in FP64,
// outputs n >= 3 in FP32 as Mhat_n = M_n / rho'^n = sum Uhat_k Mt_{n-k} with
// Uhat_k = Upsilon_k((z - z')/rho'), Mt_j = M_j(z) / rho'^j.  One block per parent and one
// warp per daughter; the daughters' contributions are then summed in daughter order.
constexpr int kM2MWarps = 8;
__host__ __device__ inline size_t m2m_warp_bytes(int p) {
    return ((size_t)2 * ncoef(p) * sizeof(float2) + 18 * sizeof(cd) + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t m2m_smem_bytes(int p) {
    const size_t nout = (size_t)(p + 1) * (p + 2) / 2;
    return kM2MWarps * m2m_warp_bytes(p) + kM2MWarps * nout * sizeof(float2) + kM2MWarps * 6 * sizeof(cd);
}
template <int MAXQ>
__global__ void __launch_bounds__(kM2MWarps * 32) k_m2m_split(Cells c, const d4* __restrict__ cen, int lev_begin,
                                                               int lev_end, int p, double* __restrict__ M,
                                                               LaneSched sched) {
    extern __shared__ __align__(16) unsigned char sraw[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nco = ncoef(p), nout = (p + 1) * (p + 2) / 2;
    const size_t per_warp = m2m_warp_bytes(p);
    float2* Yh = (float2*)(sraw + wid * per_warp);
    float2* Mt = Yh + nco;
    cd* Y64 = (cd*)(Mt + nco);
    cd* M64 = Y64 + 9;
    float2* r32 = (float2*)(sraw + kM2MWarps * per_warp);  // [kM2MWarps][nout]
    cd* r64 = (cd*)(r32 + kM2MWarps * nout);                // [kM2MWarps][6]
    __shared__ double pwi[kMaxP + 1], pwr[kMaxP + 1];        // rho^-n, rho^n
    const int cell = lev_begin + blockIdx.x;
    if (cell >= lev_end) return;
    const int nch = c.nchild[cell];
    if (nch == 0) return;  // leaves
    const d4 zp = cen[cell];
    const double rho = zp.w, inv = rho > 0 ? 1.0 / rho : 0.0;
    if (wid == 0) warp_pow_table(inv, p, lane, pwi);
    if (wid == 1) warp_pow_table(rho, p, lane, pwr);
    __syncthreads();
    if (wid < nch) {
        const int cnt = sched.cnt[lane];
        const int d = c.child[cell] + wid;
        const d4 z = cen[d];
        const double vx = z.x - zp.x, vy = z.y - zp.y, vz = z.z - zp.z;
        if (lane <= p) upsilon_column_f(p, lane, (float)(vx * inv), (float)(vy * inv), (float)(vz * inv), Yh, false);
        const double* Md = M + (size_t)d * nco;
        for (int i = lane; i < nco; i += 32) {
            const int n = n_of(i);
            const cd v = load_real_storage(Md, n, i - n * n - n);
            const double sc = pwi[n];
            Mt[i] = make_float2((float)(v.re * sc), (float)(v.im * sc));
            if (i < 9) M64[i] = v;
        }
        if (lane == 0) upsilon_low_full(vx, vy, vz, Y64, false);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < MAXQ; ++q) {
            if (q < cnt) {
                const int n = sched.n[lane][q], m = sched.m[lane][q];
                const int o = n * (n + 1) / 2 + m;
                if (n <= 2) {
                    cd sum = mkc(0.0, 0.0);
                    for (int k = 0; k <= n; ++k) {
                        const int nn = n - k;
                        for (int l = max(-k, m - nn); l <= min(k, m + nn); ++l)
                            cmac(sum, Y64[cix(k, l)], M64[cix(nn, m - l)]);
                    }
                    r64[wid * 6 + o] = sum;
                } else {
                    float2 sum = make_float2(0.f, 0.f);
                    if (rho > 0)
                        for (int k = 0; k <= n; ++k) {
                            const int nn = n - k;
                            for (int l = max(-k, m - nn); l <= min(k, m + nn); ++l)
                                cmacf(sum, Yh[cix(k, l)], Mt[cix(nn, m - l)]);
                        }
                    r32[wid * nout + o] = sum;
                }
            }
        }
    }
    __syncthreads();
    // the parent's moments: the daughters' terms summed in daughter order
    double* out = M + (size_t)cell * nco;
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= o) ++n;
        const int m = o - n * (n + 1) / 2;
        cd v;
        if (n <= 2) {
            v = mkc(0.0, 0.0);
            for (int j = 0; j < nch; ++j) v = v + r64[j * 6 + o];
        } else {
            float2 a = make_float2(0.f, 0.f);
            for (int j = 0; j < nch; ++j) {
                a.x += r32[j * nout + o].x;
                a.y += r32[j * nout + o].y;
            }
            const double sc = pwr[n];
            v = mkc((double)a.x * sc, (double)a.y * sc);
        }
        out[cix(n, m)] = v.re;
        if (m) out[cix(n, -m)] = v.im;
    }
}

void launch_m2m_split(Cells c, const d4* cen, int lev_begin, int lev_end, int p, double* M, cudaStream_t s) {
    const int ncl = lev_end - lev_begin;
    if (ncl <= 0) return;
    if (p < 3) {
        launch_m2m_level(c, cen, lev_begin, lev_end, p, M, s);
        return;
    }
    init_split_up_tables();
    LaneSched sched = make_lane_sched(p, kSchedUp);
    int maxq = 0;
    for (int l = 0; l < 32; ++l) maxq = sched.cnt[l] > maxq ? sched.cnt[l] : maxq;
    const size_t sm = m2m_smem_bytes(p);
    const unsigned g = (unsigned)ncl;  // one block per cell of the level (leaves return at once)
    if (maxq <= 4) {
        cudaFuncSetAttribute(k_m2m_split<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_m2m_split<4><<<g, kM2MWarps * 32, sm, s>>>(c, cen, lev_begin, lev_end, p, M, sched);
    } else if (maxq <= 8) {
        cudaFuncSetAttribute(k_m2m_split<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_m2m_split<8><<<g, kM2MWarps * 32, sm, s>>>(c, cen, lev_begin, lev_end, p, M, sched);
    } else {
        cudaFuncSetAttribute(k_m2m_split<24>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_m2m_split<24><<<g, kM2MWarps * 32, sm, s>>>(c, cen, lev_begin, lev_end, p, M, sched);
    }
    note_launch();
}

// ---------------------------------------------------------------- L2L
// F_n^m(s') += sum_{k<=p-n} sum_l Upsilon_k^{l*}(s - s') F_{n+k}^{m+l}(s): terms with n+k <= 2
// in FP64, the others in FP32 as rho^-n sum Uhat_k^{l*} Fhat_{n+k}^{m+l} with
// Uhat_k = Upsilon_k((s - s')/rho), Fhat_j = F_j(s) rho^j (rho: the parent's radius).
template <int MAXQ>
__global__ void __launch_bounds__(128) k_l2l_split(Cells c, const d4* __restrict__ cen, int lev_begin, int lev_end,
                                                   int p, double* __restrict__ F, LaneSched sched) {
    extern __shared__ unsigned char sraw[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nco = ncoef(p);
    const size_t per_warp = ((size_t)2 * nco * sizeof(float2) + 18 * sizeof(cd) + 15) & ~(size_t)15;
    float2* Yh = (float2*)(sraw + wid * per_warp);
    float2* Fh = Yh + nco;
    cd* Y64 = (cd*)(Fh + nco);
    cd* F64 = Y64 + 9;
    const int cell = lev_begin + blockIdx.x * 4 + wid;
    if (cell >= lev_end || !cell_active(c, cell)) return;
    const int par = c.parent[cell];
    const d4 s = cen[par], sp = cen[cell];
    const double rho = s.w;
    double* out = F + (size_t)cell * nco;
    const double* Fp = F + (size_t)par * nco;
    if (!(rho > 0)) {  // all particles at the parent's centre: the shift is the identity
        for (int i = lane; i < nco; i += 32) out[i] += Fp[i];
        return;
    }
    const double inv = 1.0 / rho;
    __shared__ double pwi_all[4][kMaxP + 1], pwr_all[4][kMaxP + 1];
    double *pwi = pwi_all[wid], *pwr = pwr_all[wid];  // rho^-n, rho^n
    warp_pow_table(inv, p, lane, pwi);
    warp_pow_table(rho, p, lane, pwr);
    __syncwarp();
    const double vx = s.x - sp.x, vy = s.y - sp.y, vz = s.z - sp.z;
    if (lane <= p) upsilon_column_f(p, lane, (float)(vx * inv), (float)(vy * inv), (float)(vz * inv), Yh, true);
    for (int i = lane; i < nco; i += 32) {
        const int n = n_of(i);
        const cd v = load_real_storage(Fp, n, i - n * n - n);
        const double sc = pwr[n];
        Fh[i] = make_float2((float)(v.re * sc), (float)(v.im * sc));
        if (i < 9) F64[i] = v;
    }
    if (lane == 0) upsilon_low_full(vx, vy, vz, Y64, true);
    __syncwarp();
    const int cnt = sched.cnt[lane];
    for (int q = 0; q < cnt; ++q) {
        const int n = sched.n[lane][q], m = sched.m[lane][q];
        cd v64 = mkc(0.0, 0.0);
        for (int k = 0; k + n <= 2 && k <= p - n; ++k)
            for (int l = -k; l <= k; ++l) cmac(v64, Y64[cix(k, l)], F64[cix(n + k, m + l)]);
        float2 v32 = make_float2(0.f, 0.f);
        for (int k = max(0, 3 - n); k <= p - n; ++k) {
            const float2* xk = Yh + k * k + k;
            const float2* yk = Fh + (n + k) * (n + k) + (n + k) + m;
            for (int l = -k; l <= k; ++l) cmacf(v32, xk[l], yk[l]);
        }
        const double sc = pwi[n];
        out[cix(n, m)] += v64.re + (double)v32.x * sc;
        if (m) out[cix(n, -m)] += v64.im + (double)v32.y * sc;
    }
}

void launch_l2l_split(Cells c, const d4* cen, int lev_begin, int lev_end, int p, double* F, cudaStream_t s) {
    const int ncl = lev_end - lev_begin;
    if (ncl <= 0) return;
    if (p < 3) {
        launch_l2l_level(c, cen, lev_begin, lev_end, p, F, s);
        return;
    }
    init_split_up_tables();
    LaneSched sched = make_lane_sched(p, kSchedDown);
    const size_t per_warp = ((size_t)2 * ncoef(p) * sizeof(float2) + 18 * sizeof(cd) + 15) & ~(size_t)15;
    k_l2l_split<4><<<(unsigned)((ncl + 3) / 4), 128, 4 * per_warp, s>>>(c, cen, lev_begin, lev_end, p, F, sched);
    note_launch();
}

}  // namespace gb3
