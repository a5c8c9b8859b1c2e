// harmonics.cuh -- device solid harmonics (eq. 2) and the shared contraction of
// the M2L, L2L and L2P kernels (eqs. 3a, 3b, 5, 7).
#pragma once
#include "common.cuh"

namespace gb3 {

// Recurrence coefficients as doubles (no integer-to-FP64 conversions in the loops):
// c_tw[n] = 2n - 1, c_inv_up[n][m] = 1 / (n^2 - m^2), c_th_b[n][m] = (n-1)^2 - m^2.
struct RecTables {
    double tw[kMaxP + 2];
    double inv_up[kMaxP + 1][kMaxP + 1];
    double th_b[kMaxP + 1][kMaxP + 1];
    double inv_2j[kMaxP + 1];  // 1 / (2j)
};
// one copy per translation unit (no relocatable device code); each unit that
// launches kernels using the recurrences calls init_rec_tables() first
static __constant__ RecTables c_rec;
static inline void init_rec_tables() {
    static DeviceOnce once;
    once_per_device(once, [] {
        RecTables t;
        memset(&t, 0, sizeof t);
        for (int n = 0; n <= kMaxP + 1; ++n) t.tw[n] = 2.0 * n - 1.0;
        for (int n = 0; n <= kMaxP; ++n)
            for (int m = 0; m <= kMaxP; ++m) {
                t.inv_up[n][m] = (n * n != m * m) ? 1.0 / (double)(n * n - m * m) : 0.0;
                t.th_b[n][m] = (double)((n - 1) * (n - 1) - m * m);
            }
        for (int j = 1; j <= kMaxP; ++j) t.inv_2j[j] = 1.0 / (2.0 * j);
        cudaMemcpyToSymbol(c_rec, &t, sizeof t);
    });
}

// One column m >= 0 of the regular harmonics Upsilon_n^m(r), n = m..p, written to
// the full complex array out[cix(n, +-m)] (negative m by X_n^{-m} = (-1)^m X_n^{m*}).
// Diagonal: Upsilon_m^m = prod_{j<=m} (x+iy)/(2j); then
// (n^2-m^2) Upsilon_n^m = (2n-1) z Upsilon_{n-1}^m - r^2 Upsilon_{n-2}^m (App. A.3.1).
// If conj_out, the conjugates are written instead.
__device__ inline void upsilon_column(int p, int m, double x, double y, double z, cd* out, bool conj_out) {
    const double r2 = x * x + y * y + z * z;
    cd d = mkc(1.0, 0.0);
    for (int j = 1; j <= m; ++j) {
        double s = c_rec.inv_2j[j];
        d = cd{s * (x * d.re - y * d.im), s * (x * d.im + y * d.re)};
    }
    cd prev2 = mkc(0.0, 0.0), prev = d;
    const double sg = (m & 1) ? -1.0 : 1.0;
    for (int n = m; n <= p; ++n) {
        cd v;
        if (n == m) v = d;
        else {
            double inv = c_rec.inv_up[n][m];
            double a = c_rec.tw[n] * z;
            v = cd{(a * prev.re - r2 * prev2.re) * inv, (a * prev.im - r2 * prev2.im) * inv};
            prev2 = prev;
            prev = v;
        }
        cd w = conj_out ? conjc(v) : v;
        out[cix(n, m)] = w;
        if (m) out[cix(n, -m)] = cd{sg * w.re, -sg * w.im};
    }
}

// One column m >= 0 of the irregular harmonics Theta_n^m(r), n = m..p:
// Theta_0^0 = 1/r, Theta_m^m = (2m-1)(x+iy)/r^2 Theta_{m-1}^{m-1},
// r^2 Theta_n^m = (2n-1) z Theta_{n-1}^m - ((n-1)^2 - m^2) Theta_{n-2}^m.
__device__ inline void theta_column(int p, int m, double x, double y, double z, cd* out) {
    const double r2 = x * x + y * y + z * z;
    const double ir2 = 1.0 / r2;
    cd d = mkc(sqrt(ir2), 0.0);
    for (int j = 1; j <= m; ++j) {
        double s = c_rec.tw[j] * ir2;
        d = cd{s * (x * d.re - y * d.im), s * (x * d.im + y * d.re)};
    }
    cd prev2 = mkc(0.0, 0.0), prev = d;
    const double sg = (m & 1) ? -1.0 : 1.0;
    for (int n = m; n <= p; ++n) {
        cd v;
        if (n == m) v = d;
        else {
            double a = c_rec.tw[n] * z;
            double b = c_rec.th_b[n][m];
            v = cd{(a * prev.re - b * prev2.re) * ir2, (a * prev.im - b * prev2.im) * ir2};
            prev2 = prev;
            prev = v;
        }
        out[cix(n, m)] = v;
        if (m) out[cix(n, -m)] = cd{sg * v.re, -sg * v.im};
    }
}

// complex FP32 multiply-accumulate: acc += a * b
__device__ inline void cmacf(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}

// expand a real-storage expansion into a full complex array (optionally conjugated)
__device__ inline void expand_real(int p, const double* R, cd* out, bool conj_out, int lane, int nlanes) {
    const int nc = ncoef(p);
    for (int i = lane; i < nc; i += nlanes) {
        int n = (int)sqrtf((float)i);
        while (n * n > i) --n;
        while ((n + 1) * (n + 1) <= i) ++n;
        int m = i - n * n - n;
        cd v = load_real_storage(R, n, m);
        out[i] = conj_out ? conjc(v) : v;
    }
}

// C_n^m = sum_{k=0}^{p-n} sum_{l=-k}^{k} X_k^l Y_{n+k}^{m+l}: the common form of
// M2L (X = M*, Y = Theta), L2L (X = Upsilon*, Y = F) and L2P (X = Upsilon*, Y = F).
__device__ inline cd contract(int p, int n, int m, const cd* __restrict__ X, const cd* __restrict__ Y) {
    cd acc = mkc(0.0, 0.0);
    for (int k = 0; k <= p - n; ++k) {
        const cd* xk = X + k * k + k;             // X_k^0
        const cd* yk = Y + (n + k) * (n + k) + (n + k) + m;  // Y_{n+k}^{m}
        for (int l = -k; l <= k; ++l) cmac(acc, xk[l], yk[l]);
    }
    return acc;
}

// Static balanced assignment of the outputs (n, m >= 0) of a contraction to the 32
// lanes of a warp, longest-processing-time first, on the cost of one output:
// (p-n+1)^2 terms for M2L/L2L (k <= p-n), (n+1)^2 for M2M (k <= n).
constexpr int kMaxPerLane = 24;
struct LaneSched {
    unsigned char n[32][kMaxPerLane];
    unsigned char m[32][kMaxPerLane];
    unsigned char cnt[32];
};
enum SchedKind { kSchedDown = 0, kSchedUp = 1 };
LaneSched make_lane_sched(int p, SchedKind kind);

}  // namespace gb3
