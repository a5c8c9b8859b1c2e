// tidal.cu -- the tidal tensor T = grad grad Psi (Sec. 7.4) as an optional output of an
// evaluation: the far part from the local expansion's Psi_2^m at each particle (eq. 7
// taken to n = 2), the near part as the direct Hessian over the P2P lists (the same
// sources as the particle's P2P), combined, multiplied by G and scattered like Psi and a.
// Reading: T_xy = +Im Psi_2^2 / 2 (with the harmonics of App. A.3, Psi_2^2 = (d_x + i d_y)^2
// Psi); the other entries as printed in Sec. 7.4.  T is stored as (xx, xy, xz, yy, yz, zz).
#include "harmonics.cuh"
#include "kernels.cuh"

namespace gb3 {

// far part: one block per leaf, F in shared memory (complex), one thread per particle
// streaming the columns of Upsilon(s - x) by their recurrences
constexpr int kTidThreads = 64;
__global__ void __launch_bounds__(kTidThreads) k_l2p_tidal(const d4* __restrict__ xm, Cells c,
                                                           const d4* __restrict__ cen,
                                                           const int* __restrict__ leaves, int nleaves, int p,
                                                           const double* __restrict__ F, double* __restrict__ T) {
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
            cd p20 = mkc(0.0, 0.0), p21 = p20, p22 = p20;
            cd d = mkc(1.0, 0.0);
            for (int l = 0; l <= p - 2; ++l) {
                if (l > 0) {
                    const double sc = 1.0 / (2.0 * l);
                    d = cd{sc * (x * d.re - y * d.im), sc * (x * d.im + y * d.re)};
                }
                const double sg = (l & 1) ? -1.0 : 1.0;
                cd prev2 = mkc(0.0, 0.0), prev = d;
                for (int k = l; k <= p - 2; ++k) {
                    cd Y;
                    if (k == l) Y = d;
                    else {
                        const double inv = 1.0 / (double)(k * k - l * l);
                        const double a = (2.0 * k - 1.0) * z;
                        Y = cd{(a * prev.re - r2 * prev2.re) * inv, (a * prev.im - r2 * prev2.im) * inv};
                        prev2 = prev;
                        prev = Y;
                    }
                    const cd Xp = conjc(Y);                 // conj(Upsilon_k^l)
                    const cd Xn = cd{sg * Y.re, sg * Y.im};  // conj(Upsilon_k^{-l}) = (-1)^l Upsilon_k^l
                    const cd* Fk = Fc + (k + 2) * (k + 2) + (k + 2);  // F_{k+2}^{.}
                    cmac(p20, Xp, Fk[l]);
                    cmac(p21, Xp, Fk[1 + l]);
                    cmac(p22, Xp, Fk[2 + l]);
                    if (l > 0) {
                        cmac(p20, Xn, Fk[-l]);
                        cmac(p21, Xn, Fk[1 - l]);
                        cmac(p22, Xn, Fk[2 - l]);
                    }
                }
            }
            double* o = T + 6 * (size_t)(first + j);
            o[0] = -0.5 * p20.re + 0.5 * p22.re;
            o[1] = 0.5 * p22.im;
            o[2] = p21.re;
            o[3] = -0.5 * p20.re - 0.5 * p22.re;
            o[4] = p21.im;
            o[5] = p20.re;
        }
    }
}

void launch_l2p_tidal(const d4* xm, Cells c, const d4* cen, const int* leaves, int nleaves, int p, const double* F,
                      double* T, cudaStream_t s) {
    if (nleaves <= 0) return;  // (p < 2: the loops are empty and T_far = 0)
    const size_t sm = sizeof(cd) * (size_t)ncoef(p);
    const unsigned g = (unsigned)std::min<long long>(nleaves, (long long)sm_count() * 16);
    k_l2p_tidal<<<g, kTidThreads, sm, s>>>(xm, c, cen, leaves, nleaves, p, F, T);
    note_launch();
}

// near part: one warp per sink leaf, lane = sink (chunks of 32), the sources of the leaf's
// own P2P segment and of its ancestors' segments through shared-memory tiles of 32.
// FP32 = true: dx from the two-float position records (hi + lo), FP32 pair terms, two-float sums
// folded per tile; false: FP64 throughout.
constexpr int kTidWarps = 4;
template <bool FP32>
__global__ void __launch_bounds__(kTidWarps * 32) k_p2p_tidal(const d4* __restrict__ xm, const float4* __restrict__ xp,
                                                              int n, Cells c,
                                                              const int2* __restrict__ list,
                                                              const int* __restrict__ seg_start,
                                                              const int* __restrict__ seg_end,
                                                              const int* __restrict__ leaves, int nleaves,
                                                              double* __restrict__ T) {
    __shared__ d4 tile64[kTidWarps][32];
    __shared__ float tile32[kTidWarps][7][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int t = blockIdx.x * kTidWarps + wid; t < nleaves; t += gridDim.x * kTidWarps) {
        const int leaf = leaves[t];
        if (!cell_active(c, leaf)) continue;
        const int first = c.first[leaf], count = c.count[leaf];
        for (int s0 = 0; s0 < count; s0 += 32) {
            const int i = first + s0 + lane;
            const bool act = s0 + lane < count;
            d4 xb = mk4(0, 0, 0, 0);
            float bh[3] = {0.f, 0.f, 0.f}, bl[3] = {0.f, 0.f, 0.f};
            if (act) {
                if (FP32) {
                    const float4 h = xp[2 * (size_t)i], l = xp[2 * (size_t)i + 1];
                    bh[0] = h.x;
                    bh[1] = h.y;
                    bh[2] = h.z;
                    bl[0] = l.x;
                    bl[1] = l.y;
                    bl[2] = l.z;
                } else {
                    xb = xm[i];
                }
            }
            double S64[6] = {0, 0, 0, 0, 0, 0};
            ff S32[6];
            for (int k = 0; k < 6; ++k) S32[k] = ff{0.f, 0.f};
            for (int cell = leaf; cell >= 0; cell = c.parent[cell]) {
                for (int e = seg_start[cell]; e < seg_end[cell]; ++e) {
                    const int A = list[e].x;
                    const int af = c.first[A], an = c.count[A];
                    for (int j0 = 0; j0 < an; j0 += 32) {
                        const int nt = min(32, an - j0);
                        __syncwarp();
                        if (lane < nt) {
                            const int j = af + j0 + lane;
                            if (FP32) {
                                const float4 h = xp[2 * (size_t)j], l = xp[2 * (size_t)j + 1];
                                tile32[wid][0][lane] = h.x;
                                tile32[wid][1][lane] = h.y;
                                tile32[wid][2][lane] = h.z;
                                tile32[wid][3][lane] = h.w;
                                tile32[wid][4][lane] = l.x;
                                tile32[wid][5][lane] = l.y;
                                tile32[wid][6][lane] = l.z;
                            } else {
                                tile64[wid][lane] = xm[j];
                            }
                        }
                        __syncwarp();
                        if (FP32) {
                            float P[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                            for (int jj = 0; jj < nt; ++jj) {
                                const float dx = (bh[0] - tile32[wid][0][jj]) + (bl[0] - tile32[wid][4][jj]);
                                const float dy = (bh[1] - tile32[wid][1][jj]) + (bl[1] - tile32[wid][5][jj]);
                                const float dz = (bh[2] - tile32[wid][2][jj]) + (bl[2] - tile32[wid][6][jj]);
                                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                                if (r2 > 0.f) {
                                    const float ri = rsqrtf(r2), ri2 = ri * ri;
                                    const float q5 = tile32[wid][3][jj] * ri * ri2 * ri2;
                                    const float q3 = 3.f * q5;
                                    const float qr = q5 * r2;
                                    P[0] = fmaf(q3 * dx, dx, P[0] - qr);
                                    P[1] = fmaf(q3 * dx, dy, P[1]);
                                    P[2] = fmaf(q3 * dx, dz, P[2]);
                                    P[3] = fmaf(q3 * dy, dy, P[3] - qr);
                                    P[4] = fmaf(q3 * dy, dz, P[4]);
                                    P[5] = fmaf(q3 * dz, dz, P[5] - qr);
                                }
                            }
                            for (int k = 0; k < 6; ++k) ff_acc(S32[k], P[k]);
                        } else {
                            for (int jj = 0; jj < nt; ++jj) {
                                const d4 q = tile64[wid][jj];
                                const double dx = xb.x - q.x, dy = xb.y - q.y, dz = xb.z - q.z;
                                const double r2 = dx * dx + dy * dy + dz * dz;
                                if (r2 > 0.0) {
                                    const double ri = rsqrt(r2), ri2 = ri * ri;
                                    const double q5 = q.w * ri * ri2 * ri2;
                                    const double q3 = 3.0 * q5, qr = q5 * r2;
                                    S64[0] += q3 * dx * dx - qr;
                                    S64[1] += q3 * dx * dy;
                                    S64[2] += q3 * dx * dz;
                                    S64[3] += q3 * dy * dy - qr;
                                    S64[4] += q3 * dy * dz;
                                    S64[5] += q3 * dz * dz - qr;
                                }
                            }
                        }
                    }
                }
            }
            if (act) {
                double* o = T + 6 * (size_t)i;
                for (int k = 0; k < 6; ++k) o[k] = FP32 ? (double)S32[k].hi + (double)S32[k].lo : S64[k];
            }
        }
    }
}

void launch_p2p_tidal(const d4* xm, const float4* xp, int n, bool fp32, Cells c, const int2* list,
                      const int* seg_start, const int* seg_end, const int* leaves, int nleaves, double* T,
                      cudaStream_t s) {
    if (nleaves <= 0) return;
    long long g = ((long long)nleaves + kTidWarps - 1) / kTidWarps;
    if (g > (long long)sm_count() * 32) g = (long long)sm_count() * 32;
    if (fp32) k_p2p_tidal<true><<<(unsigned)g, kTidWarps * 32, 0, s>>>(xm, xp, n, c, list, seg_start, seg_end,
                                                                      leaves, nleaves, T);
    else k_p2p_tidal<false><<<(unsigned)g, kTidWarps * 32, 0, s>>>(xm, xp, n, c, list, seg_start, seg_end, leaves,
                                                                   nleaves, T);
    note_launch();
}

// T_caller = G (far + near), active particles only
__global__ void k_finish_tidal(const double* __restrict__ Tf, const double* __restrict__ Tn,
                               const int* __restrict__ perm, int n, double G, const unsigned char* __restrict__ pact,
                               double* __restrict__ T, const int* __restrict__ e) {
    const int kt = e ? e[1] - 3 * e[0] : 0;  // the tidal tensor ~ mu / x^3 in the working units
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (pact && !pact[i]) continue;
        const int o = perm[i];
        for (int k = 0; k < 6; ++k)
            T[6 * (size_t)o + k] = ldexp(G * (Tf[6 * (size_t)i + k] + Tn[6 * (size_t)i + k]), kt);
    }
}
void launch_finish_tidal(const double* Tf, const double* Tn, const int* perm, int n, double G,
                         const unsigned char* pact, double* T, cudaStream_t s, const int* e) {
    if (n > 0) k_finish_tidal<<<grid_for(n, 256), 256, 0, s>>>(Tf, Tn, perm, n, G, pact, T, e); note_launch();
}

}  // namespace gb3
