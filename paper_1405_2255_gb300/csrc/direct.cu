// direct.cu -- direct summation of eq. (1) (and f_b of eq. 6) on the GPU in FP64:
// the truth generator for large N and the "GPU FP64 direct summation" baseline.
#include "kernels.cuh"

namespace gb3 {

constexpr int kDirThreads = 128;

template <bool WANT_F>
__global__ void __launch_bounds__(kDirThreads) k_direct(const double* __restrict__ x, const double* __restrict__ mu,
                                                        int n, double G, const int64_t* __restrict__ sinks,
                                                        int nsinks, double* __restrict__ psi,
                                                        double* __restrict__ acc, double* __restrict__ f) {
    __shared__ d4 tile[kDirThreads];
    for (int b0 = blockIdx.x * kDirThreads; b0 < nsinks; b0 += gridDim.x * kDirThreads) {
        const int t = b0 + threadIdx.x;
        const bool active = t < nsinks;
        long long bi = active ? (sinks ? sinks[t] : t) : 0;
        const double bx = x[3 * bi], by = x[3 * bi + 1], bz = x[3 * bi + 2];
        double ps = 0, ax = 0, ay = 0, az = 0, fs = 0;
        for (int j0 = 0; j0 < n; j0 += kDirThreads) {
            __syncthreads();
            int j = j0 + threadIdx.x;
            if (j < n) tile[threadIdx.x] = mk4(x[3 * (long long)j], x[3 * (long long)j + 1], x[3 * (long long)j + 2], mu[j]);
            __syncthreads();
            int nt = min(kDirThreads, n - j0);
            if (active)
                for (int k = 0; k < nt; ++k) {
                    const d4 q = tile[k];
                    const double dx = q.x - bx, dy = q.y - by, dz = q.z - bz;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 > 0.0) {
                        const double rinv = rsqrt(r2);
                        const double qm = q.w * rinv;
                        const double q3 = qm * rinv * rinv;
                        ps += qm;
                        if (WANT_F) fs += q.w * rinv * rinv;
                        ax = fma(q3, dx, ax);
                        ay = fma(q3, dy, ay);
                        az = fma(q3, dz, az);
                    }
                }
        }
        if (active) {
            psi[t] = G * ps;
            acc[3 * (long long)t] = G * ax;
            acc[3 * (long long)t + 1] = G * ay;
            acc[3 * (long long)t + 2] = G * az;
            if (WANT_F) f[t] = G * fs;
        }
    }
}

void launch_direct(const double* x, const double* mu, int n, double G, const int64_t* sinks, int nsinks,
                   double* psi, double* acc, double* f, cudaStream_t s) {
    if (nsinks <= 0) return;
    unsigned g = grid_for(nsinks, kDirThreads, 32);
    if (f) k_direct<true><<<g, kDirThreads, 0, s>>>(x, mu, n, G, sinks, nsinks, psi, acc, f);
    else k_direct<false><<<g, kDirThreads, 0, s>>>(x, mu, n, G, sinks, nsinks, psi, acc, f);
    note_launch();
}

}  // namespace gb3
