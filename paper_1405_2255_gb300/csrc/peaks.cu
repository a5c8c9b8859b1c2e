// peaks.cu -- ALU throughput probes (FP64 DFMA, FP32 FFMA) used as the roofline
// denominators of the FP64 expansion kernels and of the FP32 P2P kernel.
#include "kernels.cuh"

namespace gb3 {

template <int ITERS>
__global__ void k_peak_dfma(double* out, double a, double b) {
    double x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
           x7 = x0 + 7;
#pragma unroll 16
    for (int i = 0; i < ITERS; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <int ITERS>
__global__ void k_peak_ffma(float* out, float a, float b) {
    float x[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = threadIdx.x * 1e-3f + j;
#pragma unroll 8
    for (int i = 0; i < ITERS; ++i) {
#pragma unroll
        for (int j = 0; j < 16; ++j) x[j] = fmaf(x[j], a, b);
    }
    float s = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) s += x[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int alu_peaks(double* fp64_tflops, double* fp32_tflops) {
    int dev, nsm;
    GB3_CUDA_TRY(cudaGetDevice(&dev));
    GB3_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 256, blocks = nsm * 8;
    const size_t nt = (size_t)threads * blocks;
    double* dd = nullptr;
    GB3_CUDA_TRY(cudaMalloc(&dd, nt * sizeof(double)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0, best64 = 1e30f, best32 = 1e30f;
    const int ID = 2048, IF = 8192;
    for (int rep = 0; rep < 3; ++rep) {
        k_peak_dfma<ID><<<blocks, threads>>>(dd, 0.999999, 1e-7);
        cudaEventRecord(e0);
        k_peak_dfma<ID><<<blocks, threads>>>(dd, 0.999999, 1e-7);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        best64 = ms < best64 ? ms : best64;
        k_peak_ffma<IF><<<blocks, threads>>>((float*)dd, 0.999f, 1e-4f);
        cudaEventRecord(e0);
        k_peak_ffma<IF><<<blocks, threads>>>((float*)dd, 0.999f, 1e-4f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        best32 = ms < best32 ? ms : best32;
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dd);
    if (err != cudaSuccess) return cuda_fail(err, "peak probe", __FILE__, __LINE__);
    *fp64_tflops = 2.0 * 8 * ID * (double)nt / (best64 * 1e-3) / 1e12;
    *fp32_tflops = 2.0 * 16 * IF * (double)nt / (best32 * 1e-3) / 1e12;
    return 0;
}

// The pair arithmetic of the mixed P2P alone (its far form: dx from FP32 offsets, packed f32x2
// operations, rsqrt.approx.ftz), sources from a shared-memory table, one sink per lane, no tile
// staging, list walking or idle lanes: the rate the P2P kernel's arithmetic can reach on this
// device.  Gpairs/s over iters passes of 1024 sources per thread.
typedef unsigned long long pf2;
__device__ __forceinline__ pf2 pp_pack(float a, float b) {
    pf2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void pp_unpack(pf2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ pf2 pp_sub(pf2 a, pf2 b) {
    pf2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ pf2 pp_add(pf2 a, pf2 b) {
    pf2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ pf2 pp_mul(pf2 a, pf2 b) {
    pf2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ pf2 pp_fma(pf2 a, pf2 b, pf2 c) {
    pf2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// one far-form pair of eq. (1) for two packed sources against one sink
__device__ __forceinline__ void peak_pair2(pf2 X, pf2 Y, pf2 Z, pf2 W, pf2 hx, pf2 hy, pf2 hz, pf2& ps, pf2& ax,
                                           pf2& ay, pf2& az) {
    const pf2 dx = pp_sub(X, hx), dy = pp_sub(Y, hy), dz = pp_sub(Z, hz);
    const pf2 r2 = pp_fma(dx, dx, pp_fma(dy, dy, pp_mul(dz, dz)));
    float a, b;
    pp_unpack(r2, a, b);
    const pf2 ri = pp_pack(rsqrt_ftz(a), rsqrt_ftz(b));
    const pf2 qm = pp_mul(W, ri), q3 = pp_mul(qm, pp_mul(ri, ri));
    ps = pp_add(ps, qm);
    ax = pp_fma(q3, dx, ax);
    ay = pp_fma(q3, dy, ay);
    az = pp_fma(q3, dz, az);
}
// the P2P kernel's inner loop: groups of four sources from shared memory (structure of
// arrays), two sinks per lane, each source pair packed against both
__global__ void __launch_bounds__(128) k_peak_pairs(float* out, int iters) {
    __shared__ float4 src[4][128];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) {
        src[0][i] = make_float4(i * 1e-3f, 1 + i * 1e-3f, 2 + i * 1e-3f, 3 + i * 1e-3f);
        src[1][i] = src[0][i];
        src[2][i] = src[0][i];
        src[3][i] = make_float4(1e-6f, 1e-6f, 1e-6f, 1e-6f);
    }
    __syncthreads();
    const float bx = threadIdx.x * 0.01f + 0.5f, by = 0.3f, bz = -0.2f;
    const pf2 hx = pp_pack(bx, bx), hy = pp_pack(by, by), hz = pp_pack(bz, bz);
    const pf2 gx = pp_pack(bx + 0.1f, bx + 0.1f), gy = pp_pack(by - 0.1f, by - 0.1f), gz = hz;
    pf2 ps = 0, ax = 0, ay = 0, az = 0, qs = 0, bx2 = 0, by2 = 0, bz2 = 0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll 2
        for (int g = 0; g < 128; ++g) {
            const ulonglong2 X = ((const ulonglong2*)src[0])[g], Y = ((const ulonglong2*)src[1])[g],
                             Z = ((const ulonglong2*)src[2])[g], W = ((const ulonglong2*)src[3])[g];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const pf2 xx = h ? X.y : X.x, yy = h ? Y.y : Y.x, zz = h ? Z.y : Z.x, ww = h ? W.y : W.x;
                peak_pair2(xx, yy, zz, ww, hx, hy, hz, ps, ax, ay, az);
                peak_pair2(xx, yy, zz, ww, gx, gy, gz, qs, bx2, by2, bz2);
            }
        }
    }
    float a, b, s = 0.f;
    for (pf2 v : {ps, ax, ay, az, qs, bx2, by2, bz2}) {
        pp_unpack(v, a, b);
        s += a + b;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int pair_peak(int warps_per_sm, double* gpairs_s) {
    if (warps_per_sm < 4 || warps_per_sm > 32 || !gpairs_s) return FMM_E_INVALID;
    int dev, nsm;
    GB3_CUDA_TRY(cudaGetDevice(&dev));
    GB3_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int threads = 128, blocks = nsm * warps_per_sm / 4, iters = 64;
    float* d = nullptr;
    GB3_CUDA_TRY(cudaMalloc(&d, (size_t)threads * blocks * sizeof(float)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f, ms = 0.f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0);
        k_peak_pairs<<<blocks, threads>>>(d, iters);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d);
    if (err != cudaSuccess) return cuda_fail(err, "pair probe", __FILE__, __LINE__);
    *gpairs_s = (double)blocks * threads * iters * 1024.0 / (best * 1e-3) / 1e9;
    return 0;
}

}  // namespace gb3
