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

}  // namespace gb3
