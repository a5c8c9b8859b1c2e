// common.cu -- error reporting and the device-wide exclusive scan.
#include <stdio.h>

#include "common.cuh"

namespace gb3 {

// set by the C-ABI layer to record the message of the last CUDA failure
thread_local char g_cuda_msg[256];

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_cuda_msg, sizeof g_cuda_msg, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    if (e == cudaErrorMemoryAllocation) return FMM_E_OOM;
    return FMM_E_CUDA;
}

// SM count per device, queried on first use (0 = not yet known)
static int g_sm_count[64] = {0};
int sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 148;  // a query that fails only sizes grid-stride loops
    }
    int n = __atomic_load_n(&g_sm_count[dev], __ATOMIC_RELAXED);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            return 148;
        }
        __atomic_store_n(&g_sm_count[dev], n, __ATOMIC_RELAXED);
    }
    return n;
}

thread_local long long g_launches = 0;
void note_launch() { ++g_launches; }
long long launches_so_far() { return g_launches; }

thread_local cudaEvent_t* g_marks = nullptr;
thread_local int g_marks_hit = 0;
void kernel_marks(cudaEvent_t* ev) {
    g_marks = ev;
    g_marks_hit = 0;
}
void mark_begin(cudaStream_t s) {
    if (g_marks && cudaEventRecord(g_marks[0], s) == cudaSuccess) g_marks_hit |= 1;
}
void mark_end(cudaStream_t s) {
    if (g_marks && cudaEventRecord(g_marks[1], s) == cudaSuccess) g_marks_hit |= 2;
}
bool marks_recorded() { return g_marks_hit == 3; }

// ---------------------------------------------------------------- scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ inline int block_exclusive_scan(int v, int* smem_warp, int& total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        int s = lane < nw ? smem_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) smem_warp[lane] = s;
    }
    __syncthreads();
    int warp_base = w ? smem_warp[w - 1] : 0;
    total = smem_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_base + x - v;
}

__global__ void k_chunk_sums(const int* __restrict__ in, long long n, int* __restrict__ sums) {
    __shared__ int sw[32];
    long long base = (long long)blockIdx.x * kScanChunk;
    int local = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + (long long)threadIdx.x * kScanItems + k;
        if (i < n) local += in[i];
    }
    int total;
    block_exclusive_scan(local, sw, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_chunk_scan(const int* __restrict__ in, int* __restrict__ out, long long n,
                             const int* __restrict__ offs, int* __restrict__ d_total, long long nchunks) {
    __shared__ int sw[32];
    long long base = (long long)blockIdx.x * kScanChunk;
    int vals[kScanItems];
    int local = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + (long long)threadIdx.x * kScanItems + k;
        vals[k] = i < n ? in[i] : 0;
        local += vals[k];
    }
    int total;
    int ex = block_exclusive_scan(local, sw, total);
    int run = ex + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long i = base + (long long)threadIdx.x * kScanItems + k;
        if (i < n) out[i] = run;
        run += vals[k];
    }
    if (d_total && blockIdx.x == nchunks - 1 && threadIdx.x == blockDim.x - 1) *d_total = run;
}

__global__ void k_zero_total(int* d_total) { *d_total = 0; }

size_t scan_tmp_ints(long long n) {
    size_t t = 0;
    while (n > kScanChunk) {
        long long c = (n + kScanChunk - 1) / kScanChunk;
        t += (size_t)2 * c + 1;
        n = c;
    }
    return t + 1;
}

void scan_exclusive_i32(const int* in, int* out, long long n, int* d_total, int* tmp, cudaStream_t s) {
    if (n <= 0) {
        if (d_total) k_zero_total<<<1, 1, 0, s>>>(d_total); note_launch();
        return;
    }
    long long nchunks = (n + kScanChunk - 1) / kScanChunk;
    if (nchunks == 1) {
        k_chunk_scan<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, d_total, 1); note_launch();
        return;
    }
    int* sums = tmp;
    int* sums_scan = tmp + nchunks;
    k_chunk_sums<<<(unsigned)nchunks, kScanThreads, 0, s>>>(in, n, sums); note_launch();
    scan_exclusive_i32(sums, sums_scan, nchunks, nullptr, tmp + 2 * nchunks + 1, s);
    k_chunk_scan<<<(unsigned)nchunks, kScanThreads, 0, s>>>(in, out, n, sums_scan, d_total, nchunks); note_launch();
}

}  // namespace gb3
