// swap_probe.cu -- measurement behind a design decision of the rotation-accelerated M2L
// (App. A.5): can the swap stage (the matrices Bhat_n of App. A.5.1, applied to one vector per
// interaction pair, orders n = 0..p) run faster on the tensor cores than as the FMA-immediate
// code the M2L kernel compiles it to?
//
// Both kernels take the same input, 32 pairs per warp staged in shared memory as columns
// S[entry][pair] (the M2L kernel's layout), and apply the swap `reps` times in place
// (Bhat_n is an involution: swapping x and z twice is the identity).
//   FMA:  one pair per lane, the order's 2n+1 values in registers, one FMA per non-zero
//         matrix entry with the entry as an immediate operand (swap_xz of m2l_rot.cuh).
//   MMA:  the parity of n+m+l splits each order's cosine and sine blocks into four dense
//         blocks of at most 8 x 8 (for n <= 14); each is one mma.sync m16n8k8 (TF32 inputs,
//         FP32 accumulation) per 16 pairs with the pairs as rows, the block's inputs as K and
//         its outputs as N, done as three products (a_hi b_hi + a_hi b_lo + a_lo b_hi, the
//         "3xTF32" split) so that the result keeps FP32 accuracy.
#include <cstring>
#include <vector>

#include "m2l_rot.cuh"

namespace gb3 {
namespace {

constexpr int kProbeP = 14;
constexpr int kProbeNco = (kProbeP + 1) * (kProbeP + 1);

// one dense block of Bhat_n: output slots rows[0..nr), input slots cols[0..nc) (real storage
// index j within order n), the entries split into TF32 high and low parts, [k][n] as the mma's
// B operand (k = input, n = output)
struct ProbeBlock {
    int n, nr, nc;
    int rows[8], cols[8];
    float bhi[8][8], blo[8][8];
};
constexpr int kProbeBlocks = 4 * (kProbeP + 1);
__constant__ ProbeBlock c_blocks[kProbeBlocks];

__device__ __forceinline__ unsigned to_tf32(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void mma_tf32(float* c, const unsigned* a, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ void stage_in(const float* __restrict__ V, size_t p0, long long npairs, float* S, int lane) {
    for (int b = 0; b < 32; ++b) {
        const long long q = (long long)p0 + b;
        for (int c = lane; c < kProbeNco; c += 32) S[c * kPad + b] = q < npairs ? V[q * kProbeNco + c] : 0.f;
    }
}
__device__ void stage_out(float* __restrict__ V, size_t p0, long long npairs, const float* S, int lane) {
    for (int b = 0; b < 32; ++b) {
        const long long q = (long long)p0 + b;
        if (q < npairs)
            for (int c = lane; c < kProbeNco; c += 32) V[q * kProbeNco + c] = S[c * kPad + b];
    }
}

template <int... N>
__device__ __forceinline__ void fma_swaps(float* Sl, iseq<N...>) {
    auto one = [&](auto nc) {
        constexpr int Nn = decltype(nc)::value;
        float v[2 * Nn + 1], t[2 * Nn + 1];
#pragma unroll
        for (int j = 0; j <= 2 * Nn; ++j) v[j] = Sl[(Nn * Nn + j) * kPad];
        swap_xz<Nn, Nn, Nn>(v, t);
#pragma unroll
        for (int j = 0; j <= 2 * Nn; ++j) Sl[(Nn * Nn + j) * kPad] = t[j];
    };
    (one(std::integral_constant<int, N>{}), ...);
}

// warps per block (one block per SM, as many warps as the shared memory holds, as in the M2L)
constexpr int kProbeWarpsFma = 7, kProbeWarpsMma = 6;
constexpr size_t kProbeWarpFloats = (size_t)kProbeNco * kPad;            // S
constexpr size_t kProbeTmpFloats = (size_t)(2 * kProbeP + 1) * kPad;     // one order's outputs

// one warp per 32 pairs
__global__ void __launch_bounds__(32 * kProbeWarpsFma) k_swap_fma(float* __restrict__ V, long long npairs, int reps) {
    extern __shared__ float sm_probe[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* S = sm_probe + (size_t)warp * kProbeWarpFloats;
    const long long nw = (npairs + 31) / 32;
    for (long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + warp; wg < nw;
         wg += (long long)gridDim.x * (blockDim.x >> 5)) {
        stage_in(V, (size_t)wg * 32, npairs, S, lane);
        __syncwarp();
        for (int r = 0; r < reps; ++r) fma_swaps(S + lane, upto<kProbeP>{});
        __syncwarp();
        stage_out(V, (size_t)wg * 32, npairs, S, lane);
        __syncwarp();
    }
}

// the four dense blocks of every order, 16 pairs per mma tile; an order's outputs go to T,
// then back into S
__global__ void __launch_bounds__(32 * kProbeWarpsMma)
    k_swap_mma(float* __restrict__ V, long long npairs, int reps, const uint4* __restrict__ frag) {
    extern __shared__ float sm_probe[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* S = sm_probe + (size_t)warp * (kProbeWarpFloats + kProbeTmpFloats);
    float* T = S + kProbeWarpFloats;
    const int g = lane >> 2, tg = lane & 3;
    const long long nw = (npairs + 31) / 32;
    for (long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + warp; wg < nw;
         wg += (long long)gridDim.x * (blockDim.x >> 5)) {
        stage_in(V, (size_t)wg * 32, npairs, S, lane);
        __syncwarp();
        for (int r = 0; r < reps; ++r) {
            for (int n = 0; n <= kProbeP; ++n) {
                const int base = n * n;
                for (int bi = 4 * n; bi < 4 * n + 4; ++bi) {
                    const ProbeBlock& B = c_blocks[bi];
                    if (B.nr == 0) continue;
                    // B operand: k = tg (b0) and tg + 4 (b1), n = g, per lane from the fragment table
                    const uint4 fb = frag[bi * 32 + lane];
                    const unsigned ubh0 = fb.x, ubh1 = fb.y, ubl0 = fb.z, ubl1 = fb.w;
                    const int k0 = tg, k1 = tg + 4;
                    const int j0 = k0 < B.nc ? base + B.cols[k0] : -1, j1 = k1 < B.nc ? base + B.cols[k1] : -1;
#pragma unroll
                    for (int tile = 0; tile < 2; ++tile) {
                        const int p0 = tile * 16 + g, p1 = p0 + 8;
                        const float x[4] = {j0 >= 0 ? S[j0 * kPad + p0] : 0.f, j0 >= 0 ? S[j0 * kPad + p1] : 0.f,
                                            j1 >= 0 ? S[j1 * kPad + p0] : 0.f, j1 >= 0 ? S[j1 * kPad + p1] : 0.f};
                        unsigned ah[4], al[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            ah[q] = to_tf32(x[q]);
                            al[q] = to_tf32(x[q] - __uint_as_float(ah[q]));
                        }
                        float c[4] = {0.f, 0.f, 0.f, 0.f};
                        mma_tf32(c, al, ubh0, ubh1);
                        mma_tf32(c, ah, ubl0, ubl1);
                        mma_tf32(c, ah, ubh0, ubh1);
                        // C: (pair g, out 2 tg), (g, 2 tg + 1), (g + 8, 2 tg), (g + 8, 2 tg + 1)
                        const int o0 = 2 * tg, o1 = 2 * tg + 1;
                        if (o0 < B.nr) {
                            T[B.rows[o0] * kPad + p0] = c[0];
                            T[B.rows[o0] * kPad + p1] = c[2];
                        }
                        if (o1 < B.nr) {
                            T[B.rows[o1] * kPad + p0] = c[1];
                            T[B.rows[o1] * kPad + p1] = c[3];
                        }
                    }
                }
                __syncwarp();
                for (int jj = 0; jj <= 2 * n; ++jj) S[(base + jj) * kPad + lane] = T[jj * kPad + lane];
                __syncwarp();
            }
        }
        stage_out(V, (size_t)wg * 32, npairs, S, lane);
        __syncwarp();
    }
}

float tf32_round(float x) {  // round to nearest (ties away), 10 explicit mantissa bits
    unsigned u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & ~0x1fffu;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}

// the dense blocks from the swap tables; false if an entry falls outside them
bool build_blocks(std::vector<ProbeBlock>& out) {
    out.assign(kProbeBlocks, ProbeBlock{});
    for (int n = 0; n <= kProbeP; ++n) {
        // covered[m][l] for the cosine (0) and sine (1) blocks
        bool cov[2][kProbeP + 1][kProbeP + 1] = {};
        for (int kind = 0; kind < 2; ++kind)
            for (int rp = 0; rp < 2; ++rp) {
                ProbeBlock& B = out[4 * n + 2 * kind + rp];
                B.n = n;
                const int m0 = kind == 0 ? 0 : 1;
                // cosine: n + m + l even; sine: odd
                const int lp = ((kind == 0 ? 0 : 1) + n + rp) & 1;
                for (int m = m0; m <= n; ++m)
                    if ((m & 1) == rp) {
                        if (B.nr == 8) return false;
                        B.rows[B.nr++] = kind == 0 ? n + m : n - m;
                    }
                for (int l = m0; l <= n; ++l)
                    if ((l & 1) == lp) {
                        if (B.nc == 8) return false;
                        B.cols[B.nc++] = kind == 0 ? n + l : n - l;
                    }
                for (int a = 0; a < B.nr; ++a)
                    for (int b = 0; b < B.nc; ++b) {
                        const int m = kind == 0 ? B.rows[a] - n : n - B.rows[a];
                        const int l = kind == 0 ? B.cols[b] - n : n - B.cols[b];
                        const double v = kind == 0 ? kSwap.cosb[n][m][l] : kSwap.sinb[n][m][l];
                        const float f = (float)v, h = tf32_round(f);
                        B.bhi[b][a] = h;
                        B.blo[b][a] = tf32_round(f - h);
                        cov[kind][m][l] = true;
                    }
                if (B.nr == 0 || B.nc == 0) B.nr = B.nc = 0;
            }
        for (int m = 0; m <= n; ++m)
            for (int l = 0; l <= n; ++l) {
                if (!cov[0][m][l] && kSwap.cosb[n][m][l] != 0.0) return false;
                if (m >= 1 && l >= 1 && !cov[1][m][l] && kSwap.sinb[n][m][l] != 0.0) return false;
            }
    }
    return true;
}

}  // namespace

int swap_probe(int npairs, int reps, double* ms, double* maxdiff) {
    if (npairs <= 0 || reps <= 0 || (reps & 1) || !ms || !maxdiff) return FMM_E_INVALID;
    std::vector<ProbeBlock> blocks;
    if (!build_blocks(blocks)) return FMM_E_INVALID;
    GB3_CUDA_TRY(cudaMemcpyToSymbol(c_blocks, blocks.data(), sizeof(ProbeBlock) * kProbeBlocks));
    const size_t nf = (size_t)npairs * kProbeNco;
    std::vector<float> h(nf);
    unsigned long long st = 0x9e3779b97f4a7c15ull;
    for (size_t i = 0; i < nf; ++i) {  // SplitMix64 values in [-1, 1)
        st += 0x9e3779b97f4a7c15ull;
        unsigned long long z = st;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        h[i] = (float)((double)(z >> 11) * 0x1p-52 - 1.0);
    }
    // the B fragments of every block for every lane: (hi k = tg, hi k = tg + 4, lo, lo), n = g
    std::vector<unsigned> hf((size_t)kProbeBlocks * 32 * 4);
    for (int bi = 0; bi < kProbeBlocks; ++bi)
        for (int ln = 0; ln < 32; ++ln) {
            const int gg = ln >> 2, tt = ln & 3;
            const float v[4] = {blocks[bi].bhi[tt][gg], blocks[bi].bhi[tt + 4][gg], blocks[bi].blo[tt][gg],
                                blocks[bi].blo[tt + 4][gg]};
            std::memcpy(&hf[((size_t)bi * 32 + ln) * 4], v, sizeof v);
        }
    float *d0 = nullptr, *d1 = nullptr;
    uint4* dfrag = nullptr;
    GB3_CUDA_TRY(cudaMalloc(&dfrag, hf.size() * sizeof(unsigned)));
    cudaMemcpy(dfrag, hf.data(), hf.size() * sizeof(unsigned), cudaMemcpyHostToDevice);
    if (cudaMalloc(&d0, nf * sizeof(float)) != cudaSuccess || cudaMalloc(&d1, nf * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d0);
        cudaFree(dfrag);
        return FMM_E_OOM;
    }
    cudaMemcpy(d0, h.data(), nf * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(d1, h.data(), nf * sizeof(float), cudaMemcpyHostToDevice);
    const size_t sm_fma = kProbeWarpsFma * kProbeWarpFloats * sizeof(float);
    const size_t sm_mma = kProbeWarpsMma * (kProbeWarpFloats + kProbeTmpFloats) * sizeof(float);
    cudaFuncSetAttribute(k_swap_fma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_fma);
    cudaFuncSetAttribute(k_swap_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_mma);
    int b_fma = 1, b_mma = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b_fma, k_swap_fma, 32 * kProbeWarpsFma, sm_fma);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b_mma, k_swap_mma, 32 * kProbeWarpsMma, sm_mma);
    const unsigned g_fma = (unsigned)(sm_count() * (b_fma > 0 ? b_fma : 1));
    const unsigned g_mma = (unsigned)(sm_count() * (b_mma > 0 ? b_mma : 1));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best[2] = {1e30f, 1e30f};
    for (int rep = 0; rep < 4; ++rep) {  // the first round warms up; reps is even, so V returns
        for (int k = 0; k < 2; ++k) {
            cudaEventRecord(e0);
            if (k == 0) k_swap_fma<<<g_fma, 32 * kProbeWarpsFma, sm_fma>>>(d0, npairs, reps);
            else k_swap_mma<<<g_mma, 32 * kProbeWarpsMma, sm_mma>>>(d1, npairs, reps, dfrag);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0 && t < best[k]) best[k] = t;
        }
    }
    // one more application of each (an odd count) to compare a non-trivial result
    k_swap_fma<<<g_fma, 32 * kProbeWarpsFma, sm_fma>>>(d0, npairs, 1);
    k_swap_mma<<<g_mma, 32 * kProbeWarpsMma, sm_mma>>>(d1, npairs, 1, dfrag);
    std::vector<float> a(nf), b(nf);
    cudaMemcpy(a.data(), d0, nf * sizeof(float), cudaMemcpyDeviceToHost);
    cudaMemcpy(b.data(), d1, nf * sizeof(float), cudaMemcpyDeviceToHost);
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d0);
    cudaFree(d1);
    cudaFree(dfrag);
    if (err != cudaSuccess) return cuda_fail(err, "swap probe", __FILE__, __LINE__);
    double md = 0.0;
    for (size_t i = 0; i < nf; ++i) md = std::max(md, (double)std::fabs(a[i] - b[i]));
    ms[0] = best[0];
    ms[1] = best[1];
    *maxdiff = md;
    return 0;
}

}  // namespace gb3
