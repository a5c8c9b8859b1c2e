// m2l_rot.cu -- host side of the rotation-accelerated M2L (App. A.5) of the mixed-precision
// path: the per-cell preparation of the scaled FP32 multipoles and the dispatch on p to
// the kernels of m2l_rot.cuh (instantiated in m2l_rot_p*.cu).
#include "m2l_rot.cuh"

namespace gb3 {
namespace {

// per cell: Mt = N_n^m M_n^m / rho^n in FP32 (real storage) and conj(M) of orders <= 2 in FP64
// (the kernel reads the orders <= kRotJ64)
__global__ void k_prep_rot(const double* __restrict__ M, const d4* __restrict__ cen, int ncells, int p,
                           float* __restrict__ Mt, cd* __restrict__ M64) {
    const int nco = ncoef(p), lane = threadIdx.x & 31;
    for (long long cell = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; cell < ncells;
         cell += ((long long)gridDim.x * blockDim.x) >> 5) {
        const double rho = cen[cell].w;
        double pw = lane == 0 ? 1.0 : 0.0;  // a source of radius 0 has no moments above the monopole
        if (rho > 0 && lane > 0 && lane <= p) {
            const double rinv = 1.0 / rho;
            pw = rinv;
            for (int k = 1; k < lane; ++k) pw *= rinv;
        }
        const double* R = M + (size_t)cell * nco;
        for (int i0 = 0; i0 < nco; i0 += 32) {  // uniform trip count: the shuffle needs every lane
            const int i = i0 + lane;
            const int n = i < nco ? (int)sqrtf((float)i) : 0;
            const double sc = __shfl_sync(0xffffffffu, pw, n);
            if (i < nco) {
                Mt[(size_t)cell * nco + i] = (float)(R[i] * c_rot_norm.v[i] * sc);
                if (i < 9) M64[(size_t)cell * 9 + i] = conjc(load_real_storage(R, n, i - n * n - n));
            }
        }
    }
}

}  // namespace

extern template void rot_launch<3>(const int2*, const int*, const int*, const int*, const int*, unsigned*, const d4*,
                             const float*, const cd*, double*, cudaStream_t);
extern template void rot_launch<4>(const int2*, const int*, const int*, const int*, const int*, unsigned*, const d4*,
                             const float*, const cd*, double*, cudaStream_t);
extern template void rot_launch<5>(const int2*, const int*, const int*, const int*, const int*, unsigned*, const d4*,
                             const float*, const cd*, double*, cudaStream_t);
extern template void rot_launch<6>(const int2*, const int*, const int*, const int*, const int*, unsigned*, const d4*,
                             const float*, const cd*, double*, cudaStream_t);
extern template void rot_launch<7>(const int2*, const int*, const int*, const int*, const int*, unsigned*, const d4*,
                             const float*, const cd*, double*, cudaStream_t);
extern template void rot_launch<8>(const int2*, const int*, const int*, const int*, const int*, unsigned*, const d4*,
                             const float*, const cd*, double*, cudaStream_t);
extern template void rot_launch<9>(const int2*, const int*, const int*, const int*, const int*, unsigned*, const d4*,
                             const float*, const cd*, double*, cudaStream_t);
extern template void rot_launch<10>(const int2*, const int*, const int*, const int*, const int*, unsigned*, const d4*,
                             const float*, const cd*, double*, cudaStream_t);
extern template void rot_launch<11>(const int2*, const int*, const int*, const int*, const int*, unsigned*, const d4*,
                             const float*, const cd*, double*, cudaStream_t);
extern template void rot_launch<12>(const int2*, const int*, const int*, const int*, const int*, unsigned*, const d4*,
                             const float*, const cd*, double*, cudaStream_t);
extern template void rot_launch<13>(const int2*, const int*, const int*, const int*, const int*, unsigned*, const d4*,
                             const float*, const cd*, double*, cudaStream_t);
extern template void rot_launch<14>(const int2*, const int*, const int*, const int*, const int*, unsigned*, const d4*,
                             const float*, const cd*, double*, cudaStream_t);
extern template void rot_launch<15>(const int2*, const int*, const int*, const int*, const int*, unsigned*, const d4*,
                             const float*, const cd*, double*, cudaStream_t);
extern template void rot_launch<16>(const int2*, const int*, const int*, const int*, const int*, unsigned*, const d4*,
                             const float*, const cd*, double*, cudaStream_t);

bool m2l_rot_supported(int p) { return p >= 3 && p <= kRotMaxP; }

void launch_m2l_rot(const int2* list, const int* seg_start, const int* seg_end, const int* order,
                    const int* item_start, unsigned* work, const d4* cen, const double* M, int ncells, int p,
                    float* Mt, cd* M64, double* part, cudaStream_t s) {
    k_prep_rot<<<grid_for((long long)ncells * 32, 256), 256, 0, s>>>(M, cen, ncells, p, Mt, M64);
    note_launch();
#define GB3_ROT(PP) \
    case PP: rot_launch<PP>(list, seg_start, seg_end, order, item_start, work, cen, Mt, M64, part, s); break;
    switch (p) {
        GB3_ROT(3) GB3_ROT(4) GB3_ROT(5) GB3_ROT(6) GB3_ROT(7) GB3_ROT(8) GB3_ROT(9) GB3_ROT(10) GB3_ROT(11)
        GB3_ROT(12) GB3_ROT(13) GB3_ROT(14) GB3_ROT(15) GB3_ROT(16)
        default: break;
    }
#undef GB3_ROT
}

}  // namespace gb3

extern "C" int fmm_swap_matrix(int n, double* B) {
    if (n < 0 || n > gb3::kRotMaxP || !B) return FMM_E_INVALID;
    for (int m = -n; m <= n; ++m)
        for (int l = -n; l <= n; ++l)
            B[(m + n) * (2 * n + 1) + (l + n)] = gb3::kSwap.full[n][gb3::kO + m][gb3::kO + l];
    return FMM_OK;
}
