// m2l_rot.cuh -- device code of the rotation-accelerated M2L of the mixed-precision
// path (A9, the M2L kernel of eq. 3b, accelerated as in App. A.5); m2l_rot.cu holds the
// host side, and the kernel for each order p is instantiated in one of the
// m2l_rot_p*.cu files so that they compile in parallel.
//
// For every accepted pair the source's multipoles are turned into a frame whose z axis
// points along the interaction, the M2L is done there with the z-axis form (eq. A31,
// O(p^3)), and the result is turned back.  A rotation does not mix orders; it is built
// from rotations about z (a phase e^{-i m alpha} per coefficient) and the constant swap
// of the x and z axes (the matrices B_n of App. A.5.1, from the recurrences given there).
//
// Frames.  For r = s_B - z_A = (x, y, z), rho = |(x, y)|, R = |r|:
//   1. rotate about z by alpha with e^{i alpha} = (y - i x)/rho   -> r = (0, rho, z)
//   2. swap x and z                                               -> r = (z, rho, 0)
//   3. rotate about z by beta with e^{i beta} = (z + i rho)/R      -> r = (R, 0, 0)
//   4. swap x and z                                               -> r = (0, 0, R)
// A rotation about z by alpha multiplies X_n^m by e^{-i m alpha}.  Multipoles turn with
// the Upsilon matrices, local coefficients with the inverse of that map (the potential
// sum_n Upsilon^* F is frame independent), so F goes back through steps 4 .. 1 with the
// same swap and the conjugate phases.
//
// Normalisation.  With N_n^m = sqrt((n-m)!(n+m)!), Theta_n^m / N_n^m and
// Upsilon_n^m N_n^m have the same angular part (an orthonormal set up to a constant), so
// the swap is the same matrix Bhat_n = diag(1/N) B_n diag(N) for the scaled multipoles
// Mhat = N M and the scaled local coefficients Fhat = F / N, and its entries are O(1).
// In the real storage (Re X_n^m at slot n^2+n+m, Im X_n^m at n^2+n-m) Bhat_n splits into
// a cosine block (m, l >= 0) and a sine block (m, l >= 1), each with the chequerboard of
// zeros that the parity of the harmonics gives; the entries are compile-time constants
// (immediate operands of the FMAs), computed below from the recurrences in FP64.
//
// Precision split: the terms of eq. (3b) with n + k <= kRotJ64 (= 1: the monopole and
// dipole couplings, which carry nearly all of the force) are summed in FP64 from the FP64
// moments; the others are summed in FP32 on the scaled quantities Mt_k = Mhat_k /
// rho_A^k, (rho_A/R)^k, unit distance, and the pair's result is scaled by
// (sigma_B/R)^{n+1}, so that every FP32 value is O(1)..O(M).  (The direct mixed-mode
// kernel also sums the order-2 couplings in FP64; in FP32 they add about 1 % to the rms
// force error at eps = 3e-7 and cost half of the FP64 work of a pair.)  The z-axis kernel
// maps each order k of the rotated multipoles to each order n of the rotated local
// expansion separately, so leaving out n + k <= kRotJ64 in the rotated frame leaves out
// exactly the same terms as in the original frame.
#pragma once
#include <utility>

#include "kernels.cuh"

namespace gb3 {

// arguments of one launch of the rotated M2L kernel (see k_m2l_rot)
struct RotArgs {
    const int2* list;
    const int* seg_start;
    const int* seg_end;
    const int* order;
    const int* item_start;
    unsigned* work;
    const d4* cen;
    const float* Mt;
    const cd* M64;
    double* part;
    double* F;
    const int* ilist;
    const unsigned* goff;
    int gq;
    unsigned* counter;
    int nco_out;
    int adapt;
    // by-sink mode (ilist == nullptr and cnt != nullptr): every warp takes units from
    // *sink_counter: units[u] = (position i of the sorted order, piece k); sink i has cnt[i]
    // items, and a sink of more than kM2LPieceItems items is cut into pieces of that many
    const int* cnt;
    unsigned* sink_counter;
    const int2* units;
    const unsigned* nunits;
};

namespace {

// ---------------------------------------------------------------- constant tables
constexpr double rfact(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}
constexpr double rsqrt_newton(double x) {  // sqrt by Newton's iteration, for constants only
    if (!(x > 0.0)) return 0.0;
    double y = x > 1.0 ? x : 1.0;
    for (int i = 0; i < 400; ++i) {
        const double z = 0.5 * (y + x / y);
        if (z == y) break;
        y = z;
    }
    return y;
}
constexpr double norm_nm(int n, int m) {  // N_n^m = sqrt((n-|m|)!(n+|m|)!)
    const int a = m < 0 ? -m : m;
    return rsqrt_newton(rfact(n - a) * rfact(n + a));
}

constexpr int kW = 2 * kRotMaxP + 1, kO = kRotMaxP;  // B_n^{ml} at b[kO + m][kO + l]

struct SwapTables {
    double cosb[kRotMaxP + 1][kRotMaxP + 1][kRotMaxP + 1];  // [n][m][l], 0 <= m, l <= n
    double sinb[kRotMaxP + 1][kRotMaxP + 1][kRotMaxP + 1];  // [n][m][l], 1 <= m, l <= n
    double full[kRotMaxP + 1][kW][kW];                     // B_n^{ml} at [n][kO + m][kO + l]
};

constexpr double b_at(const double (&b)[kW][kW], int n, int m, int l) {
    return (m < -n || m > n || l < -n || l > n) ? 0.0 : b[kO + m][kO + l];
}

constexpr SwapTables make_swap_tables() {
    SwapTables t{};
    double b[kW][kW] = {};
    double nb[kW][kW] = {};
    b[kO][kO] = 1.0;  // B_0 = 1
    for (int n = 0; n <= kRotMaxP; ++n) {
        for (int i = 0; i < kW; ++i)
            for (int j = 0; j < kW; ++j) t.full[n][i][j] = b[i][j];
        // real blocks of Bhat_n = diag(1/N) B_n diag(N): a complex vector with
        // X^{-l} = (-1)^l conj(X^l) maps to Re Y^m = sum_{l>=0} C_ml Re X^l and
        // Im Y^m = sum_{l>=1} S_ml Im X^l
        for (int m = 0; m <= n; ++m)
            for (int l = 0; l <= n; ++l) {
                const double f = norm_nm(n, l) / norm_nm(n, m);
                const double bp = b_at(b, n, m, l) * f, bm = b_at(b, n, m, -l) * f;
                const double sg = (l & 1) ? -1.0 : 1.0;
                t.cosb[n][m][l] = l == 0 ? bp : bp + sg * bm;
                if (m >= 1 && l >= 1) t.sinb[n][m][l] = bp - sg * bm;
            }
        if (n == kRotMaxP) break;
        // recurrences of App. A.5.1 for swapping x and z:
        //   2 B_{n+1}^{m l}     = B_n^{m,l-1} - B_n^{m,l+1}                 (|m| <= n)
        //   2 B_{n+1}^{m+-1, l} = B_n^{m,l-1} + B_n^{m,l+1} +- 2 B_n^{m l}   (m = +-n)
        for (int i = 0; i < kW; ++i)
            for (int j = 0; j < kW; ++j) nb[i][j] = 0.0;
        for (int m = -n; m <= n; ++m)
            for (int l = -(n + 1); l <= n + 1; ++l)
                nb[kO + m][kO + l] = 0.5 * (b_at(b, n, m, l - 1) - b_at(b, n, m, l + 1));
        for (int l = -(n + 1); l <= n + 1; ++l) {
            nb[kO + n + 1][kO + l] = 0.5 * (b_at(b, n, n, l - 1) + b_at(b, n, n, l + 1)) + b_at(b, n, n, l);
            nb[kO - n - 1][kO + l] = 0.5 * (b_at(b, n, -n, l - 1) + b_at(b, n, -n, l + 1)) - b_at(b, n, -n, l);
        }
        for (int i = 0; i < kW; ++i)
            for (int j = 0; j < kW; ++j) b[i][j] = nb[i][j];
    }
    return t;
}

constexpr SwapTables kSwap = make_swap_tables();

template <int N, int M, int L>
constexpr float kCos = (float)kSwap.cosb[N][M][L];
template <int N, int M, int L>
constexpr float kSin = (float)kSwap.sinb[N][M][L];

// z-axis M2L (eq. A31) on the scaled coefficients: Fhat_n^m = sum_k Z(n,k,m) Mhat_k^m / R^{n+k+1}
// with Z(n,k,m) = (-1)^m (n+k)! / (N_k^m N_n^m)
constexpr double zcoef(int n, int k, int m) {
    return ((m & 1) ? -1.0 : 1.0) * rfact(n + k) / (norm_nm(k, m) * norm_nm(n, m));
}
template <int N, int K, int M>
constexpr float kZ = (float)zcoef(N, K, M);

template <int... I>
using iseq = std::integer_sequence<int, I...>;
template <int N>
using upto = std::make_integer_sequence<int, N + 1>;  // 0 .. N

constexpr int imin(int a, int b) { return a < b ? a : b; }
constexpr int imax(int a, int b) { return a > b ? a : b; }

// ---------------------------------------------------------------- one order, in registers
// v holds order N in real storage: v[N + m] = Re X^m (m >= 0), v[N - m] = Im X^m (m >= 1).

// X^m *= c[m] (or conj(c[m])) for m = 1..N
template <int N, bool CONJ, int M>
__host__ __device__ __forceinline__ void zrot_one(float* v, const float2* c) {
    const float re = v[N + M], im = v[N - M];
    const float cx = c[M].x, cy = CONJ ? -c[M].y : c[M].y;
    v[N + M] = fmaf(re, cx, -(im * cy));
    v[N - M] = fmaf(re, cy, im * cx);
}
template <int N, bool CONJ, int... M>
__host__ __device__ __forceinline__ void zrot_seq(float* v, const float2* c, iseq<M...>) {
    (zrot_one<N, CONJ, M + 1>(v, c), ...);
}
template <int N, bool CONJ>
__host__ __device__ __forceinline__ void zrot(float* v, const float2* c) {
    zrot_seq<N, CONJ>(v, c, std::make_integer_sequence<int, N>{});
}

// out = Bhat_N in, for output rows |m| <= RL, reading input entries |l| <= CL only
template <int N, int CL, int M, int L>
__host__ __device__ __forceinline__ void cos_term(float& acc, const float* in) {
    if constexpr (L <= CL && kCos<N, M, L> != 0.0f) acc = fmaf(kCos<N, M, L>, in[N + L], acc);
}
template <int N, int CL, int M, int L>
__host__ __device__ __forceinline__ void sin_term(float& acc, const float* in) {
    if constexpr (L >= 1 && L <= CL && kSin<N, M, L> != 0.0f) acc = fmaf(kSin<N, M, L>, in[N - L], acc);
}
template <int N, int RL, int CL, int M, int... L>
__host__ __device__ __forceinline__ void swap_row(const float* in, float* out, iseq<L...>) {
    if constexpr (M <= RL) {
        float a = 0.f;
        (cos_term<N, CL, M, L>(a, in), ...);
        out[N + M] = a;
        if constexpr (M >= 1) {
            float b = 0.f;
            (sin_term<N, CL, M, L>(b, in), ...);
            out[N - M] = b;
        }
    }
}
template <int N, int RL, int CL, int... M>
__host__ __device__ __forceinline__ void swap_seq(const float* in, float* out, iseq<M...>) {
    (swap_row<N, RL, CL, M>(in, out, upto<N>{}), ...);
}
template <int N, int RL, int CL>
__host__ __device__ __forceinline__ void swap_xz(const float* in, float* out) {
    swap_seq<N, RL, CL>(in, out, upto<N>{});
}

constexpr int kPad = 33;  // column stride of the per-lane shared-memory vectors (words)
// terms of eq. (3b) with n + k <= kRotJ64 are summed in FP64, the others in FP32
constexpr int kRotJ64 = 1;
constexpr int kRotLow = (kRotJ64 + 1) * (kRotJ64 + 2) / 2;  // FP64 outputs (n <= kRotJ64, m >= 0)
constexpr int kRotLowM = (kRotJ64 + 1) * (kRotJ64 + 1);     // FP64 moments per cell (orders <= kRotJ64)

// forward: scaled multipoles of order K -> rotated frame, entries |m| <= min(K, P-K), times (rho_A/R)^K
template <int P, int K>
__host__ __device__ __forceinline__ void fwd_order(float* S, const float2* cw, const float2* cu, float tk) {
    constexpr int L = imin(K, P - K);
    float v[2 * K + 1], t[2 * K + 1];
#pragma unroll
    for (int j = 0; j <= 2 * K; ++j) v[j] = S[(K * K + j) * kPad];
    zrot<K, false>(v, cw);
    swap_xz<K, K, K>(v, t);
    zrot<K, false>(t, cu);
    swap_xz<K, L, K>(t, v);
#pragma unroll
    for (int j = K - L; j <= K + L; ++j) S[(K * K + j) * kPad] = v[j] * tk;
}
// warps of a block meet after every kRotSyncOrders orders (0: only between the phases)
constexpr int kRotSyncOrders = 0;
template <int K>
__host__ __device__ __forceinline__ void order_sync() {
#ifdef __CUDA_ARCH__
    if constexpr (kRotSyncOrders > 0 && K % (kRotSyncOrders > 0 ? kRotSyncOrders : 1) == 0) __syncthreads();
#endif
}
template <int P, int... K>
__host__ __device__ __forceinline__ void fwd_all(float* S, const float2* cw, const float2* cu, float tA, iseq<K...>) {
    float tk = 1.f;
    ((fwd_order<P, K>(S, cw, cu, tk), tk *= tA, order_sync<K + 1>()), ...);
}

// z-axis M2L for column m = M (SG = +1: real parts, -1: imaginary parts), in place.
// MASK: the lane's pair has its own order q <= P (adaptive walk): only terms n + k <= q
template <int P, int M, int SG, bool MASK, int N, int... K>
__host__ __device__ __forceinline__ void zm2l_out(float* S, const float* x, int q, iseq<K...>) {
    if constexpr (N >= M && N <= P - M) {
        float acc = 0.f;
        ((K >= M && K <= P - N && N + K > kRotJ64
              ? (void)(acc = fmaf(kZ<N, K, M>, (!MASK || N + K <= q) ? x[K] : 0.f, acc))
              : (void)0),
         ...);
        S[(N * N + N + SG * M) * kPad] = acc;
    }
}
template <int P, int M, int SG, bool MASK, int... I>
__host__ __device__ __forceinline__ void zm2l_col(float* S, int q, iseq<I...>) {
    float x[P + 1];
    ((I >= M && I <= P - M ? (void)(x[I] = S[(I * I + I + SG * M) * kPad]) : (void)0), ...);
    (zm2l_out<P, M, SG, MASK, I>(S, x, q, upto<P>{}), ...);
}
template <int P, bool MASK, int... M>
__host__ __device__ __forceinline__ void zm2l_all(float* S, int q, iseq<M...>) {
    ((zm2l_col<P, M, 1, MASK>(S, q, upto<P>{}), (M >= 1 ? zm2l_col<P, M, -1, MASK>(S, q, upto<P>{}) : (void)0)), ...);
}

// backward: rotated local coefficients of order N (entries |m| <= min(N, P-N)) -> original
// frame, times (sigma_B/R)^{N+1}
template <int P, int N>
__host__ __device__ __forceinline__ void bwd_order(float* S, const float2* cw, const float2* cu, float tn) {
    constexpr int L = imin(N, P - N);
    float v[2 * N + 1], t[2 * N + 1];
#pragma unroll
    for (int j = N - L; j <= N + L; ++j) v[j] = S[(N * N + j) * kPad];
    swap_xz<N, N, L>(v, t);
    zrot<N, true>(t, cu);
    swap_xz<N, N, N>(t, v);
    zrot<N, true>(v, cw);
#pragma unroll
    for (int j = 0; j <= 2 * N; ++j) S[(N * N + j) * kPad] = v[j] * tn;
}
template <int P, int... N>
__host__ __device__ __forceinline__ void bwd_all(float* S, const float2* cw, const float2* cu, float tB, iseq<N...>) {
    float tn = tB;
    ((bwd_order<P, N>(S, cw, cu, tn), tn *= tB, order_sync<N + 1>()), ...);
}

// N_n^{|m|} by slot n^2+n+m (a constant-initialised copy in every translation unit)
struct RotNorm {
    double v[(kRotMaxP + 1) * (kRotMaxP + 1)];
};
constexpr RotNorm make_rot_norm() {
    RotNorm t{};
    for (int n = 0; n <= kRotMaxP; ++n)
        for (int m = -n; m <= n; ++m) t.v[n * n + n + m] = norm_nm(n, m);
    return t;
}
static __constant__ RotNorm c_rot_norm = make_rot_norm();

// 4-byte asynchronous global -> shared copy; nbytes = 0 writes a zero
__device__ __forceinline__ void rot_cp_async4(float* smem, const float* gmem, unsigned nbytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(nbytes) : "memory");
}
__device__ __forceinline__ void rot_cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void rot_cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Theta_j^m(r) for j <= 2 and m >= 0 in closed form (FP64)
__device__ inline cd theta_low_rot(int j, int m, double x, double y, double z, double rinv) {
    const double r2i = rinv * rinv, r3 = rinv * r2i, r5 = r3 * r2i;
    if (j == 0) return mkc(rinv, 0.0);
    if (j == 1) return m == 0 ? mkc(z * r3, 0.0) : mkc(x * r3, y * r3);
    if (m == 0) return mkc((3.0 * z * z - (x * x + y * y + z * z)) * r5, 0.0);
    if (m == 1) return mkc(3.0 * z * x * r5, 3.0 * z * y * r5);
    return mkc(3.0 * (x * x - y * y) * r5, 6.0 * x * y * r5);
}

// Shared memory of one warp: the per-lane vectors S[NCO][kPad] (floats), sigma^-n and
// the FP64 low-order outputs; then the sink's accumulated expansion (NCO doubles, by-sink mode).
template <int P>
constexpr int rot_warp_core_bytes() {
    return (((P + 1) * (P + 1) * kPad * 4 + 15) & ~15) + (((P + 2) * 8 + kRotLow * 16 + 15) & ~15);
}
template <int P>
constexpr int rot_warp_bytes() {
    return rot_warp_core_bytes<P>() + (((P + 1) * (P + 1) * 8 + 15) & ~15);
}
// warps per block: as many as the shared memory of one SM holds (at most 8); they step
// through the (long, straight-line) code of the orders together, so that they share its
// instruction fetches
template <int P>
constexpr int rot_warps() {
    return imin(8, imax(1, (227 * 1024) / rot_warp_bytes<P>()));
}

// One warp per work item: up to kM2LChunk pairs of one sink, lane = pair.  By sink (cnt !=
// nullptr, every pair at p): a warp takes a unit from *sink_counter (longest lists first) --
// a whole sink, or a piece of kM2LPieceItems items of a longer one -- and its items one after
// the other, adds their expansions in item order into its shared-memory accumulator and writes
// it once: to F + B * nco_out for a whole sink, to the part slot of the piece's first item for
// a piece.  By item (the adaptive walk's
// groups): the items are ilist[goff[gq] .. goff[gq + 1]) taken from *counter; item w's partial
// expansion goes to part + w * nco_out, nco_out = (p+1)^2 of the global order p >= P, which is
// also the row length of Mt (a sink whose whole list is one item has its expansion written to F
// directly; F starts at zero).  adapt: the pairs carry their own orders q <= P (adaptive walk)
// and each lane keeps only the terms n + k <= q of its pair.
template <int P>
__global__ void __launch_bounds__(32 * rot_warps<P>(), 1) k_m2l_rot(const RotArgs args) {
    const int2* __restrict__ list = args.list;
    const int* __restrict__ seg_start = args.seg_start;
    const int* __restrict__ seg_end = args.seg_end;
    const int* __restrict__ order = args.order;
    const int* __restrict__ item_start = args.item_start;
    const unsigned* __restrict__ work = args.work;
    const d4* __restrict__ cen = args.cen;
    const float* __restrict__ Mt = args.Mt;
    const cd* __restrict__ M64g = args.M64;
    const int* __restrict__ ilist = args.ilist;
    const unsigned* __restrict__ goff = args.goff;
    const int gq = args.gq, nco_out = args.nco_out, adapt = args.adapt;
    unsigned* __restrict__ counter = args.counter;
    constexpr int NCO = (P + 1) * (P + 1), W = rot_warps<P>();
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ unsigned s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char* base = sm_raw + (size_t)warp * rot_warp_bytes<P>();
    float* S = (float*)base;                                          // [NCO][kPad]
    double* pws = (double*)(base + ((NCO * kPad * 4 + 15) & ~15));    // sigma^-n, n <= P+1
    cd* lowF = (cd*)(pws + P + 2);                                    // FP64 outputs (n <= kRotJ64, m >= 0)
    float* Sl = S + lane;
    double* accF = (double*)(base + rot_warp_core_bytes<P>());  // the sink's expansion (by sink)
    const unsigned nsinks = work[1];
    const unsigned lbase = ilist ? goff[gq] : 0u, nlist = ilist ? goff[gq + 1] - goff[gq] : work[2];
    const bool by_sink = !ilist && args.cnt;
    // by sink: the warp's sink position, item cursor and end, and where its sum goes
    int cur = -1, cur_it = 0, cur_end = 0, cur_first = 0;
    bool cur_piece = false, done = false;
    const unsigned nunits = by_sink ? *args.nunits : 0u;
    for (;;) {
        bool has;
        unsigned w;
        int pos = 0;
        if (by_sink) {
            // the warp's sink is used up: write its expansion, take the next sink
            while (!done && cur_it >= cur_end) {
                if (cur >= 0) {
                    double* o = cur_piece ? args.part + (size_t)cur_first * nco_out
                                          : args.F + (size_t)order[cur] * nco_out;
                    for (int c = lane; c < NCO; c += 32) o[c] = accF[c];
                }
                unsigned nx = 0;
                if (lane == 0) nx = atomicAdd(args.sink_counter, 1u);
                nx = __shfl_sync(0xffffffffu, nx, 0);
                if (nx >= nunits) {
                    done = true;
                    cur = -1;
                    break;
                }
                const int2 un = args.units[nx];
                cur = un.x;
                const int c0 = item_start[cur], nit = args.cnt[cur];
                cur_it = c0 + un.y * kM2LPieceItems;
                cur_end = min(cur_it + kM2LPieceItems, c0 + nit);
                cur_first = cur_it;
                cur_piece = nit > kM2LPieceItems;
                for (int c = lane; c < NCO; c += 32) accF[c] = 0.0;
                __syncwarp();
            }
            has = !done;
            w = has ? (unsigned)cur_it : 0u;
            pos = has ? cur : 0;
            if (!__syncthreads_or(has)) break;  // every warp runs every barrier
        } else {
            // the block takes W consecutive list entries, one per warp (every warp runs every barrier)
            if (threadIdx.x == 0) s_item = atomicAdd(counter, (unsigned)W);
            __syncthreads();
            const unsigned w0 = s_item;
            __syncthreads();
            if (w0 >= nlist) break;
            has = w0 + warp < nlist;
            w = has ? (ilist ? (unsigned)ilist[lbase + w0 + warp] : w0 + warp) : 0u;
            if (has) {
                int lo_i = 0, hi_i = (int)nsinks - 1;
                while (lo_i < hi_i) {
                    const int mid = (lo_i + hi_i + 1) >> 1;
                    if ((unsigned)item_start[mid] <= w) lo_i = mid;
                    else hi_i = mid - 1;
                }
                pos = lo_i;
            }
        }
        int e0 = 0, e1 = 0, s0 = 0, s1 = 0, B = 0;
        d4 sB = mk4(0.0, 0.0, 0.0, 1.0);
        if (has) {
            const int lo_i = pos;
            B = order[lo_i];
            s0 = seg_start[B];
            s1 = seg_end[B];
            e0 = s0 + (int)(w - (unsigned)item_start[lo_i]) * kM2LChunk;
            e1 = min(e0 + kM2LChunk, s1);
            sB = cen[B];
        }
        double sigma = sB.w;
        if (!(sigma > 0)) {  // radius 0: half the closest source distance (over the whole list)
            double rmin = INFINITY;
            for (int e = s0 + lane; e < s1; e += 32) {
                const d4 zA = cen[m2l_src(list[e].x)];
                const double dx = sB.x - zA.x, dy = sB.y - zA.y, dz = sB.z - zA.z;
                rmin = fmin(rmin, sqrt(dx * dx + dy * dy + dz * dz));
            }
            sigma = 0.5 * warp_min(rmin);
        }
        // the lane's pair: rotation phases e^{-i alpha}, e^{-i beta} and the scale factors
        const int e = e0 + lane;
        const bool act = e < e1;
        const int xe = act ? list[e].x : 0;
        const int A = act ? m2l_src(xe) : -1;
        const int qlane = act ? m2l_order(xe, P) : P;
        float tA = 0.f, tB = 0.f;
        float2 wv = make_float2(1.f, 0.f), uv = make_float2(1.f, 0.f);
        if (act) {  // FP64 differences, then FP32 (the quantities feed FP32 arithmetic only)
            const d4 zA = cen[A];
            const float x = (float)(sB.x - zA.x), y = (float)(sB.y - zA.y), z = (float)(sB.z - zA.z);
            const float rxy2 = x * x + y * y, rxy = sqrtf(rxy2), Rinv = 1.f / sqrtf(rxy2 + z * z);
            if (rxy > 0.f) {
                const float ri = 1.f / rxy;
                wv = make_float2(y * ri, x * ri);
            }
            uv = make_float2(z * Rinv, -rxy * Rinv);
            tA = (float)zA.w * Rinv;
            tB = (float)sigma * Rinv;
        }
        float2 cw[P + 1], cu[P + 1];
        cw[0] = make_float2(1.f, 0.f);
        cu[0] = cw[0];
#pragma unroll
        for (int m = 1; m <= P; ++m) {
            cw[m] = make_float2(cw[m - 1].x * wv.x - cw[m - 1].y * wv.y, cw[m - 1].x * wv.y + cw[m - 1].y * wv.x);
            cu[m] = make_float2(cu[m - 1].x * uv.x - cu[m - 1].y * uv.y, cu[m - 1].x * uv.y + cu[m - 1].y * uv.x);
        }
        // stage the chunk's scaled multipoles, column b = pair b (zeros for missing pairs),
        // by asynchronous copies that complete while the FP64 terms below are summed
        for (int b = 0; b < 32; ++b) {
            const int Ab = __shfl_sync(0xffffffffu, A, b);
            const float* src = Mt + (size_t)(Ab < 0 ? 0 : Ab) * nco_out;  // rows of the global order
            const unsigned nbytes = Ab >= 0 ? 4u : 0u;  // 0: zero fill
            for (int c = lane; c < NCO; c += 32) rot_cp_async4(S + c * kPad + b, src + c, nbytes);
        }
        rot_cp_async_commit();
        // FP64 terms of orders n + k <= kRotJ64, then their sums over the pairs (fixed butterfly)
        cd lo[kRotLow];
#pragma unroll
        for (int i = 0; i < kRotLow; ++i) lo[i] = mkc(0.0, 0.0);
        if (act) {
            const d4 zA = cen[A];
            const double x = sB.x - zA.x, y = sB.y - zA.y, z = sB.z - zA.z;
            const double Rinv = rsqrt(x * x + y * y + z * z);
            cd T[kRotLowM], Mx[kRotLowM];
#pragma unroll
            for (int j = 0; j <= kRotJ64; ++j)
#pragma unroll
                for (int m = 0; m <= j; ++m) {
                    const cd v = theta_low_rot(j, m, x, y, z, Rinv);
                    T[cix(j, m)] = v;
                    if (m) T[cix(j, -m)] = (m & 1) ? mkc(-v.re, v.im) : mkc(v.re, -v.im);
                }
#pragma unroll
            for (int i = 0; i < kRotLowM; ++i) Mx[i] = M64g[(size_t)A * 9 + i];
#pragma unroll
            for (int n = 0; n <= kRotJ64; ++n)
#pragma unroll
                for (int m = 0; m <= n; ++m)
#pragma unroll
                    for (int k = 0; k + n <= kRotJ64; ++k)
#pragma unroll
                        for (int l = -k; l <= k; ++l) cmac(lo[n * (n + 1) / 2 + m], Mx[cix(k, l)], T[cix(n + k, m + l)]);
        }
#pragma unroll
        for (int i = 0; i < kRotLow; ++i) {
            lo[i].re = warp_sum(lo[i].re);
            lo[i].im = warp_sum(lo[i].im);
        }
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < kRotLow; ++i) lowF[i] = lo[i];
        }
        rot_cp_async_wait_all();
        __syncthreads();
        fwd_all<P>(Sl, cw, cu, tA, upto<P>{});
        __syncthreads();
        if (adapt) zm2l_all<P, true>(Sl, qlane, upto<P / 2>{});
        else zm2l_all<P, false>(Sl, P, upto<P / 2>{});
        __syncthreads();
        bwd_all<P>(Sl, cw, cu, tB, upto<P>{});
        warp_pow_table(1.0 / sigma, P + 1, lane, pws);
        __syncwarp();
        if (has) {
            double* out = by_sink ? accF
                          : (s1 - s0 <= kM2LChunk ? args.F + (size_t)B * nco_out : args.part + (size_t)w * nco_out);
            for (int c = lane; c < NCO; c += 32) {
                const float* row = S + c * kPad;
                float s = 0.f;
#pragma unroll 8
                for (int b = 0; b < 32; ++b) s += row[b];
                const int n = (int)sqrtf((float)c), m = c - n * n - n;
                double v = (double)s * c_rot_norm.v[c] * pws[n + 1];
                if (n <= kRotJ64) {
                    const cd lv = lowF[n * (n + 1) / 2 + (m < 0 ? -m : m)];
                    v += m >= 0 ? lv.re : lv.im;
                }
                if (by_sink) out[c] += v;
                else out[c] = v;
            }
            if (by_sink) ++cur_it;
        }
        __syncwarp();
    }
}

}  // namespace

template <int P>
void rot_launch(const RotArgs& args, cudaStream_t s) {
    constexpr int W = rot_warps<P>();
    const size_t sm = (size_t)W * rot_warp_bytes<P>();
    cudaFuncSetAttribute(k_m2l_rot<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int dev = 0, nsm = 152, bps = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_m2l_rot<P>, 32 * W, sm);
    const unsigned g = (unsigned)(nsm * (bps > 0 ? bps : 1));
    k_m2l_rot<P><<<g, 32 * W, sm, s>>>(args);
    note_launch();
}

}  // namespace gb3
