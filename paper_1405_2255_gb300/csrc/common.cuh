// common.cuh -- shared device types and helpers of the GB300 FMM library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "../../include/gb3fmm.h"

namespace gb3 {

// Run an initialisation (an upload of __constant__ tables, which every device holds
// separately) once per device, safely from several host threads.
struct DeviceOnce {
    std::mutex m;
    unsigned long long done = 0;
};
template <class F>
inline void once_per_device(DeviceOnce& o, F&& init) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(o.m);
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (o.done & bit) return;
    init();
    o.done |= bit;
}

constexpr int kMaxP = 20;        // largest expansion order supported (p <= 20, Sec. 6.1)
constexpr int kMaxLevel = 21;    // 21 bits per axis in a 63-bit Morton key
constexpr int kWarp = 32;

__host__ __device__ inline int ncoef(int p) { return (p + 1) * (p + 1); }
// index of (n, m), -n <= m <= n, in a (p+1)^2 array of real or complex coefficients
__host__ __device__ inline int cix(int n, int m) { return n * n + n + m; }

// t[k] = x^k for k = 0..n (n < 32), lane k forming its power by repeated products (the
// rounding of a serial loop); the caller synchronises the warp before reading t
__device__ inline void warp_pow_table(double x, int n, int lane, double* t) {
    if (lane <= n) {
        double v = 1.0;
        for (int k = 0; k < lane; ++k) v *= x;
        t[lane] = v;
    }
}

// device status word bits (OR-ed by kernels, read by the host)
enum : unsigned {
    kStatInvalid = 1u,      // NaN/Inf position or negative mass
    kStatOverflow = 2u,     // a list or frontier capacity was exceeded
    kStatMeb = 4u,          // a smallest-ball computation found no valid support set
};

// 32-byte aligned quadruple of doubles (one 256-bit load)
struct __align__(32) d4 {
    double x, y, z, w;
};
__host__ __device__ inline d4 mk4(double x, double y, double z, double w) { return d4{x, y, z, w}; }

// ---------------------------------------------------------------- complex FP64
struct cd {
    double re, im;
};
__host__ __device__ inline cd mkc(double r, double i) { return cd{r, i}; }
__host__ __device__ inline cd operator+(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
__host__ __device__ inline cd operator-(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
__host__ __device__ inline cd operator*(cd a, cd b) {
    return cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ inline cd operator*(double s, cd a) { return cd{s * a.re, s * a.im}; }
__host__ __device__ inline cd conjc(cd a) { return cd{a.re, -a.im}; }
// a += x * y
__host__ __device__ inline void cmac(cd& a, cd x, cd y) {
    a.re = fma(x.re, y.re, a.re);
    a.re = fma(-x.im, y.im, a.re);
    a.im = fma(x.re, y.im, a.im);
    a.im = fma(x.im, y.re, a.im);
}

// Real storage of (p+1)^2 coefficients (App. A.3.2): slot cix(n, m) holds
// Re X_n^m for m >= 0 and Im X_n^{|m|} for m < 0.  Complex values for any m
// follow from the symmetry X_n^{-m} = (-1)^m conj(X_n^m).
__host__ __device__ inline cd load_real_storage(const double* R, int n, int m) {
    int am = m < 0 ? -m : m;
    cd v = cd{R[cix(n, am)], am ? R[cix(n, -am)] : 0.0};
    if (m < 0) {
        v.im = -v.im;
        if (am & 1) { v.re = -v.re; v.im = -v.im; }
    }
    return v;
}

// ---------------------------------------------------------------- error helpers
#define GB3_CUDA_TRY(expr)                                                          \
    do {                                                                            \
        cudaError_t _e = (expr);                                                    \
        if (_e != cudaSuccess) return ::gb3::cuda_fail(_e, #expr, __FILE__, __LINE__); \
    } while (0)

int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

// count of kernels launched by this host thread (reported in fmm_stats.launches)
void note_launch();
long long launches_so_far();

// kernel marks: while a pair of events is set for this host thread, the launchers of the
// main P2P and M2L kernels record the first event right before the kernel and the second
// right after it, so that the kernel's own device time can be read; nullptr turns it off
void kernel_marks(cudaEvent_t* ev);
void mark_begin(cudaStream_t s);
void mark_end(cudaStream_t s);
bool marks_recorded();  // both events were recorded since the last kernel_marks()

// a length on a logarithmic scale of eight steps per octave, 0 for 0 and 1..255 otherwise:
// sort keys of work lists ordered longest first (one 8-bit radix pass instead of one per byte
// of the exact length; the order within a step stays that of the indices)
__host__ __device__ inline unsigned qlen8(unsigned len) {
    if (len == 0) return 0;
    int lg = 31;
    while (!(len >> lg)) --lg;                                 // floor(log2 len)
    const unsigned frac = lg >= 3 ? (len >> (lg - 3)) & 7u : (len << (3 - lg)) & 7u;
    const unsigned q = 1u + 8u * (unsigned)lg + frac;          // 1 .. 256
    return q > 255u ? 255u : q;
}

// streaming multiprocessors of the current device (queried once per device)
int sm_count();

// blocks for n items of `block` threads, at most per_sm blocks per SM (grid-stride loops)
inline unsigned grid_for(long long n, int block, int per_sm = 64) {
    long long g = (n + block - 1) / block;
    const long long cap = (long long)sm_count() * per_sm;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

// ---------------------------------------------------------------- scans
// Exclusive prefix sum of n int32 values (device) into out (device); the total is
// written to *d_total (device) when not NULL.  tmp must hold scan_tmp_ints(n) ints.
size_t scan_tmp_ints(long long n);
void scan_exclusive_i32(const int* in, int* out, long long n, int* d_total, int* tmp, cudaStream_t s);

// ---------------------------------------------------------------- warp helpers
__device__ inline double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ inline double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ---------------------------------------------------------------- two-float sums
// (hi, lo) with hi + lo the sum to about 2^-48 relative: TwoSum (Knuth) of the running sum
// and each FP32 partial, in explicit round-to-nearest operations
struct ff {
    float hi, lo;
};
__device__ inline ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff{s, e};
}
__device__ inline void ff_add_shfl(ff& a, int o) {
    float h = __shfl_xor_sync(0xffffffffu, a.hi, o), l = __shfl_xor_sync(0xffffffffu, a.lo, o);
    ff s = two_sum(a.hi, h);
    float lo = __fadd_rn(__fadd_rn(a.lo, l), s.lo);
    a.hi = __fadd_rn(s.hi, lo);
    a.lo = __fsub_rn(lo, __fsub_rn(a.hi, s.hi));
}
// a += the (hi, lo) of lane src
__device__ inline void ff_add_lane(ff& a, int src) {
    float h = __shfl_sync(0xffffffffu, a.hi, src), l = __shfl_sync(0xffffffffu, a.lo, src);
    ff s = two_sum(a.hi, h);
    float lo = __fadd_rn(__fadd_rn(a.lo, l), s.lo);
    a.hi = __fadd_rn(s.hi, lo);
    a.lo = __fsub_rn(lo, __fsub_rn(a.hi, s.hi));
}
__device__ inline void ff_acc(ff& a, float v) {
    ff s = two_sum(a.hi, v);
    float lo = __fadd_rn(a.lo, s.lo);
    a.hi = __fadd_rn(s.hi, lo);
    a.lo = __fsub_rn(lo, __fsub_rn(a.hi, s.hi));
}

// 1/sqrt(x) by the hardware approximation with subnormal inputs flushed to zero (an x below
// 2^-126 would be a pair closer than 1e-19 in the working units); the non-flushing form spends
// extra instructions per call on rescaling such inputs
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 2^k as a double for |k| <= 1022, from its bits (exact)
__device__ inline double pow2i(int k) {
    k = k < -1022 ? -1022 : (k > 1023 ? 1023 : k);
    return __longlong_as_double((long long)(k + 1023) << 52);
}

// order-preserving map of a double to uint64 (for atomicMin/atomicMax on doubles)
__device__ inline unsigned long long dbl_key(double d) {
    unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ inline double key_dbl(unsigned long long k) {
    unsigned long long u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)u);
}
__host__ inline double key_dbl_host(unsigned long long k) {
    unsigned long long u = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
    double d;
    memcpy(&d, &u, sizeof d);
    return d;
}

}  // namespace gb3
