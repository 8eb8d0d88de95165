// Device-side helpers shared by the CUDA translation units: complex amplitude
// types for the packed FP32x2 / FP64 arithmetic, and the mbarrier and bulk-copy
// primitives (inline PTX) with bounded waits.
#pragma once
#include <cuda_runtime.h>

namespace osmps {

constexpr unsigned long long kWaitNs = 2000000000ull;   // bounded waits: 2 s

template <typename T> struct Cx;
// complex64: an amplitude is one 64-bit register pair {re, im} used directly by
// the packed FP32x2 instructions; a 16-byte vector holds two amplitudes.
template <> struct Cx<float> {
    typedef ulonglong2 v16;
    typedef unsigned long long amp;
    typedef unsigned long long coef;   // {f, f}
    static constexpr int VE = 2;       // amplitudes per 16-byte vector
    static constexpr int LOGVE = 1;
};
// complex128: one amplitude per 16-byte vector, FP64 arithmetic
template <> struct Cx<double> {
    typedef double2 v16;
    typedef double2 amp;
    typedef double coef;
    static constexpr int VE = 1;
    static constexpr int LOGVE = 0;
};

__device__ __forceinline__ void unpackv(const ulonglong2 &v, unsigned long long *a) {
    a[0] = v.x;
    a[1] = v.y;
}
__device__ __forceinline__ ulonglong2 packv(const unsigned long long *a) { return make_ulonglong2(a[0], a[1]); }
__device__ __forceinline__ void unpackv(const double2 &v, double2 *a) { a[0] = v; }
__device__ __forceinline__ double2 packv(const double2 *a) { return a[0]; }

__device__ __forceinline__ unsigned long long mkcoef(float f) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(f));
    return r;
}
__device__ __forceinline__ double mkcoef(double f) { return f; }
__device__ __forceinline__ unsigned long long azero(float) { return 0ull; }
__device__ __forceinline__ double2 azero(double) { return make_double2(0.0, 0.0); }

// acc += f * x on complex amplitudes (f real): one fma.rn.f32x2, or two FP64 FMAs
__device__ __forceinline__ void afma(unsigned long long f, unsigned long long x, unsigned long long &acc) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(f), "l"(x));
}
__device__ __forceinline__ void afma(double f, const double2 &x, double2 &acc) {
    acc.x = fma(f, x.x, acc.x);
    acc.y = fma(f, x.y, acc.y);
}
// a *= f
__device__ __forceinline__ void amul(unsigned long long f, unsigned long long &a) {
    asm("mul.rn.f32x2 %0, %1, %0;" : "+l"(a) : "l"(f));
}
__device__ __forceinline__ void amul(double f, double2 &a) {
    a.x *= f;
    a.y *= f;
}
__device__ __forceinline__ float2 tocx(unsigned long long a) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a));
    return r;
}
__device__ __forceinline__ double2 tocx(const double2 &a) { return a; }

// fixed-order sum of partials[i*stride + k], i < n, done by one warp (every lane
// returns the sum; the same order in every CTA and kernel that calls it)
static __device__ __forceinline__ double warp_sum_partials(const double *partials, int n, int stride, int k) {
    double s = 0.0;
    for (int i = threadIdx.x & 31; i < n; i += 32) s += partials[(size_t)i * stride + k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    return s;
}

// ---- complex128 flip sums in 64-bit fixed point ----
// All amplitudes of a tile go on one grid of unit 2^(et - 1080), et the largest
// biased FP64 exponent in the tile, so every |X| < 2^58 and the sum of a
// partner per flipped bit (at most 12) is exact in 64-bit integers.  Onto the
// grid by integer operations; back by one conversion, the unit folded into the
// field: the FP64 pipe (2 lanes per clock per SM on this part) is left to the
// diagonal, the partial sum and the epilogue.
static __device__ __forceinline__ unsigned fx_expo(double x) {
    return (unsigned)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFu;
}
// x on the grid, truncated toward zero (error below one unit, i.e. below
// 2^-57 of the tile's largest magnitude); zero and subnormals give 0
static __device__ __forceinline__ long long fx_from(double x, int et) {
    const long long b = __double_as_longlong(x);
    const int e = (int)(((unsigned long long)b >> 52) & 0x7FFull);
    const unsigned long long M = (((unsigned long long)b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull) << 5;
    const int sh = et - e;  // >= 0
    unsigned long long a = sh < 64 ? (M >> sh) : 0ull;
    if (e == 0) a = 0ull;
    const long long sg = b >> 63;  // 0 or -1
    return ((long long)a ^ sg) - sg;
}
// the field times the grid unit: one FP64 multiply per value turns an integer
// sum (converted with rounding to nearest) into its term; tiles whose largest
// magnitude is under 2^-960 get 0, a non-finite amplitude in the tile NaN
static __device__ __forceinline__ double fx_scale(double h, int et) {
    if (et >= 2047) return __longlong_as_double(0x7FF8000000000000ll);
    if (et <= 57) return 0.0;
    return h * __longlong_as_double((long long)(et - 57) << 52);
}

// ---- mbarrier / TMA primitives (PTX) ----
__device__ __forceinline__ unsigned smem_u32(const void *ptr) { return (unsigned)__cvta_generic_to_shared(ptr); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of the given parity.  try_wait itself suspends the
// thread for a while; the timer (and the error flag raised by another warp)
// is consulted only every 64 polls, so a completed phase is seen at once.
// Gives up after limit_ns (kWaitNs for the kernels of this library).
static __device__ __noinline__ bool mbar_wait_ns(unsigned long long *bar, unsigned parity, const int *err,
                                                 unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0) {
            if (*(volatile const int *)err != 0) return false;
            if (global_ns() - t0 > limit_ns) return false;
        }
    }
}
static __device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, const int *err) {
    return mbar_wait_ns(bar, parity, err, kWaitNs);
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

}  // namespace osmps
