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
