// Two-site reduced density matrices of every pair of sites (Sec. IV: reduced
// density matrices of a pure state by tracing out the rest of the rank-L
// tensor), i.e. every two-point Pauli correlator <s^a_i s^b_j>.
//
//   rho_ij[v'][v] = sum_rest psi(v', rest) conj(psi(v, rest)),  v = 2 sigma_i + sigma_j,
//
// One launch covers all L(L-1)/2 pairs (blockIdx.y = pair).  A thread takes
// groups of the four amplitudes that differ only in the pair's two bits (the
// group index with two zero bits inserted) and accumulates the Hermitian
// 4 x 4 outer product x x^H: 4 real diagonal and 6 complex upper entries,
// compensated sums in the working precision per thread, FP64 across threads
// and blocks (fixed order).
#include <cuda_runtime.h>

#include "ed_internal.h"

namespace osmps {
namespace rdm {

constexpr int kRdmThreads = 256;
constexpr int kRdmBlocks = 48;  // blocks per pair
constexpr int kRdmVals = 16;    // 4 diagonal + 6 (re, im) upper entries
constexpr int kRdmBatch = 4;    // amplitude quadruples loaded together per thread
constexpr int kRdmRuns = 4;     // batches summed in FP32 before the FP64 accumulators

template <typename T> struct Cr;
template <> struct Cr<float> { typedef float2 C; };
template <> struct Cr<double> { typedef double2 C; };

// pair index p -> sites (i, j), 1 <= i < j <= L, row-major (1,2), (1,3), ..., (L-1, L)
__device__ __forceinline__ void pair_sites(int p, int L, int &i, int &j) {
    i = 1;
    while (p >= L - i) {
        p -= L - i;
        ++i;
    }
    j = i + 1 + p;
}

template <typename T>
__global__ void __launch_bounds__(kRdmThreads, sizeof(T) == 4 ? 2 : 1) pair_rdm_kernel(const typename Cr<T>::C *psi, int L, double *partials) {
    typedef typename Cr<T>::C C;
    int si, sj;
    pair_sites(blockIdx.y, L, si, sj);
    const int bh = L - si, bl = L - sj;  // bit of site i (higher) and of site j
    const uint64_t ngroups = (1ull << L) >> 2;
    const uint64_t mlo = (1ull << bl) - 1ull;          // bits below bl
    const uint64_t mmid = ((1ull << (bh - 1)) - 1ull) & ~mlo;  // group bits that land between bl and bh
    // per-thread sums: compensated (Kahan) in the working precision, so that
    // the long per-thread runs keep full accuracy without FP64 work in the
    // loop (the FP64 pipe of this part is narrow); FP64 from the thread sums on
    T acc[kRdmVals], comp[kRdmVals];
#pragma unroll
    for (int q = 0; q < kRdmVals; ++q) acc[q] = comp[q] = (T)0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // kRdmBatch groups are loaded at once (independent loads in flight),
    // kRdmRuns batches are summed plainly, then added to the compensated sums
    for (uint64_t g0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g0 < ngroups;
         g0 += (uint64_t)kRdmRuns * kRdmBatch * stride) {
        T a[kRdmVals];
#pragma unroll
        for (int q = 0; q < kRdmVals; ++q) a[q] = (T)0;
#pragma unroll
        for (int run = 0; run < kRdmRuns; ++run) {
            C x[kRdmBatch][4];
#pragma unroll
            for (int rr = 0; rr < kRdmBatch; ++rr) {
                const uint64_t g = g0 + (uint64_t)(run * kRdmBatch + rr) * stride;
                // insert zero bits at bl and bh
                const uint64_t base = (g & mlo) | ((g & mmid) << 1) | ((g & ~(mlo | mmid)) << 2);
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    x[rr][v].x = (T)0;
                    x[rr][v].y = (T)0;
                    if (g < ngroups) x[rr][v] = psi[base | ((uint64_t)(v >> 1) << bh) | ((uint64_t)(v & 1) << bl)];
                }
            }
#pragma unroll
            for (int rr = 0; rr < kRdmBatch; ++rr) {
#pragma unroll
                for (int v = 0; v < 4; ++v) a[v] += x[rr][v].x * x[rr][v].x + x[rr][v].y * x[rr][v].y;
                int q = 4;
#pragma unroll
                for (int v1 = 0; v1 < 4; ++v1)
#pragma unroll
                    for (int v2 = v1 + 1; v2 < 4; ++v2) {  // x[v1] conj(x[v2])
                        a[q] += x[rr][v1].x * x[rr][v2].x + x[rr][v1].y * x[rr][v2].y;
                        a[q + 1] += x[rr][v1].y * x[rr][v2].x - x[rr][v1].x * x[rr][v2].y;
                        q += 2;
                    }
            }
        }
#pragma unroll
        for (int q = 0; q < kRdmVals; ++q) {
            const T y = a[q] - comp[q];
            const T t = acc[q] + y;
            comp[q] = (t - acc[q]) - y;
            acc[q] = t;
        }
    }
    __shared__ double red[kRdmVals][kRdmThreads / 32];
#pragma unroll
    for (int q = 0; q < kRdmVals; ++q) {
        double v = (double)acc[q] - (double)comp[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < kRdmVals) {
        double s = 0.0;
        for (int w = 0; w < kRdmThreads / 32; ++w) s += red[threadIdx.x][w];
        partials[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kRdmVals + threadIdx.x] = s;
    }
}

// out[p][q] = sum over the blocks of pair p (fixed order)
__global__ void pair_rdm_finish_kernel(const double *partials, int nblocks, int npairs, double *out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npairs * kRdmVals) return;
    const int p = t / kRdmVals, q = t % kRdmVals;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[((size_t)p * nblocks + b) * kRdmVals + q];
    out[t] = s;
}

}  // namespace rdm

// 16 reals per pair into out_dev (device, npairs x 16): diag |.|^2 for v = 0..3,
// then x[v1] conj(x[v2]) (re, im) for (v1, v2) = (0,1), (0,2), (0,3), (1,2), (1,3), (2,3).
// scratch_dev: npairs * kRdmBlocks * 16 doubles.
cudaError_t launch_pair_rdm(Handle *h, const void *psi, double *scratch_dev, double *out_dev) {
    using namespace rdm;
    const int L = h->L;
    const int npairs = L * (L - 1) / 2;
    const dim3 grid(kRdmBlocks, npairs);
    if (h->prec == OSMPS_FP64)
        pair_rdm_kernel<double><<<grid, kRdmThreads, 0, h->stream>>>((const double2 *)psi, L, scratch_dev);
    else
        pair_rdm_kernel<float><<<grid, kRdmThreads, 0, h->stream>>>((const float2 *)psi, L, scratch_dev);
    pair_rdm_finish_kernel<<<(npairs * kRdmVals + 255) / 256, 256, 0, h->stream>>>(scratch_dev, kRdmBlocks, npairs,
                                                                                     out_dev);
    h->launches += 2;
    return cudaGetLastError();
}

size_t pair_rdm_scratch_doubles(int L) { return (size_t)(L * (L - 1) / 2) * (rdm::kRdmBlocks + 1) * rdm::kRdmVals; }

}  // namespace osmps
