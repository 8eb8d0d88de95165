// Measurements of a pure state (Sec. IV):
//   * <sz_k> and <sz_i sz_j> from p_b = |psi_b|^2 in one streaming pass,
//   * the half-chain reduced density matrix rho = M M^dagger (bond entropy)
//     and its spectrum, S = -sum_j Lambda_j ln Lambda_j.
//
// Correlators: with b = (hi, lo) split at t low bits, per tile of fixed hi the
// CTA forms P(hi) = sum_lo p and M_j(hi) = sum_lo s_j(lo) p (j < t).  Then
//   <sz_i sz_i'> (both high) = sum_hi s_i s_i' P,   <sz_i sz_j> = sum_hi s_i M_j,
//   <sz_j sz_j'> (both low)  = sum_lo s_j s_j' G(lo),  G(lo) = sum_hi p(hi, lo),
// so every amplitude costs O(1) FP64 work while the L^2 outputs are updated
// once per tile.  All sums are FP64 in a fixed order.
#include <cuda_runtime.h>
#include <cublas_v2.h>  // types and prototypes only: the library is loaded at first use
#include <cusolverDn.h>
#include <dlfcn.h>
#include <math.h>

#include <cmath>

#include <mutex>
#include <vector>

#include "ed_internal.h"

namespace osmps {

constexpr int kZThreads = 256;
constexpr int kZTileBits = 12;                  // 4096 amplitudes per tile
constexpr int kZPer = (1 << kZTileBits) / kZThreads;  // amplitudes per thread (16)

template <typename T> struct ZV;
template <> struct ZV<float> {
    typedef float2 c;
};
template <> struct ZV<double> {
    typedef double2 c;
};

// number of per-CTA accumulators: C (L*L) + m (L) + total
__host__ __device__ inline int zacc_count(int L) { return L * L + L + 1; }

// One streaming pass over p_b = |psi_b|^2.  Per thread: 16 amplitudes at
// li = tid + 256 k; sums over a thread and warp in T (FP32 in mixed mode),
// across warps, tiles and CTAs in FP64.  The low-bit marginal G(lo) runs over
// every tile a CTA visits (thousands at L = 30 on a small grid), so in FP32 it
// is a compensated (Kahan) sum: its error stays at a few units of FP32
// rounding of G instead of growing with the number of tiles.
template <typename T>
__global__ void __launch_bounds__(kZThreads) zstats_kernel(const typename ZV<T>::c *psi, int L, int t,
                                                           long long ntiles, double *blockacc, double *Gpart) {
    const int nel = 1 << t;
    const int nacc = zacc_count(L);
    const int nown = (nacc + kZThreads - 1) / kZThreads;  // <= 4 for L <= 30
    double own[4] = {0, 0, 0, 0};
    T G[kZPer], Gc[kZPer];  // running marginal and its Kahan compensation (unused in FP64)
#pragma unroll
    for (int k = 0; k < kZPer; ++k) G[k] = Gc[k] = (T)0;
    __shared__ double red[kZTileBits + 1][kZThreads / 32];
    __shared__ double stat[kZTileBits + 1];  // P, M_0..M_{t-1}
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t base = (uint64_t)tile << t;
        T pk[kZPer];
#pragma unroll
        for (int k = 0; k < kZPer; ++k) {
            const int li = threadIdx.x + k * kZThreads;
            T pv = (T)0;
            if (li < nel) {
                const typename ZV<T>::c a = __ldcs(&psi[base + li]);
                pv = a.x * a.x + a.y * a.y;
            }
            pk[k] = pv;
            if (sizeof(T) == sizeof(float)) {
                const T y = pv - Gc[k];
                const T tsum = G[k] + y;
                Gc[k] = (tsum - G[k]) - y;
                G[k] = tsum;
            } else {
                G[k] += pv;
            }
        }
        // per-thread moments: v[0] = sum p, v[1+j] = sum s_j p
        T v[kZTileBits + 1];
        T Pt = (T)0;
#pragma unroll
        for (int k = 0; k < kZPer; ++k) Pt += pk[k];
        v[0] = Pt;
#pragma unroll
        for (int j = 0; j < 8; ++j) v[1 + j] = ((threadIdx.x >> j) & 1) ? -Pt : Pt;
#pragma unroll
        for (int j = 8; j < kZTileBits; ++j) {
            T s = (T)0;
#pragma unroll
            for (int k = 0; k < kZPer; ++k) s += (((k << 8) >> j) & 1) ? -pk[k] : pk[k];
            v[1 + j] = s;
        }
#pragma unroll
        for (int j = 0; j <= kZTileBits; ++j) {
            T x = v[j];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
            if (lane == 0) red[j][wid] = (double)x;
        }
        __syncthreads();
        if (threadIdx.x <= t) {
            double sacc = 0.0;
            for (int w = 0; w < kZThreads / 32; ++w) sacc += red[threadIdx.x][w];
            stat[threadIdx.x] = sacc;
        }
        __syncthreads();
        const double P = stat[0];
        for (int k = 0; k < nown; ++k) {
            const int e = threadIdx.x + k * kZThreads;
            if (e >= nacc) break;
            double add = 0.0;
            if (e < L * L) {
                const int i = e / L, j = e % L;  // bit indices
                if (i >= t && j >= t) {
                    const int si = 1 - 2 * (int)((tile >> (i - t)) & 1);
                    const int sj = 1 - 2 * (int)((tile >> (j - t)) & 1);
                    add = (double)(si * sj) * P;
                } else if (i >= t && j < t) {
                    const int si = 1 - 2 * (int)((tile >> (i - t)) & 1);
                    add = (double)si * stat[1 + j];
                } else if (i < t && j >= t) {
                    const int sj = 1 - 2 * (int)((tile >> (j - t)) & 1);
                    add = (double)sj * stat[1 + i];
                }
            } else if (e < L * L + L) {
                const int i = e - L * L;
                if (i >= t) {
                    const int si = 1 - 2 * (int)((tile >> (i - t)) & 1);
                    add = (double)si * P;
                } else {
                    add = stat[1 + i];
                }
            } else {
                add = P;
            }
            own[k] += add;
        }
        __syncthreads();
    }
    for (int k = 0; k < nown; ++k) {
        const int e = threadIdx.x + k * kZThreads;
        if (e < nacc) blockacc[(size_t)blockIdx.x * nacc + e] = own[k];
    }
#pragma unroll
    for (int k = 0; k < kZPer; ++k) {
        const int li = threadIdx.x + k * kZThreads;
        if (li < nel) Gpart[(size_t)blockIdx.x * nel + li] = (double)G[k] - (double)Gc[k];
    }
}

// Sum the per-CTA partials in a fixed order, one warp per entry:
// red[0..nacc) accumulators, red[nacc..nacc+nel) the low-bit marginal G.
__global__ void zstats_reduce_kernel(const double *blockacc, const double *Gpart, int nblk, int nacc, int nel,
                                     double *red) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= nacc + nel) return;
    double s = 0.0;
    if (w < nacc) {
        for (int b = lane; b < nblk; b += 32) s += blockacc[(size_t)b * nacc + w];
    } else {
        const int li = w - nacc;
        for (int b = lane; b < nblk; b += 32) s += Gpart[(size_t)b * nel + li];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) red[w] = s;
}

// Outputs in site order, one warp per output: out[0..L) = <sz_k>,
// out[L..L+L*L) = <sz_i sz_j>.
__global__ void zstats_assemble_kernel(const double *red, int L, int t, double *out) {
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= L + L * L) return;
    const int nacc = zacc_count(L);
    const int nel = 1 << t;
    double s = 0.0;
    if (w < L) {
        const int bit = L - (w + 1);
        s = red[L * L + bit];
    } else {
        const int q = w - L;
        const int bi = L - (q / L + 1), bj = L - (q % L + 1);
        if (bi == bj) {
            s = red[L * L + L];
        } else if (bi < t && bj < t) {
            double part = 0.0;
            for (int lo = lane; lo < nel; lo += 32) {
                const int sg = (((lo >> bi) ^ (lo >> bj)) & 1) ? -1 : 1;
                part += (double)sg * red[nacc + lo];
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            s = part;
        } else {
            s = red[bi * L + bj];
        }
    }
    if (lane == 0) out[w] = s;
}

template <typename T>
static cudaError_t zstats_t(Handle *h, const void *psi, double *out_dev) {
    const int L = h->L;
    const int t = L < kZTileBits ? L : kZTileBits;
    const long long ntiles = 1ll << (L - t);
    long long cap = (long long)h->nsm * 4;
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    const int nacc = zacc_count(L), nel = 1 << t;
    const size_t need = (size_t)grid * (nacc + nel) + nacc + nel;
    if (need > h->partials2_cap) return cudaErrorMemoryAllocation;
    double *blockacc = h->partials2;
    double *Gpart = h->partials2 + (size_t)grid * nacc;
    double *red = Gpart + (size_t)grid * nel;
    zstats_kernel<T><<<grid, kZThreads, 0, h->stream>>>(reinterpret_cast<const typename ZV<T>::c *>(psi), L, t,
                                                         ntiles, blockacc, Gpart);
    const int nw1 = nacc + nel;
    zstats_reduce_kernel<<<(nw1 + 7) / 8, 256, 0, h->stream>>>(blockacc, Gpart, grid, nacc, nel, red);
    const int nw2 = L + L * L;
    zstats_assemble_kernel<<<(nw2 + 7) / 8, 256, 0, h->stream>>>(red, L, t, out_dev);
    h->launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_zstats(Handle *h, const void *psi, double *out_dev) {
    return h->prec == OSMPS_FP64 ? zstats_t<double>(h, psi, out_dev) : zstats_t<float>(h, psi, out_dev);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the measurement pass.
//
// Its per-CTA partial sums live in one file-scope device array instead of
// handle-owned memory.  Every GPU that loads this library holds the array
// (kNoAllocScratch doubles, 3.75 MiB) until the process exits.  Host code must
// not pass the array's name to a kernel (on the host it is only a stand-in
// symbol); the device address is looked up once per device with
// cudaGetSymbolAddress and cached.
// ---------------------------------------------------------------------------
constexpr int kNoAllocGrid = 96;  // CTAs of the measurement pass
constexpr size_t kNoAllocScratch = 491520;  // >= 96 * (931 + 4096) + 931 + 4096 for L <= 30
static_assert((size_t)kNoAllocGrid * (30 * 30 + 30 + 1 + (1u << kZTileBits)) + 30 * 30 + 30 + 1 +
                      (1u << kZTileBits) <=
                  kNoAllocScratch,
              "scratch too small for L = 30");
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

static std::mutex g_noalloc_mutex;
static double *g_noalloc_ptr[128];  // device address of g_noalloc_scratch per device ordinal

template <typename T>
static cudaError_t zstats_noalloc_t(int L, const void *psi, double *out_dev, double *scratch, cudaStream_t st) {
    const int t = L < kZTileBits ? L : kZTileBits;
    const long long ntiles = 1ll << (L - t);
    const int grid = (int)(ntiles < kNoAllocGrid ? ntiles : kNoAllocGrid);
    const int nacc = zacc_count(L), nel = 1 << t;
    double *blockacc = scratch;
    double *Gpart = scratch + (size_t)grid * nacc;
    double *red = Gpart + (size_t)grid * nel;
    zstats_kernel<T><<<grid, kZThreads, 0, st>>>(reinterpret_cast<const typename ZV<T>::c *>(psi), L, t, ntiles,
                                                  blockacc, Gpart);
    const int nw1 = nacc + nel;
    zstats_reduce_kernel<<<(nw1 + 7) / 8, 256, 0, st>>>(blockacc, Gpart, grid, nacc, nel, red);
    const int nw2 = L + L * L;
    zstats_assemble_kernel<<<(nw2 + 7) / 8, 256, 0, st>>>(red, L, t, out_dev);
    return cudaGetLastError();
}

}  // namespace osmps

extern "C" osmps_status osmps_ed_measure_zz_noalloc(int L, int prec, const void *psi, double *out_dev,
                                                    void *cuda_stream) {
    using namespace osmps;
    if (L < 1 || L > OSMPS_MAX_L) return OSMPS_EINVAL;
    if (prec != OSMPS_FP64 && prec != OSMPS_MIXED) return OSMPS_EINVAL;
    if (psi == nullptr || out_dev == nullptr || ((uintptr_t)psi & 15u) != 0 || ((uintptr_t)out_dev & 7u) != 0)
        return OSMPS_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        cudaGetLastError();
        return OSMPS_ECUDA;
    }
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (g_noalloc_ptr[dev] == nullptr) {
            void *addr = nullptr;
            if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || addr == nullptr) {
                cudaGetLastError();
                return OSMPS_ECUDA;
            }
            g_noalloc_ptr[dev] = (double *)addr;
        }
        scratch = g_noalloc_ptr[dev];
    }
    cudaError_t err = (prec == OSMPS_FP64)
                          ? zstats_noalloc_t<double>(L, psi, out_dev, scratch, (cudaStream_t)cuda_stream)
                          : zstats_noalloc_t<float>(L, psi, out_dev, scratch, (cudaStream_t)cuda_stream);
    return err == cudaSuccess ? OSMPS_OK : OSMPS_ECUDA;
}

namespace osmps {

// ---------------------------------------------------------------------------
// Gram product rho[x][y] = sum_k A[x,k] conj(A[y,k]),  A[x,k] = psi[x*sx + k*sk]
// (half-chain reduced density matrix, Sec. IV bond entropy).  Tiled on CUDA
// cores: 64x64 output tile per CTA, 16-deep K slices staged in shared memory,
// 4x4 complex outputs per thread.
// ---------------------------------------------------------------------------
constexpr int kGT = 64, kGK = 16;

// Split K (blockIdx.z = split): split z sums k in [z*kchunk, min(K, (z+1)*kchunk))
// into its own n x n slice of rho (slices summed afterwards in a fixed order).
template <typename T>
__global__ void __launch_bounds__(256) gram_kernel(const typename ZV<T>::c *psi, int n, long long K, long long sx,
                                                   long long sk, long long kchunk, typename ZV<T>::c *rho) {
    typedef typename ZV<T>::c C;
    __shared__ C As[kGK][kGT + 1];
    __shared__ C Bs[kGK][kGT + 1];
    const int x0 = blockIdx.y * kGT, y0 = blockIdx.x * kGT;
    const long long kbeg = (long long)blockIdx.z * kchunk;
    const long long kend = kbeg + kchunk < K ? kbeg + kchunk : K;
    rho += (size_t)blockIdx.z * n * n;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T accr[4][4], acci[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) accr[i][j] = acci[i][j] = (T)0;
    for (long long k0 = kbeg; k0 < kend; k0 += kGK) {
        // load 64 x 16 slices of rows x0.. and y0..
        for (int idx = threadIdx.x; idx < kGT * kGK; idx += 256) {
            int r, kk;
            if (sk == 1) {  // contiguous along k: vary k fastest
                r = idx / kGK;
                kk = idx % kGK;
            } else {        // contiguous along rows
                kk = idx / kGT;
                r = idx % kGT;
            }
            const long long k = k0 + kk;
            C a = C{(T)0, (T)0}, b = C{(T)0, (T)0};
            if (k < kend) {
                if (x0 + r < n) a = psi[(long long)(x0 + r) * sx + k * sk];
                if (y0 + r < n) b = psi[(long long)(y0 + r) * sx + k * sk];
            }
            As[kk][r] = a;
            Bs[kk][r] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            C a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // a * conj(b)
                    accr[i][j] = fma(a[i].x, b[j].x, fma(a[i].y, b[j].y, accr[i][j]));
                    acci[i][j] = fma(a[i].y, b[j].x, fma(-a[i].x, b[j].y, acci[i][j]));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int x = x0 + ty + 16 * i, y = y0 + tx + 16 * j;
            if (x < n && y < n) rho[(size_t)x * n + y] = C{accr[i][j], acci[i][j]};
        }
}

// rho = sum over the nsplit slices of part (fixed order, FP64 accumulation)
template <typename T>
__global__ void gram_split_sum_kernel(const typename ZV<T>::c *part, int nsplit, size_t nn, typename ZV<T>::c *rho) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int z = 0; z < nsplit; ++z) {
            const typename ZV<T>::c v = part[(size_t)z * nn + i];
            re += (double)v.x;
            im += (double)v.y;
        }
        rho[i] = typename ZV<T>::c{(T)re, (T)im};
    }
}

cudaError_t launch_gram(Handle *h, const void *psi, int cut, void *rho, int *n_out) {
    const int L = h->L;
    const int l = cut;
    int n;
    long long K, sx, sk;
    if (l <= L - l) {
        n = 1 << l;
        K = 1ll << (L - l);
        sx = K;
        sk = 1;
    } else {
        n = 1 << (L - l);
        K = 1ll << l;
        sx = 1;
        sk = n;
    }
    *n_out = n;
    // tensor cores (tcgen05, 3xTF32) for complex64 rows; CUDA cores otherwise
    const bool tc_ok = (h->prec == OSMPS_MIXED) && (sk == 1) && gram_tc_supported(n, K);
    if (h->gram_mode == 2 && !tc_ok) return cudaErrorNotSupported;
    if (tc_ok && h->gram_mode != 1) {
        const size_t need = sizeof(float) * ((size_t)n * 4 * (size_t)K + (size_t)n * n);
        if (need > h->gram_aux_bytes) {
            dev_free(h, h->gram_aux, h->gram_aux_bytes);
            h->gram_aux = nullptr;
            h->gram_aux_bytes = 0;
            cudaError_t err;
            h->gram_aux = dev_alloc(h, need, &err);
            if (err != cudaSuccess) return err;
            h->gram_aux_bytes = need;
        }
        float *planes = (float *)h->gram_aux;
        float *G = planes + (size_t)n * 4 * (size_t)K;
        return gram_tc_launch(h, psi, n, K, rho, planes, G);
    }
    // few output tiles (small n, long K): split K so that the grid fills the GPU
    const long long tiles = (long long)((n + kGT - 1) / kGT) * ((n + kGT - 1) / kGT);
    long long nsplit = (4ll * h->nsm + tiles - 1) / tiles;
    if (nsplit > K / 1024) nsplit = K / 1024;
    if (nsplit < 1) nsplit = 1;
    const long long kchunk = ((K + nsplit - 1) / nsplit + kGK - 1) / kGK * kGK;
    nsplit = (K + kchunk - 1) / kchunk;
    void *out = rho;
    const size_t nn = (size_t)n * n;
    if (nsplit > 1) {
        const size_t need = (size_t)nsplit * nn * h->esize;
        if (need > h->gram_aux_bytes) {
            dev_free(h, h->gram_aux, h->gram_aux_bytes);
            h->gram_aux = nullptr;
            h->gram_aux_bytes = 0;
            cudaError_t err;
            h->gram_aux = dev_alloc(h, need, &err);
            if (err != cudaSuccess) return err;
            h->gram_aux_bytes = need;
        }
        out = h->gram_aux;
    }
    dim3 grid((n + kGT - 1) / kGT, (n + kGT - 1) / kGT, (unsigned)nsplit);
    if (h->prec == OSMPS_FP64)
        gram_kernel<double><<<grid, 256, 0, h->stream>>>((const double2 *)psi, n, K, sx, sk, kchunk, (double2 *)out);
    else
        gram_kernel<float><<<grid, 256, 0, h->stream>>>((const float2 *)psi, n, K, sx, sk, kchunk, (float2 *)out);
    h->launches += 1;
    if (nsplit > 1) {
        const unsigned g = (unsigned)((nn + 255) / 256 < 4096 ? (nn + 255) / 256 : 4096);
        if (h->prec == OSMPS_FP64)
            gram_split_sum_kernel<double><<<g, 256, 0, h->stream>>>((const double2 *)out, (int)nsplit, nn,
                                                                     (double2 *)rho);
        else
            gram_split_sum_kernel<float><<<g, 256, 0, h->stream>>>((const float2 *)out, (int)nsplit, nn,
                                                                    (float2 *)rho);
        h->launches += 1;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Spectrum of rho by cuSOLVER heevd (loaded at first use) and the entropy
// ---------------------------------------------------------------------------
struct SolverLib {
    bool tried = false;
    bool ok = false;
    void *so = nullptr;
    cusolverDnHandle_t handle = nullptr;
    decltype(&cusolverDnCreate) create = nullptr;
    decltype(&cusolverDnSetStream) set_stream = nullptr;
    decltype(&cusolverDnDestroy) destroy = nullptr;
    decltype(&cusolverDnZheevd_bufferSize) z_bufsize = nullptr;
    decltype(&cusolverDnZheevd) z_eig = nullptr;
    decltype(&cusolverDnCheevd_bufferSize) c_bufsize = nullptr;
    decltype(&cusolverDnCheevd) c_eig = nullptr;
    // 64-bit API (workspace sizes beyond 2^31 elements, e.g. n = 32768)
    decltype(&cusolverDnCreateParams) create_params = nullptr;
    decltype(&cusolverDnXsyevd_bufferSize) x_bufsize = nullptr;
    decltype(&cusolverDnXsyevd) x_eig = nullptr;
    decltype(&cusolverDnXgesvd_bufferSize) x_svd_bufsize = nullptr;
    decltype(&cusolverDnXgesvd) x_svd = nullptr;
    // Householder QR and its explicit Q (the dominant-subspace route)
    decltype(&cusolverDnCgeqrf_bufferSize) c_geqrf_bufsize = nullptr;
    decltype(&cusolverDnCgeqrf) c_geqrf = nullptr;
    decltype(&cusolverDnCungqr_bufferSize) c_ungqr_bufsize = nullptr;
    decltype(&cusolverDnCungqr) c_ungqr = nullptr;
    decltype(&cusolverDnZgeqrf_bufferSize) z_geqrf_bufsize = nullptr;
    decltype(&cusolverDnZgeqrf) z_geqrf = nullptr;
    decltype(&cusolverDnZungqr_bufferSize) z_ungqr_bufsize = nullptr;
    decltype(&cusolverDnZungqr) z_ungqr = nullptr;
    cusolverDnParams_t params = nullptr;  // default options, read-only after creation
};
static SolverLib g_solver;

static bool load_solver() {
    if (g_solver.tried) return g_solver.ok;
    g_solver.tried = true;
    const char *names[] = {"libcusolver.so.12", "libcusolver.so", "libcusolver.so.11"};
    for (const char *nm : names) {
        g_solver.so = dlopen(nm, RTLD_NOW | RTLD_LOCAL);
        if (g_solver.so) break;
    }
    if (!g_solver.so) return false;
    g_solver.create = (decltype(g_solver.create))dlsym(g_solver.so, "cusolverDnCreate");
    g_solver.set_stream = (decltype(g_solver.set_stream))dlsym(g_solver.so, "cusolverDnSetStream");
    g_solver.destroy = (decltype(g_solver.destroy))dlsym(g_solver.so, "cusolverDnDestroy");
    g_solver.z_bufsize = (decltype(g_solver.z_bufsize))dlsym(g_solver.so, "cusolverDnZheevd_bufferSize");
    g_solver.z_eig = (decltype(g_solver.z_eig))dlsym(g_solver.so, "cusolverDnZheevd");
    g_solver.c_bufsize = (decltype(g_solver.c_bufsize))dlsym(g_solver.so, "cusolverDnCheevd_bufferSize");
    g_solver.c_eig = (decltype(g_solver.c_eig))dlsym(g_solver.so, "cusolverDnCheevd");
    if (!g_solver.create || !g_solver.set_stream || !g_solver.z_bufsize || !g_solver.z_eig || !g_solver.c_bufsize ||
        !g_solver.c_eig)
        return false;
    if (g_solver.create(&g_solver.handle) != CUSOLVER_STATUS_SUCCESS) return false;
    g_solver.create_params = (decltype(g_solver.create_params))dlsym(g_solver.so, "cusolverDnCreateParams");
    g_solver.x_bufsize = (decltype(g_solver.x_bufsize))dlsym(g_solver.so, "cusolverDnXsyevd_bufferSize");
    g_solver.x_eig = (decltype(g_solver.x_eig))dlsym(g_solver.so, "cusolverDnXsyevd");
    g_solver.x_svd_bufsize = (decltype(g_solver.x_svd_bufsize))dlsym(g_solver.so, "cusolverDnXgesvd_bufferSize");
    g_solver.x_svd = (decltype(g_solver.x_svd))dlsym(g_solver.so, "cusolverDnXgesvd");
    if (!g_solver.create_params || !g_solver.x_bufsize || !g_solver.x_eig ||
        g_solver.create_params(&g_solver.params) != CUSOLVER_STATUS_SUCCESS)
        g_solver.params = nullptr;
    g_solver.c_geqrf_bufsize = (decltype(g_solver.c_geqrf_bufsize))dlsym(g_solver.so, "cusolverDnCgeqrf_bufferSize");
    g_solver.c_geqrf = (decltype(g_solver.c_geqrf))dlsym(g_solver.so, "cusolverDnCgeqrf");
    g_solver.c_ungqr_bufsize = (decltype(g_solver.c_ungqr_bufsize))dlsym(g_solver.so, "cusolverDnCungqr_bufferSize");
    g_solver.c_ungqr = (decltype(g_solver.c_ungqr))dlsym(g_solver.so, "cusolverDnCungqr");
    g_solver.z_geqrf_bufsize = (decltype(g_solver.z_geqrf_bufsize))dlsym(g_solver.so, "cusolverDnZgeqrf_bufferSize");
    g_solver.z_geqrf = (decltype(g_solver.z_geqrf))dlsym(g_solver.so, "cusolverDnZgeqrf");
    g_solver.z_ungqr_bufsize = (decltype(g_solver.z_ungqr_bufsize))dlsym(g_solver.so, "cusolverDnZungqr_bufferSize");
    g_solver.z_ungqr = (decltype(g_solver.z_ungqr))dlsym(g_solver.so, "cusolverDnZungqr");
    g_solver.ok = true;
    return true;
}

// cuBLAS, loaded at first use like the solver; only complex GEMM is used
// (default math mode: FP32 or FP64 arithmetic as named, no TF32)
struct BlasLib {
    bool tried = false;
    bool ok = false;
    void *so = nullptr;
    cublasHandle_t handle = nullptr;
    decltype(&cublasCreate_v2) create = nullptr;
    decltype(&cublasSetStream_v2) set_stream = nullptr;
    decltype(&cublasCgemm_v2) cgemm = nullptr;
    decltype(&cublasZgemm_v2) zgemm = nullptr;
};
static BlasLib g_blas;

static bool load_blas() {
    if (g_blas.tried) return g_blas.ok;
    g_blas.tried = true;
    const char *names[] = {"libcublas.so.13", "libcublas.so", "libcublas.so.12"};
    for (const char *nm : names) {
        g_blas.so = dlopen(nm, RTLD_NOW | RTLD_LOCAL);
        if (g_blas.so) break;
    }
    if (!g_blas.so) return false;
    g_blas.create = (decltype(g_blas.create))dlsym(g_blas.so, "cublasCreate_v2");
    g_blas.set_stream = (decltype(g_blas.set_stream))dlsym(g_blas.so, "cublasSetStream_v2");
    g_blas.cgemm = (decltype(g_blas.cgemm))dlsym(g_blas.so, "cublasCgemm_v2");
    g_blas.zgemm = (decltype(g_blas.zgemm))dlsym(g_blas.so, "cublasZgemm_v2");
    if (!g_blas.create || !g_blas.set_stream || !g_blas.cgemm || !g_blas.zgemm) return false;
    if (g_blas.create(&g_blas.handle) != CUBLAS_STATUS_SUCCESS) return false;
    g_blas.ok = true;
    return true;
}

// S = -sum lambda ln lambda over lambda > 0; lambda (ascending, T) -> descending FP64
template <typename T>
__global__ void entropy_kernel(const T *w, int n, double *lambda, double *S) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double l = (double)w[i];
        lambda[n - 1 - i] = l;
        if (l > 0.0) s -= l * log(l);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        *S = t;
    }
}

// flag = 1 when the library solver reported a failure (info != 0) or returned
// a non-finite eigenvalue
template <typename T>
__global__ void eig_check_kernel(const int *info, const T *w, int n, int *flag) {
    int bad = (threadIdx.x == 0 && *info != 0) ? 1 : 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        if (!isfinite((double)w[i])) bad = 1;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) *flag = bad;
}

// One cuSOLVER handle serves the process; its use (and its lazy loading) is
// serialised, so that an asynchronous measurement on a worker thread and a
// synchronous one never share it at the same time.
static std::mutex g_solver_mu;

#define CKS_(expr)                          \
    do {                                    \
        const osmps_status _s = (expr);     \
        if (_s != OSMPS_OK) return _s;      \
    } while (0)

// Device buffer of at least `need` bytes in *ws_p (counted in the handle's bytes when tracked).
static osmps_status grow_ws(Handle *h, void **ws_p, size_t *ws_bytes_p, bool tracked, size_t need) {
    if (need <= *ws_bytes_p) return OSMPS_OK;
    if (*ws_p) {
        if (tracked)
            dev_free(h, *ws_p, *ws_bytes_p);
        else
            cudaFree(*ws_p);
    }
    *ws_p = nullptr;
    *ws_bytes_p = 0;
    cudaError_t err = cudaSuccess;
    if (tracked) {
        *ws_p = dev_alloc(h, need, &err);
    } else if ((err = cudaMalloc(ws_p, need)) != cudaSuccess) {
        cudaGetLastError();
        *ws_p = nullptr;
    }
    if (err != cudaSuccess) return OSMPS_ENOMEM;
    *ws_bytes_p = need;
    return OSMPS_OK;
}

void *solver_handle_new() {
    std::lock_guard<std::mutex> lock(g_solver_mu);
    if (!load_solver() || g_solver.destroy == nullptr) return nullptr;
    cusolverDnHandle_t sh = nullptr;
    if (g_solver.create(&sh) != CUSOLVER_STATUS_SUCCESS) return nullptr;
    return sh;
}

void solver_handle_free(void *solver) {
    if (solver != nullptr && g_solver.destroy != nullptr) g_solver.destroy((cusolverDnHandle_t)solver);
}

osmps_status schmidt_eig_on(Handle *h, cudaStream_t stream, void *solver, void **ws_p, size_t *ws_bytes_p,
                            bool tracked, int64_t *launches, void *rho, int n, double *lambda_dev, double *S_dev) {
    // the process-wide handle is shared: hold the lock for the whole call; a
    // caller's own handle needs none (the library was loaded when it was made)
    std::unique_lock<std::mutex> lock(g_solver_mu, std::defer_lock);
    if (solver == nullptr) {
        lock.lock();
        if (!load_solver()) return OSMPS_EUNSUPPORTED;
    }
    const cusolverDnHandle_t hs = solver ? (cusolverDnHandle_t)solver : g_solver.handle;
    if (g_solver.set_stream(hs, stream) != CUSOLVER_STATUS_SUCCESS) return OSMPS_ECUDA;
    const bool dbl = (h->prec == OSMPS_FP64);
    const bool x64 = g_solver.params != nullptr;
    const cudaDataType ta = dbl ? CUDA_C_64F : CUDA_C_32F, tw = dbl ? CUDA_R_64F : CUDA_R_32F;
    const size_t cs = dbl ? sizeof(cuDoubleComplex) : sizeof(cuComplex);
    const size_t wbytes = (dbl ? sizeof(double) : sizeof(float)) * (size_t)n;
    const size_t o_work = 16 + ((wbytes + 15) & ~(size_t)15);
    // the size queries get real buffers: info and the eigenvalue array first
    CKS_(grow_ws(h, ws_p, ws_bytes_p, tracked, o_work + 256));
    cusolverStatus_t st;
    size_t work_bytes = 0, host_bytes = 0;
    int lwork = 0;
    if (x64) {
        st = g_solver.x_bufsize(hs, g_solver.params, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, (int64_t)n,
                                ta, rho, (int64_t)n, tw, (char *)*ws_p + 16, ta, &work_bytes, &host_bytes);
    } else if (dbl) {
        st = g_solver.z_bufsize(hs, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                (const cuDoubleComplex *)rho, n, (const double *)((char *)*ws_p + 16), &lwork);
        work_bytes = (size_t)lwork * cs;
    } else {
        st = g_solver.c_bufsize(hs, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n,
                                (const cuComplex *)rho, n, (const float *)((char *)*ws_p + 16), &lwork);
        work_bytes = (size_t)lwork * cs;
    }
    if (st != CUSOLVER_STATUS_SUCCESS) return OSMPS_ECUDA;
    if (work_bytes < 256) work_bytes = 256;
    // workspace: info and the failure flag, eigenvalues, the solver's work
    // array, a copy of rho and the workspace of this library's reduction,
    // which takes over when the library solver fails on the copy
    const int G = trd_ctas(n, h->prec, h->nsm, h->device);
    const size_t o_copy = o_work + ((work_bytes + 255) & ~(size_t)255);
    const size_t copy_bytes = G > 0 ? (size_t)n * n * cs : 0;
    const size_t o_trd = o_copy + ((copy_bytes + 255) & ~(size_t)255);
    const size_t trd_bytes = G > 0 ? trd_workspace_bytes(n, h->prec, G) : 0;
    CKS_(grow_ws(h, ws_p, ws_bytes_p, tracked, o_trd + trd_bytes + 64));
    std::vector<char> host_ws;
    try {
        host_ws.resize(host_bytes > 0 ? host_bytes : 1);
    } catch (...) {
        return OSMPS_ENOMEM;
    }
    char *ws = (char *)*ws_p;
    int *info = (int *)ws;
    int *flag = info + 1;
    void *wvals = ws + 16;
    void *work = ws + o_work;
    if (copy_bytes > 0 && cudaMemcpyAsync(ws + o_copy, rho, copy_bytes, cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
        return OSMPS_ECUDA;
    if (x64)
        st = g_solver.x_eig(hs, g_solver.params, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, (int64_t)n, ta, rho,
                            (int64_t)n, tw, wvals, ta, work, work_bytes, host_ws.data(), host_bytes, info);
    else if (dbl)
        st = g_solver.z_eig(hs, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n,
                            (cuDoubleComplex *)rho, n, (double *)wvals, (cuDoubleComplex *)work, lwork, info);
    else
        st = g_solver.c_eig(hs, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, n, (cuComplex *)rho,
                            n, (float *)wvals, (cuComplex *)work, lwork, info);
    if (st != CUSOLVER_STATUS_SUCCESS) return OSMPS_ECUDA;
    if (dbl)
        eig_check_kernel<double><<<1, 1024, 0, stream>>>(info, (const double *)wvals, n, flag);
    else
        eig_check_kernel<float><<<1, 1024, 0, stream>>>(info, (const float *)wvals, n, flag);
    *launches += 1;
    int bad = 0;
    if (cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return OSMPS_ECUDA;
    if (bad == 0) {
        if (dbl)
            entropy_kernel<double><<<1, 1024, 0, stream>>>((const double *)wvals, n, lambda_dev, S_dev);
        else
            entropy_kernel<float><<<1, 1024, 0, stream>>>((const float *)wvals, n, lambda_dev, S_dev);
        *launches += 1;
        return cudaGetLastError() == cudaSuccess ? OSMPS_OK : OSMPS_ECUDA;
    }
    // the library solver failed (seen on nearly rank-one complex64 matrices):
    // this library's reduction on the saved copy of rho
    if (G == 0) return OSMPS_ECUDA;
    if (cudaMemsetAsync(flag, 0, sizeof(int), stream) != cudaSuccess) return OSMPS_ECUDA;
    TrdRun run{h->prec, h->device, stream, G, ws + o_trd, trd_bytes, flag, launches};
    double *w = nullptr;
    if (trd_eigvals(run, ws + o_copy, n, &w) != cudaSuccess) return OSMPS_ECUDA;
    entropy_kernel<double><<<1, 1024, 0, stream>>>(w, n, lambda_dev, S_dev);
    *launches += 1;
    if (cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return OSMPS_ECUDA;
    return bad == 0 ? OSMPS_OK : OSMPS_ETIMEOUT;
}

cudaError_t launch_entropy(cudaStream_t stream, const double *w, int n, double *lambda_dev, double *S_dev) {
    entropy_kernel<double><<<1, 1024, 0, stream>>>(w, n, lambda_dev, S_dev);
    return cudaGetLastError();
}

osmps_status schmidt_eig(Handle *h, void *rho, int n, double *lambda_dev, double *S_dev) {
    return schmidt_eig_on(h, h->stream, nullptr, &h->solver_ws, &h->solver_ws_bytes, true, &h->launches, rho, n,
                          lambda_dev, S_dev);
}

// ---------------------------------------------------------------------------
// Schmidt values from the singular values of M itself (no Gram product):
// lambda = sigma^2 keeps an absolute error of ~2 sigma eps, so tiny Schmidt
// values stay accurate in complex64, where forming rho = M M^H would give
// every lambda an error of ~eps.
// ---------------------------------------------------------------------------

// A[a + c*m] = psi[a*nc + c]: the row-major m x nc block matrix, column-major
template <typename C>
__global__ void transpose_kernel(const C *psi, long long m, long long nc, C *A) {
    __shared__ C t[32][33];
    const long long a0 = (long long)blockIdx.x * 32, c0 = (long long)blockIdx.y * 32;  // rows on x (up to 2^29)
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const long long a = a0 + r, c = c0 + threadIdx.x;
        if (a < m && c < nc) t[r][threadIdx.x] = psi[a * nc + c];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const long long c = c0 + r, a = a0 + threadIdx.x;
        if (a < m && c < nc) A[a + c * m] = t[threadIdx.x][r];
    }
}

// lambda_i = sigma_i^2 (descending as returned), S = -sum lambda ln lambda;
// flag = 1 on a reported failure or a non-finite value
template <typename T>
__global__ void sv_entropy_kernel(const T *sv, int n, const int *info, double *lambda, double *S, int *flag) {
    __shared__ double red[32];
    double s = 0.0;
    int bad = (threadIdx.x == 0 && *info != 0) ? 1 : 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double x = (double)sv[i];
        if (!isfinite(x)) bad = 1;
        const double l = x * x;
        lambda[i] = l;
        if (l > 0.0) s -= l * log(l);
    }
    bad = __syncthreads_or(bad);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        *S = t;
        *flag = bad;
    }
}

osmps_status schmidt_svd(Handle *h, const void *psi, int cut, double *lambda_dev, double *S_dev) {
    std::lock_guard<std::mutex> lock(g_solver_mu);
    if (!load_solver() || g_solver.params == nullptr || !g_solver.x_svd || !g_solver.x_svd_bufsize)
        return OSMPS_EUNSUPPORTED;
    if (g_solver.set_stream(g_solver.handle, h->stream) != CUSOLVER_STATUS_SUCCESS) return OSMPS_ECUDA;
    const int L = h->L;
    const bool dbl = (h->prec == OSMPS_FP64);
    // column-major m x nc with m >= nc
    const bool left_small = cut <= L - cut;
    const long long m = 1ll << (left_small ? L - cut : cut), nc = 1ll << (left_small ? cut : L - cut);
    const cudaDataType ta = dbl ? CUDA_C_64F : CUDA_C_32F, tr = dbl ? CUDA_R_64F : CUDA_R_32F;
    const size_t cs = h->esize, rs = dbl ? sizeof(double) : sizeof(float);
    const size_t abytes = (size_t)m * (size_t)nc * cs;
    // layout: info, flag | singular values | U, VT (not referenced: jobu = jobvt = 'N') | A | work
    const size_t o_s = 256, o_u = o_s + ((nc * rs + 255) & ~(size_t)255), o_vt = o_u + 256, o_a = o_vt + 256;
    const size_t o_work = o_a + ((abytes + 255) & ~(size_t)255);
    CKS_(grow_ws(h, &h->solver_ws, &h->solver_ws_bytes, true, o_work + 256));
    size_t work_bytes = 0, host_bytes = 0;
    {
        char *ws = (char *)h->solver_ws;
        if (g_solver.x_svd_bufsize(g_solver.handle, g_solver.params, 'N', 'N', m, nc, ta, ws + o_a, m, tr, ws + o_s, ta,
                                   ws + o_u, m, ta, ws + o_vt, nc, ta, &work_bytes, &host_bytes) !=
            CUSOLVER_STATUS_SUCCESS)
            return OSMPS_ECUDA;
    }
    if (work_bytes < 256) work_bytes = 256;
    CKS_(grow_ws(h, &h->solver_ws, &h->solver_ws_bytes, true, o_work + work_bytes + 64));
    std::vector<char> host_ws;
    try {
        host_ws.resize(host_bytes > 0 ? host_bytes : 1);
    } catch (...) {
        return OSMPS_ENOMEM;
    }
    char *ws = (char *)h->solver_ws;
    int *info = (int *)ws, *flag = info + 1;
    if (left_small) {
        // the row-major block matrix read column-major is already m x nc with lda = m
        if (cudaMemcpyAsync(ws + o_a, psi, abytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
            return OSMPS_ECUDA;
    } else {
        const dim3 grid((unsigned)((m + 31) / 32), (unsigned)((nc + 31) / 32)), block(32, 8);
        if (dbl)
            transpose_kernel<double2><<<grid, block, 0, h->stream>>>((const double2 *)psi, m, nc, (double2 *)(ws + o_a));
        else
            transpose_kernel<float2><<<grid, block, 0, h->stream>>>((const float2 *)psi, m, nc, (float2 *)(ws + o_a));
        h->launches += 1;
    }
    if (g_solver.x_svd(g_solver.handle, g_solver.params, 'N', 'N', m, nc, ta, ws + o_a, m, tr, ws + o_s, ta, ws + o_u,
                       m, ta, ws + o_vt, nc, ta, ws + o_work, work_bytes, host_ws.data(), host_bytes, info) !=
        CUSOLVER_STATUS_SUCCESS)
        return OSMPS_ECUDA;
    if (dbl)
        sv_entropy_kernel<double><<<1, 1024, 0, h->stream>>>((const double *)(ws + o_s), (int)nc, info, lambda_dev,
                                                             S_dev, flag);
    else
        sv_entropy_kernel<float><<<1, 1024, 0, h->stream>>>((const float *)(ws + o_s), (int)nc, info, lambda_dev,
                                                            S_dev, flag);
    h->launches += 1;
    int bad = 0;
    if (cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
        return OSMPS_ECUDA;
    return bad == 0 ? OSMPS_OK : OSMPS_ECUDA;
}


// ---------------------------------------------------------------------------
// Schmidt values as Rayleigh quotients of the Gram product's eigenvectors
// (complex64).  The eigenvalues of rho = A A^H carry absolute errors of order
// eps |rho| in FP32, which dominate S of a weakly entangled state; the
// eigenvectors u_i do not square anything, and |u_i^H A|^2 formed from A
// itself keeps the small Schmidt values to their own relative accuracy.  The
// tensor cores' truncating accumulation leaves every value with nearly the same
// relative deficit (~1e-6), so the values are rescaled to sum to |psi|^2 (FP64):
// the Schmidt values sum to the norm (Sec. IV, bond entropy).
// ---------------------------------------------------------------------------
constexpr int kRayMaxN = 8192;  // one CTA sorts the spectrum in shared memory

// lambda_i = sum_t part_re[i][t] + part_im[i][t] (fixed order), sorted descending,
// rescaled by |psi|^2 / sum_i lambda_i (norm partials: 4 doubles per CTA, the
// first is |x|^2), S = -sum lambda ln lambda.  One CTA, n a power of two.  A
// non-finite value or norm (the library eigen-solver has returned non-finite
// eigenvectors for nearly rank-one rho with FP32-subnormal entries) makes S NaN,
// which sends the caller to the singular values of M.
__global__ void __launch_bounds__(1024) rayleigh_entropy_kernel(const double *part_re, const double *part_im, int n,
                                                                 int ntx, const double *norm_parts, int nparts,
                                                                 double *lambda, double *S) {
    extern __shared__ double lam_s[];
    __shared__ double red[32];
    __shared__ double trace_s;
    int bad = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v = 0.0;
        for (int t = 0; t < ntx; ++t) v += part_re[(size_t)i * ntx + t] + part_im[(size_t)i * ntx + t];
        lam_s[i] = v;
        if (!isfinite(v)) bad = 1;
    }
    if (threadIdx.x < 32) {
        double t = 0.0;
        for (int p = threadIdx.x; p < nparts; p += 32) t += norm_parts[4 * (size_t)p];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (threadIdx.x == 0) trace_s = t;
        if (!isfinite(t)) bad = 1;
    }
    bad = __syncthreads_or(bad);
    // bitonic sort, descending
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const double a = lam_s[i], b = lam_s[ixj];
                    const bool desc = (i & k) == 0;
                    if (desc ? (a < b) : (a > b)) {
                        lam_s[i] = b;
                        lam_s[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    // sum of all values, fixed order
    double r = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) r += lam_s[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        trace_s = tot > 0.0 ? trace_s / tot : 1.0;  // now the rescaling factor
    }
    __syncthreads();
    const double scale = trace_s;
    double e = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double l = lam_s[i] * scale;
        lambda[i] = l;
        if (l > 0.0) e -= l * log(l);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *S = bad ? __longlong_as_double(0x7FF8000000000000ll) : t;
    }
}

bool rayleigh_applicable(const Handle *h, int cut) {
    const int L = h->L;
    const int ls = cut < L - cut ? cut : L - cut;
    const int n = 1 << ls;
    const long long K = 1ll << (L - ls);
    return h->prec == OSMPS_MIXED && n <= kRayMaxN && rayleigh_tc_supported(n, K);
}

osmps_status schmidt_rayleigh(Handle *h, const void *psi, int cut, void *rho, double *lambda_dev, double *S_dev) {
    if (!rayleigh_applicable(h, cut)) return OSMPS_EUNSUPPORTED;
    const int L = h->L;
    int n;
    long long K, sx, sk;
    if (cut <= L - cut) {
        n = 1 << cut;
        K = 1ll << (L - cut);
        sx = K;
        sk = 1;
    } else {
        n = 1 << (L - cut);
        K = 1ll << cut;
        sx = 1;
        sk = n;
    }
    const int ntx = (int)(K / 128);
    // scratch: the Gram product's planes and the Rayleigh planes share gram_aux
    const size_t gram_need = sizeof(float) * ((size_t)n * 4 * (size_t)K + (size_t)n * n);
    const size_t ray_need = sizeof(float) * rayleigh_tc_plane_floats(n, K) + 2 * sizeof(double) * (size_t)n * ntx;
    const size_t need = gram_need > ray_need ? gram_need : ray_need;
    if (need > h->gram_aux_bytes) {
        dev_free(h, h->gram_aux, h->gram_aux_bytes);
        h->gram_aux = nullptr;
        h->gram_aux_bytes = 0;
        cudaError_t err;
        h->gram_aux = dev_alloc(h, need, &err);
        if (err != cudaSuccess) return OSMPS_ENOMEM;
        h->gram_aux_bytes = need;
    }
    int nn = 0;
    if (launch_gram(h, psi, cut, rho, &nn) != cudaSuccess || nn != n) return OSMPS_ECUDA;
    // eigenvectors of the Hermitian rho (read as the column-major lower triangle
    // of conj(rho), so column i is conj(u_i); rho is overwritten by them)
    {
        std::lock_guard<std::mutex> lock(g_solver_mu);
        if (!load_solver() || g_solver.params == nullptr) return OSMPS_EUNSUPPORTED;
        if (g_solver.set_stream(g_solver.handle, h->stream) != CUSOLVER_STATUS_SUCCESS) return OSMPS_ECUDA;
        const size_t o_work = 16 + (((size_t)n * sizeof(float) + 255) & ~(size_t)255);
        CKS_(grow_ws(h, &h->solver_ws, &h->solver_ws_bytes, true, o_work + 256));
        size_t work_bytes = 0, host_bytes = 0;
        if (g_solver.x_bufsize(g_solver.handle, g_solver.params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                               (int64_t)n, CUDA_C_32F, rho, (int64_t)n, CUDA_R_32F, (char *)h->solver_ws + 16,
                               CUDA_C_32F, &work_bytes, &host_bytes) != CUSOLVER_STATUS_SUCCESS)
            return OSMPS_ECUDA;
        if (work_bytes < 256) work_bytes = 256;
        CKS_(grow_ws(h, &h->solver_ws, &h->solver_ws_bytes, true, o_work + work_bytes + 64));
        std::vector<char> host_ws;
        try {
            host_ws.resize(host_bytes > 0 ? host_bytes : 1);
        } catch (...) {
            return OSMPS_ENOMEM;
        }
        char *ws = (char *)h->solver_ws;
        int *info = (int *)ws, *flag = info + 1;
        if (g_solver.x_eig(g_solver.handle, g_solver.params, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER,
                           (int64_t)n, CUDA_C_32F, rho, (int64_t)n, CUDA_R_32F, ws + 16, CUDA_C_32F, ws + o_work,
                           work_bytes, host_ws.data(), host_bytes, info) != CUSOLVER_STATUS_SUCCESS)
            return OSMPS_ECUDA;
        eig_check_kernel<float><<<1, 1024, 0, h->stream>>>(info, (const float *)(ws + 16), n, flag);
        h->launches += 1;
        int bad = 0;
        if (cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            return OSMPS_ECUDA;
        if (bad != 0) return OSMPS_ENOCONV;  // the caller falls back to the singular values of M
    }
    float *planes = (float *)h->gram_aux;
    double *part_re = (double *)((char *)h->gram_aux + sizeof(float) * rayleigh_tc_plane_floats(n, K));
    double *part_im = part_re + (size_t)n * ntx;
    if (rayleigh_tc_launch(h, rho, psi, n, K, sx, sk, planes, part_re, part_im) != cudaSuccess) return OSMPS_ECUDA;
    int np = 0;
    if (launch_norm2(h, psi, h->partials, &np) != cudaSuccess) return OSMPS_ECUDA;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(rayleigh_entropy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kRayMaxN * sizeof(double)));
        attr = true;
    }
    rayleigh_entropy_kernel<<<1, 1024, (size_t)n * sizeof(double), h->stream>>>(part_re, part_im, n, ntx, h->partials,
                                                                                 np, lambda_dev, S_dev);
    h->launches += 1;
    return cudaGetLastError() == cudaSuccess ? OSMPS_OK : OSMPS_ECUDA;
}

// ---------------------------------------------------------------------------
// Schmidt values from the dominant subspace (complex64; Sec. IV bond entropy).
// A weakly entangled state has few Schmidt values above 1e-10 (~100 of 4096 on
// the L = 24 quench to t = 2.5); the rest carry < 1e-8 of weight.  With M the
// n x K block matrix of psi and G a K x p random block: Y = M G, Q = orth(Y)
// (Householder), B = Q^dag M (FP32 GEMMs); the Schmidt values are the squared
// singular values of B, taken as the eigenvalues of C = B B^dag formed (own
// split-K kernel) and diagonalised in FP64 (the FP32 products are exact there, so no value is lost
// to squaring: each keeps the error 2 sigma |dB| of the singular-value route).
// The weight left outside the subspace, |M - Q B|_F^2, is measured directly
// (not by subtraction from the trace) and must stay at or below 1e-9 of the
// trace; otherwise p doubles, and beyond n/2 the caller takes the full route.
// ---------------------------------------------------------------------------
constexpr int kSubResBlocks = 608;  // CTAs of the residual-norm partial sums
constexpr int kSubMaxP = 768;       // largest subspace tried
constexpr int kSubSkip = 4;         // calls that go straight to the full route after one that needed more

// uniform complex entries in [-1, 1)^2: the SplitMix64 output function (Steele,
// Lea & Flood 2014) of seed + i * golden gamma, 24 bits per component
template <typename V2>
__global__ void sub_random_kernel(V2 *G, long long count, unsigned long long seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + (unsigned long long)i * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const float a = (float)(z >> 40) * (1.0f / 8388608.0f) - 1.0f;
        const float b = (float)((z >> 16) & 0xFFFFFFull) * (1.0f / 8388608.0f) - 1.0f;
        G[i].x = a;
        G[i].y = b;
    }
}
__device__ __forceinline__ double2 to_d2(const float2 v) { return make_double2((double)v.x, (double)v.y); }
__device__ __forceinline__ double2 to_d2(const double2 v) { return v; }

// C = B B^dag in FP64 from B (column-major p x K, FP32 or FP64): the products of
// FP32 values are exact in FP64.  One CTA per 32 x 32 tile of the lower triangle and
// per chunk of K (split so the grid fills the GPU), the chunk of both row
// blocks staged in shared memory as FP64; partial tiles to part[split], summed
// in a fixed order by sub_gram_sum_kernel.
constexpr int kG64T = 32;   // tile edge
constexpr int kG64K = 32;   // K staged per step (2 x 16 KB of FP64 in shared memory)
template <typename V2>
__global__ void __launch_bounds__(256) sub_gram64_kernel(const V2 *B, int p, long long K, int nsplit,
                                                         double2 *part) {
    __shared__ double2 As[kG64K][kG64T], Bs[kG64K][kG64T];
    // lower-triangle tile index -> (ti, tj), ti >= tj
    int t = blockIdx.x, ti = 0;
    while (t > ti) {
        t -= ti + 1;
        ++ti;
    }
    const int tj = t;
    const int split = blockIdx.y;
    const long long k0 = K * split / nsplit, k1 = K * (split + 1) / nsplit;
    const int r = threadIdx.x & 31, c0 = threadIdx.x >> 5;  // rows r, columns c0 + 8 m
    double cr[4] = {0, 0, 0, 0}, ci[4] = {0, 0, 0, 0};
    for (long long kb = k0; kb < k1; kb += kG64K) {
        const int kn = (int)((k1 - kb) < kG64K ? (k1 - kb) : kG64K);
        for (int e = threadIdx.x; e < kG64K * kG64T; e += 256) {
            const int kk = e / kG64T, ii = e % kG64T;
            double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
            if (kk < kn) {
                const int ia = ti * kG64T + ii, ib = tj * kG64T + ii;
                if (ia < p) a = to_d2(B[(size_t)ia + (size_t)(kb + kk) * p]);
                if (ib < p) b = to_d2(B[(size_t)ib + (size_t)(kb + kk) * p]);
            }
            As[kk][ii] = a;
            Bs[kk][ii] = b;
        }
        __syncthreads();
        for (int kk = 0; kk < kn; ++kk) {
            const double2 a = As[kk][r];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const double2 b = Bs[kk][c0 + 8 * m];
                // a conj(b)
                cr[m] = fma(a.x, b.x, fma(a.y, b.y, cr[m]));
                ci[m] = fma(a.y, b.x, fma(-a.x, b.y, ci[m]));
            }
        }
        __syncthreads();
    }
    const int i = ti * kG64T + r;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int j = tj * kG64T + c0 + 8 * m;
        if (i < p && j < p) part[(size_t)split * p * p + (size_t)i + (size_t)j * p] = make_double2(cr[m], ci[m]);
    }
}
// C[i + j p] = sum over splits (fixed order) for i >= j
__global__ void sub_gram_sum_kernel(const double2 *part, int p, int nsplit, double2 *C) {
    const long long total = (long long)p * p;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % p), j = (int)(e / p);
        if (i < j) continue;
        double2 s = make_double2(0.0, 0.0);
        for (int q = 0; q < nsplit; ++q) {
            const double2 v = part[(size_t)q * total + e];
            s.x += v.x;
            s.y += v.y;
        }
        C[e] = s;
    }
}

// part[block] = sum of |R_k|^2 over the block's grid-stride share (in the
// element type per thread over 32 elements, FP64 across, fixed order)
template <typename V2>
__global__ void __launch_bounds__(256) sub_frob_kernel(const V2 *R, long long count, double *part) {
    typedef decltype(R->x) E;
    __shared__ double red[8];
    double acc = 0.0;
    E s = 0;
    int k = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const V2 r = R[i];
        s = fma(r.x, r.x, fma(r.y, r.y, s));
        if (++k == 32) {
            acc += (double)s;
            s = 0;
            k = 0;
        }
    }
    acc += (double)s;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// theta: the p ascending FP64 eigenvalues of C; lambda[0..n) = theta descending
// (values below 0, FP64 rounding of zero ones, as 0) and zeros after, rescaled so
// that they and the residual weight sum to |psi|^2 (FP64 norm partials, 4
// doubles per CTA; the FP32 products leave a common relative deficit or excess
// of order 1e-7); S = -sum lambda ln lambda; stats = {residual weight, sum of
// lambda, values above 1e-12}.  A non-zero solver status or a non-finite value
// makes S NaN.  One CTA.
__global__ void __launch_bounds__(1024) sub_entropy_kernel(const double *theta, int p, const double *res_part,
                                                           int nres, const double *norm_parts, int nnorm,
                                                           const int *infos, int ninfo, int n, double *lambda,
                                                           double *S, double *stats) {
    __shared__ double red[32];
    __shared__ double res_s, trace_s, scale_s;
    int bad = 0;
    if (threadIdx.x < 32) {
        double t = 0.0, r = 0.0;
        for (int b = threadIdx.x; b < nres; b += 32) r += res_part[b];
        for (int b = threadIdx.x; b < nnorm; b += 32) t += norm_parts[4 * (size_t)b];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            r += __shfl_xor_sync(0xffffffffu, r, off);
            t += __shfl_xor_sync(0xffffffffu, t, off);
        }
        if (threadIdx.x == 0) {
            res_s = r;
            trace_s = t;
        }
        if (!isfinite(r) || !isfinite(t)) bad = 1;
        for (int q = threadIdx.x; q < ninfo; q += 32)
            if (infos[q] != 0) bad = 1;
    }
    // sum of the captured values (fixed order)
    double tot = 0.0;
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        const double l = theta[p - 1 - i];
        if (!isfinite(l)) bad = 1;
        if (l > 0.0) tot += l;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tot;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        const double want = trace_s - res_s;
        scale_s = (t > 0.0 && want > 0.0) ? want / t : 1.0;
    }
    __syncthreads();
    const double scale = scale_s;
    double e = 0.0, cnt = 0.0;
    tot = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double l = 0.0;
        if (i < p) {
            l = theta[p - 1 - i] * scale;
            if (!(l > 0.0)) l = 0.0;
        }
        lambda[i] = l;
        if (l > 0.0) {
            e -= l * log(l);
            tot += l;
        }
        if (l > 1e-12) cnt += 1.0;
    }
    double vals[3] = {e, tot, cnt};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) vals[q] += __shfl_xor_sync(0xffffffffu, vals[q], off);
    }
    for (int q = 0; q < 3; ++q) {
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = vals[q];
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            vals[q] = t;
        }
    }
    if (threadIdx.x == 0) {
        *S = bad ? __longlong_as_double(0x7FF8000000000000ll) : vals[0];
        stats[0] = res_s;
        stats[1] = vals[1];
        stats[2] = vals[2];
    }
}

bool subspace_applicable(const Handle *h, int cut) {
    const int L = h->L;
    const int ls = cut < L - cut ? cut : L - cut;
    const int n = 1 << ls;
    return n >= 512 && n <= kRayMaxN;
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// library entry points of the route per precision; the residual bound keeps the
// uncaptured share of S below the precision's tolerance (1e-5 and 1e-10):
// w (1 + ln(n / w)) < 1e-7 for w = 1e-9, < 1e-10 for w = 2e-12
template <typename T> struct SubLib;
template <> struct SubLib<float> {
    typedef cuComplex C;
    typedef float2 V2;
    static constexpr double kResTol = 1e-9;
    static bool loaded() {
        return g_solver.c_geqrf && g_solver.c_ungqr && g_solver.c_geqrf_bufsize && g_solver.c_ungqr_bufsize;
    }
    static C scal(float r) { return make_cuComplex(r, 0.0f); }
    static cublasStatus_t gemm(cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, const C *al,
                               const C *A, int lda, const C *B, int ldb, const C *be, C *Cm, int ldc) {
        return g_blas.cgemm(g_blas.handle, ta, tb, m, n, k, al, A, lda, B, ldb, be, Cm, ldc);
    }
    static bool qr_sizes(int m, int n, C *A, int *lw) {
        int a = 0, b = 0;
        if (g_solver.c_geqrf_bufsize(g_solver.handle, m, n, A, m, &a) != CUSOLVER_STATUS_SUCCESS ||
            g_solver.c_ungqr_bufsize(g_solver.handle, m, n, n, A, m, A, &b) != CUSOLVER_STATUS_SUCCESS)
            return false;
        *lw = a > b ? a : b;
        return true;
    }
    static bool qr(int m, int n, C *A, C *tau, C *w, int lw, int *info) {
        return g_solver.c_geqrf(g_solver.handle, m, n, A, m, tau, w, lw, info) == CUSOLVER_STATUS_SUCCESS &&
               g_solver.c_ungqr(g_solver.handle, m, n, n, A, m, tau, w, lw, info + 1) == CUSOLVER_STATUS_SUCCESS;
    }
};
template <> struct SubLib<double> {
    typedef cuDoubleComplex C;
    typedef double2 V2;
    static constexpr double kResTol = 2e-12;
    static bool loaded() {
        return g_solver.z_geqrf && g_solver.z_ungqr && g_solver.z_geqrf_bufsize && g_solver.z_ungqr_bufsize;
    }
    static C scal(double r) { return make_cuDoubleComplex(r, 0.0); }
    static cublasStatus_t gemm(cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, const C *al,
                               const C *A, int lda, const C *B, int ldb, const C *be, C *Cm, int ldc) {
        return g_blas.zgemm(g_blas.handle, ta, tb, m, n, k, al, A, lda, B, ldb, be, Cm, ldc);
    }
    static bool qr_sizes(int m, int n, C *A, int *lw) {
        int a = 0, b = 0;
        if (g_solver.z_geqrf_bufsize(g_solver.handle, m, n, A, m, &a) != CUSOLVER_STATUS_SUCCESS ||
            g_solver.z_ungqr_bufsize(g_solver.handle, m, n, n, A, m, A, &b) != CUSOLVER_STATUS_SUCCESS)
            return false;
        *lw = a > b ? a : b;
        return true;
    }
    static bool qr(int m, int n, C *A, C *tau, C *w, int lw, int *info) {
        return g_solver.z_geqrf(g_solver.handle, m, n, A, m, tau, w, lw, info) == CUSOLVER_STATUS_SUCCESS &&
               g_solver.z_ungqr(g_solver.handle, m, n, n, A, m, tau, w, lw, info + 1) == CUSOLVER_STATUS_SUCCESS;
    }
};

template <typename T>
static osmps_status schmidt_subspace_t(Handle *h, const void *psi, int cut, double *lambda_dev, double *S_dev) {
    typedef SubLib<T> Lib;
    typedef typename Lib::C C;
    typedef typename Lib::V2 V2;
    const int L = h->L;
    // M[x][k] = psi[x sx + k sk]: column-major n x K (sx = 1, ld n) or its
    // transpose, column-major K x n (sk = 1, ld K)
    const bool colM = cut > L - cut;
    const int ls = colM ? L - cut : cut;
    const int n = 1 << ls;
    const int K = 1 << (L - ls);
    std::lock_guard<std::mutex> lock(g_solver_mu);
    if (!load_solver() || !Lib::loaded() || !load_blas()) return OSMPS_EUNSUPPORTED;
    if (g_solver.set_stream(g_solver.handle, h->stream) != CUSOLVER_STATUS_SUCCESS ||
        g_blas.set_stream(g_blas.handle, h->stream) != CUBLAS_STATUS_SUCCESS)
        return OSMPS_ECUDA;
    const C one = Lib::scal(1), zero = Lib::scal(0), mone = Lib::scal(-1);
    C *A = (C *)const_cast<void *>(psi);
    // largest subspace worth trying: the FP64 eigenvalues of a p x p matrix cost
    // about as much as the full FP32 route at p ~ 800 on this part
    const int pmax = (n / 2 < kSubMaxP) ? n / 2 : kSubMaxP;
    if (h->sub_skip > 0) {  // the last call needed more: the full route for a few calls
        --h->sub_skip;
        return OSMPS_ENOCONV;
    }
    int p = h->sub_hint > 0 ? h->sub_hint : 128;
    p = ((p + 63) / 64) * 64;
    if (p > pmax) p = pmax;
    for (;;) {
        // workspace sizes for this p (queries touch no memory)
        int lw = 0, lw_e = 0;
        if (!Lib::qr_sizes(n, p, A, &lw) ||
            g_solver.z_bufsize(g_solver.handle, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, p,
                               (const cuDoubleComplex *)A, p, (const double *)A, &lw_e) != CUSOLVER_STATUS_SUCCESS)
            return OSMPS_ECUDA;
        // lower-triangle tiles of C and the K split with the shortest makespan: waves of
        // one CTA per SM, each CTA a 1/nsplit share of K (a split that leaves a few
        // SMs a second CTA doubles the kernel's time)
        const int nt = (p + kG64T - 1) / kG64T, ntl = nt * (nt + 1) / 2;
        int nsplit = 1;
        double best = 1e300;
        for (int ns = 1; ns <= 16; ++ns) {
            const long long waves = ((long long)ntl * ns + h->nsm - 1) / h->nsm;
            const double cost = (double)waves / ns;
            if (cost < best - 1e-12) {
                best = cost;
                nsplit = ns;
            }
        }
        const size_t gpart = sizeof(cuDoubleComplex) * (size_t)nsplit * p * p;
        const size_t gk = sizeof(C) * (size_t)p * K;  // G (K x p) before B
        const size_t o_Y = 0;
        const size_t o_tau = o_Y + al256(sizeof(C) * (size_t)n * p);
        const size_t o_B = o_tau + al256(sizeof(C) * (size_t)p);
        const size_t o_GP = o_B + al256(sizeof(C) * (size_t)p * K);  // G, then the Gram partials
        const size_t o_C = o_GP + al256(gpart > gk ? gpart : gk);
        const size_t o_Mc = o_C + al256(sizeof(cuDoubleComplex) * (size_t)p * p);
        const size_t o_th = o_Mc + al256(sizeof(C) * (size_t)n * K);
        const size_t o_rp = o_th + al256(sizeof(double) * (size_t)p);
        const size_t o_st = o_rp + al256(sizeof(double) * kSubResBlocks);
        const size_t o_inf = o_st + al256(sizeof(double) * 4);
        const size_t o_wq = o_inf + al256(sizeof(int) * 4);
        const size_t o_we = o_wq + al256(sizeof(C) * (size_t)(lw > 0 ? lw : 1));
        const size_t need = o_we + al256(sizeof(cuDoubleComplex) * (size_t)(lw_e > 0 ? lw_e : 1));
        CKS_(grow_ws(h, &h->sub_ws, &h->sub_ws_bytes, true, need));
        char *ws = (char *)h->sub_ws;
        C *Y = (C *)(ws + o_Y), *tau = (C *)(ws + o_tau), *B = (C *)(ws + o_B);
        C *G = (C *)(ws + o_GP), *Mc = (C *)(ws + o_Mc);
        cuDoubleComplex *GP = (cuDoubleComplex *)(ws + o_GP), *Cm = (cuDoubleComplex *)(ws + o_C);
        double *th = (double *)(ws + o_th), *rp = (double *)(ws + o_rp), *st = (double *)(ws + o_st);
        int *inf = (int *)(ws + o_inf);
        C *wq = (C *)(ws + o_wq);
        cuDoubleComplex *we = (cuDoubleComplex *)(ws + o_we);
        if (cudaMemsetAsync(inf, 0, sizeof(int) * 4, h->stream) != cudaSuccess) return OSMPS_ECUDA;
        // G (K x p), Y = M G
        sub_random_kernel<V2><<<h->nsm * 4, 256, 0, h->stream>>>((V2 *)G, (long long)K * p, 0x5EEDull + (unsigned)p);
        h->launches += 1;
        cublasStatus_t bs = colM ? Lib::gemm(CUBLAS_OP_N, CUBLAS_OP_N, n, p, K, &one, A, n, G, K, &zero, Y, n)
                                 : Lib::gemm(CUBLAS_OP_T, CUBLAS_OP_N, n, p, K, &one, A, K, G, K, &zero, Y, n);
        if (bs != CUBLAS_STATUS_SUCCESS) return OSMPS_ECUDA;
        // Q = orth(Y), in place
        if (!Lib::qr(n, p, Y, tau, wq, lw, inf)) return OSMPS_ECUDA;
        // B = Q^dag M (p x K)
        bs = colM ? Lib::gemm(CUBLAS_OP_C, CUBLAS_OP_N, p, K, n, &one, Y, n, A, n, &zero, B, p)
                  : Lib::gemm(CUBLAS_OP_C, CUBLAS_OP_T, p, K, n, &one, Y, n, A, K, &zero, B, p);
        if (bs != CUBLAS_STATUS_SUCCESS) return OSMPS_ECUDA;
        // C = B B^dag in FP64 (lower triangle) and its eigenvalues
        sub_gram64_kernel<V2><<<dim3((unsigned)ntl, (unsigned)nsplit), 256, 0, h->stream>>>((const V2 *)B, p,
                                                                                           (long long)K, nsplit,
                                                                                           (double2 *)GP);
        sub_gram_sum_kernel<<<h->nsm * 4, 256, 0, h->stream>>>((const double2 *)GP, p, nsplit, (double2 *)Cm);
        h->launches += 2;
        if (g_solver.z_eig(g_solver.handle, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, p, Cm, p, th, we,
                           lw_e, inf + 2) != CUSOLVER_STATUS_SUCCESS)
            return OSMPS_ECUDA;
        // the weight outside the subspace: |M - Q B|_F^2
        if (cudaMemcpyAsync(Mc, A, sizeof(C) * (size_t)n * K, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
            return OSMPS_ECUDA;
        bs = colM ? Lib::gemm(CUBLAS_OP_N, CUBLAS_OP_N, n, K, p, &mone, Y, n, B, p, &one, Mc, n)
                  : Lib::gemm(CUBLAS_OP_T, CUBLAS_OP_T, K, n, p, &mone, B, p, Y, n, &one, Mc, K);
        if (bs != CUBLAS_STATUS_SUCCESS) return OSMPS_ECUDA;
        sub_frob_kernel<V2><<<kSubResBlocks, 256, 0, h->stream>>>((const V2 *)Mc, (long long)n * K, rp);
        h->launches += 1;
        int np = 0;
        if (launch_norm2(h, psi, h->partials, &np) != cudaSuccess) return OSMPS_ECUDA;
        sub_entropy_kernel<<<1, 1024, 0, h->stream>>>(th, p, rp, kSubResBlocks, h->partials, np, inf, 3, n, lambda_dev,
                                                      S_dev, st);
        h->launches += 1;
        double hs[4] = {0, 0, 0, 0};
        if (cudaMemcpyAsync(hs, st, sizeof(double) * 3, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            cudaMemcpyAsync(hs + 3, S_dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            return OSMPS_ECUDA;
        if (!std::isfinite(hs[3])) return OSMPS_ENOCONV;  // solver status or a non-finite value
        const double trace = hs[0] + hs[1];
        if (hs[0] <= Lib::kResTol * trace) {
            // the next call starts from the values that mattered here, plus a quarter and 64
            const int cnt = (int)hs[2];
            h->sub_hint = cnt + cnt / 4 + 64;
            return OSMPS_OK;
        }
        if (p >= pmax) {
            h->sub_hint = pmax;
            h->sub_skip = kSubSkip;
            return OSMPS_ENOCONV;  // too much weight outside any affordable subspace: the full route
        }
        p = 2 * p < pmax ? 2 * p : pmax;
    }
}

osmps_status schmidt_subspace(Handle *h, const void *psi, int cut, double *lambda_dev, double *S_dev) {
    if (!subspace_applicable(h, cut)) return OSMPS_EUNSUPPORTED;
    return h->prec == OSMPS_FP64 ? schmidt_subspace_t<double>(h, psi, cut, lambda_dev, S_dev)
                                 : schmidt_subspace_t<float>(h, psi, cut, lambda_dev, S_dev);
}

}  // namespace osmps
