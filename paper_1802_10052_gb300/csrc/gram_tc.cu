// Half-chain reduced density matrix rho = M M^dagger on the 5th-generation
// tensor cores (Sec. IV, bond entropy: the one dense contraction of the path).
//
// M is the state reshaped to (n, K) with rows contiguous (complex64).  With
// P = [Re M | Im M] (n x 2K real, split into TF32 hi and lo parts):
//   Re rho = P P^T                      (K' = 2K)
//   Im rho = G^T - G,  G = Re M (Im M)^T  (K' = K)
// Each product uses three TF32 MMAs per K-step (hi*hi + hi*lo + lo*hi), the
// "3xTF32" split that recovers FP32-level accuracy on TF32 tensor cores
// (Ootomo & Yokota 2022).  A CTA owns one 128 x 128 output tile:
//   warp 0  TMA producer (128-byte-swizzled 128 x 32 tiles of P_hi, P_lo for
//           the row and column blocks, 3-stage ring) and TMEM allocator;
//   warp 1  one thread issues tcgen05.mma (cta_group::1, kind::tf32,
//           M = N = 128, K = 8) and returns stages with tcgen05.commit;
//   warps 2..5 read each K-chunk's FP32 accumulator back with tcgen05.ld
//           and add it into registers (the tensor cores' accumulation
//           truncates; chunking keeps that bias near 2^-24 x 48).
// Only the tiles of the upper triangle (row block <= column block) of Re rho
// are formed: that is the triangle the eigenvalue solver reads.
//
// The same kernel forms the cross product of two different row sets (mode 2)
// for the Schmidt values as Rayleigh quotients: B = U^H A with U the
// eigenvectors of rho, |B_i|^2 = u_i^H rho u_i, formed from A itself (no
// squared matrix), and only the row sums of |B|^2 leave the chip.  All waits are
// bounded; on timeout the kernel raises the error flag, lets the MMAs it
// issued finish, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "ed_internal.h"

namespace osmps {

namespace gtc {

constexpr int kTile = 128;                 // output tile (M = N)
constexpr int kKc = 32;                    // floats per stage row (128 bytes)
constexpr int kStages = 3;
constexpr int kOpBytes = kTile * kKc * 4;  // one operand tile: 16 KiB
constexpr int kStageBytes = 4 * kOpBytes;  // A_hi, A_lo, B_hi, B_lo
constexpr int kThreads = 192;                // warp 0 TMA, warp 1 MMA, warps 2..5 epilogue
constexpr int kChunk = 4;                    // stages accumulated in TMEM before a register readout

__device__ __forceinline__ void tma2d(void *dst, const CUtensorMap *tm, int c0, int c1, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// tcgen05 shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row core-matrix groups 1024 bytes apart (stride byte offset), leading
// byte offset unused for swizzled K-major layouts (encoded 1), version 1.
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFFu);
    d |= (unsigned long long)1 << 16;                 // leading byte offset (ignored)
    d |= (unsigned long long)(1024 >> 4) << 32;       // stride byte offset
    d |= (unsigned long long)1 << 46;                 // descriptor version
    d |= (unsigned long long)2 << 61;                 // SWIZZLE_128B
    return d;
}
// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major,
// N = 128, M = 128.
constexpr unsigned kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(kTile >> 3) << 17) |
                            ((unsigned)(kTile >> 4) << 24);

__device__ __forceinline__ void mma_tf32(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// planes: P[x][k] = Re M[x][k], P[x][K + k] = Im M[x][k]; hi = TF32 rounding, lo = rest
__global__ void split_planes_kernel(const float2 *psi, int n, long long K, float *Phi, float *Plo) {
    const long long total = (long long)n * K;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long x = i / K, k = i % K;
        const float2 a = psi[i];
        unsigned ur, ui;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(ur) : "f"(a.x));
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(ui) : "f"(a.y));
        const float hr = __uint_as_float(ur), hi_ = __uint_as_float(ui);
        const long long row = x * 2 * K;
        Phi[row + k] = hr;
        Plo[row + k] = a.x - hr;
        Phi[row + K + k] = hi_;
        Plo[row + K + k] = a.y - hi_;
    }
}

__device__ __forceinline__ void tf32_split(float v, float &hi, float &lo) {
    unsigned u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
    hi = __uint_as_float(u);
    lo = v - hi;
}

// Rows of the left factor of the Rayleigh images: R (row-major n x n complex,
// R[i][x] = conj(u_i[x])) as PX[i] = [Re R_i | Im R_i] and QX[i] = [Im R_i | -Re R_i],
// so that Re (R A)[i][k] = PX_i . PY_k and Im (R A)[i][k] = QX_i . PY_k.
__global__ void x_planes_kernel(const float2 *R, int n, float *Phi, float *Plo, float *Qhi, float *Qlo) {
    const long long total = (long long)n * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / n, x = i % n;
        const float2 a = R[i];
        float hr, lr, hi_, li;
        tf32_split(a.x, hr, lr);
        tf32_split(a.y, hi_, li);
        const long long row = r * 2 * n;
        Phi[row + x] = hr;
        Plo[row + x] = lr;
        Phi[row + n + x] = hi_;
        Plo[row + n + x] = li;
        Qhi[row + x] = hi_;
        Qlo[row + x] = li;
        Qhi[row + n + x] = -hr;
        Qlo[row + n + x] = -lr;
    }
}

// Rows of the right factor: Y[k][x] = conj(A[x][k]), A[x][k] = psi[x * sx + k * sk]
// (sx = 1 or sk = 1), as PY[k] = [Re Y_k | Im Y_k]; 32 x 32 tiles through shared
// memory so that the reads run along the contiguous index of psi and the
// writes along x.
__global__ void y_planes_kernel(const float2 *psi, int n, long long sx, long long sk, float *Phi, float *Plo) {
    __shared__ float2 t[32][33];  // t[k - k0][x - x0]
    const int x0 = blockIdx.x * 32;
    const long long k0 = (long long)blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int xl = (sx == 1) ? (int)threadIdx.x : r, kl = (sx == 1) ? r : (int)threadIdx.x;
        t[kl][xl] = psi[(long long)(x0 + xl) * sx + (k0 + kl) * sk];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const long long row = (k0 + r) * 2 * n;
        const int x = x0 + threadIdx.x;
        const float2 a = t[r][threadIdx.x];
        float h, l;
        tf32_split(a.x, h, l);
        Phi[row + x] = h;
        Plo[row + x] = l;
        tf32_split(-a.y, h, l);
        Phi[row + n + x] = h;
        Plo[row + n + x] = l;
    }
}

// One 128 x 128 tile of  mode 0: Re rho = P P^T (upper-triangle tiles)
//                        mode 1: G = P[:, :K] P[:, K:]^T (all tiles)
// The tensor cores accumulate in FP32 with truncation, so a long K-loop into
// one TMEM accumulator is biased low (about 2^-24 per accumulation).  The
// K-loop is therefore cut into chunks of kChunk stages, each accumulated in
// one of two TMEM buffers and added by the epilogue warps into FP32 registers
// (round to nearest) while the next chunk is computed.
//                        mode 2: rows x of A (ahi, alo) against rows y of B (bhi,
//                                the same K offset 0, nk stages); each output row's
//                                sum of squares over the tile goes to
//                                part[x * ntx + tile column] in FP64
__global__ void __launch_bounds__(kThreads, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap ahi, const __grid_constant__ CUtensorMap alo,
                   const __grid_constant__ CUtensorMap bhi, const __grid_constant__ CUtensorMap blo, int mode,
                   int n, int nk, int kb, int ntx, float2 *rho, float *G, double *part, int *err) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned stages (128-byte swizzle atoms)
    const unsigned raw = smem_u32(smem_raw);
    unsigned char *smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    unsigned long long *full = reinterpret_cast<unsigned long long *>(smem + kStages * kStageBytes);
    unsigned long long *empty = full + kStages;
    unsigned long long *chunk_done = empty + kStages;  // [2]
    unsigned long long *acc_free = chunk_done + 2;     // [2]
    unsigned long long *drain = acc_free + 2;
    unsigned *tmem_slot = reinterpret_cast<unsigned *>(drain + 1);

    const int T = n / kTile;
    int ty, tx;
    if (mode == 0) {  // upper triangle: ty <= tx
        int t = blockIdx.x;
        ty = 0;
        while (t >= T - ty) {
            t -= T - ty;
            ++ty;
        }
        tx = ty + t;
    } else if (mode == 1) {
        ty = blockIdx.x / T;
        tx = blockIdx.x % T;
    } else {
        ty = blockIdx.x / ntx;
        tx = blockIdx.x % ntx;
    }
    const int x0 = ty * kTile, y0 = tx * kTile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&chunk_done[b], 1);
            mbar_init(&acc_free[b], 4);
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * kTile)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;

    const int nchunks = (nk + kChunk - 1) / kChunk;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer ----
            int issued = 0;
            for (int s = 0; s < nk; ++s) {
                const int st = s % kStages;
                if (s >= kStages && !mbar_wait(&empty[st], (unsigned)(((s / kStages) - 1) & 1), err)) {
                    atomicExch(err, 1);
                    break;
                }
                unsigned char *base = smem + st * kStageBytes;
                mbar_arrive_expect_tx(&full[st], kStageBytes);
                tma2d(base, &ahi, s * kKc, x0, &full[st]);
                tma2d(base + kOpBytes, &alo, s * kKc, x0, &full[st]);
                tma2d(base + 2 * kOpBytes, &bhi, kb + s * kKc, y0, &full[st]);
                tma2d(base + 3 * kOpBytes, &blo, kb + s * kKc, y0, &full[st]);
                ++issued;
            }
            // every copy issued has landed before the CTA moves on
            for (int s = issued > kStages ? issued - kStages : 0; s < issued; ++s)
                mbar_wait(&full[s % kStages], (unsigned)((s / kStages) & 1), err);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            for (int s = 0; s < nk; ++s) {
                const int st = s % kStages;
                const int c = s / kChunk, buf = c & 1;
                if (s % kChunk == 0 && c >= 2 &&
                    !mbar_wait(&acc_free[buf], (unsigned)(((c / 2) - 1) & 1), err)) {
                    atomicExch(err, 1);
                    break;
                }
                if (!mbar_wait(&full[st], (unsigned)((s / kStages) & 1), err)) {
                    atomicExch(err, 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned base = smem_u32(smem + st * kStageBytes);
                const unsigned dcol = tmem + (unsigned)(buf * kTile);
#pragma unroll
                for (int kk = 0; kk < kKc / 8; ++kk) {
                    const unsigned off = kk * 32;  // 8 tf32 = 32 bytes along K
                    const unsigned long long ahi = smem_desc(base + off), alo = smem_desc(base + kOpBytes + off);
                    const unsigned long long bhi = smem_desc(base + 2 * kOpBytes + off);
                    const unsigned long long blo = smem_desc(base + 3 * kOpBytes + off);
                    mma_tf32(dcol, ahi, bhi, ((s % kChunk) | kk) != 0 ? 1u : 0u);
                    mma_tf32(dcol, ahi, blo, 1u);
                    mma_tf32(dcol, alo, bhi, 1u);
                }
                mma_commit(&empty[st]);  // stage free once these MMAs have read it
                if (s % kChunk == kChunk - 1 || s == nk - 1) mma_commit(&chunk_done[buf]);
            }
            // no MMA of this CTA is in flight past this point
            mma_commit(drain);
            mbar_wait(drain, 0u, err);
        }
    } else {
        // ---- epilogue warps: TMEM chunk -> FP32 registers ----
        const int lg = warp & 3;  // TMEM lane group this warp may access
        float sum[kTile];
#pragma unroll
        for (int j = 0; j < kTile; ++j) sum[j] = 0.0f;
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            const int buf = c & 1;
            if (!mbar_wait(&chunk_done[buf], (unsigned)((c / 2) & 1), err)) {
                atomicExch(err, 1);
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int q = 0; q < kTile / 32; ++q) {
                unsigned v[32];
                const unsigned taddr = tmem + ((unsigned)(lg * 32) << 16) + (unsigned)(buf * kTile + q * 32);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, "
                    "%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                      "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                      "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 32; ++j) sum[q * 32 + j] += __uint_as_float(v[j]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_free[buf])) : "memory");
        }
        if (ok) {
            const int row = lg * 32 + lane;
            const long long o = (long long)(x0 + row) * n + y0;
            if (mode == 0) {
#pragma unroll
                for (int j = 0; j < kTile; ++j) rho[o + j].x = sum[j];
            } else if (mode == 2) {
                double s2 = 0.0;
#pragma unroll
                for (int j = 0; j < kTile; ++j) s2 = fma((double)sum[j], (double)sum[j], s2);
                part[(long long)(x0 + row) * ntx + tx] = s2;
            } else {
#pragma unroll
                for (int j = 0; j < kTile; j += 4)
                    *reinterpret_cast<float4 *>(&G[o + j]) = make_float4(sum[j], sum[j + 1], sum[j + 2], sum[j + 3]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTile) : "memory");
}

// Im rho[x][y] = G[y][x] - G[x][y] on the upper triangle (x <= y); 32 x 32
// tiles through shared memory so that both reads are coalesced.
__global__ void gram_assemble_kernel(const float *G, float2 *rho, int n) {
    __shared__ float Gt[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;  // tile rows x in [by, by+32), cols y in [bx, bx+32)
    if (bx + 31 < by) return;                               // wholly below the diagonal
    // load G[y][x] for y in [bx, bx+32), x in [by, by+32) (transposed tile)
    for (int i = threadIdx.y; i < 32; i += blockDim.y) Gt[i][threadIdx.x] = G[(long long)(bx + i) * n + by + threadIdx.x];
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int x = by + i, y = bx + threadIdx.x;
        if (x <= y) {
            const long long o = (long long)x * n + y;
            rho[o].y = (x == y) ? 0.0f : Gt[threadIdx.x][i] - G[o];
        }
    }
}

}  // namespace gtc

size_t gram_tc_smem() { return (size_t)gtc::kStages * gtc::kStageBytes + 1024 + 256; }

// Encoder of the TMA maps (runtime driver entry point)
typedef CUresult (*GtcEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static GtcEncodeFn gtc_encoder() {
    static GtcEncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (GtcEncodeFn)ptr;
        else
            cudaGetLastError();
    }
    return fn;
}

bool gram_tc_supported(int n, long long K) {
    return n >= gtc::kTile && n % gtc::kTile == 0 && K % gtc::kKc == 0 && K <= (1ll << 30) && gtc_encoder() != nullptr;
}

// rho (n x n complex64, row-major, upper triangle filled) of the rows of psi
// viewed as (n, K); scratch: two planes of n x 2K floats and G (n x n floats)
cudaError_t gram_tc_launch(Handle *h, const void *psi, int n, long long K, void *rho, float *planes, float *G) {
    GtcEncodeFn enc = gtc_encoder();
    if (enc == nullptr) return cudaErrorNotSupported;
    float *Phi = planes, *Plo = planes + (size_t)n * 2 * K;
    gtc::split_planes_kernel<<<h->nsm * 8, 256, 0, h->stream>>>((const float2 *)psi, n, K, Phi, Plo);
    CUtensorMap thi, tlo;
    cuuint64_t dims[2] = {(cuuint64_t)(2 * K), (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)(2 * K * 4)};
    cuuint32_t box[2] = {gtc::kKc, gtc::kTile}, es[2] = {1, 1};
    if (enc(&thi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Phi, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        enc(&tlo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Plo, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gtc::gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_tc_smem());
        attr = true;
    }
    const int T = n / gtc::kTile;
    gtc::gram_tc_kernel<<<T * (T + 1) / 2, gtc::kThreads, gram_tc_smem(), h->stream>>>(
        thi, tlo, thi, tlo, 0, n, (int)(2 * K / gtc::kKc), 0, T, (float2 *)rho, G, nullptr, &h->ctl->error);
    gtc::gram_tc_kernel<<<T * T, gtc::kThreads, gram_tc_smem(), h->stream>>>(
        thi, tlo, thi, tlo, 1, n, (int)(K / gtc::kKc), (int)K, T, (float2 *)rho, G, nullptr, &h->ctl->error);
    dim3 g2(n / 32, n / 32), b2(32, 8);
    gtc::gram_assemble_kernel<<<g2, b2, 0, h->stream>>>(G, (float2 *)rho, n);
    h->launches += 4;
    return cudaGetLastError();
}

bool rayleigh_tc_supported(int n, long long K) {
    return n >= gtc::kTile && n % gtc::kTile == 0 && K % gtc::kTile == 0 && K >= n && K / gtc::kTile <= (1ll << 24) &&
           gtc_encoder() != nullptr;
}

size_t rayleigh_tc_plane_floats(int n, long long K) { return 8 * (size_t)n * n + 4 * (size_t)n * (size_t)K; }

// Row sums of |B|^2 for B = R A: R row-major n x n complex64 (R[i][x] = conj(u_i[x])),
// A[x][k] = psi[x * sx + k * sk] (n x K).  planes: rayleigh_tc_plane_floats(n, K)
// floats; part_re / part_im: n x (K / 128) doubles, the sums over each 128-column
// tile of (Re B)^2 and (Im B)^2.
cudaError_t rayleigh_tc_launch(Handle *h, const void *R, const void *psi, int n, long long K, long long sx,
                               long long sk, float *planes, double *part_re, double *part_im) {
    GtcEncodeFn enc = gtc_encoder();
    if (enc == nullptr || !rayleigh_tc_supported(n, K)) return cudaErrorNotSupported;
    const size_t xp = 2 * (size_t)n * n, yp = 2 * (size_t)n * (size_t)K;
    float *PXhi = planes, *PXlo = PXhi + xp, *QXhi = PXlo + xp, *QXlo = QXhi + xp;
    float *PYhi = QXlo + xp, *PYlo = PYhi + yp;
    gtc::x_planes_kernel<<<h->nsm * 8, 256, 0, h->stream>>>((const float2 *)R, n, PXhi, PXlo, QXhi, QXlo);
    {
        const dim3 g((unsigned)(n / 32), (unsigned)(K / 32)), b(32, 8);
        gtc::y_planes_kernel<<<g, b, 0, h->stream>>>((const float2 *)psi, n, sx, sk, PYhi, PYlo);
    }
    CUtensorMap m[6];
    float *base[6] = {PXhi, PXlo, QXhi, QXlo, PYhi, PYlo};
    for (int i = 0; i < 6; ++i) {
        cuuint64_t dims[2] = {(cuuint64_t)(2 * n), (cuuint64_t)(i < 4 ? n : K)};
        cuuint64_t strides[1] = {(cuuint64_t)(2 * (size_t)n * 4)};
        cuuint32_t box[2] = {gtc::kKc, gtc::kTile}, es[2] = {1, 1};
        if (enc(&m[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base[i], dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    }
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(gtc::gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_tc_smem());
        attr = true;
    }
    const int ntx = (int)(K / gtc::kTile), nty = n / gtc::kTile;
    const int nk = 2 * n / gtc::kKc;
    gtc::gram_tc_kernel<<<nty * ntx, gtc::kThreads, gram_tc_smem(), h->stream>>>(
        m[0], m[1], m[4], m[5], 2, n, nk, 0, ntx, nullptr, nullptr, part_re, &h->ctl->error);
    gtc::gram_tc_kernel<<<nty * ntx, gtc::kThreads, gram_tc_smem(), h->stream>>>(
        m[2], m[3], m[4], m[5], 2, n, nk, 0, ntx, nullptr, nullptr, part_im, &h->ctl->error);
    h->launches += 4;
    return cudaGetLastError();
}

}  // namespace osmps
