// Matrix-free H.psi for the spin chain H = sum_{i<j} J(j-i) sz_i sz_j + sum_k h_k sx_k.
//
// Paper: Sec. III.D (Krylov mode 2: the rule set is applied to the state
// without building H; cost Eq. OKrylov) with the Hamiltonian of Eq. genericH.
// The paper contracts each rule with the rank-L tensor one site at a time
// (L tensordot passes over psi); here the whole product is one streaming pass
// per group of bits:
//
//   w[b] = E(b) psi[b] + sum_k h_k psi[b ^ 2^k]
//
// * The state is cut into tiles staged in shared memory.  A tile spans a set
//   of bits: every sigma^x on one of those bits pairs two amplitudes of the
//   same tile, so its term is formed on chip.
// * Pass 1 takes the a1 lowest bits (a contiguous 64 KiB tile) and also adds
//   the diagonal; later passes take a chunk of c contiguous low bits (for
//   coalesced 32..128-byte segments, not flipped again) plus a group of g high
//   bits (flipped), accumulating into the partial sum of the previous pass.
// * The diagonal uses the tile structure: with b = (hi, lo),
//       E(b) = E_ll(lo) + E_hh(hi) + sum_{j<a1} s_j(lo) F_j(hi)
//   where F_j(hi) = sum_{i>=a1} J(i-j) s_i(hi).  E_ll is a global table over
//   lo (L1-resident), F and E_hh a per-tile table; per tile the sum over j is
//   folded into two small tables TA (low half of lo, plus E_hh) and TB (high
//   half), so each amplitude costs three lookups and two adds.
// * The last pass optionally fuses the Lanczos/Krylov epilogue
//       w = sv*H u - a*sv*u - b*uprev
//   and the inner products <sv u, w> and |w|^2 (FP32 per thread and tile,
//   FP64 across tiles and CTAs, fixed reduction order).
#include <cuda.h>  // CUtensorMap types; the encoder is fetched through the runtime's driver entry point
#include <cuda_runtime.h>

#include "ed_internal.h"
#include "device_common.cuh"

namespace osmps {

constexpr int kBV = 16;                                 // 16-byte vectors per consumer thread per tile
constexpr int kHB = kBV / 2;                            // processed in two halves
constexpr int kTileV = 1 << (kTileBytesLog2 - 4);       // 16-byte vectors per tile
constexpr int kTab = 192;                               // TA (<= 64) + TB (<= 128) per stage
constexpr int kStages = 2;                              // shared-memory ring of u tiles
constexpr int kConsumerWarps = kPassThreads / 32;       // 8
constexpr int kIBits = 4;                               // log2 kBV: vector-index bits held in registers
constexpr int kTBits = 8;                               // log2 kPassThreads
constexpr int kHpsiThreads = kPassThreads;              // warp 0 also issues the copies
static_assert(kTileV == kBV * kPassThreads && (1 << kIBits) == kBV && (1 << kTBits) == kPassThreads,
              "sixteen vectors per consumer thread per tile");

template <typename T>
struct PassParams {
    const typename Cx<T>::v16 *stream;  // elementwise input: previous Lanczos vector (first pass) or partial sum
    typename Cx<T>::v16 *out;
    const T *Ell;
    const T *Tab;                       // per-tile diagonal tables: TA[64] then TB[128] (first pass)
    const double *epi;                  // sv, a, b (device) or null
    double *partials;                   // 4 doubles per consumer warp
    const int *m_eff;
    int *err;                           // set to 1 when a bounded wait gives up
    long long ntiles;
    int stop_index;
    int L, c, o, g, ta, first, last, epilogue, rank;
    int pf;                             // L2 prefetch distance in tiles beyond the shared-memory stages
    unsigned tile_bytes;
    int df;                             // complex128 with one field on every flipped bit: flip sums on FP32 pairs
    double dfh;                         // that field
    T hb[kMaxL + 1];
};

// ---- complex128 flip sums on the FP32 pipes ----
// x = hi + lo exactly up to 2^-48 |x| with hi, lo FP32 (hi: the top 24 bits of
// the mantissa, lo: the next 24 of the remaining 29), by integer operations
// only; |x| below 2^-126 is flushed to zero (an absolute error < 1.2e-38).
__device__ __forceinline__ void split_df(double x, float &hi, float &lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ffull);
    const int e32 = e - 1023 + 127;
    if (e32 <= 0) {
        hi = 0.0f;
        lo = 0.0f;
        return;
    }
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    hi = __uint_as_float(sign | ((unsigned)(e32 < 255 ? e32 : 255) << 23) | (unsigned)(m >> 29));
    const unsigned rem = (unsigned)(m & 0x1FFFFFFFull);  // x - hi = rem 2^(e - 1075)
    if (rem == 0u) {
        lo = 0.0f;
        return;
    }
    const int pl = 31 - __clz(rem);  // leading one of rem
    const int le = pl + e - 1075 + 127;
    if (le <= 0) {
        lo = 0.0f;
        return;
    }
    const unsigned mant = pl >= 23 ? (rem >> (pl - 23)) : (rem << (23 - pl));
    lo = __uint_as_float(sign | ((unsigned)le << 23) | (mant & 0x7FFFFFu));
}
// exact FP32 -> FP64 by integer operations (FP32 denormals flushed to zero)
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xFFu;
    if (e == 0u) return 0.0;
    const unsigned long long d = ((unsigned long long)(b & 0x80000000u) << 32) |
                                 ((unsigned long long)(e - 127u + 1023u) << 52) |
                                 ((unsigned long long)(b & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)d);
}
// Sum of the hi parts with the exact rounding error of every addition (Knuth's
// TwoSum, no condition on the order of magnitudes) accumulated beside it (the
// cascaded summation of Ogita, Rump and Oishi 2005), plain FP32 sum of the lo
// parts: error O((n u)^2) of the sum of magnitudes, u = 2^-24.
struct DfAcc {
    float s, c, l;
};
__device__ __forceinline__ void df_add(DfAcc &a, float hi, float lo) {
    const float t = a.s + hi;
    const float bp = t - a.s;
    const float ap = t - bp;
    a.c += (a.s - ap) + (hi - bp);
    a.s = t;
    a.l += lo;
}
__device__ __forceinline__ double df_value(const DfAcc &a) { return f2d_bits(a.s) + (f2d_bits(a.c) + f2d_bits(a.l)); }

__device__ __forceinline__ void tma_load(void *dst, const CUtensorMap *tm, int rank, const int *crd,
                                         unsigned long long *bar) {
    const unsigned long long tmp = reinterpret_cast<unsigned long long>(tm);
    if (rank == 3) {
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4}], [%5];" ::"r"(smem_u32(dst)),
            "l"(tmp), "r"(crd[0]), "r"(crd[1]), "r"(crd[2]), "r"(smem_u32(bar))
            : "memory");
    } else {
        asm volatile(
            "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
            "%4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
            "l"(tmp), "r"(crd[0]), "r"(crd[1]), "r"(crd[2]), "r"(crd[3]), "r"(crd[4]), "r"(smem_u32(bar))
            : "memory");
    }
}
__device__ __forceinline__ void tma_prefetch_l2(const CUtensorMap *tm, int rank, const int *crd) {
    const unsigned long long tmp = reinterpret_cast<unsigned long long>(tm);
    if (rank == 3) {
        asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(tmp), "r"(crd[0]),
                     "r"(crd[1]), "r"(crd[2])
                     : "memory");
    } else {
        asm volatile("cp.async.bulk.prefetch.tensor.5d.L2.global.tile [%0, {%1, %2, %3, %4, %5}];" ::"l"(tmp),
                     "r"(crd[0]), "r"(crd[1]), "r"(crd[2]), "r"(crd[3]), "r"(crd[4])
                     : "memory");
    }
}

template <typename V>
__device__ __forceinline__ void st_stream(V *ptr, const V &v) {
    __stcs(ptr, v);
}
// read-only table load that asks L1 to keep the line (the E_ll table is
// re-read by every tile of the first pass)
__device__ __forceinline__ float ld_keep(const float *ptr) {
    float v;
    asm("ld.global.nc.L1::evict_last.f32 %0, [%1];" : "=f"(v) : "l"(ptr));
    return v;
}
__device__ __forceinline__ double ld_keep(const double *ptr) {
    double v;
    asm("ld.global.nc.L1::evict_last.f64 %0, [%1];" : "=d"(v) : "l"(ptr));
    return v;
}

// One pass of the product, warp-specialized and persistent (one CTA per SM):
//  * warp 0 fills a 2-stage shared-memory ring with tiles of u and a third
//    stage with the tile of the elementwise stream (previous Lanczos vector in
//    the first pass, partial sum later), all by TMA (cp.async.bulk.tensor,
//    completion on mbarriers), as soon as the stage is released, and builds
//    the first pass's per-tile diagonal tables;
//  * all 8 warps own the vectors q = tid + 256 i (i < 16) of a
//    tile: flips of the amplitude bit inside a vector and of the four bits of
//    i are formed in registers, flips of the eight bits of tid from shared
//    memory; the stream is read from its stage; results go to global memory
//    with lane-coalesced stores.
// All waits are bounded (2 s); on timeout the error flag is raised, warp 0
// waits for the copies it issued, and the kernel returns.
template <typename T>
__global__ void __launch_bounds__(kHpsiThreads, 1)
    hpsi_pass_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_s,
                     PassParams<T> p) {
    typedef typename Cx<T>::v16 V;
    typedef typename Cx<T>::amp A;
    typedef typename Cx<T>::coef K;
    constexpr int VE = Cx<T>::VE;
    constexpr int LOGVE = Cx<T>::LOGVE;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    V *U = reinterpret_cast<V *>(smem_raw);   // kStages tiles of u
    V *S = U + kStages * kTileV;              // one tile of the stream
    T *tab = reinterpret_cast<T *>(S + kTileV);
    unsigned long long *fullU = reinterpret_cast<unsigned long long *>(tab + kStages * kTab);
    unsigned long long *emptyU = fullU + kStages;
    unsigned long long *fullS = emptyU + kStages;
    unsigned long long *emptyS = fullS + 1;

    if (p.m_eff != nullptr && *p.m_eff <= p.stop_index) return;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&fullU[s], 1);
            mbar_init(&emptyU[s], kConsumerWarps);
        }
        mbar_init(fullS, 1);
        mbar_init(emptyS, kConsumerWarps);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int tbits = p.c + p.g;
    const int nvec = (1 << tbits) >> LOGVE;
    const uint64_t cmask = (1ull << p.c) - 1ull;
    const int oc = p.o - p.c;
    const uint64_t ocmask = (1ull << oc) - 1ull;
    const bool has_stream = p.stream != nullptr;
    const bool dfm = (sizeof(T) == sizeof(double)) && p.df != 0;  // FP32-pair flip sums

    auto coords = [&](long long t, int *crd) {
        if (p.rank == 3) {
            crd[0] = 0;
            crd[1] = 0;
            crd[2] = (int)t;
        } else {
            crd[0] = 0;
            crd[1] = (int)(t & (long long)ocmask);
            crd[2] = 0;
            crd[3] = 0;
            crd[4] = (int)(t >> oc);
        }
    };

    // Copies are issued by warp 0: u of tile k into stage k % kStages once all
    // warps released the stage's previous tile, the stream of tile k once all
    // warps consumed the stream of tile k-1.
    long long nu = 0, ns = 0;
    auto issue_u = [&](long long k, long long t) -> bool {
        const int s = (int)(k % kStages);
        if (k >= kStages) {
            bool w = true;
            if (lane == 0) w = mbar_wait(&emptyU[s], (unsigned)(((k / kStages) & 1) ^ 1), p.err);
            if (!__shfl_sync(0xffffffffu, w ? 1 : 0, 0)) return false;
        }
        if (lane == 0) {
            int crd[5];
            coords(t, crd);
            const unsigned tab_bytes = p.first ? (unsigned)(kTab * sizeof(T)) : 0u;
            mbar_arrive_expect_tx(&fullU[s], p.tile_bytes + tab_bytes);
            tma_load(U + (size_t)s * kTileV, &tm_u, p.rank, crd, &fullU[s]);
            // first pass: the tile's diagonal tables (precomputed per tile) ride on the same barrier
            if (p.first) bulk_load(tab + s * kTab, p.Tab + (size_t)t * kTab, tab_bytes, &fullU[s]);
        }
        return true;
    };
    auto issue_s = [&](long long k, long long t) -> bool {
        if (k >= 1) {
            bool w = true;
            if (lane == 0) w = mbar_wait(emptyS, (unsigned)((k - 1) & 1), p.err);
            if (!__shfl_sync(0xffffffffu, w ? 1 : 0, 0)) return false;
        }
        if (lane == 0) {
            int crd[5];
            coords(t, crd);
            mbar_arrive_expect_tx(fullS, p.tile_bytes);
            tma_load(S, &tm_s, p.rank, crd, fullS);
        }
        return true;
    };
    if (warp == 0) {
        for (long long t = blockIdx.x; t < p.ntiles && nu < kStages; t += gridDim.x) issue_u(nu++, t);
        if (has_stream && blockIdx.x < p.ntiles) issue_s(ns++, blockIdx.x);
    }

    // ------------------------------ consumers ------------------------------
    const int tid = threadIdx.x;
    double sv = 1.0, ea = 0.0, eb = 0.0;
    if (p.epi != nullptr) {
        sv = p.epi[0];
        ea = p.epi[1];
        eb = p.epi[2];
    }
    // first pass: r = H_inner u - a u + bs uprev with bs = -b/sv; later: r = flips + partial
    const T aT = (T)ea;
    const T bsT = (p.first && has_stream) ? (T)(-eb / sv) : (T)1;
    const T svT = (T)sv;
    const int nmine =
        tid < nvec ? ((nvec - 1 - tid) / kPassThreads + 1 < kBV ? (nvec - 1 - tid) / kPassThreads + 1 : kBV) : 0;
    const bool full_tile = (nmine == kBV);
    auto gidx = [&](uint64_t base, int q) -> uint64_t {  // global 16-byte vector index of tile vector q
        const int li = q << LOGVE;
        return (base | ((uint64_t)(li >> p.c) << p.o) | ((uint64_t)li & cmask)) >> LOGVE;
    };

    // E_ll of this thread's amplitudes: they sit at the same low bits in every
    // tile of the first pass, so the table is read once per launch
    T ell[kBV * VE];
#pragma unroll
    for (int e = 0; e < kBV * VE; ++e) {
        const int li = (((e / VE) * kPassThreads + tid) << LOGVE) + (e % VE);
        ell[e] = (p.first && li < (nvec << LOGVE)) ? __ldg(&p.Ell[li]) : (T)0;
    }
    double acc_d0 = 0.0, acc_d1 = 0.0, acc_n = 0.0;
    long long n = 0;
    bool failed = false;
    for (long long t = blockIdx.x; t < p.ntiles; t += gridDim.x, ++n) {
        const int s = (int)(n % kStages);
        if (warp == 0 && n >= 1) {
            // u of tile n-1+kStages into the stage released by tile n-1; stream of tile n
            const long long tu = t + (long long)(kStages - 1) * gridDim.x;
            bool ok = true;
            if (nu == n - 1 + kStages && tu < p.ntiles) ok = issue_u(nu++, tu);
            if (ok && has_stream && ns == n) ok = issue_s(ns++, t);
            if (!ok) {
                if (lane == 0) atomicExch(p.err, 1);
                failed = true;
                if (!dfm) break;  // FP32-pair mode: every thread leaves together at the tile barrier
            }
        }
        if (warp == 0 && lane == 0 && p.pf > 0) {
            // warm L2 up to pf tiles beyond what the shared-memory stages hold:
            // u of the pf-th tile after the ring, the stream pf tiles ahead
            // (the nearer ones were requested by the previous iterations)
            int crd[5];
            const long long tp = t + (long long)(kStages - 1 + p.pf) * gridDim.x;
            if (tp < p.ntiles) {
                coords(tp, crd);
                tma_prefetch_l2(&tm_u, p.rank, crd);
            }
            const long long tq = t + (long long)p.pf * gridDim.x;
            if (has_stream && tq < p.ntiles) {
                coords(tq, crd);
                tma_prefetch_l2(&tm_s, p.rank, crd);
            }
            if (n == 0) {  // the first iteration also requests the nearer tiles
                for (int k = 1; k < p.pf; ++k) {
                    const long long tu = t + (long long)(kStages - 1 + k) * gridDim.x;
                    if (tu < p.ntiles) {
                        coords(tu, crd);
                        tma_prefetch_l2(&tm_u, p.rank, crd);
                    }
                    const long long ts = t + (long long)k * gridDim.x;
                    if (has_stream && ts < p.ntiles) {
                        coords(ts, crd);
                        tma_prefetch_l2(&tm_s, p.rank, crd);
                    }
                }
            }
        }
        const V *Ucur = U + (size_t)s * kTileV;
        const T *tcur = tab + s * kTab;
        const uint64_t tt = (uint64_t)t;
        const uint64_t base = ((tt >> oc) << (p.o + p.g)) | ((tt & ocmask) << p.c);
        {
            const bool okw = mbar_wait(&fullU[s], (unsigned)((n / kStages) & 1), p.err);
            if (dfm) {
                if (__syncthreads_or(!okw || failed)) {
                    atomicExch(p.err, 1);
                    failed = true;
                    break;
                }
            } else if (!okw) {
                atomicExch(p.err, 1);
                break;
            }
        }
        const T *trow = tcur;
        T pd0 = 0, pd1 = 0, pn = 0;
        bool stream_ready = false;
        A self[kBV * VE];
#pragma unroll
        for (int i = 0; i < kBV; ++i) {
            if (full_tile || i < nmine) unpackv(Ucur[i * kPassThreads + tid], &self[i * VE]);
            else unpackv(V{}, &self[i * VE]);
        }
        if constexpr (sizeof(T) == sizeof(double)) {
            if (dfm) {
                // this thread's amplitudes to (re_hi, re_lo, im_hi, im_lo) in place; the
                // flips below read every partner in that form
                float4 *Uf = reinterpret_cast<float4 *>(const_cast<V *>(Ucur));
#pragma unroll
                for (int i = 0; i < kBV; ++i) {
                    if (full_tile || i < nmine) {
                        const double2 a = self[i];
                        float4 f;
                        split_df(a.x, f.x, f.y);
                        split_df(a.y, f.z, f.w);
                        Uf[i * kPassThreads + tid] = f;
                    }
                }
                __syncthreads();
            }
        }
        // accumulate in two halves of eight vectors; all four bits of i are
        // flipped in registers
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            constexpr int NH = kBV / 2;
            A r[NH * VE];
#pragma unroll
            for (int e = 0; e < NH * VE; ++e) r[e] = azero(T(0));
            if constexpr (sizeof(T) == sizeof(double)) {
                if (dfm) {
                    // complex128, one field on every flipped bit: sum of the flipped
                    // partners on FP32 pairs with exact error terms, then one FP64 multiply
                    const float4 *Uf = reinterpret_cast<const float4 *>(Ucur);
                    DfAcc ar[NH], ai[NH];
#pragma unroll
                    for (int i = 0; i < NH; ++i) ar[i] = ai[i] = DfAcc{0.0f, 0.0f, 0.0f};
                    for (int lb = p.c; lb < tbits; ++lb) {
#pragma unroll
                        for (int i = 0; i < NH; ++i) {
                            const int ii = hh * NH + i;
                            if (full_tile || ii < nmine) {
                                const float4 v = Uf[(ii * kPassThreads + tid) ^ (1 << lb)];
                                df_add(ar[i], v.x, v.y);
                                df_add(ai[i], v.z, v.w);
                            }
                        }
                    }
#pragma unroll
                    for (int i = 0; i < NH; ++i) {
                        r[i].x = p.dfh * df_value(ar[i]);
                        r[i].y = p.dfh * df_value(ai[i]);
                    }
                }
            }
            if (!dfm && VE == 2 && p.c == 0) {
                // bit 0 lives inside the 16-byte vector
                const K f = mkcoef(p.hb[p.o]);
#pragma unroll
                for (int i = 0; i < NH; ++i) {
                    const int ii = hh * NH + i;
                    afma(f, self[ii * VE + VE - 1], r[i * VE]);
                    afma(f, self[ii * VE], r[i * VE + VE - 1]);
                }
            }
#pragma unroll
            for (int j = 0; j < kIBits; ++j) {
                const int lb = LOGVE + kTBits + j;  // local bit carried by bit j of i
                if (!dfm && lb >= p.c && lb < tbits) {
                    const K f = mkcoef(p.hb[p.o + lb - p.c]);
#pragma unroll
                    for (int i = 0; i < NH; ++i) {
                        const int ii = hh * NH + i;
#pragma unroll
                        for (int e = 0; e < VE; ++e) afma(f, self[(ii ^ (1 << j)) * VE + e], r[i * VE + e]);
                    }
                }
            }
            // flips of the eight bits of tid: neighbour vectors from shared memory
            if (!dfm) {
                const int lb0 = p.c > LOGVE ? p.c : LOGVE;
                const int lb1 = tbits < LOGVE + kTBits ? tbits : LOGVE + kTBits;
                for (int lb = lb0; lb < lb1; ++lb) {
                    const K f = mkcoef(p.hb[p.o + lb - p.c]);
                    const int flip = 1 << (lb - LOGVE);
#pragma unroll
                    for (int h4 = 0; h4 < NH / kHB; ++h4) {
                        V v[kHB];
#pragma unroll
                        for (int i = 0; i < kHB; ++i) {
                            const int ii = hh * NH + h4 * kHB + i;
                            if (full_tile || ii < nmine) v[i] = Ucur[(ii * kPassThreads + tid) ^ flip];
                            else v[i] = V{};
                        }
#pragma unroll
                        for (int i = 0; i < kHB; ++i) {
                            A x[VE];
                            unpackv(v[i], x);
#pragma unroll
                            for (int e = 0; e < VE; ++e) afma(f, x[e], r[(h4 * kHB + i) * VE + e]);
                        }
                    }
                }
            }
            if (p.first) {
                // E(b) - a = E_ll (registers) + TA (low ta bits) + TB (bits above ta) - a
                const int tmask = (1 << p.ta) - 1;
#pragma unroll
                for (int i = 0; i < NH; ++i) {
                    const int ii = hh * NH + i;
                    if (full_tile || ii < nmine) {
                        const int li = (ii * kPassThreads + tid) << LOGVE;
                        const T tbv = trow[64 + (li >> p.ta)] - aT;
#pragma unroll
                        for (int e = 0; e < VE; ++e) {
                            const T E = ell[ii * VE + e] + trow[(li + e) & tmask] + tbv;
                            afma(mkcoef(E), self[ii * VE + e], r[i * VE + e]);
                        }
                    }
                }
            }
            if (hh == 1) {
                // u stage s is no longer read by this warp (its FP32-pair stores
                // are ordered before the next bulk copy into the stage)
                if (dfm) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&emptyU[s]);
            }
            if (has_stream) {
                if (!stream_ready) {
                    if (!mbar_wait(fullS, (unsigned)(n & 1), p.err)) {
                        atomicExch(p.err, 1);
                        failed = true;
                        if (!dfm) break;  // FP32-pair mode: leave at the next tile barrier
                    }
                    stream_ready = true;
                }
                const K bsK = mkcoef(bsT);
#pragma unroll
                for (int i = 0; i < NH; ++i) {
                    const int ii = hh * NH + i;
                    if (full_tile || ii < nmine) {
                        A x[VE];
                        unpackv(S[ii * kPassThreads + tid], x);
#pragma unroll
                        for (int e = 0; e < VE; ++e) afma(bsK, x[e], r[i * VE + e]);
                    }
                }
                if (hh == 1) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(emptyS);
                }
            }
            if (p.last && p.epilogue != EPI_ENERGY && svT != (T)1) {
                const K svK = mkcoef(svT);
#pragma unroll
                for (int e = 0; e < NH * VE; ++e) amul(svK, r[e]);
            }
            if (!p.last || p.epilogue != EPI_ENERGY) {
#pragma unroll
                for (int i = 0; i < NH; ++i) {
                    const int ii = hh * NH + i;
                    if (full_tile || ii < nmine) {
                        if (p.last) st_stream(&p.out[gidx(base, ii * kPassThreads + tid)], packv(&r[i * VE]));
                        else p.out[gidx(base, ii * kPassThreads + tid)] = packv(&r[i * VE]);
                    }
                }
            }
            if (p.last && p.epilogue == EPI_ENERGY) {
#pragma unroll
                for (int e = 0; e < NH * VE; ++e) {
                    const auto u = tocx(self[hh * NH * VE + e]), w = tocx(r[e]);
                    pd0 = fma(u.x, w.x, fma(u.y, w.y, pd0));
                    pd1 = fma(u.x, w.y, fma(-u.y, w.x, pd1));
                    pn = fma(u.x, u.x, fma(u.y, u.y, pn));
                }
            } else if (p.last && p.epilogue == EPI_KRYLOV) {
#pragma unroll
                for (int e = 0; e < NH * VE; ++e) {
                    const auto u = tocx(self[hh * NH * VE + e]), w = tocx(r[e]);
                    pd0 = fma(u.x, w.x, fma(u.y, w.y, pd0));
                    pd1 = fma(u.x, w.y, fma(-u.y, w.x, pd1));
                    pn = fma(w.x, w.x, fma(w.y, w.y, pn));
                }
            }
        }
        if (failed && !dfm) break;
        acc_d0 += (double)pd0;
        acc_d1 += (double)pd1;
        acc_n += (double)pn;
    }

    if (failed && warp == 0 && lane == 0) {
        // every copy this CTA issued lands before it exits (bounded)
        const long long fu = nu > kStages ? nu - kStages : 0;
        for (long long k = fu; k < nu; ++k)
            mbar_wait(&fullU[(int)(k % kStages)], (unsigned)((k / kStages) & 1), p.err);
        if (ns > 0) mbar_wait(fullS, (unsigned)((ns - 1) & 1), p.err);
    }
    if (p.last && p.epilogue != EPI_PLAIN && p.partials != nullptr) {
        // per-warp partials (fixed order, no CTA barrier so early exits cannot hang)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            acc_d0 += __shfl_xor_sync(0xffffffffu, acc_d0, off);
            acc_d1 += __shfl_xor_sync(0xffffffffu, acc_d1, off);
            acc_n += __shfl_xor_sync(0xffffffffu, acc_n, off);
        }
        if (lane == 0) {
            double *dst = p.partials + 4 * ((size_t)blockIdx.x * kConsumerWarps + warp);
            dst[0] = acc_d0 * sv;
            dst[1] = acc_d1 * sv;
            dst[2] = acc_n;
            dst[3] = 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// Diagonal-energy tables (built once per handle, FP64 then rounded to T)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void ell_table_kernel(T *Ell, int a1, const double *Jr) {
    const int lo = blockIdx.x * blockDim.x + threadIdx.x;
    if (lo >= (1 << a1)) return;
    double E = 0.0;
    for (int j = 0; j < a1; ++j) {
        const int sj = 1 - 2 * ((lo >> j) & 1);
        for (int jj = j + 1; jj < a1; ++jj) {
            const int sjj = 1 - 2 * ((lo >> jj) & 1);
            E += Jr[jj - j] * (double)(sj * sjj);
        }
    }
    Ell[lo] = (T)E;
}

template <typename T>
__global__ void fhh_table_kernel(T *Fhh, int L, int a1, const double *Jr, long long ntiles) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ntiles * (a1 + 1)) return;
    const long long t = idx / (a1 + 1);
    const int j = (int)(idx % (a1 + 1));
    double s = 0.0;
    if (j < a1) {
        for (int i = a1; i < L; ++i) {
            const int si = 1 - 2 * (int)((t >> (i - a1)) & 1);
            s += Jr[i - j] * (double)si;
        }
    } else {
        for (int i = a1; i < L; ++i) {
            const int si = 1 - 2 * (int)((t >> (i - a1)) & 1);
            for (int ii = i + 1; ii < L; ++ii) {
                const int sii = 1 - 2 * (int)((t >> (ii - a1)) & 1);
                s += Jr[ii - i] * (double)(si * sii);
            }
        }
    }
    Fhh[idx] = (T)s;
}

// Per-tile tables of the first pass: TA[x] = E_hh + sum_{j<ta} s_j(x) F_j and
// TB[y] = sum_{j<a1-ta} s_j(y) F_{ta+j} for every tile (row of Fhh).
template <typename T>
__global__ void tab_table_kernel(T *Tab, const T *Fhh, long long ntiles, int a1, int ta) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ntiles * kTab) return;
    const long long t = idx / kTab;
    const int x = (int)(idx % kTab);
    const T *F = Fhh + (size_t)t * (size_t)(a1 + 1);
    const int tb = a1 - ta;
    double v = 0.0;
    if (x < 64) {
        if (x < (1 << ta)) {
            v = (double)F[a1];
            for (int j = 0; j < ta; ++j) v += ((x >> j) & 1) ? -(double)F[j] : (double)F[j];
        }
    } else {
        const int y = x - 64;
        if (y < (1 << tb))
            for (int j = 0; j < tb; ++j) v += ((y >> j) & 1) ? -(double)F[ta + j] : (double)F[ta + j];
    }
    Tab[idx] = (T)v;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
PassPlan make_plan(int L, int prec) {
    PassPlan pl{};
    const int logE = (prec == OSMPS_FP64) ? 4 : 3;       // log2 bytes per amplitude
    const int TB = kTileBytesLog2 - logE;                  // tile bits (64 KiB tile)
    const int cmin = 5 - logE;                             // chunk >= one 32-byte sector
    const int cmax = 11 - logE;                            // chunk <= 256 eight-byte words (TMA box)
    pl.a1 = L < TB ? L : TB;
    pl.ta = pl.a1 / 2;
    pl.p[0] = PassDesc{0, 0, pl.a1, 1, 1ll << (L - pl.a1)};
    pl.npass = 1;
    const int rest = L - pl.a1;
    if (rest > 0) {
        const int room = TB - cmin;
        const int k = (rest + room - 1) / room;
        int o = pl.a1;
        int left = rest;
        for (int i = 0; i < k; ++i) {
            const int g = (left + (k - i) - 1) / (k - i);
            // fill the tile: carry as many contiguous low bits as fit
            int c = TB - g;
            if (c > cmax) c = cmax;
            if (c > pl.a1) c = pl.a1;
            if (c < cmin) c = cmin;
            pl.p[pl.npass++] = PassDesc{c, o, g, 0, 1ll << (L - c - g)};
            o += g;
            left -= g;
        }
    }
    return pl;
}

static size_t pass_smem() {
    return (size_t)(kStages + 1) * (1u << kTileBytesLog2) + (size_t)kStages * kTab * sizeof(double) +
           (2 * kStages + 2) * sizeof(unsigned long long);
}

template <typename T>
static int grid_for(Handle *h, long long ntiles) {
    static int occ = -1;
    if (occ < 0) {
        cudaFuncSetAttribute(hpsi_pass_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem());
        // smallest shared-memory carve-out that fits (the rest stays L1 for the E_ll table)
        int maxsm = 0;
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device);
        if (maxsm > 0) {
            int pct = (int)((pass_smem() + 2048) * 100 / (size_t)maxsm) + 1;
            if (pct > 100) pct = 100;
            cudaFuncSetAttribute(hpsi_pass_kernel<T>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
        }
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hpsi_pass_kernel<T>, kHpsiThreads, pass_smem());
        occ = n > 0 ? n : 1;
    }
    long long g = (long long)occ * h->nsm;
    return (int)(ntiles < g ? ntiles : g);
}

int hpsi_grid(Handle *h, int pass) {
    const long long nt = h->plan.p[pass].ntiles;
    return h->prec == OSMPS_FP64 ? grid_for<double>(h, nt) : grid_for<float>(h, nt);
}

int hpsi_partials_per_cta() { return kConsumerWarps; }

// ---- tensor maps ----
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)ptr;
        else
            cudaGetLastError();
    }
    return fn;
}

// Tensor map of the tiles of one pass over the vector at base (8-byte words).
//  first pass : 3-D (256-word rows, rows per tile, tiles)
//  later      : 5-D (chunk words, low other bits, low group bits, high group
//               bits, high other bits); the box is one tile, landing in shared
//               memory as local index (group << c) | chunk.
static cudaError_t encode_pass_map(Handle *h, const PassDesc &d, const void *base, CUtensorMap *tm, int *rank) {
    EncodeTiledFn enc = encoder();
    if (enc == nullptr) return cudaErrorNotSupported;
    const uint64_t e = h->esize / 8;  // words per amplitude
    cuuint64_t dims[5], strides[4];
    cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
    if (d.first) {
        const uint64_t W = (1ull << d.g) * e;
        const uint64_t d0 = W < 256 ? W : 256;
        dims[0] = d0;
        dims[1] = W / d0;
        dims[2] = (cuuint64_t)d.ntiles;
        strides[0] = d0 * 8;
        strides[1] = W * 8;
        box[0] = (cuuint32_t)d0;
        box[1] = (cuuint32_t)(W / d0);
        box[2] = 1;
        *rank = 3;
    } else {
        const int g1 = d.g < 8 ? d.g : 8, g2 = d.g - g1;
        const uint64_t X = (1ull << d.c) * e;
        dims[0] = X;
        dims[1] = 1ull << (d.o - d.c);
        dims[2] = 1ull << g1;
        dims[3] = 1ull << g2;
        dims[4] = 1ull << (h->L - d.o - d.g);
        strides[0] = (1ull << d.c) * h->esize;
        strides[1] = (1ull << d.o) * h->esize;
        strides[2] = (1ull << (d.o + g1)) * h->esize;
        strides[3] = (1ull << (d.o + d.g)) * h->esize;
        box[0] = (cuuint32_t)X;
        box[1] = 1;
        box[2] = 1u << g1;
        box[3] = 1u << g2;
        box[4] = 1;
        *rank = 5;
    }
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT64, (cuuint32_t)*rank, const_cast<void *>(base), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t build_tables_t(Handle *h) {
    cudaError_t err = cudaSuccess;
    const int a1 = h->plan.a1;
    const long long nt = 1ll << (h->L - a1);
    const size_t ell_bytes = sizeof(T) << a1;
    const size_t fhh_bytes = sizeof(T) * (size_t)nt * (size_t)(a1 + 1);
    h->Ell = dev_alloc(h, ell_bytes, &err);
    if (err != cudaSuccess) return err;
    h->Fhh = dev_alloc(h, fhh_bytes, &err);
    if (err != cudaSuccess) return err;
    double *Jd = nullptr;
    err = cudaMalloc(&Jd, sizeof(double) * (kMaxL + 1));
    if (err != cudaSuccess) return err;
    err = cudaMemcpyAsync(Jd, h->Jr, sizeof(double) * (kMaxL + 1), cudaMemcpyHostToDevice, h->stream);
    if (err == cudaSuccess) {
        ell_table_kernel<T><<<((1 << a1) + 255) / 256, 256, 0, h->stream>>>((T *)h->Ell, a1, Jd);
        const long long n = nt * (a1 + 1);
        fhh_table_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>((T *)h->Fhh, h->L, a1, Jd, nt);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) {
        h->Tab = dev_alloc(h, sizeof(T) * (size_t)nt * kTab, &err);
        if (err == cudaSuccess) {
            const long long n2 = nt * kTab;
            tab_table_kernel<T><<<(unsigned)((n2 + 255) / 256), 256, 0, h->stream>>>((T *)h->Tab,
                                                                                     (const T *)h->Fhh, nt, a1,
                                                                                     h->plan.ta);
            err = cudaGetLastError();
        }
    }
    cudaError_t e2 = cudaStreamSynchronize(h->stream);
    cudaFree(Jd);
    return err != cudaSuccess ? err : e2;
}

cudaError_t build_tables(Handle *h) {
    return h->prec == OSMPS_FP64 ? build_tables_t<double>(h) : build_tables_t<float>(h);
}

template <typename T>
static cudaError_t launch_hpsi_t(Handle *h, const HpsiArgs &a, int *nparts_out) {
    typedef typename Cx<T>::v16 V;
    const PassPlan &pl = h->plan;
    int nparts = 0;
    for (int i = 0; i < pl.npass; ++i) {
        const PassDesc &d = pl.p[i];
        PassParams<T> p{};
        const bool last = (i == pl.npass - 1);
        // ping-pong: pass i reads the partial written by pass i-1
        const void *src_acc = nullptr;
        void *dst = nullptr;
        if (pl.npass == 1) {
            dst = a.out;
        } else {
            // passes alternate between tmp and out so that the last one lands in out
            const int from_end = pl.npass - 1 - i;
            dst = (from_end % 2 == 0) ? a.out : a.tmp;
            if (i > 0) src_acc = ((from_end + 1) % 2 == 0) ? a.out : a.tmp;
        }
        if (last && a.epilogue == EPI_ENERGY) dst = nullptr;
        const void *stream = (i == 0) ? a.uprev : src_acc;
        CUtensorMap tm_u, tm_s;
        int rank = 0, rank_s = 0;
        cudaError_t err = encode_pass_map(h, d, a.u, &tm_u, &rank);
        if (err != cudaSuccess) return err;
        if (stream != nullptr) {
            err = encode_pass_map(h, d, stream, &tm_s, &rank_s);
            if (err != cudaSuccess) return err;
        } else {
            tm_s = tm_u;
        }
        p.stream = reinterpret_cast<const V *>(stream);
        p.out = reinterpret_cast<V *>(dst);
        p.Ell = reinterpret_cast<const T *>(h->Ell);
        p.Tab = reinterpret_cast<const T *>(h->Tab);
        p.epi = a.epi;
        p.partials = a.partials;
        p.m_eff = a.m_eff;
        p.err = &h->ctl->error;
        p.stop_index = a.stop_index;
        p.ntiles = d.ntiles;
        p.L = h->L;
        p.c = d.c;
        p.o = d.o;
        p.g = d.g;
        p.ta = pl.ta;
        p.first = d.first;
        p.last = last ? 1 : 0;
        p.epilogue = a.epilogue;
        p.rank = rank;
        p.pf = h->prefetch;
        p.tile_bytes = (unsigned)((1u << (d.c + d.g)) * h->esize);
        for (int k = 0; k <= kMaxL; ++k) p.hb[k] = (T)h->hbit[k];
        // complex128 passes that flip many bits sharing one field sum on FP32 pairs:
        // the split and recombination cost about as much as six FP64 flips, and
        // the FP32-pair code is issue-bound at this kernel's 8 warps per SM, so
        // only the passes of ten or more flipped bits (the first) gain
        p.df = 0;
        p.dfh = 0.0;
        if (sizeof(T) == sizeof(double) && h->flip_pairs && d.g >= 10) {
            bool uniform = true;
            for (int k = d.o + 1; k < d.o + d.g; ++k) uniform = uniform && (h->hbit[k] == h->hbit[d.o]);
            if (uniform) {
                p.df = 1;
                p.dfh = h->hbit[d.o];
            }
        }
        const int grid = grid_for<T>(h, d.ntiles);
        hpsi_pass_kernel<T><<<grid, kHpsiThreads, pass_smem(), h->stream>>>(tm_u, tm_s, p);
        h->launches += 1;
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        if (last) nparts = grid * kConsumerWarps;
    }
    if (nparts_out) *nparts_out = nparts;
    return cudaSuccess;
}

cudaError_t launch_hpsi(Handle *h, const HpsiArgs &a, int *nparts_out) {
    return h->prec == OSMPS_FP64 ? launch_hpsi_t<double>(h, a, nparts_out)
                                 : launch_hpsi_t<float>(h, a, nparts_out);
}

}  // namespace osmps
