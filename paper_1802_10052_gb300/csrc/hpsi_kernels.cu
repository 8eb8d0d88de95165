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
//   and the inner products <sv u, w> and |w|^2 (FP32 per thread, tile and
//   warp, FP64 across tiles and CTAs, fixed reduction order).
#include <cuda.h>  // CUtensorMap types; the encoder is fetched through the runtime's driver entry point
#include <cuda_runtime.h>

#include "ed_internal.h"
#include "device_common.cuh"

namespace osmps {

constexpr int kTileV = 1 << (kTileBytesLog2 - 4);       // 16-byte vectors per tile
constexpr int kTab = 192;                               // TA (<= 64) + TB (<= 128) per stage
constexpr int kStages = 2;                              // shared-memory ring of u tiles
constexpr int kMaxPassWarps = kTileV / 8 / 32;          // 16: the 512-thread shape
__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }
// Two CTA shapes over the same 64 KiB tile: BV = 16 vectors per thread (256
// threads: four vector-index bits flipped in registers, eight thread bits from
// shared memory) or BV = 8 (512 threads: three in registers, nine from shared
// memory, twice the warps to hide latency with half the registers).
static_assert(kTileV / 16 == kPassThreads, "the 256-thread shape holds sixteen vectors per thread");

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
    KrylovCtl *fold_ctl;                // first pass of Lanczos step stop_index >= 1: beta, scale and the
    const double *fold_parts;           //   epilogue scalars from the update's partial |u|^2 (else null)
    int fold_nparts;
    int fx;                             // complex128 with one field on every flipped bit: flip sums in fixed point
    double fxh;                         // that field
    T hb[kMaxL + 1];
};

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
//  * all warps own the vectors q = tid + NT i (i < BV) of a tile: flips of
//    the amplitude bit inside a vector and of the bits of i are formed in
//    registers, flips of the bits of tid from shared memory; the stream is
//    read from its stage; results go to global memory with lane-coalesced
//    stores.
// All waits are bounded (2 s); on timeout the error flag is raised, warp 0
// waits for the copies it issued, and the kernel returns.
template <typename T, int BV>
__global__ void __launch_bounds__(kTileV / BV, 1)
    hpsi_pass_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_s,
                     PassParams<T> p) {
    constexpr int NT = kTileV / BV;      // threads; all of them consume, warp 0 also issues the copies
    constexpr int NW = NT / 32;          // consumer warps
    constexpr int IBITS = ilog2c(BV);    // vector-index bits held in registers
    constexpr int TBITS = ilog2c(NT);    // thread bits, flipped through shared memory
    constexpr int HB = BV / 2;           // vectors per batch of shared-memory loads
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
    unsigned *fxe = reinterpret_cast<unsigned *>(emptyS + 1);  // per stage: the tile's largest FP64 exponent

    if (p.m_eff != nullptr && *p.m_eff <= p.stop_index) return;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Lanczos control of this step folded in (as a control kernel would do it
    // between the update and this product): beta_j = |u_j| from the update's
    // partials in a fixed order, breakdown test, scale and epilogue scalars;
    // every CTA computes the same values, CTA 0 stores them for the later passes
    __shared__ double fold_s[3];
    __shared__ int fold_stop;
    const bool fold = p.fold_parts != nullptr;
    if (fold && warp == 0) {
        const int jj = p.stop_index;
        KrylovCtl *ctl = p.fold_ctl;
        const double n2 = warp_sum_partials(p.fold_parts, p.fold_nparts, 4, 0);
        if (lane == 0) {
            const double b = sqrt(n2);
            const double ref = fabs(ctl->alpha[jj - 1]) + ctl->beta[jj - 1];
            const bool brk = !(b > ctl->bd_tol * ref) || !(b > 0.0);
            fold_stop = brk ? 1 : 0;
            fold_s[0] = brk ? 0.0 : 1.0 / b;
            fold_s[1] = 0.0;
            fold_s[2] = brk ? 0.0 : b * ctl->scale[jj - 1];
            if (blockIdx.x == 0) {
                ctl->beta[jj] = b;
                if (brk) {
                    ctl->m_eff = jj;  // invariant subspace: the basis ends with v_{jj-1}
                    ctl->scale[jj] = 0.0;
                } else {
                    ctl->scale[jj] = 1.0 / b;
                    ctl->epi[0] = 1.0 / b;
                    ctl->epi[1] = 0.0;
                    ctl->epi[2] = b * ctl->scale[jj - 1];
                }
            }
        }
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&fullU[s], 1);
            mbar_init(&emptyU[s], NW);
        }
        mbar_init(fullS, 1);
        mbar_init(emptyS, NW);
        for (int s = 0; s < kStages; ++s) fxe[s] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (fold && fold_stop) return;  // breakdown: this step is not taken

    const int tbits = p.c + p.g;
    const int nvec = (1 << tbits) >> LOGVE;
    const uint64_t cmask = (1ull << p.c) - 1ull;
    const int oc = p.o - p.c;
    const uint64_t ocmask = (1ull << oc) - 1ull;
    const bool has_stream = p.stream != nullptr;
    const bool fxm = (sizeof(T) == sizeof(double)) && p.fx != 0;  // fixed-point flip sums
    const bool fx_defer = fxm && !p.first && has_stream;            // flips x field + partial in one FMA

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
    if (fold) {
        sv = fold_s[0];
        ea = fold_s[1];
        eb = fold_s[2];
    } else if (p.epi != nullptr) {
        sv = p.epi[0];
        ea = p.epi[1];
        eb = p.epi[2];
    }
    // first pass: r = H_inner u - a u + bs uprev with bs = -b/sv; later: r = flips + partial
    const T aT = (T)ea;
    const T bsT = (p.first && has_stream) ? (T)(-eb / sv) : (T)1;
    const T svT = (T)sv;
    const int nmine =
        tid < nvec ? ((nvec - 1 - tid) / NT + 1 < BV ? (nvec - 1 - tid) / NT + 1 : BV) : 0;
    const bool full_tile = (nmine == BV);
    // Output vector index of tile vector ii*NT + tid.  The local-to-global bit map
    // li -> ((li >> c) << o) | (li & cmask) sends disjoint bit sets to disjoint
    // ones, and the ii part (a multiple of NT*VE >= 2^c, checked at launch) to
    // ii * (NT*VE << (o - c)): one part per thread, one uniform stride.
    const uint64_t tli = (uint64_t)tid << LOGVE;
    const uint64_t gtid = (((tli >> p.c) << p.o) | (tli & cmask)) >> LOGVE;
    const uint64_t gstep = (((uint64_t)NT << LOGVE) << (p.o - p.c)) >> LOGVE;

    // E_ll of this thread's amplitudes: they sit at the same low bits in every
    // tile of the first pass, so the table is read once per launch
    T ell[BV * VE];
#pragma unroll
    for (int e = 0; e < BV * VE; ++e) {
        const int li = (((e / VE) * NT + tid) << LOGVE) + (e % VE);
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
                if (!fxm) break;  // fixed-point mode: every thread leaves together at the tile barrier
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
        const uint64_t gt = (base >> LOGVE) + gtid;  // base has no bits below c >= LOGVE (or is a multiple of the tile)
        const bool okw = mbar_wait(&fullU[s], (unsigned)((n / kStages) & 1), p.err);
        if (!fxm && !okw) {
            atomicExch(p.err, 1);
            break;
        }
        const T *trow = tcur;
        T pd0 = 0, pd1 = 0, pn = 0;
        bool stream_ready = false;
        // Loads and flips need no guard in a partial tile (L below the tile's bits):
        // every index stays inside the stage, and the partners of an in-range vector
        // are in range.  Stores, table indices and sums are guarded below.
        A self[BV * VE];
#pragma unroll
        for (int i = 0; i < BV; ++i) unpackv(Ucur[i * NT + tid], &self[i * VE]);
        int et = 0;
        double fxs = 0.0;
        if constexpr (sizeof(T) == sizeof(double)) {
            if (fxm) {
                // the tile's largest exponent (every thread, then every warp, then the CTA)
                unsigned em = 0u;
#pragma unroll
                for (int i = 0; i < BV; ++i) {
                    if (full_tile || i < nmine) {
                        const unsigned a = fx_expo(self[i].x), b = fx_expo(self[i].y);
                        em = max(em, max(a, b));
                    }
                }
                em = __reduce_max_sync(0xffffffffu, em);
                if (lane == 0) atomicMax(&fxe[s], em);
                if (__syncthreads_or(!okw || failed)) {
                    atomicExch(p.err, 1);
                    failed = true;
                    break;
                }
                et = (int)*reinterpret_cast<volatile unsigned *>(&fxe[s]);
                fxs = fx_scale(p.fxh, et);
                // this thread's amplitudes onto the tile's grid, in place; the flips
                // below read every partner in that form
                longlong2 *Ux = reinterpret_cast<longlong2 *>(const_cast<V *>(Ucur));
#pragma unroll
                for (int i = 0; i < BV; ++i) {
                    if (full_tile || i < nmine) {
                        longlong2 f;
                        f.x = fx_from(self[i].x, et);
                        f.y = fx_from(self[i].y, et);
                        Ux[i * NT + tid] = f;
                    }
                }
                __syncthreads();
                if (tid == 0) fxe[s] = 0u;  // every thread has read it; stage s is refilled after the next tile's barriers
            }
        }
        // accumulate in two halves of eight vectors; all four bits of i are
        // flipped in registers
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            constexpr int NH = BV / 2;
            A r[NH * VE];
#pragma unroll
            for (int e = 0; e < NH * VE; ++e) r[e] = azero(T(0));
            if constexpr (sizeof(T) == sizeof(double)) {
                if (fxm) {
                    // complex128, one field on every flipped bit: exact integer sum of
                    // the flipped partners, then one FP64 multiply by the field
                    const longlong2 *Ux = reinterpret_cast<const longlong2 *>(Ucur);
                    long long ar[NH], ai[NH];
#pragma unroll
                    for (int i = 0; i < NH; ++i) ar[i] = ai[i] = 0ll;
                    // thread bits: the partner of vector ii*NT + tid is ii*NT + (tid ^ 2^lb)
                    const int tb1 = tbits < TBITS ? tbits : TBITS;
                    for (int lb = p.c; lb < tb1; ++lb) {
                        const longlong2 *Uf = Ux + (tid ^ (1 << lb));
#pragma unroll
                        for (int i = 0; i < NH; ++i) {
                            const longlong2 v = Uf[(hh * NH + i) * NT];
                            ar[i] += v.x;
                            ai[i] += v.y;
                        }
                    }
                    // vector-index bits: the partner of ii is ii ^ 2^j
#pragma unroll
                    for (int j = 0; j < IBITS; ++j) {
                        const int lb = TBITS + j;
                        if (lb >= p.c && lb < tbits) {
#pragma unroll
                            for (int i = 0; i < NH; ++i) {
                                const longlong2 v = Ux[((hh * NH + i) ^ (1 << j)) * NT + tid];
                                ar[i] += v.x;
                                ai[i] += v.y;
                            }
                        }
                    }
                    if (fx_defer) {  // later passes: the field is applied with the partial sum below
#pragma unroll
                        for (int i = 0; i < NH; ++i) {
                            r[i].x = __ll2double_rn(ar[i]);
                            r[i].y = __ll2double_rn(ai[i]);
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < NH; ++i) {
                            r[i].x = fxs * __ll2double_rn(ar[i]);
                            r[i].y = fxs * __ll2double_rn(ai[i]);
                        }
                    }
                }
            }
            if (!fxm && VE == 2 && p.c == 0) {
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
            for (int j = 0; j < IBITS; ++j) {
                const int lb = LOGVE + TBITS + j;  // local bit carried by bit j of i
                if (!fxm && lb >= p.c && lb < tbits) {
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
            if (!fxm) {
                const int lb0 = p.c > LOGVE ? p.c : LOGVE;
                const int lb1 = tbits < LOGVE + TBITS ? tbits : LOGVE + TBITS;
                for (int lb = lb0; lb < lb1; ++lb) {
                    const K f = mkcoef(p.hb[p.o + lb - p.c]);
                    // the flipped bit is a thread bit: the partner of ii*NT + tid is ii*NT + (tid ^ flip)
                    const V *Uf = Ucur + (tid ^ (1 << (lb - LOGVE)));
#pragma unroll
                    for (int h4 = 0; h4 < NH / HB; ++h4) {
                        V v[HB];
#pragma unroll
                        for (int i = 0; i < HB; ++i) {
                            v[i] = Uf[(hh * NH + h4 * HB + i) * NT];
                        }
#pragma unroll
                        for (int i = 0; i < HB; ++i) {
                            A x[VE];
                            unpackv(v[i], x);
#pragma unroll
                            for (int e = 0; e < VE; ++e) afma(f, x[e], r[(h4 * HB + i) * VE + e]);
                        }
                    }
                }
            }
            if (p.first) {
                // E(b) - a = E_ll (registers) + TA (low ta bits) + TB (bits above ta) - a;
                // the low ta <= 6 bits of li are those of (tid << LOGVE) + e for every ii
                const int tmask = (1 << p.ta) - 1;
                T tav[VE];
#pragma unroll
                for (int e = 0; e < VE; ++e) tav[e] = trow[((tid << LOGVE) + e) & tmask];
#pragma unroll
                for (int i = 0; i < NH; ++i) {
                    const int ii = hh * NH + i;
                    if (full_tile || ii < nmine) {
                        const int li = (ii * NT + tid) << LOGVE;
                        const T tbv = trow[64 + (li >> p.ta)] - aT;
#pragma unroll
                        for (int e = 0; e < VE; ++e) {
                            const T E = ell[ii * VE + e] + tav[e] + tbv;
                            afma(mkcoef(E), self[ii * VE + e], r[i * VE + e]);
                        }
                    }
                }
            }
            if (hh == 1) {
                // u stage s is no longer read by this warp (its fixed-point stores
                // are ordered before the next bulk copy into the stage)
                if (fxm) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&emptyU[s]);
            }
            if (has_stream) {
                if (!stream_ready) {
                    if (!mbar_wait(fullS, (unsigned)(n & 1), p.err)) {
                        atomicExch(p.err, 1);
                        failed = true;
                        if (!fxm) break;  // fixed-point mode: leave at the next tile barrier
                    }
                    stream_ready = true;
                }
                const K bsK = mkcoef(bsT);
#pragma unroll
                for (int i = 0; i < NH; ++i) {
                    const int ii = hh * NH + i;
                    A x[VE];
                    unpackv(S[ii * NT + tid], x);
                    if constexpr (sizeof(T) == sizeof(double)) {
                        if (fx_defer) {
                            // r = field x unit x (integer flip sum) + partial
                            r[i].x = fma(fxs, r[i].x, x[0].x);
                            r[i].y = fma(fxs, r[i].y, x[0].y);
                            continue;
                        }
                    }
#pragma unroll
                    for (int e = 0; e < VE; ++e) afma(bsK, x[e], r[i * VE + e]);
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
                        const uint64_t gi = gt + (uint64_t)ii * gstep;
                        if (p.last) st_stream(&p.out[gi], packv(&r[i * VE]));
                        else p.out[gi] = packv(&r[i * VE]);
                    }
                }
            }
            if (p.last && p.epilogue != EPI_PLAIN && !full_tile) {
                // partial tile: the vectors past the end hold stale shared memory
#pragma unroll
                for (int i = 0; i < NH; ++i) {
                    if (hh * NH + i >= nmine) {
#pragma unroll
                        for (int e = 0; e < VE; ++e) {
                            r[i * VE + e] = azero(T(0));
                            self[(hh * NH + i) * VE + e] = azero(T(0));
                        }
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
        if (failed && !fxm) break;
        if (p.last && p.epilogue != EPI_PLAIN) {
            if constexpr (sizeof(T) == sizeof(float)) {
                // the tile's FP32 sums of the warp first (fixed order), then one FP64
                // add per warp: FP64 issues at 2 lanes per clock per SM on this part
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    pd0 += __shfl_xor_sync(0xffffffffu, pd0, off);
                    pd1 += __shfl_xor_sync(0xffffffffu, pd1, off);
                    pn += __shfl_xor_sync(0xffffffffu, pn, off);
                }
                if (lane == 0) {
                    acc_d0 += (double)pd0;
                    acc_d1 += (double)pd1;
                    acc_n += (double)pn;
                }
            } else {
                acc_d0 += (double)pd0;
                acc_d1 += (double)pd1;
                acc_n += (double)pn;
            }
        }
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
            double *dst = p.partials + 4 * ((size_t)blockIdx.x * NW + warp);
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
           (2 * kStages + 2) * sizeof(unsigned long long) + 16;
}

template <typename T, int BV>
static int grid_for(Handle *h, long long ntiles) {
    static int occ = -1;
    if (occ < 0) {
        cudaFuncSetAttribute(hpsi_pass_kernel<T, BV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem());
        // smallest shared-memory carve-out that fits (the rest stays L1 for the E_ll table)
        int maxsm = 0;
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device);
        if (maxsm > 0) {
            int pct = (int)((pass_smem() + 2048) * 100 / (size_t)maxsm) + 1;
            if (pct > 100) pct = 100;
            cudaFuncSetAttribute(hpsi_pass_kernel<T, BV>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
        }
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hpsi_pass_kernel<T, BV>, kTileV / BV, pass_smem());
        occ = n > 0 ? n : 1;
    }
    long long g = (long long)occ * h->nsm;
    return (int)(ntiles < g ? ntiles : g);
}

static int pass_bv(const Handle *h) { return h->pass_threads == 512 ? 8 : 16; }

int hpsi_grid(Handle *h, int pass) {
    const long long nt = h->plan.p[pass].ntiles;
    const bool w = pass_bv(h) == 8;
    if (h->prec == OSMPS_FP64) return w ? grid_for<double, 8>(h, nt) : grid_for<double, 16>(h, nt);
    return w ? grid_for<float, 8>(h, nt) : grid_for<float, 16>(h, nt);
}

int hpsi_partials_per_cta() { return kMaxPassWarps; }

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
        if (i == 0 && a.fold_parts != nullptr) {
            p.fold_ctl = a.fold_ctl;
            p.fold_parts = a.fold_parts;
            p.fold_nparts = a.fold_nparts;
        }
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
        // complex128 passes whose flipped bits share one field sum the partners in
        // fixed point (flip_fixed = the fewest flipped bits for which it is used; 0 = never)
        p.fx = 0;
        p.fxh = 0.0;
        if (sizeof(T) == sizeof(double) && h->flip_fixed > 0 && d.g >= h->flip_fixed) {
            bool uniform = true;
            for (int k = d.o + 1; k < d.o + d.g; ++k) uniform = uniform && (h->hbit[k] == h->hbit[d.o]);
            if (uniform) {
                p.fx = 1;
                p.fxh = h->hbit[d.o];
            }
        }
        // the kernel's output indexing needs the vector-index bits above the carried chunk
        if (((kTileV / pass_bv(h)) * (int)(16 / h->esize)) < (1 << d.c)) return cudaErrorInvalidValue;
        int grid = 0, nw = 0;
        if (pass_bv(h) == 8) {
            grid = grid_for<T, 8>(h, d.ntiles);
            nw = kTileV / 8 / 32;
            hpsi_pass_kernel<T, 8><<<grid, kTileV / 8, pass_smem(), h->stream>>>(tm_u, tm_s, p);
        } else {
            grid = grid_for<T, 16>(h, d.ntiles);
            nw = kTileV / 16 / 32;
            hpsi_pass_kernel<T, 16><<<grid, kTileV / 16, pass_smem(), h->stream>>>(tm_u, tm_s, p);
        }
        h->launches += 1;
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        if (last) nparts = grid * nw;
    }
    if (nparts_out) *nparts_out = nparts;
    return cudaSuccess;
}

cudaError_t launch_hpsi(Handle *h, const HpsiArgs &a, int *nparts_out) {
    return h->prec == OSMPS_FP64 ? launch_hpsi_t<double>(h, a, nparts_out)
                                 : launch_hpsi_t<float>(h, a, nparts_out);
}

}  // namespace osmps
