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
#include <cuda_runtime.h>

#include "ed_internal.h"

namespace osmps {

template <typename T> struct Cx;
template <> struct Cx<float> {
    typedef float2 c;
    typedef float4 v16;
    static constexpr int VE = 2;     // amplitudes per 16-byte vector
    static constexpr int LOGVE = 1;
    static constexpr int BLOG = 4;   // log2 amplitudes per register block (8 vectors)
};
template <> struct Cx<double> {
    typedef double2 c;
    typedef double2 v16;
    static constexpr int VE = 1;
    static constexpr int LOGVE = 0;
    static constexpr int BLOG = 3;
};

constexpr int kBV = 8;                                  // 16-byte vectors per register block
constexpr int kTileV = 1 << (kTileBytesLog2 - 4);       // 16-byte vectors per tile
constexpr int kTab = 256;                               // TA (<= 64) + TB (<= 128) per stage
static_assert(kTileV == kBV * kPassThreads, "eight vectors per thread per tile");

template <typename T>
struct PassParams {
    const typename Cx<T>::v16 *u;       // vector being multiplied (tile staged in shared memory)
    const typename Cx<T>::v16 *stream;  // elementwise input: previous Lanczos vector (first pass) or partial sum
    typename Cx<T>::v16 *out;
    const T *Ell;
    const T *Fhh;
    const double *epi;                  // sv, a, b (device) or null
    double *partials;
    const int *m_eff;
    long long ntiles;
    int stop_index;
    int L, c, o, g, ta, first, last, epilogue;
    T hb[kMaxL + 1];
};

__device__ __forceinline__ void unpack(const float4 &v, float2 *e) {
    e[0] = make_float2(v.x, v.y);
    e[1] = make_float2(v.z, v.w);
}
__device__ __forceinline__ float4 pack(const float2 *e) { return make_float4(e[0].x, e[0].y, e[1].x, e[1].y); }
__device__ __forceinline__ void unpack(const double2 &v, double2 *e) { e[0] = v; }
__device__ __forceinline__ double2 pack(const double2 *e) { return e[0]; }

// acc += f * x on a complex amplitude: one packed FP32x2 FMA, or two FP64 FMAs
__device__ __forceinline__ void cfma(float f, const float2 &x, float2 &acc) {
    unsigned long long X = ((unsigned long long)__float_as_uint(x.y) << 32) | __float_as_uint(x.x);
    unsigned long long F = ((unsigned long long)__float_as_uint(f) << 32) | __float_as_uint(f);
    unsigned long long A = ((unsigned long long)__float_as_uint(acc.y) << 32) | __float_as_uint(acc.x);
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(A) : "l"(F), "l"(X));
    acc.x = __uint_as_float((unsigned)A);
    acc.y = __uint_as_float((unsigned)(A >> 32));
}
__device__ __forceinline__ void cfma(double f, const double2 &x, double2 &acc) {
    acc.x = fma(f, x.x, acc.x);
    acc.y = fma(f, x.y, acc.y);
}

template <typename V>
__device__ __forceinline__ void st_stream(V *p, const V &v) {
    __stcs(p, v);
}

template <typename T>
__device__ __forceinline__ void block_reduce3(double v0, double v1, double v2, double *dst) {
    __shared__ double red[3][kPassThreads / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, off);
        v1 += __shfl_xor_sync(0xffffffffu, v1, off);
        v2 += __shfl_xor_sync(0xffffffffu, v2, off);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        red[0][w] = v0;
        red[1][w] = v1;
        red[2][w] = v2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, s1 = 0, s2 = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            s0 += red[0][i];
            s1 += red[1][i];
            s2 += red[2][i];
        }
        dst[0] = s0;
        dst[1] = s1;
        dst[2] = s2;
        dst[3] = 0.0;
    }
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One pass of the product.  Persistent: one 512-thread CTA per SM walks the
// tiles.  Thread tid owns the 16-byte vectors q = tid + 512 i (i < 8) of every
// tile, so all global loads and stores are lane-coalesced.  The tile of u for
// the next iteration is copied asynchronously into the second shared-memory
// stage while the current one is computed; the elementwise stream (previous
// vector or partial sum) of the thread's own vectors is copied one tile ahead
// by the thread that consumes it.
template <typename T>
__global__ void __launch_bounds__(kPassThreads, 1) hpsi_pass_kernel(PassParams<T> p) {
    typedef typename Cx<T>::c C;
    typedef typename Cx<T>::v16 V;
    constexpr int VE = Cx<T>::VE;
    constexpr int LOGVE = Cx<T>::LOGVE;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *U0 = reinterpret_cast<V *>(smem_raw);
    V *U1 = U0 + kTileV;
    V *S = U1 + kTileV;
    T *tab0 = reinterpret_cast<T *>(S + kTileV);
    T *tab1 = tab0 + kTab;

    if (p.m_eff != nullptr && *p.m_eff <= p.stop_index) return;

    const int tid = threadIdx.x;
    const int tbits = p.c + p.g;
    const int nvec = (1 << tbits) >> LOGVE;
    const uint64_t cmask = (1ull << p.c) - 1ull;
    const int oc = p.o - p.c;
    const uint64_t ocmask = (1ull << oc) - 1ull;
    const bool has_stream = p.stream != nullptr;

    double sv = 1.0, ea = 0.0, eb = 0.0;
    if (p.epi != nullptr) {
        sv = p.epi[0];
        ea = p.epi[1];
        eb = p.epi[2];
    }
    // first pass: r = H_inner u - a u - (b/sv) uprev ;  last pass: w = sv * r
    const T aT = (T)ea;
    const T bsT = (p.first && has_stream) ? (T)(-eb / sv) : (T)1;
    const T svT = (T)sv;

    auto tile_base = [&](long long t) -> uint64_t {
        const uint64_t tt = (uint64_t)t;
        return ((tt >> oc) << (p.o + p.g)) | ((tt & ocmask) << p.c);
    };
    auto gidx = [&](uint64_t base, int q) -> uint64_t {  // global 16-byte vector index of tile vector q
        const int li = q << LOGVE;
        return (base | ((uint64_t)(li >> p.c) << p.o) | ((uint64_t)li & cmask)) >> LOGVE;
    };
    auto issue_u = [&](long long t, V *buf) {
        const uint64_t base = tile_base(t);
#pragma unroll
        for (int i = 0; i < kBV; ++i) {
            const int q = i * kPassThreads + tid;
            if (q < nvec) cp_async16(&buf[q], &p.u[gidx(base, q)]);
        }
    };
    auto issue_s = [&](long long t) {
        const uint64_t base = tile_base(t);
#pragma unroll
        for (int i = 0; i < kBV; ++i) {
            const int q = i * kPassThreads + tid;
            if (q < nvec) cp_async16(&S[q], &p.stream[gidx(base, q)]);
        }
    };
    auto build_tab = [&](long long t, T *tab) {
        const int a = p.g, ta = p.ta, tb = a - ta;
        const T *F = p.Fhh + (size_t)t * (size_t)(a + 1);
        if (tid < (1 << ta)) {
            T s = F[a];
            for (int j = 0; j < ta; ++j) s += ((tid >> j) & 1) ? -F[j] : F[j];
            tab[tid] = s;
        } else if (tid < (1 << ta) + (1 << tb)) {
            const int y = tid - (1 << ta);
            T s = (T)0;
            for (int j = 0; j < tb; ++j) s += ((y >> j) & 1) ? -F[ta + j] : F[ta + j];
            tab[64 + y] = s;
        }
    };

    double acc_d0 = 0.0, acc_d1 = 0.0, acc_n = 0.0;
    long long t = blockIdx.x;
    if (t < p.ntiles) {
        issue_u(t, U0);
        cp_async_commit();
        if (has_stream) issue_s(t);
        cp_async_commit();
        if (p.first) build_tab(t, tab0);
    }
    int stage = 0;
    // vectors of this thread that exist in a tile (small chains have tiles < 4096 vectors)
    const int nmine = tid < nvec ? ((nvec - 1 - tid) / kPassThreads + 1 < kBV ? (nvec - 1 - tid) / kPassThreads + 1 : kBV)
                                 : 0;
    for (; t < p.ntiles; t += gridDim.x, stage ^= 1) {
        const long long tn = t + gridDim.x;
        V *Ucur = stage ? U1 : U0;
        V *Unext = stage ? U0 : U1;
        T *tcur = stage ? tab1 : tab0;
        T *tnext = stage ? tab0 : tab1;
        cp_async_wait<1>();
        __syncthreads();
        if (tn < p.ntiles) {
            issue_u(tn, Unext);
            if (p.first) build_tab(tn, tnext);
        }
        cp_async_commit();

        const uint64_t base = tile_base(t);
        T pd0 = 0, pd1 = 0, pn = 0;
        C self[kBV * VE], r[kBV * VE];
#pragma unroll
        for (int i = 0; i < kBV; ++i) {
            if (i < nmine) unpack(Ucur[i * kPassThreads + tid], &self[i * VE]);
            else unpack(V{}, &self[i * VE]);
        }
#pragma unroll
        for (int e = 0; e < kBV * VE; ++e) r[e] = C{(T)0, (T)0};
        int k0 = 0;
        if (VE == 2 && p.c == 0) {
            // bit 0 lives inside the 16-byte vector
            const T f = p.hb[p.o];
#pragma unroll
            for (int i = 0; i < kBV; ++i) {
                cfma(f, self[i * VE + VE - 1], r[i * VE]);
                cfma(f, self[i * VE], r[i * VE + VE - 1]);
            }
            k0 = 1;
        }
        for (int k = k0; k < p.g; ++k) {
            const T f = p.hb[p.o + k];
            const int flip = 1 << (p.c + k - LOGVE);
#pragma unroll
            for (int i = 0; i < kBV; ++i) {
                if (i < nmine) {
                    C x[VE];
                    unpack(Ucur[(i * kPassThreads + tid) ^ flip], x);
#pragma unroll
                    for (int e = 0; e < VE; ++e) cfma(f, x[e], r[i * VE + e]);
                }
            }
        }
        if (p.first) {
            const int tmask = (1 << p.ta) - 1;
#pragma unroll
            for (int i = 0; i < kBV; ++i) {
                if (i < nmine) {
#pragma unroll
                    for (int e = 0; e < VE; ++e) {
                        const int li = ((i * kPassThreads + tid) << LOGVE) + e;
                        const T E = __ldg(&p.Ell[li]) + tcur[li & tmask] + tcur[64 + (li >> p.ta)] - aT;
                        cfma(E, self[i * VE + e], r[i * VE + e]);
                    }
                }
            }
        }
        if (has_stream) {
            cp_async_wait<1>();  // this thread's stream copies of tile t have landed
#pragma unroll
            for (int i = 0; i < kBV; ++i) {
                if (i < nmine) {
                    C x[VE];
                    unpack(S[i * kPassThreads + tid], x);
#pragma unroll
                    for (int e = 0; e < VE; ++e) cfma(bsT, x[e], r[i * VE + e]);
                }
            }
        }
        if (!p.last) {
#pragma unroll
            for (int i = 0; i < kBV; ++i)
                if (i < nmine) p.out[gidx(base, i * kPassThreads + tid)] = pack(&r[i * VE]);
        } else if (p.epilogue == EPI_ENERGY) {
#pragma unroll
            for (int e = 0; e < kBV * VE; ++e) {
                pd0 = fma(self[e].x, r[e].x, fma(self[e].y, r[e].y, pd0));
                pd1 = fma(self[e].x, r[e].y, fma(-self[e].y, r[e].x, pd1));
                pn = fma(self[e].x, self[e].x, fma(self[e].y, self[e].y, pn));
            }
        } else {
#pragma unroll
            for (int e = 0; e < kBV * VE; ++e) {
                r[e].x *= svT;
                r[e].y *= svT;
            }
#pragma unroll
            for (int i = 0; i < kBV; ++i)
                if (i < nmine) st_stream(&p.out[gidx(base, i * kPassThreads + tid)], pack(&r[i * VE]));
            if (p.epilogue == EPI_KRYLOV) {
#pragma unroll
                for (int e = 0; e < kBV * VE; ++e) {
                    pd0 = fma(self[e].x, r[e].x, fma(self[e].y, r[e].y, pd0));
                    pd1 = fma(self[e].x, r[e].y, fma(-self[e].y, r[e].x, pd1));
                    pn = fma(r[e].x, r[e].x, fma(r[e].y, r[e].y, pn));
                }
            }
        }
        acc_d0 += (double)pd0;
        acc_d1 += (double)pd1;
        acc_n += (double)pn;
        if (has_stream && tn < p.ntiles) issue_s(tn);
        cp_async_commit();
    }
    cp_async_wait<0>();

    if (p.last && p.epilogue != EPI_PLAIN && p.partials != nullptr) {
        block_reduce3<T>(acc_d0 * sv, acc_d1 * sv, acc_n, p.partials + 4 * (size_t)blockIdx.x);
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

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
PassPlan make_plan(int L, int prec) {
    PassPlan pl{};
    const int logE = (prec == OSMPS_FP64) ? 4 : 3;       // log2 bytes per amplitude
    const int TB = kTileBytesLog2 - logE;                  // tile bits
    const int cdef = kChunkBytesLog2 - logE;               // 128-byte chunk
    const int cmin = 5 - logE;                             // 32-byte sector
    pl.a1 = L < TB ? L : TB;
    pl.ta = pl.a1 / 2;
    pl.p[0] = PassDesc{0, 0, pl.a1, 1, 1ll << (L - pl.a1)};
    pl.npass = 1;
    const int rest = L - pl.a1;
    if (rest > 0) {
        const int room = TB - cmin;
        const int k = (rest + room - 1) / room;
        int gmax = (rest + k - 1) / k;
        int c = cdef < TB - gmax ? cdef : TB - gmax;
        if (c < cmin) c = cmin;
        int o = pl.a1;
        int left = rest;
        for (int i = 0; i < k; ++i) {
            const int g = (left + (k - i) - 1) / (k - i);
            pl.p[pl.npass++] = PassDesc{c, o, g, 0, 1ll << (L - c - g)};
            o += g;
            left -= g;
        }
    }
    return pl;
}

static size_t pass_smem() { return 3u * (1u << kTileBytesLog2) + 2 * kTab * sizeof(double); }

template <typename T>
static int grid_for(Handle *h, long long ntiles) {
    static int occ = -1;
    if (occ < 0) {
        cudaFuncSetAttribute(hpsi_pass_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem());
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hpsi_pass_kernel<T>, kPassThreads, pass_smem());
        occ = n > 0 ? n : 1;
    }
    long long g = (long long)occ * h->nsm;
    return (int)(ntiles < g ? ntiles : g);
}

int hpsi_grid(Handle *h, int pass) {
    const long long nt = h->plan.p[pass].ntiles;
    return h->prec == OSMPS_FP64 ? grid_for<double>(h, nt) : grid_for<float>(h, nt);
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
        p.u = reinterpret_cast<const V *>(a.u);
        p.stream = reinterpret_cast<const V *>(i == 0 ? a.uprev : src_acc);
        p.out = reinterpret_cast<V *>(dst);
        p.Ell = reinterpret_cast<const T *>(h->Ell);
        p.Fhh = reinterpret_cast<const T *>(h->Fhh);
        p.epi = a.epi;
        p.partials = a.partials;
        p.m_eff = a.m_eff;
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
        for (int k = 0; k <= kMaxL; ++k) p.hb[k] = (T)h->hbit[k];
        const int grid = grid_for<T>(h, d.ntiles);
        hpsi_pass_kernel<T><<<grid, kPassThreads, pass_smem(), h->stream>>>(p);
        h->launches += 1;
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        if (last) nparts = grid;
    }
    if (nparts_out) *nparts_out = nparts;
    return cudaSuccess;
}

cudaError_t launch_hpsi(Handle *h, const HpsiArgs &a, int *nparts_out) {
    return h->prec == OSMPS_FP64 ? launch_hpsi_t<double>(h, a, nparts_out)
                                 : launch_hpsi_t<float>(h, a, nparts_out);
}

}  // namespace osmps
