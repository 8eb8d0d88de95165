// Batched Lanczos ground states: many independent chains in one persistent launch.
//
// Paper: the ground state of the Hamiltonian of Eq. genericH found by the
// Lanczos method (statics, Sec. II; the Krylov construction of Sec. III.D),
// here for many long-range Ising chains (Sec. VII) of different length and
// parameters at once.
//
// * One CTA takes one chain at a time from a work queue (largest chains first)
//   and runs that chain's whole Lanczos iteration by itself, so there is no
//   grid-wide synchronisation and every chain stops at its own convergence.
// * Vectors are complex64 (or complex128); alpha, beta, every reduction and the
//   tridiagonal problem are FP64.
// * No Krylov basis is stored.  Sweep 1 runs the three-term recurrence
//       w = H v_j - alpha_j v_j - beta_j v_{j-1},   beta_{j+1} = |w|,
//   with vectors kept unnormalised (v_j = s_j u_j, s_j = 1/beta_j), and every
//   few steps finds the lowest Ritz pair (theta, y) of T_{j+1}; it stops when
//   beta_{j+1} |y_{j+1}| <= tol (or, with complex64 vectors, when theta is
//   stationary in FP64; see sweep 1).  Sweep 2 regenerates the same vectors from the
//   stored alpha, beta (the same arithmetic, so bit-identical) and accumulates
//   x = sum_j y_j v_j.  A last product forms the true residual |H x - theta x|.
// * H v of one chain: pass A stages contiguous tiles of the TB low bits in
//   shared memory (bulk copies completing on an mbarrier ring) and adds the
//   diagonal E(b) = E_ll(lo) + TA(lo) + TB(lo) (E_ll a per-chain table read
//   into registers once per pass, TA/TB per tile); pass B stages gathered tiles (2^g segments of 2^c amplitudes) for
//   the g = L - TB high bits and adds their flips to the partial sum.  Pass C
//   is the streaming update of the recurrence.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "ed_internal.h"

namespace osmps {
namespace batch {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kStages = 3;
constexpr int kVPT = 16;                   // 16-byte vectors per thread per tile
constexpr int kTileVec = kThreads * kVPT;  // 4096 vectors = 64 KiB per tile
constexpr int kTA = 64, kTB = 128, kTabN = kTA + kTB;
constexpr unsigned kTileBytes = kTileVec * 16u;

enum Mode { MODE_STORE = 0, MODE_ALPHA = 1, MODE_RESID = 2 };

template <typename T>
struct BatchParams {
    typedef typename Cx<T>::v16 V;
    const BatchInst *inst;
    const int *order;
    V *psi, *R0, *R1, *R2, *X;
    double *energy, *residual;
    int *iters, *status;
    double *scratch;  // per CTA: 8 * max_iter + 8 + kBatchEllScratch doubles
    int *counter;     // [0] queue of the large chains, [1] queue of the others
    int *err;
    double tol;
    int n, max_iter;
    int nbig;         // order[0..nbig) are solved by whole clusters (cluster launches only)
    int small_first;  // first order index of the one-CTA queue
};

// ---------------------------------------------------------------------------
// small helpers

__device__ __forceinline__ float adot(unsigned long long u, unsigned long long w) {
    const float2 a = tocx(u), b = tocx(w);
    return fmaf(a.x, b.x, a.y * b.y);
}
__device__ __forceinline__ double adot(const double2 &a, const double2 &b) { return fma(a.x, b.x, a.y * b.y); }
__device__ __forceinline__ float anorm(unsigned long long u) {
    const float2 a = tocx(u);
    return fmaf(a.x, a.x, a.y * a.y);
}
__device__ __forceinline__ double anorm(const double2 &a) { return fma(a.x, a.x, a.y * a.y); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Sum of one value per thread over the CTA, fixed order; every thread gets it.
__device__ __forceinline__ double cta_sum(double v, double *red) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) r += red[w];
    __syncthreads();
    return r;
}
__device__ __forceinline__ void cta_sum2(double &a, double &b, double *red) {
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = a;
        red[kWarps + (threadIdx.x >> 5)] = b;
    }
    __syncthreads();
    double ra = 0.0, rb = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        ra += red[w];
        rb += red[kWarps + w];
    }
    __syncthreads();
    a = ra;
    b = rb;
}

// ---------------------------------------------------------------------------
// Tridiagonal T_k (diagonal a[0..k-1], off-diagonal b[1..k-1]) in FP64.

// Number of eigenvalues of T_k below x (Sturm count from the LDL^T pivots).
__device__ int sturm_count(const double *a, const double *b, int k, double x, double pivmin) {
    int cnt = 0;
    double d = a[0] - x;
    if (fabs(d) < pivmin) d = -pivmin;
    if (d < 0.0) ++cnt;
    for (int i = 1; i < k; ++i) {
        d = (a[i] - x) - b[i] * b[i] / d;
        if (fabs(d) < pivmin) d = -pivmin;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// Lowest eigenvalue of T_k by multisection on the 32 lanes of one warp:
// each round evaluates 32 points of the bracket [lo, hi] and keeps the
// sub-interval where the count first becomes non-zero.  The bracket starts at
// [guess_lo, hi] when guess_lo lies below the spectrum (checked by lane 0),
// else at the Gershgorin lower bound.  Call with the whole warp.
__device__ double lowest_eig_warp(const double *a, const double *b, int k, double guess_lo, double hi) {
    const int lane = threadIdx.x & 31;
    double glo = a[0], tnorm = fabs(a[0]);
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? fabs(b[i]) : 0.0) + (i + 1 < k ? fabs(b[i + 1]) : 0.0);
        glo = fmin(glo, a[i] - r);
        tnorm = fmax(tnorm, fabs(a[i]) + r);
        hi = fmin(hi, a[i]);  // every diagonal entry is a Rayleigh quotient
    }
    const double pivmin = 1e-300 + 1e-30 * tnorm * tnorm;
    double lo = glo;
    if (guess_lo > glo && guess_lo < hi) {
        const int c = (lane == 0) ? sturm_count(a, b, k, guess_lo, pivmin) : 0;
        if (__shfl_sync(0xffffffffu, c, 0) == 0) lo = guess_lo;
    }
    const double tolx = 2.2e-16 * fmax(tnorm, 1e-300);
    for (int round = 0; round < 64 && hi - lo > tolx; ++round) {
        const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
        const int c = sturm_count(a, b, k, x, pivmin);
        const unsigned bal = __ballot_sync(0xffffffffu, c >= 1);
        const double xl = __shfl_sync(0xffffffffu, x, 31);
        if (bal == 0u) {
            lo = xl;
        } else {
            const int f = __ffs((int)bal) - 1;
            const double xf = __shfl_sync(0xffffffffu, x, f);
            const double xp = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
            hi = xf;
            if (f > 0) lo = xp;
        }
    }
    return 0.5 * (lo + hi);
}

// Eigenvector of T_k for the eigenvalue theta by two steps of inverse
// iteration, solving (T - theta I) z = r by Gaussian elimination with partial
// pivoting (the tridiagonal factor gains one extra super-diagonal).
// work holds 5k doubles.  Writes the normalised y with y[0] >= 0.  One thread.
__device__ void ritz_vector(const double *a, const double *b, int k, double theta, double *y, double *work) {
    double *d = work, *du = work + k, *du2 = work + 2 * k, *ml = work + 3 * k, *sw = work + 4 * k;
    double tnorm = 0.0;
    for (int i = 0; i < k; ++i)
        tnorm = fmax(tnorm, fabs(a[i]) + (i > 0 ? fabs(b[i]) : 0.0) + (i + 1 < k ? fabs(b[i + 1]) : 0.0));
    const double tiny = 1e-14 * fmax(tnorm, 1e-300);
    for (int i = 0; i < k; ++i) {
        d[i] = a[i] - theta;
        du[i] = (i + 1 < k) ? b[i + 1] : 0.0;
        du2[i] = 0.0;
    }
    for (int i = 0; i + 1 < k; ++i) {
        const double sub = b[i + 1];  // T(i+1, i)
        if (fabs(d[i]) >= fabs(sub)) {
            if (fabs(d[i]) < tiny) d[i] = tiny;
            const double mlt = sub / d[i];
            ml[i] = mlt;
            sw[i] = 0.0;
            d[i + 1] -= mlt * du[i];
        } else {  // rows i and i+1 swap
            const double mlt = d[i] / sub;
            ml[i] = mlt;
            sw[i] = 1.0;
            d[i] = sub;
            const double old_du = du[i];
            du[i] = d[i + 1];
            d[i + 1] = old_du - mlt * d[i + 1];
            if (i + 2 < k) {
                du2[i] = du[i + 1];
                du[i + 1] = -mlt * du[i + 1];
            }
        }
    }
    if (fabs(d[k - 1]) < tiny) d[k - 1] = tiny;
    for (int i = 0; i < k; ++i) y[i] = 1.0;
    for (int it = 0; it < 2; ++it) {
        for (int i = 0; i + 1 < k; ++i) {  // apply the row swaps and L^{-1}
            if (sw[i] != 0.0) {
                const double t = y[i];
                y[i] = y[i + 1];
                y[i + 1] = t - ml[i] * y[i];
            } else {
                y[i + 1] -= ml[i] * y[i];
            }
        }
        y[k - 1] /= d[k - 1];  // U z = y
        if (k >= 2) y[k - 2] = (y[k - 2] - du[k - 2] * y[k - 1]) / d[k - 2];
        for (int i = k - 3; i >= 0; --i) y[i] = (y[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) / d[i];
        double nrm = 0.0;
        for (int i = 0; i < k; ++i) nrm = fma(y[i], y[i], nrm);
        const double sc = (y[0] < 0.0 ? -1.0 : 1.0) / sqrt(nrm);
        for (int i = 0; i < k; ++i) y[i] *= sc;
    }
}

// Bounded wait that ignores the error flag (used only to let copies already in
// flight land before the CTA leaves after a failure).
__device__ __forceinline__ void drain_wait(unsigned long long *bar, unsigned parity) {
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > kWaitNs) return;
}

// Lowest Ritz pair bookkeeping shared by the convergence checks.
struct RitzState {
    double theta, theta_prev, dtheta, est;
};

// ---- thread-block cluster primitives (C CTAs sharing one chain) ----
__device__ __forceinline__ int cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}
__device__ __forceinline__ int cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return (int)r;
}
// Every thread of every CTA of the cluster; release/acquire orders the global
// and shared memory accesses before it with those after it, cluster-wide.
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned dsmem_addr(const void *ptr, int rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(ptr)), "r"(rank));
    return r;
}
__device__ __forceinline__ double ld_dsmem(const double *ptr, int rank) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(dsmem_addr(ptr, rank)) : "memory");
    return v;
}
__device__ __forceinline__ void st_dsmem(int *ptr, int rank, int v) {
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(dsmem_addr(ptr, rank)), "r"(v) : "memory");
}

// Launched either without clusters (every CTA solves one chain at a time) or
// with clusters of C CTAs: the C CTAs of a cluster first solve the large
// chains order[0..nbig) together (tiles and vector ranges split by rank,
// reductions exchanged through distributed shared memory, a cluster barrier
// after each pass), then take the remaining chains one CTA each.
template <typename T>
__global__ void __launch_bounds__(kThreads, 1) lanczos_batch_kernel(BatchParams<T> p) {
    typedef typename Cx<T>::v16 V;
    typedef typename Cx<T>::amp A;
    typedef typename Cx<T>::coef K;
    constexpr int VE = Cx<T>::VE;
    constexpr int LOGVE = Cx<T>::LOGVE;
    constexpr int TBITS = 12 + LOGVE;  // amplitude bits of one 64 KiB tile
    constexpr int NE = kVPT * VE;      // amplitudes per thread per tile

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    V *U = reinterpret_cast<V *>(smem_raw);  // kStages tiles
    T *tab = reinterpret_cast<T *>(U + kStages * kTileVec);  // two (TA, TB) buffers
    unsigned long long *full = reinterpret_cast<unsigned long long *>(tab + 2 * kTabN);
    double *red = reinterpret_cast<double *>(full + kStages);  // 2 * kWarps
    T *Jt = reinterpret_cast<T *>(red + 2 * kWarps);           // J(r) for r <= kMaxL
    __shared__ int s_int[2];
    __shared__ double s_dbl[2];
    __shared__ double s_slot[2][4];  // cluster reductions, double-buffered
    __shared__ unsigned s_fxe;       // complex128: the current tile's largest FP64 exponent

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int csize = cluster_size(), crank = cluster_rank();
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fxe = 0u;
    }
    __syncthreads();
    if (csize > 1) cluster_barrier();  // peers' shared memory exists before any remote access
    unsigned ph = 0u;  // parity of the next wait on each stage (bit s)
    int par = 0;       // slot set of the next cluster reduction
    const int mi = p.max_iter;
    double *alpha = p.scratch + (size_t)blockIdx.x * (size_t)(8 * mi + 8 + kBatchEllScratch);
    double *beta = alpha + mi;         // beta[0..mi]
    double *yv = beta + mi + 1;        // Ritz vector in the Lanczos basis
    double *work = yv + mi;            // 5 * mi
    double *ell_scr = work + 5 * mi;   // kBatchEllScratch doubles: E_ll table of the current chain

    // Solves chain k with cc CTAs (this one has rank cr); false when a bounded
    // wait gave up (the decision is the same on every CTA of the group).
    auto solve = [&](const int k, const int cc, const int cr) -> bool {
        const BatchInst &in = p.inst[k];
        const int L = in.L;
        const int g = L - TBITS, c = TBITS - g;  // pass B: g flipped bits, chunks of 2^c amplitudes
        const int nt = 1 << g;                   // tiles per pass
        const int ntl = (nt - cr + cc - 1) / cc; // this CTA's tiles per pass: t = cr + l cc
        const long long nvec = (1ll << L) >> LOGVE;
        const long long vlen = nvec / cc, vbeg = vlen * cr;  // this CTA's range of the streaming passes
        const long long voff = in.off >> LOGVE;
        if (tid <= kMaxL) Jt[tid] = (T)in.J[tid];
        const T hT = (T)in.h;
        __syncthreads();

        // sums over the group: CTA sums, then (cc > 1) the CTAs' slots read in rank order
        auto gsum = [&](double &a, double &b, double &f) {
            cta_sum2(a, b, red);
            if (cc > 1) {
                if (tid == 0) {
                    s_slot[par][0] = a;
                    s_slot[par][1] = b;
                    s_slot[par][2] = f;
                }
                cluster_barrier();
                double sa = 0.0, sb = 0.0, sf = 0.0;
                for (int r = 0; r < cc; ++r) {
                    sa += ld_dsmem(&s_slot[par][0], r);
                    sb += ld_dsmem(&s_slot[par][1], r);
                    sf += ld_dsmem(&s_slot[par][2], r);
                }
                a = sa;
                b = sb;
                f = sf;
                par ^= 1;
            }
        };
        auto gbar = [&]() {
            if (cc > 1)
                cluster_barrier();
            else
                __syncthreads();
        };

        // E_ll over the TBITS low bits (same in every tile), a per-CTA table
        // read into registers at the start of every pass A
        T *ell_tab = reinterpret_cast<T *>(ell_scr);
        for (int li = tid; li < (1 << TBITS); li += kThreads) {
            double E = 0.0;
            for (int r = 1; r < TBITS; ++r)
                E += in.J[r] * (double)((TBITS - r) - 2 * __popc((li ^ (li >> r)) & ((1 << (TBITS - r)) - 1)));
            ell_tab[li] = (T)E;
        }
        __syncthreads();

        // per-tile tables: TA[x] = E_hh(hi) + sum_{j<6} s_j(x) F_j(hi), TB[y] = sum_j s_j(y) F_{6+j}(hi)
        // with F_j(hi) = sum_{q<g} J(TBITS+q-j) s_q(hi)
        auto build_tab = [&](int hi, int bsel) {
            if (tid < kTabN) {
                T v = (T)0;
                if (tid < kTA) {
                    for (int q = 0; q < g; ++q)
                        for (int q2 = q + 1; q2 < g; ++q2)
                            v += ((((hi >> q) ^ (hi >> q2)) & 1) ? -Jt[q2 - q] : Jt[q2 - q]);
                    for (int j = 0; j < 6; ++j) {
                        T F = (T)0;
                        for (int q = 0; q < g; ++q) F += ((hi >> q) & 1) ? -Jt[TBITS + q - j] : Jt[TBITS + q - j];
                        v += ((tid >> j) & 1) ? -F : F;
                    }
                } else {
                    const int y = tid - kTA;
                    if (y < (1 << (TBITS - 6)))
                        for (int j = 0; j < TBITS - 6; ++j) {
                            T F = (T)0;
                            for (int q = 0; q < g; ++q)
                                F += ((hi >> q) & 1) ? -Jt[TBITS + q - 6 - j] : Jt[TBITS + q - 6 - j];
                            v += ((y >> j) & 1) ? -F : F;
                        }
                }
                tab[bsel * kTabN + tid] = v;
            }
        };

        // Loop over this CTA's tiles l = 0..ntl-1 (tile t = cr + l cc): warp 0
        // keeps kStages copies in flight; body(t, l, s) runs on all threads.
        auto run_tiles = [&](auto issue, auto body) -> bool {
            const int pre = ntl < kStages ? ntl : kStages;
            if (warp == 0)
                for (int l = 0; l < pre; ++l) issue(cr + l * cc, l);
            for (int l = 0; l < ntl; ++l) {
                const int s = l % kStages;
                const bool ok = mbar_wait(&full[s], (ph >> s) & 1u, p.err);
                ph ^= 1u << s;
                if (__syncthreads_or(!ok)) {
                    if (tid == 0) {
                        atomicExch(p.err, 1);
                        drain_wait(&full[s], ((ph >> s) & 1u) ^ 1u);
                        for (int u = l + 1; u < ntl && u < l + kStages; ++u)
                            drain_wait(&full[u % kStages], (ph >> (u % kStages)) & 1u);
                    }
                    return false;
                }
                body(cr + l * cc, l, s);
                __syncthreads();
                if (warp == 0 && l + kStages < ntl) issue(cr + (l + kStages) * cc, l + kStages);
            }
            return true;
        };
        auto issue_contig = [&](const V *src, int t, int l) {
            const int s = l % kStages;
            if (lane == 0) {
                mbar_arrive_expect_tx(&full[s], kTileBytes);
                bulk_load(U + (size_t)s * kTileVec, src + (size_t)t * kTileVec, kTileBytes, &full[s]);
            }
        };
        auto issue_gather = [&](const V *src, int m, int l) {
            // segment hi: 2^c amplitudes at (hi << TBITS) + (m << c), to tile offset hi << c
            const int s = l % kStages;
            const unsigned seg = (unsigned)(2 * sizeof(T)) << c;
            if (lane == 0) mbar_arrive_expect_tx(&full[s], kTileBytes);
            __syncwarp();
            const unsigned char *sb = reinterpret_cast<const unsigned char *>(src);
            unsigned char *db = reinterpret_cast<unsigned char *>(U + (size_t)s * kTileVec);
            for (int hi = lane; hi < nt; hi += 32)
                bulk_load(db + (size_t)hi * seg, sb + (((size_t)hi << TBITS) + ((size_t)m << c)) * (2 * sizeof(T)), seg,
                          &full[s]);
        };

        // Pass A: w = sc * (E u + h sum_{bits < TBITS} flips of u), tile by tile.
        // MODE_ALPHA adds sc Re<u, w> to acc1; MODE_RESID (sc = 1, no store)
        // adds |w - theta u|^2 to acc1 and Re<u, w> to acc2.
        auto passA = [&](const V *src, V *dst, double sc, int mode, double theta, double &acc1, double &acc2) -> bool {
            const T scT = (T)sc;
            const K hk = mkcoef(hT * scT);
            const T thT = (T)theta;
            T ell[NE];
#pragma unroll
            for (int i = 0; i < kVPT; ++i)
#pragma unroll
                for (int e = 0; e < VE; ++e) ell[i * VE + e] = ell_tab[((tid + kThreads * i) << LOGVE) + e];
            build_tab(cr, 0);
            __syncthreads();
            return run_tiles([&](int t, int l) { issue_contig(src, t, l); },
                             [&](int t, int l, int s) {
                const V *Us = U + (size_t)s * kTileVec;
                const T *ta = tab + (l & 1) * kTabN;
                const T *tb = ta + kTA;
                A self[NE];
#pragma unroll
                for (int i = 0; i < kVPT; ++i) unpackv(Us[tid + kThreads * i], &self[i * VE]);
                constexpr int HV = kVPT / 2;  // vectors per half
                T part1 = (T)0, part2 = (T)0;
                V *dt = dst + (size_t)t * kTileVec;
                // complex128: the flip sums in 64-bit fixed point on the tile's grid
                // (exact integer adds; the FP64 pipe keeps the diagonal and the dots)
                int et = 0;
                double fxs = 0.0;
                if constexpr (sizeof(T) == sizeof(double)) {
                    unsigned em = 0u;
#pragma unroll
                    for (int q = 0; q < NE; ++q) em = max(em, max(fx_expo(tocx(self[q]).x), fx_expo(tocx(self[q]).y)));
                    em = __reduce_max_sync(0xffffffffu, em);
                    if (lane == 0) atomicMax(&s_fxe, em);
                    __syncthreads();
                    et = (int)*reinterpret_cast<volatile unsigned *>(&s_fxe);
                    fxs = fx_scale((double)hT * sc, et);
                    longlong2 *Ux = reinterpret_cast<longlong2 *>(const_cast<V *>(Us));
#pragma unroll
                    for (int i = 0; i < kVPT; ++i) {
                        const double2 a = tocx(self[i]);
                        longlong2 f;
                        f.x = fx_from(a.x, et);
                        f.y = fx_from(a.y, et);
                        Ux[tid + kThreads * i] = f;
                    }
                    // generic-proxy stores ordered before the stage's next bulk copy
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncthreads();
                    if (tid == 0) s_fxe = 0u;  // read by every thread; the next tile starts after a barrier
                }
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    A acc[HV * VE];
#pragma unroll
                    for (int i = 0; i < HV; ++i)
#pragma unroll
                        for (int e = 0; e < VE; ++e) {
                            const int gi = hh * HV + i;
                            const int li = ((tid + kThreads * gi) << LOGVE) + e;
                            const T E = (ell[gi * VE + e] + ta[li & (kTA - 1)] + tb[li >> 6]) * scT;
                            acc[i * VE + e] = self[gi * VE + e];
                            amul(mkcoef(E), acc[i * VE + e]);
                        }
                    if (VE == 2) {
#pragma unroll
                        for (int i = 0; i < HV; ++i) {
                            const int gi = hh * HV + i;
                            afma(hk, self[gi * VE + VE - 1], acc[i * VE]);
                            afma(hk, self[gi * VE], acc[i * VE + VE - 1]);
                        }
                    }
                    if constexpr (sizeof(T) == sizeof(double)) {
                        const longlong2 *Ux = reinterpret_cast<const longlong2 *>(Us);
                        long long ar[HV], ai[HV];
#pragma unroll
                        for (int i = 0; i < HV; ++i) ar[i] = ai[i] = 0ll;
#pragma unroll
                        for (int kb = 0; kb < 4; ++kb)
#pragma unroll
                            for (int i = 0; i < HV; ++i) {
                                const longlong2 v = Ux[tid + kThreads * ((hh * HV + i) ^ (1 << kb))];
                                ar[i] += v.x;
                                ai[i] += v.y;
                            }
#pragma unroll 1
                        for (int kb = 0; kb < 8; ++kb) {
                            const longlong2 *Uf = Ux + (tid ^ (1 << kb));
#pragma unroll
                            for (int i = 0; i < HV; ++i) {
                                const longlong2 v = Uf[kThreads * (hh * HV + i)];
                                ar[i] += v.x;
                                ai[i] += v.y;
                            }
                        }
#pragma unroll
                        for (int i = 0; i < HV; ++i) {
                            double2 a = tocx(acc[i]);
                            a.x = fma(fxs, __ll2double_rn(ar[i]), a.x);
                            a.y = fma(fxs, __ll2double_rn(ai[i]), a.y);
                            acc[i] = a;
                        }
                    } else {
#pragma unroll
                        for (int kb = 0; kb < 4; ++kb)
#pragma unroll
                            for (int i = 0; i < HV; ++i)
#pragma unroll
                                for (int e = 0; e < VE; ++e)
                                    afma(hk, self[((hh * HV + i) ^ (1 << kb)) * VE + e], acc[i * VE + e]);
#pragma unroll 1
                        for (int kb = 0; kb < 8; ++kb) {
                            const int pt = tid ^ (1 << kb);
#pragma unroll
                            for (int i = 0; i < HV; ++i) {
                                A pv[VE];
                                unpackv(Us[pt + kThreads * (hh * HV + i)], pv);
#pragma unroll
                                for (int e = 0; e < VE; ++e) afma(hk, pv[e], acc[i * VE + e]);
                            }
                        }
                    }
                    if (mode == MODE_RESID) {
                        const K mth = mkcoef(-thT);
#pragma unroll
                        for (int i = 0; i < HV; ++i)
#pragma unroll
                            for (int e = 0; e < VE; ++e) {
                                const A u = self[(hh * HV + i) * VE + e];
                                part2 += adot(u, acc[i * VE + e]);
                                A r = acc[i * VE + e];
                                afma(mth, u, r);
                                part1 += anorm(r);
                            }
                    } else {
#pragma unroll
                        for (int i = 0; i < HV; ++i) dt[tid + kThreads * (hh * HV + i)] = packv(&acc[i * VE]);
                        if (mode == MODE_ALPHA) {
#pragma unroll
                            for (int i = 0; i < HV; ++i)
#pragma unroll
                                for (int e = 0; e < VE; ++e) part1 += adot(self[(hh * HV + i) * VE + e], acc[i * VE + e]);
                        }
                    }
                }
                if (l + 1 < ntl) build_tab(t + cc, (l + 1) & 1);
                acc1 += (mode == MODE_ALPHA ? sc : 1.0) * (double)part1;
                acc2 += (double)part2;
            });
        };

        // Pass B: w += sc * h sum_{g high bits} flips of u, on gathered tiles
        // (tile-local index li = (hi << c) | chunk <-> amplitude (hi << TBITS) | (m << c) | chunk).
        const size_t cmask = ((size_t)1 << c) - 1;
        auto gvec = [&](int m, int i) -> size_t {
            const size_t li = (size_t)(tid + kThreads * i) << LOGVE;
            return (((li >> c) << TBITS) | ((size_t)m << c) | (li & cmask)) >> LOGVE;
        };
        auto passB = [&](const V *src, V *dst, double sc, int mode, double theta, double &acc1, double &acc2) -> bool {
            const T scT = (T)sc;
            const K hk = mkcoef(hT * scT);
            const T thT = (T)theta;
            return run_tiles([&](int m, int l) { issue_gather(src, m, l); },
                             [&](int m, int l, int s) {
                const V *Us = U + (size_t)s * kTileVec;
                A wv[NE], f[NE];
#pragma unroll
                for (int i = 0; i < kVPT; ++i) unpackv(dst[gvec(m, i)], &wv[i * VE]);  // partial sum of pass A
#pragma unroll
                for (int q = 0; q < NE; ++q) f[q] = azero((T)0);
                bool fx_done = false;
                if constexpr (sizeof(T) == sizeof(double)) {
                    if (TBITS - c >= 4) {
                        // complex128, four or more gathered bits: the flip sums in
                        // 64-bit fixed point on the tile's grid, as in pass A
                        unsigned em = 0u;
#pragma unroll
                        for (int i = 0; i < kVPT; ++i) {
                            const double2 a = tocx(Us[tid + kThreads * i]);
                            em = max(em, max(fx_expo(a.x), fx_expo(a.y)));
                        }
                        em = __reduce_max_sync(0xffffffffu, em);
                        if (lane == 0) atomicMax(&s_fxe, em);
                        __syncthreads();
                        const int et = (int)*reinterpret_cast<volatile unsigned *>(&s_fxe);
                        const double fxs = fx_scale((double)hT * sc, et);
                        longlong2 *Ux = reinterpret_cast<longlong2 *>(const_cast<V *>(Us));
                        longlong2 own[kVPT];
#pragma unroll
                        for (int i = 0; i < kVPT; ++i) {
                            const double2 a = tocx(Us[tid + kThreads * i]);
                            own[i].x = fx_from(a.x, et);
                            own[i].y = fx_from(a.y, et);
                        }
                        __syncthreads();  // every thread has read its doubles before any is overwritten
#pragma unroll
                        for (int i = 0; i < kVPT; ++i) Ux[tid + kThreads * i] = own[i];
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncthreads();
                        if (tid == 0) s_fxe = 0u;
                        long long ar[kVPT], ai[kVPT];
#pragma unroll
                        for (int i = 0; i < kVPT; ++i) ar[i] = ai[i] = 0ll;
#pragma unroll 1
                        for (int kb = c; kb < TBITS; ++kb) {
                            const int pb = kb < 8 ? (1 << kb) : (kThreads << (kb - 8));  // partner offset in vectors
#pragma unroll
                            for (int i = 0; i < kVPT; ++i) {
                                const longlong2 v = Ux[(tid + kThreads * i) ^ pb];
                                ar[i] += v.x;
                                ai[i] += v.y;
                            }
                        }
#pragma unroll
                        for (int i = 0; i < kVPT; ++i) {
                            double2 a = tocx(wv[i]);
                            a.x = fma(fxs, __ll2double_rn(ar[i]), a.x);
                            a.y = fma(fxs, __ll2double_rn(ai[i]), a.y);
                            wv[i] = a;
                        }
                        fx_done = true;
                    }
                }
                if (!fx_done) {
                    // flips of tile-local bits c .. TBITS-1, partners read from shared memory
#pragma unroll 1
                    for (int kb = 0; kb < 12; ++kb) {
                        if (LOGVE + kb < c) continue;
                        const int pb = kb < 8 ? (1 << kb) : (kThreads << (kb - 8));  // partner offset in vectors
#pragma unroll
                        for (int i = 0; i < kVPT; ++i) {
                            A pv[VE];
                            unpackv(Us[(tid + kThreads * i) ^ pb], pv);
#pragma unroll
                            for (int e = 0; e < VE; ++e) afma(hk, pv[e], f[i * VE + e]);
                        }
                    }
                    const K one = mkcoef((T)1);
#pragma unroll
                    for (int q = 0; q < NE; ++q) afma(one, f[q], wv[q]);
                }
                T part1 = (T)0, part2 = (T)0;
                if (mode == MODE_RESID) {
                    const K mth = mkcoef(-thT);
#pragma unroll
                    for (int i = 0; i < kVPT; ++i) {
                        A sv[VE];
                        // the tile holds integers after a fixed-point pass: u from global
                        // memory then (the same values, just staged from there)
                        unpackv(fx_done ? src[gvec(m, i)] : Us[tid + kThreads * i], sv);
#pragma unroll
                        for (int e = 0; e < VE; ++e) {
                            part2 += adot(sv[e], wv[i * VE + e]);
                            A r = wv[i * VE + e];
                            afma(mth, sv[e], r);
                            part1 += anorm(r);
                        }
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < kVPT; ++i) dst[gvec(m, i)] = packv(&wv[i * VE]);
                    if (mode == MODE_ALPHA) {
#pragma unroll
                        for (int i = 0; i < kVPT; ++i) {
                            A sv[VE];
                            unpackv(fx_done ? src[gvec(m, i)] : Us[tid + kThreads * i], sv);
#pragma unroll
                            for (int e = 0; e < VE; ++e) part1 += adot(sv[e], wv[i * VE + e]);
                        }
                    }
                }
                acc1 += (mode == MODE_ALPHA ? sc : 1.0) * (double)part1;
                acc2 += (double)part2;
            });
        };

        // Pass C (streaming over this CTA's range): w <- w - a u - b up and |w|^2;
        // x <- x + y u (or y u) and |x|^2.
        auto passC = [&](V *w, const V *u, const V *up, T a, T b, bool use_up, bool do_w, V *x, T y, bool x_init,
                         bool do_x, double &nw, double &nx) {
            const K ka = mkcoef(-a), kb = mkcoef(-b), ky = mkcoef(y);
            for (long long v0 = vbeg + tid; v0 < vbeg + vlen; v0 += 4 * kThreads) {
                V uv[4], wv[4], pv[4], xv[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const long long v = v0 + q * kThreads;
                    uv[q] = u[v];
                    if (do_w) wv[q] = w[v];
                    if (do_w && use_up) pv[q] = up[v];
                    if (do_x && !x_init) xv[q] = x[v];
                }
                T pw = (T)0, px = (T)0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const long long v = v0 + q * kThreads;
                    A ua[VE];
                    unpackv(uv[q], ua);
                    if (do_w) {
                        A wa[VE], pa[VE];
                        unpackv(wv[q], wa);
                        if (use_up) unpackv(pv[q], pa);
#pragma unroll
                        for (int e = 0; e < VE; ++e) {
                            afma(ka, ua[e], wa[e]);
                            if (use_up) afma(kb, pa[e], wa[e]);
                            pw += anorm(wa[e]);
                        }
                        w[v] = packv(wa);
                    }
                    if (do_x) {
                        A xa[VE];
                        if (x_init) {
#pragma unroll
                            for (int e = 0; e < VE; ++e) {
                                xa[e] = ua[e];
                                amul(ky, xa[e]);
                            }
                        } else {
                            unpackv(xv[q], xa);
#pragma unroll
                            for (int e = 0; e < VE; ++e) afma(ky, ua[e], xa[e]);
                        }
#pragma unroll
                        for (int e = 0; e < VE; ++e) px += anorm(xa[e]);
                        x[v] = packv(xa);
                    }
                }
                nw += (double)pw;
                nx += (double)px;
            }
            // later bulk copies (async proxy) read what these generic stores wrote
            asm volatile("fence.proxy.async.global;" ::: "memory");
        };

        // one H.psi product (passes A and B) into w; false, the same on every
        // CTA of the group, when a bounded wait gave up
        auto hpsi = [&](const V *u, V *w, double sc, bool want_alpha, double &al) -> bool {
            double a1 = 0.0, a2 = 0.0;
            bool ok = passA(u, w, sc, (want_alpha && g == 0) ? MODE_ALPHA : MODE_STORE, 0.0, a1, a2);
            if (g > 0) {
                if (cc > 1) {  // pass B reads partial sums written by every CTA of the group
                    double z1 = 0.0, z2 = 0.0, f = ok ? 0.0 : 1.0;
                    gsum(z1, z2, f);
                    ok = f == 0.0;
                }
                if (!ok) return false;
                ok = passB(u, w, sc, want_alpha ? MODE_ALPHA : MODE_STORE, 0.0, a1, a2);
            }
            al = a1;
            return ok;
        };

        V *const u0 = p.psi + voff;
        V *const Rb[3] = {p.R0 + voff, p.R1 + voff, p.R2 + voff};
        V *const Xb = p.X + voff;
        // chk: steps between convergence checks (small chains check less often: the
        // tridiagonal work is then comparable to a step)
        const int chk = L >= 17 ? 1 : (L == 16 ? 2 : (L == 15 ? 4 : 8));
        int status = 0;
        const bool lead = (cr == 0 && tid == 0);

        // |psi|^2 of the start vector
        double n0 = 0.0, zz = 0.0, f0 = 0.0;
        for (long long v0 = vbeg + tid; v0 < vbeg + vlen; v0 += 4 * kThreads) {
            T part = (T)0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                A a[VE];
                unpackv(u0[v0 + q * kThreads], a);
#pragma unroll
                for (int e = 0; e < VE; ++e) part += anorm(a[e]);
            }
            n0 += (double)part;
        }
        gsum(n0, zz, f0);
        if (!(n0 > 0.0) || !isfinite(n0)) {
            if (lead) {
                p.status[k] = OSMPS_EINVAL;
                p.energy[k] = 0.0;
                p.residual[k] = 0.0;
                p.iters[k] = 0;
            }
            return true;
        }
        const double s0 = 1.0 / sqrt(n0);

        // ---- sweep 1: the recurrence and T ----
        // Stopping: beta_{j+1} |y_j| <= tol, or (complex64 vectors only, whose
        // recurrence estimate stalls near eps32 |H| once ghost copies of the
        // converged Ritz value form) the lowest Ritz value moved by at most
        // tol max(1, |theta|) since the previous check while the estimate is
        // below sqrt(tol) max(1, |theta|).  The Ritz vector is taken from the
        // T_m with the smallest estimate seen (before any ghost copy).
        double sc = s0, sp = 0.0, bcur = 0.0;
        RitzState rs{0.0, INFINITY, INFINITY, INFINITY};
        double est_best = INFINITY, theta_best = 0.0;
        int m = 0, m_best = 0;
        bool conv = false;
        for (int j = 0; j < mi; ++j) {
            const V *uc = j == 0 ? u0 : Rb[(j - 1) % 3];
            const V *upv = j <= 1 ? u0 : Rb[(j - 2) % 3];
            V *w = Rb[j % 3];
            double al = 0.0, z = 0.0;
            double f = hpsi(uc, w, sc, true, al) ? 0.0 : 1.0;
            gsum(al, z, f);
            if (f != 0.0) return false;
            double nw = 0.0, nx = 0.0, z2 = 0.0;
            passC(w, uc, upv, (T)(al * sc), (T)(bcur * sp), j > 0, true, nullptr, (T)0, false, false, nw, nx);
            gsum(nw, nx, z2);
            const double bn = sqrt(nw);
            if (tid == 0) {
                alpha[j] = al;
                beta[j + 1] = bn;
            }
            m = j + 1;
            __syncthreads();
            const bool breakdown = !(bn > 1e-300);
            if (m == mi || breakdown || m == 1 || m % chk == 0) {
                if (warp == 0) {
                    const double guess = rs.theta_prev - fmax(8.0 * rs.dtheta, 1e-9 * fmax(1.0, fabs(rs.theta_prev)));
                    const double th = lowest_eig_warp(alpha, beta, m, isfinite(guess) ? guess : -INFINITY,
                                                      isfinite(rs.theta_prev) ? rs.theta_prev : INFINITY);
                    if (lane == 0) {
                        ritz_vector(alpha, beta, m, th, yv, work);
                        s_dbl[0] = th;
                        s_dbl[1] = bn * fabs(yv[m - 1]);
                    }
                }
                __syncthreads();
                const double th = s_dbl[0];
                rs.est = s_dbl[1];
                rs.dtheta = isfinite(rs.theta_prev) ? fabs(rs.theta_prev - th) : INFINITY;
                rs.theta_prev = th;
                rs.theta = th;
                if (rs.est < est_best) {
                    est_best = rs.est;
                    theta_best = th;
                    m_best = m;
                }
                __syncthreads();
                const double scale = fmax(1.0, fabs(th));
                constexpr bool kStall = sizeof(T) == 4;  // complex64 vectors: stationarity rule
                if (rs.est <= p.tol || breakdown ||
                    (kStall && rs.est <= sqrt(p.tol) * scale && rs.dtheta <= p.tol * scale)) {
                    conv = true;
                    break;
                }
            }
            sp = sc;
            sc = 1.0 / bn;
            bcur = bn;
        }
        if (!conv) status = OSMPS_ENOCONV;
        if (m_best != m) {  // Ritz vector of T_{m_best}
            if (tid == 0) ritz_vector(alpha, beta, m_best, theta_best, yv, work);
            __syncthreads();
        }
        const int mv = m_best;

        // ---- sweep 2: regenerate v_0..v_{mv-1}, accumulate x = sum_j y_j v_j ----
        sc = s0;
        sp = 0.0;
        bcur = 0.0;
        double nxs = 0.0;
        for (int j = 0; j < mv; ++j) {
            const V *uc = j == 0 ? u0 : Rb[(j - 1) % 3];
            const V *upv = j <= 1 ? u0 : Rb[(j - 2) % 3];
            V *w = Rb[j % 3];
            const T yT = (T)(yv[j] * sc);
            double nw = 0.0, nx = 0.0;
            if (j == mv - 1) {
                double z = 0.0, zf = 0.0;
                passC(w, uc, upv, (T)0, (T)0, false, false, Xb, yT, j == 0, true, nw, nx);
                gsum(nx, z, zf);
                nxs = nx;
                break;
            }
            double al = 0.0, z1 = 0.0, z2 = 0.0;
            double f = hpsi(uc, w, sc, false, al) ? 0.0 : 1.0;
            if (cc > 1) gsum(z1, z2, f);  // pass C reads w of every CTA's tiles
            if (f != 0.0) return false;
            passC(w, uc, upv, (T)(alpha[j] * sc), (T)(bcur * sp), j > 0, true, Xb, yT, j == 0, true, nw, nx);
            gbar();  // the next pass A reads u written by every CTA of the group
            const double bn = beta[j + 1];
            sp = sc;
            sc = 1.0 / bn;
            bcur = bn;
        }

        // psi <- x / |x|
        {
            const K kx = mkcoef((T)(1.0 / sqrt(nxs)));
            for (long long v = vbeg + tid; v < vbeg + vlen; v += kThreads) {
                A a[VE];
                unpackv(Xb[v], a);
#pragma unroll
                for (int e = 0; e < VE; ++e) amul(kx, a[e]);
                u0[v] = packv(a);
            }
            asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        gbar();

        // true residual |H psi - theta psi| and <psi, H psi>
        double r2 = 0.0, rq = 0.0;
        bool ok = passA(u0, Rb[0], 1.0, g == 0 ? MODE_RESID : MODE_STORE, rs.theta, r2, rq);
        if (g > 0) {
            if (cc > 1) {
                double z1 = 0.0, z2 = 0.0, f = ok ? 0.0 : 1.0;
                gsum(z1, z2, f);
                ok = f == 0.0;
            }
            if (!ok) return false;
            ok = passB(u0, Rb[0], 1.0, MODE_RESID, rs.theta, r2, rq);
        }
        double fr = ok ? 0.0 : 1.0;
        gsum(r2, rq, fr);
        if (fr != 0.0) return false;
        if (lead) {
            p.energy[k] = rs.theta;
            p.residual[k] = sqrt(fmax(r2, 0.0));
            p.iters[k] = m;
            p.status[k] = status;
        }
        __syncthreads();
        return true;
    };

    // ---- work queues: large chains per cluster, then one chain per CTA ----
    bool big = csize > 1 && p.nbig > 0;
    for (;;) {
        int idx, cc, cr;
        if (big) {
            if (crank == 0 && tid == 0) {
                const int v = atomicAdd(&p.counter[0], 1);
                for (int r = 0; r < csize; ++r) st_dsmem(&s_int[0], r, v);
            }
            cluster_barrier();
            idx = s_int[0];
            cluster_barrier();
            if (idx >= p.nbig) {
                big = false;
                continue;
            }
            cc = csize;
            cr = crank;
        } else {
            if (tid == 0) s_int[1] = atomicAdd(&p.counter[1], 1);
            __syncthreads();
            idx = p.small_first + s_int[1];
            __syncthreads();
            if (idx >= p.n) break;
            cc = 1;
            cr = 0;
        }
        const int k = p.order[idx];
        if (!solve(k, cc, cr)) {
            if (cr == 0 && tid == 0) p.status[k] = OSMPS_ETIMEOUT;
            break;
        }
    }
    if (csize > 1) cluster_barrier();  // no CTA leaves while a peer may still read its shared memory
}

// ---------------------------------------------------------------------------
// Host side

size_t batch_smem_bytes(int prec) {
    const size_t t = prec == OSMPS_FP64 ? sizeof(double) : sizeof(float);
    return (size_t)kStages * kTileBytes + 2 * kTabN * t + kStages * 8 + 2 * kWarps * 8 + (kMaxL + 1) * t;
}

template <typename T>
static cudaError_t launch_batch_t(BatchHandle *b, void *psi, double tol, double *energy, double *residual,
                                  int *iters, int *status) {
    typedef typename Cx<T>::v16 V;
    BatchParams<T> p;
    p.inst = b->d_inst;
    p.order = b->d_order;
    p.psi = reinterpret_cast<V *>(psi);
    p.R0 = reinterpret_cast<V *>(b->R[0]);
    p.R1 = reinterpret_cast<V *>(b->R[1]);
    p.R2 = reinterpret_cast<V *>(b->R[2]);
    p.X = reinterpret_cast<V *>(b->X);
    p.energy = energy;
    p.residual = residual;
    p.iters = iters;
    p.status = status;
    p.scratch = b->scratch;
    p.counter = b->counter;
    p.err = b->err;
    p.tol = tol;
    p.n = b->n;
    p.max_iter = b->max_iter;
    p.nbig = b->csize > 1 ? b->nbig : 0;
    p.small_first = p.nbig;
    const size_t smem = batch_smem_bytes(b->prec);
    cudaError_t err = cudaMemsetAsync(b->counter, 0, 2 * sizeof(int), b->stream);
    if (err != cudaSuccess) return err;
    if (b->csize > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)b->grid);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = b->stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)b->csize;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        err = cudaLaunchKernelEx(&cfg, lanczos_batch_kernel<T>, p);
        if (err != cudaSuccess) return err;
    } else {
        lanczos_batch_kernel<T><<<b->grid, kThreads, smem, b->stream>>>(p);
    }
    b->launches++;
    return cudaGetLastError();
}

// Opt in to the dynamic shared memory of the launch (once, at create; not a
// stream operation, so it stays out of captured graphs).
cudaError_t batch_prepare(int prec) {
    const int smem = (int)batch_smem_bytes(prec);
    return prec == OSMPS_FP64
               ? cudaFuncSetAttribute(lanczos_batch_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
               : cudaFuncSetAttribute(lanczos_batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// Clusters of csize CTAs that can be resident at once (one CTA per SM).
cudaError_t batch_max_clusters(int prec, int csize, int nsm, int *out) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(csize * (nsm / csize)));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = batch_smem_bytes(prec);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return prec == OSMPS_FP64
               ? cudaOccupancyMaxActiveClusters(out, (void *)lanczos_batch_kernel<double>, &cfg)
               : cudaOccupancyMaxActiveClusters(out, (void *)lanczos_batch_kernel<float>, &cfg);
}

cudaError_t launch_batch(BatchHandle *b, void *psi, double tol, double *energy, double *residual, int *iters,
                         int *status) {
    return b->prec == OSMPS_FP64 ? launch_batch_t<double>(b, psi, tol, energy, residual, iters, status)
                                 : launch_batch_t<float>(b, psi, tol, energy, residual, iters, status);
}

int batch_tile_bits(int prec) { return prec == OSMPS_FP64 ? 12 : 13; }

}  // namespace batch
}  // namespace osmps
