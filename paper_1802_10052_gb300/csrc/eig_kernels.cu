// Eigenvalues of the half-chain density matrix rho_A (Hermitian, n x n):
// the Schmidt spectrum Lambda_j of Sec. IV (bond entropy).
//
// Householder reduction to real symmetric tridiagonal form, blocked by panels
// of kNb columns (the Dongarra-Sorensen-Hammarling blocked form of the
// reduction), then the eigenvalues of the tridiagonal matrix by Sturm-sequence
// bisection.  Every step runs in the kernels of this file:
//
// * trd_panel_kernel: one cooperative launch per panel.  Each CTA owns a slice
//   of rows (and keeps its rows of the panel's V and W in shared memory); per
//   column c of the panel (three grid barriers with bounded waits):
//     A  update column c by the panel's earlier reflectors,
//            a = A[:,c] - V W[c,:]^H - W V[c,:]^H,
//        partial |a_{c+2:}|^2                                    -- barrier
//     B  beta, tau, v = (1, a_{c+2:} / (alpha - beta)) (every CTA, in shared
//        memory); p = A v over the CTA's rows (the lower triangle read along
//        rows and along columns); partials of W^H v and V^H v    -- barrier
//     C  p~ = p - V (W^H v) - W (V^H v); partial p~^H v         -- barrier
//     D  w = tau p~ - (|tau|^2 / 2)(p~^H v) v
//   A holds the lower triangle column-major (column c contiguous below the
//   diagonal); the trailing matrix is not touched inside a panel.  Partial
//   sums are stored value-major and reduced in a fixed order, so every CTA
//   computes bit-identical scalars.
// * her2k_lower_kernel: A22 -= V W^H + W V^H on the lower triangle after each
//   panel (register-tiled SIMT contraction, K = kNb).
// * msect_kernel: the k-th smallest eigenvalue of the tridiagonal (d, e) for
//   every k, one warp each, by 32-way multisection on a division-free Sturm
//   count in the working precision (FP32 for complex64, FP64 for complex128).
//
// The input is the row-major upper triangle written by the Gram product; read
// column-major it is the lower triangle of conj(rho), which has the same
// eigenvalues.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "ed_internal.h"

namespace osmps {
namespace eig {

constexpr int kNb = 32;             // panel width
constexpr int kThreads = 512;       // threads per CTA of the panel kernel
constexpr int kWarps = kThreads / 32;
constexpr int kPart = 4 + 4 * kNb;  // partial values per CTA
constexpr int kSmemV = 8192;        // v is kept in shared memory up to this order (else per CTA in global)
constexpr int kHT = 64;             // tile edge of the trailing update

template <typename T> struct Cp;
template <> struct Cp<float> { typedef float2 C; };
template <> struct Cp<double> { typedef double2 C; };

template <typename C> __device__ __forceinline__ C cmk(double re, double im) {
    C r;
    r.x = re;
    r.y = im;
    return r;
}
// acc += b * c
template <typename C> __device__ __forceinline__ void cfma(C &acc, C b, C c) {
    acc.x += b.x * c.x - b.y * c.y;
    acc.y += b.x * c.y + b.y * c.x;
}
// acc += conj(b) * c
template <typename C> __device__ __forceinline__ void cjfma(C &acc, C b, C c) {
    acc.x += b.x * c.x + b.y * c.y;
    acc.y += b.x * c.y - b.y * c.x;
}

struct TrdCtl {
    unsigned count;  // grid-barrier arrivals
    unsigned gen;    // grid-barrier generation
    int err;         // raised when a bounded wait gave up
    int pad;
};

template <typename T>
struct TrdArgs {
    typedef typename Cp<T>::C C;
    C *A;            // n x n, lower triangle column-major (lda = n)
    C *V, *W;        // n x kNb each, column-major (ld = n), panel-local column index
    C *col;          // n: the updated current column
    C *pv;           // n: p~ of the current column
    C *vg;           // gridDim.x x n: per-CTA copy of v when n > kSmemV
    double *part;    // kPart x gridDim.x (value-major: a value's partials are contiguous)
    double *d, *e;   // the tridiagonal (global indices)
    TrdCtl *ctl;
    int n, k0, ncol; // panel start and its columns (the last panel includes c = n-1)
};

// Grid-wide barrier for a cooperative launch.  Thread 0 of each CTA arrives
// on a global counter; the last arrival resets it and advances the
// generation.  The wait is bounded (kWaitNs): on timeout, or when another CTA
// already raised the error flag, it stops waiting (the results are then
// garbage and the host reports OSMPS_ETIMEOUT).
__device__ __forceinline__ void grid_sync(TrdCtl *ctl) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &ctl->gen;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->count, 1u) + 1u;
        if (arrived == gridDim.x) {
            ctl->count = 0u;
            __threadfence();
            atomicAdd(&ctl->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*vgen == g) {
                if (*(volatile int *)&ctl->err != 0) break;
                if (global_ns() - t0 > kWaitNs) {
                    atomicExch(&ctl->err, 1);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the CTA of one double per thread; thread 0 gets the result.
__device__ __forceinline__ double block_sum(double v, double *red) {
    v = warp_sum_d(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kWarps; ++w) r += red[w];
    return r;
}

// Sum over the G CTAs' partials part[off * G + q], the same fixed order on
// every CTA: each lane loads its kPL strided partials at once (independent
// loads), sums them, then a fixed shuffle tree.  Called by one whole warp;
// every lane gets the sum.  G <= 32 * kPL.
constexpr int kPL = 8;
__device__ __forceinline__ double warp_sum_parts(const double *part, int G, int off) {
    const int lane = threadIdx.x & 31;
    const double *p = part + (size_t)off * G;
    double x[kPL];
#pragma unroll
    for (int k = 0; k < kPL; ++k) x[k] = (lane + 32 * k < G) ? p[lane + 32 * k] : 0.0;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kPL; ++k) s += x[k];
    return warp_sum_d(s);
}

// One value per group of 8 lanes; every lane of the group gets its value's
// sum.  Each lane loads its ceil(G / 8) partials at once.  G <= 8 * kPL8.
constexpr int kPL8 = 24;
__device__ __forceinline__ double group8_sum_parts(const double *part, int G, int off) {
    const int sub = threadIdx.x & 7;
    const double *p = part + (size_t)off * G;
    double x[kPL8];
#pragma unroll
    for (int k = 0; k < kPL8; ++k) x[k] = (sub + 8 * k < G) ? p[sub + 8 * k] : 0.0;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kPL8; ++k) s += x[k];
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    return s;
}

// One panel of the blocked reduction (columns k0 .. k0+ncol-1).  Cooperative
// launch: every CTA of the grid is resident (grid_sync relies on it).  The
// CTA keeps its rows of the panel's V and W in shared memory (and writes them
// to global memory for the other CTAs and for the trailing update).
template <typename T>
__global__ void __launch_bounds__(kThreads, 1) trd_panel_kernel(TrdArgs<T> a) {
    typedef typename Cp<T>::C C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n, G = gridDim.x, b = blockIdx.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t N = (size_t)n;
    const int rows_max = (n + G - 1) / G;  // slice capacity (first panel)
    const int rows_per = (n - a.k0 + G - 1) / G;
    const int r_lo = a.k0 + b * rows_per;
    const int r_hi = min(n, r_lo + rows_per);
    C *pr = reinterpret_cast<C *>(smem_raw);  // rows_max: A v, then p~, of the own rows
    C *Vs = pr + rows_max;                    // kNb x rows_max: own rows of V (column j at j * rows_max)
    C *Ws = Vs + kNb * rows_max;              // kNb x rows_max: own rows of W
    C *whv = Ws + kNb * rows_max;             // kNb: W^H v
    C *vhv = whv + kNb;                       // kNb: V^H v
    C *vc = vhv + kNb;                        // kNb: row c of V
    C *wc = vc + kNb;                         // kNb: row c of W
    C *t1 = wc + kNb;                         // kWarps x 32: part-1 sums of the hemv
    C *v = (n <= kSmemV) ? (t1 + kWarps * 32) : (a.vg + (size_t)b * N);  // v_s for s >= c+1
    __shared__ double sc[8];
    __shared__ double red[2 * kWarps];
    __shared__ double red2[4 * kNb];
    C w_next = cmk<C>(0.0, 0.0);  // W[c][i-1] for the current column c (known on every CTA)

    for (int i = 0; i < a.ncol; ++i) {
        const int c = a.k0 + i;
        // ---- A: column c after the panel's earlier reflectors ----
        if (tid < i) {
            vc[tid] = (tid == i - 1) ? cmk<C>(1.0, 0.0) : a.V[(size_t)tid * N + c];
            wc[tid] = (tid == i - 1) ? w_next : a.W[(size_t)tid * N + c];
        }
        __syncthreads();
        double s2 = 0.0;
        for (int r = max(r_lo, c) + tid; r < r_hi; r += kThreads) {
            const int q = r - r_lo;
            C x = a.A[(size_t)c * N + r];
            for (int j = 0; j < i; ++j) {  // x -= V[r][j] conj(W[c][j]) + W[r][j] conj(V[c][j])
                const C vr = Vs[j * rows_max + q], wr = Ws[j * rows_max + q];
                x.x -= vr.x * wc[j].x + vr.y * wc[j].y + wr.x * vc[j].x + wr.y * vc[j].y;
                x.y -= vr.y * wc[j].x - vr.x * wc[j].y + wr.y * vc[j].x - wr.x * vc[j].y;
            }
            a.col[r] = x;
            if (r == c) a.d[c] = (double)x.x;
            if (r >= c + 2) s2 += (double)x.x * x.x + (double)x.y * x.y;
        }
        s2 = block_sum(s2, red);
        if (tid == 0) a.part[b] = s2;
        if (c == n - 1) break;  // the last diagonal entry has no reflector
        grid_sync(a.ctl);

        // ---- B: reflector (every CTA), v, and p = A v over the own rows ----
        if (warp == 0) {
            const double sig2 = warp_sum_parts(a.part, G, 0);
            if (lane == 0) {
                const C al = a.col[c + 1];
                const double ar = al.x, ai = al.y;
                double beta, tr, ti, sr, si;
                if (sig2 == 0.0 && ai == 0.0) {  // nothing to annihilate: H = I
                    beta = ar;
                    tr = ti = sr = si = 0.0;
                } else {
                    const double nrm = sqrt(ar * ar + ai * ai + sig2);
                    beta = ar >= 0.0 ? -nrm : nrm;
                    tr = (beta - ar) / beta;
                    ti = -ai / beta;
                    const double dr = ar - beta, di = ai, den = dr * dr + di * di;  // 1 / (alpha - beta)
                    sr = dr / den;
                    si = -di / den;
                }
                sc[0] = beta;
                sc[1] = tr;
                sc[2] = ti;
                sc[3] = sr;
                sc[4] = si;
                if (b == 0) a.e[c] = beta;
            }
        }
        __syncthreads();
        const double tr = sc[1], ti = sc[2], sr = sc[3], si = sc[4];
        for (int s = c + 1 + tid; s < n; s += kThreads) {
            if (s == c + 1) {
                v[s] = cmk<C>(1.0, 0.0);
            } else {
                const C x = a.col[s];
                v[s] = cmk<C>(x.x * sr - x.y * si, x.x * si + x.y * sr);
            }
        }
        __syncthreads();
        for (int r = r_lo + tid; r < r_hi; r += kThreads) {
            const C vr = r > c ? v[r] : cmk<C>(0.0, 0.0);
            Vs[i * rows_max + (r - r_lo)] = vr;
            a.V[(size_t)i * N + r] = vr;
        }
        const int rb = max(r_lo, c + 1);
        // p_r = sum_{s>c} A[r][s] v_s: for s <= r the lower triangle along row r
        // (column s, lanes = rows), for s > r the conjugate of column r below the
        // diagonal (lanes = s)
        constexpr int kB = 8;  // independent loads in flight per lane
        for (int g0 = rb; g0 < r_hi; g0 += 32) {
            const int r = g0 + lane;
            const bool rv = r < r_hi;
            const int rmax = min(r_hi, g0 + 32) - 1;
            C acc = cmk<C>(0.0, 0.0);
            for (int s0 = c + 1 + warp; s0 <= rmax; s0 += kWarps * kB) {
                C x[kB];
#pragma unroll
                for (int k = 0; k < kB; ++k) {
                    const int s = s0 + k * kWarps;
                    x[k] = (rv && s <= r) ? a.A[(size_t)s * N + r] : cmk<C>(0.0, 0.0);
                }
#pragma unroll
                for (int k = 0; k < kB; ++k) {
                    const int s = s0 + k * kWarps;
                    if (rv && s <= r) cfma(acc, x[k], v[s]);
                }
            }
            t1[warp * 32 + lane] = acc;
            __syncthreads();
            if (warp == 0 && rv) {
                C sum = cmk<C>(0.0, 0.0);
                for (int w = 0; w < kWarps; ++w) {
                    sum.x += t1[w * 32 + lane].x;
                    sum.y += t1[w * 32 + lane].y;
                }
                pr[r - r_lo] = sum;
            }
            __syncthreads();
        }
        for (int r = rb + warp; r < r_hi; r += kWarps) {
            C acc = cmk<C>(0.0, 0.0);
            const C *col_r = a.A + (size_t)r * N;
            for (int s0 = r + 1 + lane; s0 < n; s0 += 32 * kB) {
                C x[kB];
#pragma unroll
                for (int k = 0; k < kB; ++k) x[k] = (s0 + 32 * k < n) ? col_r[s0 + 32 * k] : cmk<C>(0.0, 0.0);
#pragma unroll
                for (int k = 0; k < kB; ++k)
                    if (s0 + 32 * k < n) cjfma(acc, x[k], v[s0 + 32 * k]);
            }
            const double xr = warp_sum_d((double)acc.x), xi = warp_sum_d((double)acc.y);
            if (lane == 0) {
                pr[r - r_lo].x += xr;
                pr[r - r_lo].y += xi;
            }
        }
        // partial W^H v and V^H v over the own rows (j < i)
        for (int jj = warp; jj < 2 * i; jj += kWarps) {
            const C *M = ((jj & 1) ? Vs : Ws) + (jj >> 1) * rows_max;
            double xr = 0.0, xi = 0.0;
            for (int r = rb + lane; r < r_hi; r += 32) {
                const C m = M[r - r_lo], vv = v[r];
                xr += (double)m.x * vv.x + (double)m.y * vv.y;
                xi += (double)m.x * vv.y - (double)m.y * vv.x;
            }
            xr = warp_sum_d(xr);
            xi = warp_sum_d(xi);
            if (lane == 0) {
                a.part[(size_t)(4 + 2 * jj) * G + b] = xr;
                a.part[(size_t)(5 + 2 * jj) * G + b] = xi;
            }
        }
        grid_sync(a.ctl);

        // ---- C: p~ = p - V (W^H v) - W (V^H v); partial p~^H v ----
        for (int base = 0; base < 4 * i; base += kThreads / 8) {  // 4i partial values, 8 lanes each
            const int val = base + (tid >> 3);
            const double x = group8_sum_parts(a.part, G, 4 + (val < 4 * i ? val : 0));
            if ((tid & 7) == 0 && val < 4 * i) red2[val] = x;
        }
        __syncthreads();
        if (tid < 2 * i) {
            const int jj = tid;
            const C z = cmk<C>(red2[2 * jj], red2[2 * jj + 1]);
            if (jj & 1)
                vhv[jj >> 1] = z;
            else
                whv[jj >> 1] = z;
        }
        __syncthreads();
        double phr = 0.0, phi = 0.0;
        for (int r = rb + tid; r < r_hi; r += kThreads) {
            const int q = r - r_lo;
            C pp = pr[q];
            for (int j = 0; j < i; ++j) {  // pp -= V[r][j] (W^H v)_j + W[r][j] (V^H v)_j
                const C vr = Vs[j * rows_max + q], wr = Ws[j * rows_max + q];
                pp.x -= vr.x * whv[j].x - vr.y * whv[j].y + wr.x * vhv[j].x - wr.y * vhv[j].y;
                pp.y -= vr.x * whv[j].y + vr.y * whv[j].x + wr.x * vhv[j].y + wr.y * vhv[j].x;
            }
            pr[q] = pp;
            a.pv[r] = pp;
            const C vv = v[r];
            phr += (double)pp.x * vv.x + (double)pp.y * vv.y;
            phi += (double)pp.x * vv.y - (double)pp.y * vv.x;
        }
        phr = block_sum(phr, red);
        phi = block_sum(phi, red + kWarps);
        if (tid == 0) {
            a.part[(size_t)G + b] = phr;
            a.part[(size_t)2 * G + b] = phi;
        }
        grid_sync(a.ctl);

        // ---- D: w = tau p~ + alpha v with alpha = -(|tau|^2 / 2) p~^H v ----
        if (warp == 0) {
            const double xr = warp_sum_parts(a.part, G, 1);
            const double xi = warp_sum_parts(a.part, G, 2);
            if (lane == 0) {
                const double hh = -0.5 * (tr * tr + ti * ti);
                sc[5] = hh * xr;
                sc[6] = hh * xi;
            }
        }
        __syncthreads();
        const double alr = sc[5], ali = sc[6];
        for (int r = r_lo + tid; r < r_hi; r += kThreads) {
            C w = cmk<C>(0.0, 0.0);
            if (r > c) {
                const C pp = pr[r - r_lo], vv = v[r];
                w = cmk<C>(tr * pp.x - ti * pp.y + alr * vv.x - ali * vv.y, tr * pp.y + ti * pp.x + alr * vv.y + ali * vv.x);
            }
            Ws[i * rows_max + (r - r_lo)] = w;
            a.W[(size_t)i * N + r] = w;
        }
        {
            const C pp = a.pv[c + 1];
            w_next = cmk<C>(tr * pp.x - ti * pp.y + alr, tr * pp.y + ti * pp.x + ali);
        }
    }
}

size_t trd_panel_smem(int n, int prec, int G) {
    const size_t cs = prec == OSMPS_FP64 ? 16 : 8;
    const size_t rows = ((size_t)n + G - 1) / G;
    return cs * (rows * (1 + 2 * kNb) + 4 * kNb + kWarps * 32 + (n <= kSmemV ? (size_t)n : 0));
}

// ---------------------------------------------------------------------------
// Trailing update after a panel: A[r][s] -= sum_j V[r][j] conj(W[s][j]) +
// W[r][j] conj(V[s][j]) for k1 <= s <= r < n (lower triangle, column-major).
// One CTA per 64 x 64 tile of the lower triangle (tile row I >= tile column
// J); each thread accumulates a 4 x 4 block.
template <typename T>
__global__ void __launch_bounds__(256) her2k_lower_kernel(typename Cp<T>::C *A, int n, int k1,
                                                          const typename Cp<T>::C *V, const typename Cp<T>::C *W,
                                                          int kc) {
    typedef typename Cp<T>::C C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *VI = reinterpret_cast<C *>(smem_raw);  // kNb x kHT each, column j contiguous over the tile's rows
    C *WI = VI + kNb * kHT;
    C *VJ = WI + kNb * kHT;
    C *WJ = VJ + kNb * kHT;
    const long long t = blockIdx.x;
    int I = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long long)(I + 1) * (I + 2) / 2 <= t) ++I;
    while ((long long)I * (I + 1) / 2 > t) --I;
    const int J = (int)(t - (long long)I * (I + 1) / 2);
    const int r0 = k1 + I * kHT, s0 = k1 + J * kHT;
    const size_t N = (size_t)n;
    for (int idx = threadIdx.x; idx < kc * kHT; idx += blockDim.x) {
        const int j = idx / kHT, q = idx % kHT;
        const C z = cmk<C>(0.0, 0.0);
        VI[idx] = r0 + q < n ? V[(size_t)j * N + r0 + q] : z;
        WI[idx] = r0 + q < n ? W[(size_t)j * N + r0 + q] : z;
        VJ[idx] = s0 + q < n ? V[(size_t)j * N + s0 + q] : z;
        WJ[idx] = s0 + q < n ? W[(size_t)j * N + s0 + q] : z;
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T ar[4][4], ai[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) ar[x][y] = ai[x][y] = (T)0;
    for (int j = 0; j < kc; ++j) {
        C vi[4], wi[4], vj[4], wj[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            vi[x] = VI[j * kHT + tx * 4 + x];
            wi[x] = WI[j * kHT + tx * 4 + x];
            vj[x] = VJ[j * kHT + ty * 4 + x];
            wj[x] = WJ[j * kHT + ty * 4 + x];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) {  // vi conj(wj) + wi conj(vj)
                ar[x][y] += vi[x].x * wj[y].x + vi[x].y * wj[y].y + wi[x].x * vj[y].x + wi[x].y * vj[y].y;
                ai[x][y] += vi[x].y * wj[y].x - vi[x].x * wj[y].y + wi[x].y * vj[y].x - wi[x].x * vj[y].y;
            }
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
        const int sc = s0 + ty * 4 + y;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int r = r0 + tx * 4 + x;
            if (r < n && sc < n && r >= sc) {
                C &el = A[(size_t)sc * N + r];
                el.x -= ar[x][y];
                el.y -= ai[x][y];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Eigenvalues of the symmetric tridiagonal (d, e): Gershgorin bounds and e^2,
// then multisection on the Sturm count for every index k.

__global__ void gersh_kernel(const double *d, const double *e, int n, double *e2, double *bounds) {
    __shared__ double slo[32], shi[32];
    double lo = 1e300, hi = -1e300;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
        lo = fmin(lo, d[i] - r);
        hi = fmax(hi, d[i] + r);
        if (i + 1 < n) e2[i] = e[i] * e[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        slo[threadIdx.x >> 5] = lo;
        shi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            lo = fmin(lo, slo[w]);
            hi = fmax(hi, shi[w]);
        }
        const double pad = 2.2e-16 * fmax(fabs(lo), fabs(hi)) * n + 1e-300;
        bounds[0] = lo - pad;
        bounds[1] = hi + pad;
    }
}

// Number of eigenvalues below x: sign changes of the leading principal minors
// p_i = det(T_i - x I), p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (no
// division; p_i / p_{i-1} is the i-th pivot of the LDL^T factorisation), in
// the precision R.  The pair (p_{i-1}, p_i) is rescaled by an exact power of
// two when |p_i| leaves [2^-S, 2^S]; an exact zero p_i is replaced by a tiny
// value of the sign that counts it as negative.
template <typename R> struct SturmScale;
template <> struct SturmScale<float> {
    static constexpr float hi = 0x1p60f, lo = 0x1p-60f, tiny = 1e-30f;
};
template <> struct SturmScale<double> {
    static constexpr double hi = 0x1p500, lo = 0x1p-500, tiny = 1e-300;
};
template <typename R>
__device__ __forceinline__ int sturm_count_poly(const R *d, const R *e2, int n, R x) {
    typedef SturmScale<R> S;
    R pm = (R)1, pc = d[0] - x;
    if (pc == (R)0) pc = -S::tiny;
    int cnt = pc < (R)0;
    for (int i = 1; i < n; ++i) {
        R pn = fma(d[i] - x, pc, -e2[i - 1] * pm);
        if (pn == (R)0) pn = (pc < (R)0 ? S::tiny : -S::tiny);
        cnt += (pn < (R)0) != (pc < (R)0);
        pm = pc;
        pc = pn;
        const R ap = fabs(pc);
        if (ap > S::hi) {
            pc *= S::lo;
            pm *= S::lo;
        } else if (ap < S::lo) {
            pc *= S::hi;
            pm *= S::hi;
        }
    }
    return cnt;
}

// w[k] = k-th smallest eigenvalue (ascending): one warp per k, 32-way
// multisection (each round evaluates 32 interior points of [lo, hi] with the
// Sturm count in precision R and keeps the sub-interval where the count first
// exceeds k) until the bracket is a few ulps of R wide.
template <typename R>
__global__ void msect_kernel(const R *d, const R *e2, int n, const double *bounds, double *w) {
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= n) return;  // whole warps leave together
    double lo = bounds[0], hi = bounds[1];
    // refine until the bracket is a few ulps of R wide relative to itself (tiny
    // eigenvalues keep their relative accuracy), at most 24 rounds (120 bits)
    const double eps = sizeof(R) == 4 ? 1.2e-7 : 2.2e-16;
    const double floor_abs = (sizeof(R) == 4 ? 1e-37 : 1e-20 * fmax(fabs(lo), fabs(hi)));
    for (int round = 0; round < 24 && hi - lo > fmax(2.0 * eps * fmax(fabs(lo), fabs(hi)), floor_abs); ++round) {
        const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
        const int cnt = sturm_count_poly<R>(d, e2, n, (R)x);
        const unsigned bal = __ballot_sync(0xffffffffu, cnt > k);
        if (bal == 0u) {
            lo = __shfl_sync(0xffffffffu, x, 31);
        } else {
            const int f = __ffs((int)bal) - 1;
            const double xf = __shfl_sync(0xffffffffu, x, f);
            const double xp = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
            hi = xf;
            if (f > 0) lo = xp;
        }
    }
    if (lane == 0) w[k] = 0.5 * (lo + hi);
}

// d, e^2 in the precision of the Sturm counts
template <typename R>
__global__ void cast_tridiag_kernel(const double *d, const double *e2, int n, R *dr, R *e2r) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        dr[i] = (R)d[i];
        e2r[i] = i + 1 < n ? (R)e2[i] : (R)0;
    }
}

// copy the barrier error flag into the handle's error word
__global__ void trd_err_kernel(const TrdCtl *ctl, int *error) {
    if (ctl->err != 0) *error = 1;
}

}  // namespace eig

// ---------------------------------------------------------------------------
// Host driver.  Workspace layout (one carve per call, 256-byte aligned
// pieces): V, W (n x kNb each), the current column and p~, per-CTA copies of v
// when n > kSmemV, partials, d, e, e^2, bounds, the barrier block, the
// eigenvalues and the Sturm inputs in the working precision.
struct TrdLayout {
    size_t oV, oW, oc, op, og, opa, od, oe, oe2, ob, octl, ow, odr, oer, total;
};

static TrdLayout trd_layout(int n, int prec, int G) {
    const size_t cs = prec == OSMPS_FP64 ? 16 : 8, rs = prec == OSMPS_FP64 ? 8 : 4, N = (size_t)n;
    TrdLayout l{};
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    l.oV = carve(cs * N * eig::kNb);
    l.oW = carve(cs * N * eig::kNb);
    l.oc = carve(cs * N);
    l.op = carve(cs * N);
    l.og = carve(n > eig::kSmemV ? cs * N * G : 0);
    l.opa = carve(sizeof(double) * G * eig::kPart);
    l.od = carve(sizeof(double) * N);
    l.oe = carve(sizeof(double) * N);
    l.oe2 = carve(sizeof(double) * N);
    l.ob = carve(2 * sizeof(double));
    l.octl = carve(sizeof(eig::TrdCtl));
    l.ow = carve(sizeof(double) * N);
    l.odr = carve(rs * N);
    l.oer = carve(rs * N);
    l.total = off;
    return l;
}

// Smallest CTA count >= want (and <= the device's SMs) whose row slices fit
// in shared memory; 0 if none does.
constexpr size_t kStaticSmemMargin = 4096;

int trd_ctas(int n, int prec, int want, int device) {
    int optin = 0, nsm = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int gmax = nsm < 8 * eig::kPL8 ? nsm : 8 * eig::kPL8;
    // the panel kernel's static shared memory (a few KB of reduction scratch) comes on top
    const size_t limit = (size_t)optin > kStaticSmemMargin ? (size_t)optin - kStaticSmemMargin : 0;
    for (int G = want < 1 ? 1 : want; G <= gmax; ++G)
        if (eig::trd_panel_smem(n, prec, G) <= limit) return G;
    return 0;
}

size_t trd_workspace_bytes(int n, int prec, int G) { return trd_layout(n, prec, G).total; }

template <typename T>
static cudaError_t trd_eigvals_t(const TrdRun &run, void *rho, int n, double **w_out) {
    using namespace eig;
    typedef typename Cp<T>::C C;
    const int prec = run.prec, G = run.G;
    cudaStream_t st = run.stream;
    const size_t smem = eig::trd_panel_smem(n, prec, G);
    int smem_optin = 0, per_sm = 0;
    cudaError_t err = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, run.device);
    if (err != cudaSuccess) return err;
    if (G < 1 || G > 8 * kPL8 || smem + kStaticSmemMargin > (size_t)smem_optin) return cudaErrorNotSupported;
    err = cudaFuncSetAttribute(trd_panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trd_panel_kernel<T>, kThreads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorNotSupported;
    const TrdLayout l = trd_layout(n, prec, G);
    if (run.ws == nullptr || run.ws_bytes < l.total) return cudaErrorInvalidValue;
    char *ws = static_cast<char *>(run.ws);
    TrdArgs<T> a;
    a.A = static_cast<C *>(rho);
    a.V = reinterpret_cast<C *>(ws + l.oV);
    a.W = reinterpret_cast<C *>(ws + l.oW);
    a.col = reinterpret_cast<C *>(ws + l.oc);
    a.pv = reinterpret_cast<C *>(ws + l.op);
    a.vg = reinterpret_cast<C *>(ws + l.og);
    a.part = reinterpret_cast<double *>(ws + l.opa);
    a.d = reinterpret_cast<double *>(ws + l.od);
    a.e = reinterpret_cast<double *>(ws + l.oe);
    a.ctl = reinterpret_cast<TrdCtl *>(ws + l.octl);
    a.n = n;
    double *e2 = reinterpret_cast<double *>(ws + l.oe2);
    double *bounds = reinterpret_cast<double *>(ws + l.ob);
    double *w = reinterpret_cast<double *>(ws + l.ow);
    *w_out = w;
    err = cudaMemsetAsync(a.ctl, 0, sizeof(TrdCtl), st);
    if (err != cudaSuccess) return err;
    const size_t hsmem = 4 * sizeof(C) * kNb * kHT;
    if (hsmem > 48 * 1024) {
        err = cudaFuncSetAttribute(her2k_lower_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem);
        if (err != cudaSuccess) return err;
    }
    int64_t nl = 0;
    for (int k0 = 0; k0 < n; k0 += kNb) {
        a.k0 = k0;
        a.ncol = n - k0 < kNb ? n - k0 : kNb;
        void *kargs[] = {&a};
        err = cudaLaunchCooperativeKernel((const void *)trd_panel_kernel<T>, dim3(G), dim3(kThreads), kargs, smem, st);
        if (err != cudaSuccess) return err;
        ++nl;
        const int k1 = k0 + kNb;
        if (k1 < n) {
            const long long mt = (n - k1 + kHT - 1) / kHT;
            her2k_lower_kernel<T><<<(unsigned)(mt * (mt + 1) / 2), 256, hsmem, st>>>(a.A, n, k1, a.V, a.W, a.ncol);
            ++nl;
        }
    }
    // Sturm counts in the working precision: the complex64 reduction carries
    // rounding of order eps32 |rho| already
    T *dr = reinterpret_cast<T *>(ws + l.odr);
    T *er = reinterpret_cast<T *>(ws + l.oer);
    gersh_kernel<<<1, 1024, 0, st>>>(a.d, a.e, n, e2, bounds);
    cast_tridiag_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(a.d, e2, n, dr, er);
    msect_kernel<T><<<(unsigned)(((size_t)n * 32 + 127) / 128), 128, 0, st>>>(dr, er, n, bounds, w);
    trd_err_kernel<<<1, 1, 0, st>>>(a.ctl, run.error);
    nl += 4;
    if (run.launches) *run.launches += nl;
    return cudaGetLastError();
}

cudaError_t trd_eigvals(const TrdRun &run, void *rho, int n, double **w) {
    return run.prec == OSMPS_FP64 ? trd_eigvals_t<double>(run, rho, n, w) : trd_eigvals_t<float>(run, rho, n, w);
}

}  // namespace osmps
