// Two-site gates on the state: the Trotter propagators of nearest-neighbour
// chains (Sec. III.C, Eqs. trotter1, trotter2, trotter4/4c) and general layers
// of two-site gates (quantum cellular automata and gates, App. C).
//
// A layer of gates on disjoint bonds is a tensor product, so its gates can be
// applied in any order.  The host cuts a layer into windows of kW = 4
// consecutive bits, each holding the gates whose two bits lie inside it; one
// streaming pass per window: every thread keeps the 16 amplitudes that differ
// only in the window bits in registers (consecutive threads take consecutive
// values of the bits below the window, so every load and store is
// coalesced), applies the window's 4 x 4 gates there and writes them back.
//
// Bits and sites: site s (1-based) is bit L - s, so the bond (s, s+1) acts on
// bits (L-s, L-s-1); a gate's matrix is taken in the basis index
// 2 sigma_s + sigma_{s+1} = 2 bit_hi + bit_lo.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "ed_internal.h"

namespace osmps {
namespace gates {

constexpr int kW = 4;                 // window bits
constexpr int kWA = 1 << kW;          // amplitudes per thread
constexpr int kMaxWinGates = kW - 1;  // gates on disjoint bonds inside a window: at most 2 (3 slots)
constexpr int kGateThreads = 256;

template <typename T> struct Cg;
template <> struct Cg<float> { typedef float2 C; };
template <> struct Cg<double> { typedef double2 C; };

template <typename T>
struct GateWin {
    int k;                        // lowest bit of the window
    int ngate;
    int q[kMaxWinGates];          // gate g acts on bits k + q[g] (lo) and k + q[g] + 1 (hi)
    T u[kMaxWinGates][32];        // 4 x 4 complex, row-major, (re, im) interleaved
};

// y = U x on the four amplitudes of one pair of window bits (Q, Q+1)
template <typename T, int Q>
__device__ __forceinline__ void apply_pair(typename Cg<T>::C (&a)[kWA], const T *u) {
    typedef typename Cg<T>::C C;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        // spread the two other window bits of r around positions Q, Q+1
        const int lowmask = (1 << Q) - 1;
        const int j0 = (r & lowmask) | ((r & ~lowmask) << 2);
        C x[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) x[c] = a[j0 | ((c >> 1) << (Q + 1)) | ((c & 1) << Q)];
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            T yr = (T)0, yi = (T)0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const T ur = u[(rr * 4 + c) * 2], ui = u[(rr * 4 + c) * 2 + 1];
                yr = fma(ur, x[c].x, fma(-ui, x[c].y, yr));
                yi = fma(ur, x[c].y, fma(ui, x[c].x, yi));
            }
            C y;
            y.x = yr;
            y.y = yi;
            a[j0 | ((rr >> 1) << (Q + 1)) | ((rr & 1) << Q)] = y;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kGateThreads) gate_window_kernel(typename Cg<T>::C *psi, uint64_t D,
                                                                    const GateWin<T> g) {
    typedef typename Cg<T>::C C;
    const uint64_t nb = D >> kW;
    const uint64_t lomask = (1ull << g.k) - 1ull;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nb; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t base = ((t & ~lomask) << kW) | (t & lomask);
        C a[kWA];
#pragma unroll
        for (int j = 0; j < kWA; ++j) a[j] = psi[base + ((uint64_t)j << g.k)];
        for (int gi = 0; gi < g.ngate; ++gi) {
            const T *u = g.u[gi];
            if (g.q[gi] == 0)
                apply_pair<T, 0>(a, u);
            else if (g.q[gi] == 1)
                apply_pair<T, 1>(a, u);
            else
                apply_pair<T, 2>(a, u);
        }
#pragma unroll
        for (int j = 0; j < kWA; ++j) psi[base + ((uint64_t)j << g.k)] = a[j];
    }
}

// ---------------------------------------------------------------------------
// Host side

// One layer of gates on disjoint bit pairs: gate i acts on bits (lo[i] + 1,
// lo[i]) with the 4 x 4 complex matrix U[32 i ..] (row-major, re/im).
template <typename T>
static cudaError_t launch_layer_t(Handle *h, void *psi, int ng, const int *lo, const double *U) {
    std::vector<int> idx(ng);
    for (int i = 0; i < ng; ++i) idx[i] = i;
    for (int i = 1; i < ng; ++i)  // sort by the low bit (few gates: insertion sort)
        for (int j = i; j > 0 && lo[idx[j - 1]] > lo[idx[j]]; --j) std::swap(idx[j - 1], idx[j]);
    const int L = h->L;
    const int grid = h->nsm * 8;
    int i = 0;
    while (i < ng) {
        GateWin<T> w{};
        const int b = lo[idx[i]];
        w.k = b < L - kW ? b : L - kW;
        w.ngate = 0;
        while (i < ng && w.ngate < kMaxWinGates && lo[idx[i]] >= w.k && lo[idx[i]] + 1 < w.k + kW) {
            w.q[w.ngate] = lo[idx[i]] - w.k;
            for (int e = 0; e < 32; ++e) w.u[w.ngate][e] = (T)U[32 * idx[i] + e];
            ++w.ngate;
            ++i;
        }
        gate_window_kernel<T><<<grid, kGateThreads, 0, h->stream>>>(static_cast<typename Cg<T>::C *>(psi), h->D, w);
        h->launches++;
        const cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

// Eigen-decomposition of a real symmetric 4 x 4 matrix by cyclic Jacobi
// rotations (a -> diagonal, v accumulates the rotations: a0 = v diag vᵀ).
static void jacobi4(double a[4][4], double v[4][4]) {
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) v[i][j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 4; ++q) off += a[p][q] * a[p][q];
        if (off < 1e-60) break;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 4; ++q) {
                if (a[p][q] == 0.0) continue;
                // rotation angle that zeroes a[p][q]
                const double theta = 0.5 * std::atan2(2.0 * a[p][q], a[q][q] - a[p][p]);
                const double c = std::cos(theta), sn = std::sin(theta);
                for (int k = 0; k < 4; ++k) {  // columns p, q
                    const double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - sn * akq;
                    a[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 4; ++k) {  // rows p, q
                    const double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - sn * aqk;
                    a[q][k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < 4; ++k) {
                    const double vkp = v[k][p], vkq = v[k][q];
                    v[k][p] = c * vkp - sn * vkq;
                    v[k][q] = sn * vkp + c * vkq;
                }
            }
    }
}

// U = exp(-i tau h_bond), h_bond = jzz sz(x)sz + fhi sx(x)1 + flo 1(x)sx in the
// basis 2 sigma_hi + sigma_lo (sz = +1 for bit 0), row-major (re, im).
static void bond_propagator(double jzz, double fhi, double flo, double tau, double *U) {
    double a[4][4] = {{0}};
    for (int r = 0; r < 4; ++r) {
        const int shi = (r >> 1) ? -1 : 1, slo = (r & 1) ? -1 : 1;
        a[r][r] = jzz * shi * slo;
        a[r][r ^ 2] += fhi;  // flip of the high (left) site
        a[r][r ^ 1] += flo;  // flip of the low (right) site
    }
    double v[4][4];
    jacobi4(a, v);
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double re = 0.0, im = 0.0;
            for (int k = 0; k < 4; ++k) {
                const double ph = -tau * a[k][k];
                re += v[r][k] * v[c][k] * std::cos(ph);
                im += v[r][k] * v[c][k] * std::sin(ph);
            }
            U[(r * 4 + c) * 2] = re;
            U[(r * 4 + c) * 2 + 1] = im;
        }
}

cudaError_t launch_gate_layer(Handle *h, void *psi, int ng, const int *lo, const double *U) {
    return h->prec == OSMPS_FP64 ? launch_layer_t<double>(h, psi, ng, lo, U) : launch_layer_t<float>(h, psi, ng, lo, U);
}

// exp(-i tau H_p) psi for the bonds (s, s+1) with s of parity p (1: odd bonds,
// H_o; 0: even bonds, H_e).  Site fields are split with weight 1/2 between the
// two bonds of a site; the first and last site keep weight 1 (open chain).
cudaError_t trotter_layer(Handle *h, void *psi, int parity, double tau) {
    const int L = h->L;
    std::vector<int> lo;
    std::vector<double> U;
    for (int s = 1; s + 1 <= L; ++s) {
        if ((s & 1) != parity) continue;
        const double hs = h->hbit[L - s], hs1 = h->hbit[L - s - 1];
        const double ws = (s == 1) ? 1.0 : 0.5, ws1 = (s + 1 == L) ? 1.0 : 0.5;
        double u[32];
        bond_propagator(h->Jr[1], ws * hs, ws1 * hs1, tau, u);
        lo.push_back(L - s - 1);
        U.insert(U.end(), u, u + 32);
    }
    if (lo.empty()) return cudaSuccess;
    return launch_gate_layer(h, psi, (int)lo.size(), lo.data(), U.data());
}

}  // namespace gates
}  // namespace osmps
