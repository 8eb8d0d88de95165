// Streaming vector kernels and the small FP64 tridiagonal problem of the
// Lanczos / Krylov recurrences (Sec. III.D; statics Sec. II).
//
// Stored Krylov vectors are unnormalised: v_j = scale[j] * u_j.  The scalars
// of the recurrence (alpha_j, beta_j, scale_j, the combination coefficients)
// live in a device control block and are produced by single-CTA "control"
// kernels that reduce the per-CTA partial sums of the streaming kernels in a
// fixed order, so that a whole Krylov step runs without a host round trip and
// reruns are bit-identical.
#include <cuda_runtime.h>
#include <math.h>

#include "ed_internal.h"
#include "device_common.cuh"

namespace osmps {

template <typename T> struct VecT;
template <> struct VecT<float> {
    typedef float4 v;
    static constexpr int VE = 2;
};
template <> struct VecT<double> {
    typedef double2 v;
    static constexpr int VE = 1;
};

// complex lanes of a 16-byte vector
__device__ __forceinline__ int nlanes(float4) { return 2; }
__device__ __forceinline__ float re(const float4 &v, int e) { return e ? v.z : v.x; }
__device__ __forceinline__ float im(const float4 &v, int e) { return e ? v.w : v.y; }
__device__ __forceinline__ double re(const double2 &v, int) { return v.x; }
__device__ __forceinline__ double im(const double2 &v, int) { return v.y; }
__device__ __forceinline__ void setc(float4 &v, int e, float a, float b) {
    if (e) {
        v.z = a;
        v.w = b;
    } else {
        v.x = a;
        v.y = b;
    }
}
__device__ __forceinline__ void setc(double2 &v, int, double a, double b) {
    v.x = a;
    v.y = b;
}

template <int K>
__device__ __forceinline__ void block_reduce(double (&v)[K], double *dst) {
    __shared__ double red[K][kVecThreads / 32];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red[k][w] = v[k];
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[threadIdx.x][i];
        dst[threadIdx.x] = s;
    }
    __syncthreads();
}


// ---------------------------------------------------------------------------
// elementary streaming kernels
// ---------------------------------------------------------------------------
template <typename T>
__global__ void fill_basis_kernel(typename VecT<T>::v *x, uint64_t nvec, uint64_t b) {
    typedef typename VecT<T>::v V;
    constexpr int VE = VecT<T>::VE;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nvec;
         q += (uint64_t)gridDim.x * blockDim.x) {
        V v;
        for (int e = 0; e < VE; ++e) setc(v, e, (q * VE + e == b) ? (T)1 : (T)0, (T)0);
        x[q] = v;
    }
}

// partial |x|^2 per CTA
template <typename T>
__global__ void __launch_bounds__(kVecThreads) norm2_kernel(const typename VecT<T>::v *x, uint64_t nvec,
                                                            double *partials) {
    typedef typename VecT<T>::v V;
    constexpr int VE = VecT<T>::VE;
    double acc[1] = {0.0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q0 < nvec; q0 += 4 * stride) {
        T s = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint64_t q = q0 + r * stride;
            if (q < nvec) {
                const V v = x[q];
#pragma unroll
                for (int e = 0; e < VE; ++e) s = fma(re(v, e), re(v, e), fma(im(v, e), im(v, e), s));
            }
        }
        acc[0] += (double)s;
    }
    block_reduce<1>(acc, partials + 4 * (size_t)blockIdx.x);
}

// partial <a, b> = sum conj(a_i) b_i (re, im) per CTA
template <typename T>
__global__ void __launch_bounds__(kVecThreads) cdot_kernel(const typename VecT<T>::v *a, const typename VecT<T>::v *b,
                                                           uint64_t nvec, double *partials) {
    typedef typename VecT<T>::v V;
    constexpr int VE = VecT<T>::VE;
    double acc[2] = {0.0, 0.0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q0 < nvec; q0 += 4 * stride) {
        T sr = 0, si = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint64_t q = q0 + r * stride;
            if (q < nvec) {
                const V x = a[q], y = b[q];
#pragma unroll
                for (int e = 0; e < VE; ++e) {
                    sr = fma(re(x, e), re(y, e), fma(im(x, e), im(y, e), sr));
                    si = fma(re(x, e), im(y, e), fma(-im(x, e), re(y, e), si));
                }
            }
        }
        acc[0] += (double)sr;
        acc[1] += (double)si;
    }
    block_reduce<2>(acc, partials + 4 * (size_t)blockIdx.x);
}

__global__ void cdot_finish_kernel(const double *partials, int nparts, double *out) {
    const double r = warp_sum_partials(partials, nparts, 4, 0);
    const double i = warp_sum_partials(partials, nparts, 4, 1);
    if (threadIdx.x == 0) {
        out[0] = r;
        out[1] = i;
    }
}

// u_{j+1} = w - alpha_j scale_j u_j (in place on w) and partial |u_{j+1}|^2.
// With hp != null, alpha_j is first summed here from the product's partials
// (the same fixed order as the control kernel it replaces, in every CTA; CTA 0
// stores it).
template <typename T>
__global__ void __launch_bounds__(kVecThreads) update_kernel(typename VecT<T>::v *w, const typename VecT<T>::v *u,
                                                             uint64_t nvec, KrylovCtl *ctl, int j,
                                                             const double *hp, int hnp, double *partials) {
    typedef typename VecT<T>::v V;
    constexpr int VE = VecT<T>::VE;
    if (ctl->m_eff <= j) return;
    __shared__ double alpha_s;
    if (hp != nullptr) {
        if (threadIdx.x < 32) {
            const double d = warp_sum_partials(hp, hnp, 4, 0);
            if (threadIdx.x == 0) {
                alpha_s = d;
                if (blockIdx.x == 0) ctl->alpha[j] = d;
            }
        }
        __syncthreads();
    }
    const double alpha = hp != nullptr ? alpha_s : ctl->alpha[j];
    const T a = (T)(alpha * ctl->scale[j]);
    double acc[1] = {0.0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q0 < nvec; q0 += 4 * stride) {
        T s = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint64_t q = q0 + r * stride;
            if (q < nvec) {
                V x = w[q];
                const V y = __ldcs(&u[q]);
#pragma unroll
                for (int e = 0; e < VE; ++e) {
                    const T xr = fma(-a, re(y, e), re(x, e));
                    const T xi = fma(-a, im(y, e), im(x, e));
                    setc(x, e, xr, xi);
                    s = fma(xr, xr, fma(xi, xi, s));
                }
                w[q] = x;
            }
        }
        acc[0] += (double)s;
    }
    block_reduce<1>(acc, partials + 4 * (size_t)blockIdx.x);
}

// partial <u_i, w> for i < nv (complex), 2*nv doubles per CTA
template <typename T>
__global__ void __launch_bounds__(kVecThreads) multidot_kernel(void *const *V_dev, int nv,
                                                               const typename VecT<T>::v *w, uint64_t nvec,
                                                               const KrylovCtl *ctl, int j, double *partials) {
    typedef typename VecT<T>::v V;
    constexpr int VE = VecT<T>::VE;
    if (ctl->m_eff <= j) return;
    __shared__ double red[2][kVecThreads / 32];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (int i = 0; i < nv; ++i) {
        const V *ui = reinterpret_cast<const V *>(V_dev[i]);
        double dr = 0.0, di = 0.0;
        for (uint64_t q0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q0 < nvec; q0 += 4 * stride) {
            T sr = 0, si = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint64_t q = q0 + r * stride;
                if (q < nvec) {
                    const V a = ui[q];
                    const V b = w[q];
#pragma unroll
                    for (int e = 0; e < VE; ++e) {
                        sr = fma(re(a, e), re(b, e), fma(im(a, e), im(b, e), sr));
                        si = fma(re(a, e), im(b, e), fma(-im(a, e), re(b, e), si));
                    }
                }
            }
            dr += (double)sr;
            di += (double)si;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            dr += __shfl_xor_sync(0xffffffffu, dr, off);
            di += __shfl_xor_sync(0xffffffffu, di, off);
        }
        const int wp = threadIdx.x >> 5, l = threadIdx.x & 31;
        if (l == 0) {
            red[0][wp] = dr;
            red[1][wp] = di;
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            double s = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[threadIdx.x][k];
            partials[(size_t)blockIdx.x * 2 * nv + 2 * i + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// w -= sum_i c_i scale_i u_i with c_i = scale_i * sum(partials); partial |w|^2
template <typename T>
__global__ void __launch_bounds__(kVecThreads) reorth_update_kernel(void *const *V_dev, int nv,
                                                                    typename VecT<T>::v *w, uint64_t nvec,
                                                                    const KrylovCtl *ctl, int j,
                                                                    const double *dots, int ndparts,
                                                                    double *partials) {
    typedef typename VecT<T>::v V;
    constexpr int VE = VecT<T>::VE;
    if (ctl->m_eff <= j) return;
    __shared__ T cr[1024], ci[1024];
    if (threadIdx.x < 32) {
        for (int i = 0; i < nv; ++i) {
            const double sr = warp_sum_partials(dots, ndparts, 2 * nv, 2 * i);
            const double si = warp_sum_partials(dots, ndparts, 2 * nv, 2 * i + 1);
            const double s2 = ctl->scale[i] * ctl->scale[i];
            if (threadIdx.x == 0) {
                cr[i] = (T)(sr * s2);
                ci[i] = (T)(si * s2);
            }
        }
    }
    __syncthreads();
    double acc[1] = {0.0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nvec; q += stride) {
        V x = w[q];
        T xr[VE], xi[VE];
#pragma unroll
        for (int e = 0; e < VE; ++e) {
            xr[e] = re(x, e);
            xi[e] = im(x, e);
        }
        for (int i = 0; i < nv; ++i) {
            const V a = reinterpret_cast<const V *>(V_dev[i])[q];
#pragma unroll
            for (int e = 0; e < VE; ++e) {
                xr[e] -= cr[i] * re(a, e) - ci[i] * im(a, e);
                xi[e] -= cr[i] * im(a, e) + ci[i] * re(a, e);
            }
        }
        T s = 0;
#pragma unroll
        for (int e = 0; e < VE; ++e) {
            setc(x, e, xr[e], xi[e]);
            s = fma(xr[e], xr[e], fma(xi[e], xi[e], s));
        }
        w[q] = x;
        acc[0] += (double)s;
    }
    block_reduce<1>(acc, partials + 4 * (size_t)blockIdx.x);
}

// out = sum_i coef_i u_i (coefficients include the vector scales); partial |out|^2
template <typename T>
__global__ void __launch_bounds__(kVecThreads) combine_kernel(void *const *V_dev, int nmax,
                                                              typename VecT<T>::v *out, uint64_t nvec,
                                                              const KrylovCtl *ctl, double *partials) {
    typedef typename VecT<T>::v V;
    constexpr int VE = VecT<T>::VE;
    __shared__ T cr[kMaxLanczos > 1024 ? 1024 : kMaxLanczos], ci[kMaxLanczos > 1024 ? 1024 : kMaxLanczos];
    __shared__ const V *ptr[kMaxLanczos > 1024 ? 1024 : kMaxLanczos];
    const int nv = ctl->m_eff < nmax ? ctl->m_eff : nmax;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        cr[i] = (T)ctl->coef_re[i];
        ci[i] = (T)ctl->coef_im[i];
        ptr[i] = reinterpret_cast<const V *>(V_dev[i]);
    }
    __syncthreads();
    double acc[1] = {0.0};
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nvec; q += stride) {
        T xr[VE], xi[VE];
#pragma unroll
        for (int e = 0; e < VE; ++e) xr[e] = xi[e] = (T)0;
        for (int i = 0; i < nv; ++i) {
            const V a = __ldcs(&ptr[i][q]);
#pragma unroll
            for (int e = 0; e < VE; ++e) {
                xr[e] = fma(cr[i], re(a, e), fma(-ci[i], im(a, e), xr[e]));
                xi[e] = fma(cr[i], im(a, e), fma(ci[i], re(a, e), xi[e]));
            }
        }
        V x;
        T s = 0;
#pragma unroll
        for (int e = 0; e < VE; ++e) {
            setc(x, e, xr[e], xi[e]);
            s = fma(xr[e], xr[e], fma(xi[e], xi[e], s));
        }
        out[q] = x;
        acc[0] += (double)s;
    }
    block_reduce<1>(acc, partials + 4 * (size_t)blockIdx.x);
}

template <typename T>
__global__ void scale_kernel(typename VecT<T>::v *x, uint64_t nvec, const double *s_dev) {
    typedef typename VecT<T>::v V;
    constexpr int VE = VecT<T>::VE;
    const T s = (T)(*s_dev);
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nvec;
         q += (uint64_t)gridDim.x * blockDim.x) {
        V v = x[q];
#pragma unroll
        for (int e = 0; e < VE; ++e) setc(v, e, re(v, e) * s, im(v, e) * s);
        x[q] = v;
    }
}

// ---------------------------------------------------------------------------
// control kernels (one warp)
// ---------------------------------------------------------------------------

// start of a step: ||psi|| from partials; v_0 = psi / ||psi||
__global__ void ctl_after_norm_kernel(KrylovCtl *ctl, const double *partials, int nparts, int m) {
    const double n2 = warp_sum_partials(partials, nparts, 4, 0);
    if (threadIdx.x == 0) {
        const double n = sqrt(n2);
        ctl->nrm = n;
        ctl->m_eff = (n > 0.0) ? m : 0;
        ctl->scale[0] = (n > 0.0) ? 1.0 / n : 0.0;
        ctl->beta[0] = 0.0;
        ctl->err = 0.0;
        ctl->epi[0] = ctl->scale[0];
        ctl->epi[1] = 0.0;
        ctl->epi[2] = 0.0;
    }
}

// alpha_j = <v_j, w> after the fused H.psi epilogue
__global__ void ctl_after_hpsi_kernel(KrylovCtl *ctl, const double *partials, int nparts, int j) {
    if (ctl->m_eff <= j) return;
    const double d = warp_sum_partials(partials, nparts, 4, 0);
    if (threadIdx.x == 0) ctl->alpha[j] = d;
}

// beta_{j+1} = ||u_{j+1}||; breakdown test; epilogue scalars of the next H.psi
__global__ void ctl_after_update_kernel(KrylovCtl *ctl, const double *partials, int nparts, int j) {
    if (ctl->m_eff <= j) return;
    const double n2 = warp_sum_partials(partials, nparts, 4, 0);
    if (threadIdx.x == 0) {
        const double b = sqrt(n2);
        ctl->beta[j + 1] = b;
        const double ref = fabs(ctl->alpha[j]) + ctl->beta[j];
        if (!(b > ctl->bd_tol * ref) || !(b > 0.0)) {
            ctl->m_eff = j + 1;  // invariant subspace: the basis ends with v_j
            ctl->scale[j + 1] = 0.0;
        } else {
            ctl->scale[j + 1] = 1.0 / b;
            ctl->epi[0] = 1.0 / b;
            ctl->epi[1] = 0.0;
            ctl->epi[2] = b * ctl->scale[j];
        }
    }
}

// Symmetric tridiagonal eigendecomposition by the implicit QL method with
// Wilkinson-type shifts (Golub & Van Loan, Sec. 8.3; Bowdler, Martin, Reinsch
// & Wilkinson 1968).  d: diagonal (in) / eigenvalues (out); e: off-diagonal,
// e[i] couples i and i+1.  Every lane of the warp runs the same scalar
// recurrence; each lane applies the plane rotations to its own rows of Z
// (row-major n x ldz in shared memory), or Z may be null.  Returns 0 on success.
__device__ int tridiag_ql(double *d, double *e, int n, double *Z, int ldz) {
    const int lane = threadIdx.x & 31;
    if (n <= 1) return 0;
    e[n - 1] = 0.0;
    for (int l = 0; l < n; ++l) {
        int iter = 0;
        while (true) {
            int mm = l;
            for (; mm < n - 1; ++mm) {
                const double dd = fabs(d[mm]) + fabs(d[mm + 1]);
                if (fabs(e[mm]) <= 1e-17 * dd) break;
            }
            if (mm == l) break;
            if (++iter > 90) return 1;
            // shift from the trailing 2x2 block at l
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = hypot(g, 1.0);
            g = d[mm] - d[l] + e[l] / (g + copysign(r, g));
            double s = 1.0, c = 1.0, p = 0.0;
            int i = mm - 1;
            bool deflated = false;
            for (; i >= l; --i) {
                const double f = s * e[i];
                const double b = c * e[i];
                r = hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= p;
                    e[mm] = 0.0;
                    deflated = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
                if (Z != nullptr) {
                    for (int k = lane; k < n; k += 32) {
                        const double zi1 = Z[k * ldz + i + 1];
                        const double zi = Z[k * ldz + i];
                        Z[k * ldz + i + 1] = s * zi + c * zi1;
                        Z[k * ldz + i] = c * zi - s * zi1;
                    }
                    __syncwarp();
                }
            }
            if (deflated) continue;
            d[l] -= p;
            e[l] = g;
            e[mm] = 0.0;
        }
    }
    return 0;
}

// xi = ||psi|| exp(-i dt T) e_1 in the Krylov basis (T real symmetric
// tridiagonal, n <= 64), by the exponential's Taylor series on the vector with
// scaling: exp(-i dt T) e_1 = (exp(-i dt T / s))^s e_1, s chosen so that
// ||dt T / s||_1 <= 1/2, 20 terms per factor (remainder < 2^-21 / 21! ~ 1e-26
// relative); Moler & Van Loan, "Nineteen dubious ways", methods 1 and 3.  One
// warp; lane i owns entries i and i + 32.  The coefficients are scaled by the
// stored-vector scales; Saad's a-posteriori estimate beta_n |xi_{n-1}| is kept.
__global__ void tridiag_exp_kernel(KrylovCtl *ctl, double dt) {
    __shared__ double a[kMaxKrylov], b[kMaxKrylov + 1];      // diag, b[i] couples i-1 and i
    __shared__ double xr[kMaxKrylov], xi[kMaxKrylov];         // running vector
    __shared__ double tr[kMaxKrylov], ti[kMaxKrylov];         // current Taylor term
    __shared__ int s_steps;
    const int lane = threadIdx.x;
    const int n = ctl->m_eff;
    if (n <= 0) {
        if (lane == 0) ctl->err = 0.0;
        return;
    }
    for (int i = lane; i < n; i += 32) {
        a[i] = ctl->alpha[i];
        b[i] = (i > 0) ? ctl->beta[i] : 0.0;
        xr[i] = (i == 0) ? 1.0 : 0.0;
        xi[i] = 0.0;
    }
    if (lane == 0) b[n] = 0.0;
    __syncwarp();
    if (lane == 0) {
        double nrm1 = 0.0;
        for (int i = 0; i < n; ++i) nrm1 = fmax(nrm1, fabs(a[i]) + fabs(b[i]) + fabs(b[i + 1]));
        const double z = fabs(dt) * nrm1;
        int s = (int)ceil(z / 0.5);
        s_steps = s < 1 ? 1 : s;
    }
    __syncwarp();
    const int s = s_steps;
    const double c = dt / (double)s;
    for (int rep = 0; rep < s; ++rep) {
        for (int i = lane; i < n; i += 32) {
            tr[i] = xr[i];
            ti[i] = xi[i];
        }
        __syncwarp();
        for (int k = 1; k <= 20; ++k) {
            // term <- (-i c T term) / k
            double nr[2], ni[2];
            for (int q = 0; q < 2; ++q) {
                const int i = lane + 32 * q;
                if (i < n) {
                    double yr = a[i] * tr[i], yi = a[i] * ti[i];
                    if (i > 0) {
                        yr = fma(b[i], tr[i - 1], yr);
                        yi = fma(b[i], ti[i - 1], yi);
                    }
                    if (i + 1 < n) {
                        yr = fma(b[i + 1], tr[i + 1], yr);
                        yi = fma(b[i + 1], ti[i + 1], yi);
                    }
                    const double f = c / (double)k;
                    nr[q] = f * yi;   // -i (yr + i yi) = yi - i yr
                    ni[q] = -f * yr;
                }
            }
            __syncwarp();
            for (int q = 0; q < 2; ++q) {
                const int i = lane + 32 * q;
                if (i < n) {
                    tr[i] = nr[q];
                    ti[i] = ni[q];
                    xr[i] += nr[q];
                    xi[i] += ni[q];
                }
            }
            __syncwarp();
        }
    }
    const double nrm = ctl->nrm;
    for (int i = lane; i < n; i += 32) {
        const double r = xr[i] * nrm, im = xi[i] * nrm;
        ctl->coef_re[i] = r * ctl->scale[i];
        ctl->coef_im[i] = im * ctl->scale[i];
        if (i == n - 1) {
            const double err = ctl->beta[n] * sqrt(r * r + im * im);
            ctl->err = err;
            ctl->err_sum += err;
        }
    }
}

// Lowest Ritz pair of T_n: theta and the last component of its eigenvector
// (convergence estimate beta_{n} |y_{n-1}|); with want_vec the eigenvector is
// obtained by inverse iteration and stored as combination coefficients.
__device__ void inverse_iteration(const double *a, const double *b, int n, double theta, double *y,
                                  double *work) {
    // solve (T - theta I) y = rhs three times by Gaussian elimination with
    // partial pivoting on the tridiagonal matrix (LU gets two super-diagonals)
    double *dd = work, *du = work + n, *du2 = work + 2 * n, *dl = work + 3 * n;
    double scale = 0.0;
    for (int i = 0; i < n; ++i) scale = fmax(scale, fabs(a[i]) + (i + 1 < n ? fabs(b[i + 1]) : 0.0));
    const double pert = 1e-15 * (scale > 0 ? scale : 1.0);
    for (int i = 0; i < n; ++i) y[i] = 1.0 + 0.01 * (double)((i * 7919) % 13);
    for (int sweep = 0; sweep < 3; ++sweep) {
        for (int i = 0; i < n; ++i) {
            dd[i] = a[i] - theta;
            du[i] = (i + 1 < n) ? b[i + 1] : 0.0;
            du2[i] = 0.0;
            dl[i] = (i + 1 < n) ? b[i + 1] : 0.0;
        }
        for (int i = 0; i < n - 1; ++i) {
            if (fabs(dd[i]) >= fabs(dl[i])) {
                if (dd[i] == 0.0) dd[i] = pert;
                const double f = dl[i] / dd[i];
                dd[i + 1] -= f * du[i];
                y[i + 1] -= f * y[i];
            } else {
                // swap rows i and i+1, then eliminate
                const double f = dd[i] / dl[i];
                const double old_dd1 = dd[i + 1];
                const double old_du1 = (i + 2 < n) ? du[i + 1] : 0.0;
                dd[i] = dl[i];
                dd[i + 1] = du[i] - f * old_dd1;
                du[i] = old_dd1;
                du2[i] = old_du1;
                if (i + 2 < n) du[i + 1] = -f * old_du1;
                const double yi = y[i];
                y[i] = y[i + 1];
                y[i + 1] = yi - f * y[i];
            }
        }
        if (dd[n - 1] == 0.0) dd[n - 1] = pert;
        y[n - 1] /= dd[n - 1];
        if (n > 1) y[n - 2] = (y[n - 2] - du[n - 2] * y[n - 1]) / dd[n - 2];
        for (int i = n - 3; i >= 0; --i) y[i] = (y[i] - du[i] * y[i + 1] - du2[i] * y[i + 2]) / dd[i];
        double nrm = 0.0;
        for (int i = 0; i < n; ++i) nrm += y[i] * y[i];
        nrm = sqrt(nrm);
        for (int i = 0; i < n; ++i) y[i] /= nrm;
    }
}

__global__ void tridiag_ground_kernel(KrylovCtl *ctl, int n_req, int want_vec) {
    // n = number of Lanczos vectors so far
    const int n = ctl->m_eff < n_req ? ctl->m_eff : n_req;
    if (threadIdx.x != 0 || n <= 0) return;
    double *d = ctl->work, *e = ctl->work + n, *y = ctl->work + 2 * n, *w = ctl->work + 3 * n;
    for (int i = 0; i < n; ++i) {
        d[i] = ctl->alpha[i];
        e[i] = (i + 1 < n) ? ctl->beta[i + 1] : 0.0;
    }
    if (tridiag_ql(d, e, n, nullptr, 0) != 0) {
        ctl->theta = nan("");
        return;
    }
    double theta = d[0];
    for (int i = 1; i < n; ++i) theta = fmin(theta, d[i]);
    inverse_iteration(ctl->alpha, ctl->beta, n, theta, y, w);
    // Rayleigh quotient of y refines theta
    double rq = 0.0;
    for (int i = 0; i < n; ++i) {
        double ty = ctl->alpha[i] * y[i];
        if (i > 0) ty += ctl->beta[i] * y[i - 1];
        if (i + 1 < n) ty += ctl->beta[i + 1] * y[i + 1];
        rq += y[i] * ty;
    }
    ctl->theta = rq;
    ctl->est = ctl->beta[n] * fabs(y[n - 1]);
    if (want_vec) {
        for (int i = 0; i < n; ++i) {
            ctl->coef_re[i] = y[i] * ctl->scale[i];
            ctl->coef_im[i] = 0.0;
        }
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
int vec_grid(Handle *h) {
    const uint64_t nvec = h->D * h->esize / 16;
    const uint64_t want = (nvec + kVecThreads - 1) / kVecThreads;
    const uint64_t cap = (uint64_t)h->nsm * 4;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

static uint64_t nvec_of(Handle *h) { return h->D * h->esize / 16; }

#define DISPATCH(h, KERNEL, GRID, BLOCK, ...)                                                     \
    do {                                                                                           \
        if ((h)->prec == OSMPS_FP64)                                                               \
            KERNEL<double><<<(GRID), (BLOCK), 0, (h)->stream>>>(__VA_ARGS__);                     \
        else                                                                                       \
            KERNEL<float><<<(GRID), (BLOCK), 0, (h)->stream>>>(__VA_ARGS__);                      \
    } while (0)

cudaError_t launch_fill_basis(Handle *h, void *psi, uint64_t b) {
    const int g = vec_grid(h);
    if (h->prec == OSMPS_FP64)
        fill_basis_kernel<double><<<g, kVecThreads, 0, h->stream>>>((double2 *)psi, nvec_of(h), b);
    else
        fill_basis_kernel<float><<<g, kVecThreads, 0, h->stream>>>((float4 *)psi, nvec_of(h), b);
    h->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_norm2(Handle *h, const void *x, double *partials, int *nparts) {
    const int g = vec_grid(h);
    if (h->prec == OSMPS_FP64)
        norm2_kernel<double><<<g, kVecThreads, 0, h->stream>>>((const double2 *)x, nvec_of(h), partials);
    else
        norm2_kernel<float><<<g, kVecThreads, 0, h->stream>>>((const float4 *)x, nvec_of(h), partials);
    *nparts = g;
    h->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_cdot(Handle *h, const void *a, const void *b, double *out_dev) {
    const int g = vec_grid(h);
    if (h->prec == OSMPS_FP64)
        cdot_kernel<double><<<g, kVecThreads, 0, h->stream>>>((const double2 *)a, (const double2 *)b, nvec_of(h),
                                                               h->partials2);
    else
        cdot_kernel<float><<<g, kVecThreads, 0, h->stream>>>((const float4 *)a, (const float4 *)b, nvec_of(h),
                                                             h->partials2);
    cdot_finish_kernel<<<1, 32, 0, h->stream>>>(h->partials2, g, out_dev);
    h->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_ctl_after_norm(Handle *h, KrylovCtl *ctl, const double *partials, int nparts, int m) {
    ctl_after_norm_kernel<<<1, 32, 0, h->stream>>>(ctl, partials, nparts, m);
    h->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_ctl_after_hpsi(Handle *h, KrylovCtl *ctl, const double *partials, int nparts, int j) {
    ctl_after_hpsi_kernel<<<1, 32, 0, h->stream>>>(ctl, partials, nparts, j);
    h->launches += 1;
    return cudaGetLastError();
}

static cudaError_t launch_update_any(Handle *h, void *w, const void *u, KrylovCtl *ctl, int j, const double *hp,
                                     int hnp, double *partials, int *nparts) {
    const int g = vec_grid(h);
    if (h->prec == OSMPS_FP64)
        update_kernel<double><<<g, kVecThreads, 0, h->stream>>>((double2 *)w, (const double2 *)u, nvec_of(h), ctl,
                                                                 j, hp, hnp, partials);
    else
        update_kernel<float><<<g, kVecThreads, 0, h->stream>>>((float4 *)w, (const float4 *)u, nvec_of(h), ctl, j,
                                                                hp, hnp, partials);
    *nparts = g;
    h->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_update(Handle *h, void *w, const void *u, KrylovCtl *ctl, int j, double *partials,
                          int *nparts) {
    return launch_update_any(h, w, u, ctl, j, nullptr, 0, partials, nparts);
}

cudaError_t launch_update_folded(Handle *h, void *w, const void *u, KrylovCtl *ctl, int j, const double *hp,
                                 int hnp, double *partials, int *nparts) {
    return launch_update_any(h, w, u, ctl, j, hp, hnp, partials, nparts);
}

cudaError_t launch_ctl_after_update(Handle *h, KrylovCtl *ctl, const double *partials, int nparts, int j, int) {
    ctl_after_update_kernel<<<1, 32, 0, h->stream>>>(ctl, partials, nparts, j);
    h->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_multidot(Handle *h, void *const *V_dev, int nvec, const void *w, KrylovCtl *ctl, int j,
                            double *partials, int *nparts) {
    const int g = vec_grid(h);
    if (h->prec == OSMPS_FP64)
        multidot_kernel<double><<<g, kVecThreads, 0, h->stream>>>(V_dev, nvec, (const double2 *)w, nvec_of(h), ctl,
                                                                   j, partials);
    else
        multidot_kernel<float><<<g, kVecThreads, 0, h->stream>>>(V_dev, nvec, (const float4 *)w, nvec_of(h), ctl, j,
                                                                  partials);
    *nparts = g;
    h->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_reorth_update(Handle *h, void *const *V_dev, int nvec, void *w, KrylovCtl *ctl, int j,
                                 const double *dots, int ndparts, double *partials, int *nparts) {
    const int g = vec_grid(h);
    if (h->prec == OSMPS_FP64)
        reorth_update_kernel<double><<<g, kVecThreads, 0, h->stream>>>(V_dev, nvec, (double2 *)w, nvec_of(h), ctl, j,
                                                                        dots, ndparts, partials);
    else
        reorth_update_kernel<float><<<g, kVecThreads, 0, h->stream>>>(V_dev, nvec, (float4 *)w, nvec_of(h), ctl, j,
                                                                       dots, ndparts, partials);
    *nparts = g;
    h->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_tridiag_exp(Handle *h, KrylovCtl *ctl, int, double dt) {
    tridiag_exp_kernel<<<1, 32, 0, h->stream>>>(ctl, dt);
    h->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_tridiag_ground(Handle *h, KrylovCtl *ctl, int m) {
    tridiag_ground_kernel<<<1, 32, 0, h->stream>>>(ctl, m, 1);
    h->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_combine(Handle *h, void *const *V_dev, int nmax, void *out, KrylovCtl *ctl, double *partials,
                           int *nparts) {
    const int g = vec_grid(h);
    if (h->prec == OSMPS_FP64)
        combine_kernel<double><<<g, kVecThreads, 0, h->stream>>>(V_dev, nmax, (double2 *)out, nvec_of(h), ctl,
                                                                  partials);
    else
        combine_kernel<float><<<g, kVecThreads, 0, h->stream>>>(V_dev, nmax, (float4 *)out, nvec_of(h), ctl,
                                                                 partials);
    *nparts = g;
    h->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_scale(Handle *h, void *x, const double *s_dev) {
    const int g = vec_grid(h);
    if (h->prec == OSMPS_FP64)
        scale_kernel<double><<<g, kVecThreads, 0, h->stream>>>((double2 *)x, nvec_of(h), s_dev);
    else
        scale_kernel<float><<<g, kVecThreads, 0, h->stream>>>((float4 *)x, nvec_of(h), s_dev);
    h->launches += 1;
    return cudaGetLastError();
}

}  // namespace osmps
