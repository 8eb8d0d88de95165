// C ABI of libosmps_ed (include/osmps_ed.h): argument checks, workspace
// management and the host-side drivers of the Lanczos and Krylov loops.  The
// drivers only enqueue kernels; every vector operation and every scalar of the
// recurrences is computed on the device (see vec_kernels.cu), and the host
// reads back a few scalars where the ABI returns them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstring>
#include <algorithm>
#include <condition_variable>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "device_common.cuh"
#include "ed_internal.h"

using namespace osmps;

namespace {

// Asynchronous bond entropy: the Gram product rho = psi_A psi_A^dag runs on the
// caller's stream (psi may be overwritten as soon as it is enqueued); the
// Hermitian eigen-solve and the entropy sum run on a lowest-priority
// non-blocking stream of one of two result slots.  With the library solver
// each slot has its own solver handle, stream and worker thread (the solver
// blocks its host thread), so two measurements can be in flight at once; with
// this library's solver the calling thread enqueues everything itself.
struct AsyncJob {
    int slot;
    int n;
    double *S_host;
    double *lambda_host;
};

struct AsyncMeas {
    std::thread worker[2];
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    bool busy[2] = {false, false};    // slot holds a measurement not yet finished
    bool queued[2] = {false, false};  // library mode: slot's job waits for its worker
    AsyncJob job[2] = {};             // the job a slot holds
    int next_slot = 0;
    osmps_status err = OSMPS_OK;      // first failure of a job, returned by the wait
    int64_t launches = 0;             // kernels launched by the workers
    cudaStream_t ss[2] = {nullptr, nullptr};  // per-slot streams (lowest priority, non-blocking)
    cudaEvent_t ready[2] = {nullptr, nullptr};
    cudaEvent_t done[2] = {nullptr, nullptr};
    void *rho[2] = {nullptr, nullptr};
    size_t rho_bytes[2] = {0, 0};
    double *lam[2] = {nullptr, nullptr};   // lambda (n) and S on the device
    size_t lam_bytes[2] = {0, 0};
    double *host[2] = {nullptr, nullptr};  // pinned staging of lambda and S
    size_t host_bytes[2] = {0, 0};
    void *sh[2] = {nullptr, nullptr};      // library mode: per-slot solver handles
    void *ws[2] = {nullptr, nullptr};      // library mode: per-slot solver workspaces
    size_t ws_bytes[2] = {0, 0};
    // own eigen-solver (osmps_ed_set_async_eigensolver > 0)
    int own_G = 0;                           // CTAs of the cooperative reduction; 0 = library solver
    void *tws[2] = {nullptr, nullptr};
    size_t tws_bytes[2] = {0, 0};
    int *err_dev = nullptr;                  // 2 ints: bounded waits of the reduction gave up
    int *err_host = nullptr;                 // pinned copies
};

}  // namespace

struct osmps_ed {
    Handle h;
    bool reorth_set;
    AsyncMeas *am;
};

namespace osmps {

void *dev_alloc(Handle *h, size_t bytes, cudaError_t *err) {
    void *p = nullptr;
    *err = cudaMalloc(&p, bytes);
    if (*err != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    h->owned_bytes += bytes;
    return p;
}

void dev_free(Handle *h, void *p, size_t bytes) {
    if (p != nullptr) {
        cudaFree(p);
        h->owned_bytes -= bytes;
    }
}

}  // namespace osmps

namespace {

osmps_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return OSMPS_OK;
    if (e == cudaErrorMemoryAllocation) return OSMPS_ENOMEM;
    return OSMPS_ECUDA;
}

#define CK(expr)                                  \
    do {                                          \
        cudaError_t _e = (expr);                  \
        if (_e != cudaSuccess) return from_cuda(_e); \
    } while (0)

#define CKS(expr)                                 \
    do {                                          \
        osmps_status _s = (expr);                 \
        if (_s != OSMPS_OK) return _s;            \
    } while (0)

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

size_t vec_bytes(const Handle *h) { return (size_t)h->D * h->esize; }

osmps_status ensure_vec(Handle *h, void **p) {
    if (*p != nullptr) return OSMPS_OK;
    cudaError_t err;
    *p = dev_alloc(h, vec_bytes(h), &err);
    return from_cuda(err);
}

// V[0] is the caller's state; V[1..nv] are owned Krylov vectors.
osmps_status ensure_basis(Handle *h, int nv) {
    if (nv <= h->Vcap) return OSMPS_OK;
    void **nV = new (std::nothrow) void *[nv + 1];
    if (nV == nullptr) return OSMPS_ENOMEM;
    for (int i = 0; i <= nv; ++i) nV[i] = nullptr;
    for (int i = 1; i <= h->Vcap; ++i) nV[i] = h->V[i];
    for (int i = h->Vcap + 1; i <= nv; ++i) {
        cudaError_t err;
        nV[i] = dev_alloc(h, vec_bytes(h), &err);
        if (err != cudaSuccess) {
            for (int k = h->Vcap + 1; k < i; ++k) dev_free(h, nV[k], vec_bytes(h));
            delete[] nV;
            return from_cuda(err);
        }
    }
    delete[] h->V;
    h->V = nV;
    if (h->V_dev != nullptr) dev_free(h, h->V_dev, sizeof(void *) * (h->Vcap + 1));
    h->V_dev = nullptr;
    h->Vcap = nv;
    cudaError_t err;
    h->V_dev = (void **)dev_alloc(h, sizeof(void *) * (nv + 1), &err);
    return from_cuda(err);
}

osmps_status upload_basis_table(Handle *h, void *psi, int nv) {
    h->V[0] = psi;
    CK(cudaMemcpyAsync(h->V_dev, h->V, sizeof(void *) * (nv + 1), cudaMemcpyHostToDevice, h->stream));
    return OSMPS_OK;
}

osmps_status read_scalars(Handle *h, size_t off, size_t bytes) {
    CK(cudaMemcpyAsync(reinterpret_cast<char *>(h->ctl_host) + off, reinterpret_cast<char *>(h->ctl) + off, bytes,
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return OSMPS_OK;
}

#define CTL_OFF(f) offsetof(KrylovCtl, f)

// Synchronise and report (then clear) a bounded device wait that gave up.
osmps_status sync_and_check(Handle *h) {
    CK(cudaStreamSynchronize(h->stream));
    int e = 0;
    CK(cudaMemcpy(&e, &h->ctl->error, sizeof(int), cudaMemcpyDeviceToHost));
    if (e != 0) {
        CK(cudaMemset(&h->ctl->error, 0, sizeof(int)));
        return OSMPS_ETIMEOUT;
    }
    return OSMPS_OK;
}

// One thread waits, with the bounded wait of the H.psi and Gram kernels, for
// the first phase of an mbarrier that nothing arrives at (complete = 0), or
// that it completed itself (complete = 1); raises the error word when the
// wait gives up.
__global__ void probe_wait_kernel(KrylovCtl *ctl, unsigned long long limit_ns, int complete) {
    __shared__ unsigned long long bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (complete) mbar_arrive(&bar);
    if (!mbar_wait_ns(&bar, 0u, &ctl->error, limit_ns)) atomicExch(&ctl->error, 1);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
}

__global__ void ctl_init_kernel(KrylovCtl *ctl, double bd_tol) {
    ctl->bd_tol = bd_tol;
    ctl->err_sum = 0.0;
    ctl->err = 0.0;
}

// x = sum y_i v_i was written with partial |x|^2; prepare the residual pass
// r = H x - theta x on the normalised x
__global__ void ctl_prepare_residual_kernel(KrylovCtl *ctl, const double *partials, int nparts) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 32) s += partials[4 * (size_t)i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) {
        const double n = sqrt(s);
        ctl->work[0] = (n > 0.0) ? 1.0 / n : 0.0;  // scale applied to x
        ctl->epi2[0] = 1.0;
        ctl->epi2[1] = ctl->theta;
        ctl->epi2[2] = 0.0;
    }
}

// residual pass reduced: work[1] = ||H x - theta x||, work[2] = <x, H x> = theta + <x, r>
__global__ void ctl_finish_residual_kernel(KrylovCtl *ctl, const double *partials, int nparts) {
    double d = 0.0, n2 = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 32) {
        d += partials[4 * (size_t)i];
        n2 += partials[4 * (size_t)i + 2];
    }
    for (int off = 16; off > 0; off >>= 1) {
        d += __shfl_xor_sync(0xffffffffu, d, off);
        n2 += __shfl_xor_sync(0xffffffffu, n2, off);
    }
    if (threadIdx.x == 0) {
        ctl->work[1] = sqrt(n2);
        ctl->work[2] = ctl->theta + d;
    }
}

// energy pass reduced: work[3] = <u, H u>, work[4] = <u, u>
__global__ void ctl_finish_energy_kernel(KrylovCtl *ctl, const double *partials, int nparts) {
    double d = 0.0, n2 = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 32) {
        d += partials[4 * (size_t)i];
        n2 += partials[4 * (size_t)i + 2];
    }
    for (int off = 16; off > 0; off >>= 1) {
        d += __shfl_xor_sync(0xffffffffu, d, off);
        n2 += __shfl_xor_sync(0xffffffffu, n2, off);
    }
    if (threadIdx.x == 0) {
        ctl->work[3] = d;
        ctl->work[4] = n2;
    }
}

// One Lanczos iteration j: w = H v_j - beta_j v_{j-1} (fused), alpha_j,
// u_{j+1} = w - alpha_j v_j, optional Gram-Schmidt against v_0..v_j, beta_{j+1}.
// Folded (allow_fold, no Gram-Schmidt pass, handle setting on): alpha_j is
// summed inside the update and beta_{j+1} inside the next product's first pass,
// so a step is three launches; lanczos_finish stores the last beta.  Every
// scalar is the same fixed-order sum as in the unfolded sequence.
osmps_status lanczos_iteration(Handle *h, int j, int reorth, bool allow_fold) {
    int np = 0;
    const bool fold = allow_fold && !reorth && h->fold_ctl;
    HpsiArgs a{};
    a.u = h->V[j];
    a.uprev = j > 0 ? h->V[j - 1] : nullptr;
    a.out = h->V[j + 1];
    a.tmp = h->tmp;
    a.epi = h->ctl->epi;
    a.partials = h->partials;
    a.m_eff = &h->ctl->m_eff;
    a.stop_index = j;
    a.epilogue = EPI_KRYLOV;
    if (fold && j > 0) {
        a.fold_ctl = h->ctl;
        a.fold_parts = h->partials_upd;
        a.fold_nparts = vec_grid(h);
    }
    CK(launch_hpsi_timed(h, a, &np));
    if (fold) {
        int nu = 0;
        CK(launch_update_folded(h, h->V[j + 1], h->V[j], h->ctl, j, h->partials, np, h->partials_upd, &nu));
        return OSMPS_OK;
    }
    CK(launch_ctl_after_hpsi(h, h->ctl, h->partials, np, j));
    CK(launch_update(h, h->V[j + 1], h->V[j], h->ctl, j, h->partials, &np));
    if (reorth) {
        int nd = 0;
        CK(launch_multidot(h, h->V_dev, j + 1, h->V[j + 1], h->ctl, j, h->partials2, &nd));
        CK(launch_reorth_update(h, h->V_dev, j + 1, h->V[j + 1], h->ctl, j, h->partials2, nd, h->partials, &np));
    }
    CK(launch_ctl_after_update(h, h->ctl, h->partials, np, j, 0));
    return OSMPS_OK;
}

// After m folded iterations: beta_m, its breakdown test and scale_m (the step
// that a next product's first pass would otherwise have done).
osmps_status lanczos_finish(Handle *h, int m, int reorth) {
    if (reorth || !h->fold_ctl) return OSMPS_OK;
    CK(launch_ctl_after_update(h, h->ctl, h->partials_upd, vec_grid(h), m - 1, 0));
    return OSMPS_OK;
}

// Krylov basis of v0 under the handle's current H (m three-term Lanczos steps;
// the basis and T stay in the handle until the next basis is built).
osmps_status krylov_basis(Handle *h, void *v0, int m) {
    CKS(ensure_basis(h, m));
    CKS(upload_basis_table(h, v0, m));
    ctl_init_kernel<<<1, 1, 0, h->stream>>>(h->ctl, 1e-12);
    h->launches += 1;
    CK(cudaGetLastError());
    int np = 0;
    CK(launch_norm2(h, v0, h->partials, &np));
    CK(launch_ctl_after_norm(h, h->ctl, h->partials, np, m));
    for (int j = 0; j < m; ++j) CKS(lanczos_iteration(h, j, h->reorth, true));
    CKS(lanczos_finish(h, m, h->reorth));
    return OSMPS_OK;
}

// out = |v0| V exp(-i tau T) e_1 from the current basis (any real tau; the
// basis is left untouched, so several tau can follow one basis).
osmps_status krylov_combine(Handle *h, int m, double tau, void *out) {
    int np = 0;
    CK(launch_tridiag_exp(h, h->ctl, m, tau));
    CK(launch_combine(h, h->V_dev, m, out, h->ctl, h->partials, &np));
    return OSMPS_OK;
}

// Gauss-Legendre nodes x and weights w on [0, 1]: Newton's method on the
// Legendre polynomial P_q (three-term recurrence), mapped from [-1, 1].
void gauss_legendre01(int q, double *x, double *w) {
    for (int i = 0; i < q; ++i) {
        double z = std::cos(3.14159265358979323846 * (i + 0.75) / (q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;  // P_0, P_1
            for (int j = 2; j <= q; ++j) {
                const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (q == 1) {
                p1 = z;
                p0 = 1.0;
            }
            dp = q * (z * p1 - p0) / (z * z - 1.0);  // P_q'(z)
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = 0.5 * (1.0 + z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  // 2 / ((1 - z^2) P'^2), times 1/2 for [0, 1]
    }
}

osmps_status check_state_ptr(const Handle *h, const void *p) {
    (void)h;
    if (p == nullptr || !aligned16(p)) return OSMPS_EINVAL;
    return OSMPS_OK;
}

osmps_status timing_flush(Handle *h) {
    if (h->tev_used == 0) return OSMPS_OK;
    CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i < h->tev_used; ++i) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, h->tev[2 * i], h->tev[2 * i + 1]));
        h->t_ms += ms;
    }
    h->t_calls += h->tev_used;
    h->tev_used = 0;
    return OSMPS_OK;
}

void destroy_handle(Handle *h) {
    cudaStreamSynchronize(h->stream);
    if (h->tev) {
        for (int i = 0; i < 2 * h->tev_cap; ++i) cudaEventDestroy(h->tev[i]);
        delete[] h->tev;
    }
    dev_free(h, h->Ell, 0);
    dev_free(h, h->Fhh, 0);
    dev_free(h, h->Tab, 0);
    dev_free(h, h->partials, 0);
    dev_free(h, h->partials_upd, 0);
    dev_free(h, h->partials2, 0);
    dev_free(h, h->dscratch, 0);
    dev_free(h, h->ctl, 0);
    if (h->ctl_host) cudaFreeHost(h->ctl_host);
    dev_free(h, h->tmp, 0);
    dev_free(h, h->xbuf, 0);
    if (h->V) {
        for (int i = 1; i <= h->Vcap; ++i) dev_free(h, h->V[i], 0);
        delete[] h->V;
    }
    dev_free(h, h->V_dev, 0);
    dev_free(h, h->gram, 0);
    dev_free(h, h->gram_aux, 0);
    dev_free(h, h->solver_ws, 0);
    dev_free(h, h->sub_ws, h->sub_ws_bytes);
    dev_free(h, h->lam_dev, 0);
}

// Library mode: the worker of slot sl solves the slot's queued job.
void async_worker(Handle *h, AsyncMeas *am, int sl) {
    cudaSetDevice(h->device);
    std::unique_lock<std::mutex> lock(am->mu);
    for (;;) {
        am->cv.wait(lock, [am, sl] { return am->stop || am->queued[sl]; });
        if (!am->queued[sl]) return;  // stop requested and nothing left
        am->queued[sl] = false;
        const AsyncJob job = am->job[sl];
        const int n = job.n;
        void *ws = am->ws[sl];
        size_t ws_bytes = am->ws_bytes[sl];
        int64_t launches = 0;
        cudaStream_t st = am->ss[sl];
        lock.unlock();
        osmps_status rs = from_cuda(cudaStreamWaitEvent(st, am->ready[sl], 0));
        if (rs == OSMPS_OK && am->sh[sl] == nullptr) {
            am->sh[sl] = solver_handle_new();
            if (am->sh[sl] == nullptr) rs = OSMPS_EUNSUPPORTED;
        }
        if (rs == OSMPS_OK)
            rs = schmidt_eig_on(h, st, am->sh[sl], &ws, &ws_bytes, false, &launches, am->rho[sl], n, am->lam[sl],
                                am->lam[sl] + n);
        if (rs == OSMPS_OK)
            rs = from_cuda(cudaMemcpyAsync(am->host[sl], am->lam[sl], sizeof(double) * (n + 1),
                                           cudaMemcpyDeviceToHost, st));
        if (rs == OSMPS_OK) rs = from_cuda(cudaStreamSynchronize(st));
        if (rs == OSMPS_OK) {
            if (job.lambda_host) std::memcpy(job.lambda_host, am->host[sl], sizeof(double) * n);
            if (job.S_host) *job.S_host = am->host[sl][n];
        }
        lock.lock();
        am->ws[sl] = ws;
        am->ws_bytes[sl] = ws_bytes;
        am->launches += launches;
        if (rs != OSMPS_OK && am->err == OSMPS_OK) am->err = rs;
        am->busy[sl] = false;
        am->cv.notify_all();
    }
}

// Stops the workers after their queued jobs and frees the slot resources.
void destroy_async(AsyncMeas *am) {
    if (am == nullptr) return;
    {
        std::lock_guard<std::mutex> lock(am->mu);
        am->stop = true;
    }
    am->cv.notify_all();
    for (int i = 0; i < 2; ++i)
        if (am->worker[i].joinable()) am->worker[i].join();
    for (int i = 0; i < 2; ++i) {
        if (am->ss[i]) cudaStreamSynchronize(am->ss[i]);
        if (am->ready[i]) cudaEventDestroy(am->ready[i]);
        if (am->done[i]) cudaEventDestroy(am->done[i]);
        if (am->rho[i]) cudaFree(am->rho[i]);
        if (am->lam[i]) cudaFree(am->lam[i]);
        if (am->host[i]) cudaFreeHost(am->host[i]);
        if (am->ws[i]) cudaFree(am->ws[i]);
        if (am->tws[i]) cudaFree(am->tws[i]);
        solver_handle_free(am->sh[i]);
        if (am->ss[i]) cudaStreamDestroy(am->ss[i]);
    }
    if (am->err_dev) cudaFree(am->err_dev);
    if (am->err_host) cudaFreeHost(am->err_host);
    delete am;
}

// Error words of the own-solver mode (created once).
osmps_status ensure_own_mode(AsyncMeas *am) {
    if (am->err_dev != nullptr) return OSMPS_OK;
    cudaError_t e = cudaMallocHost((void **)&am->err_host, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&am->err_dev, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(am->err_dev, 0, 2 * sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (am->err_dev) cudaFree(am->err_dev);
        am->err_dev = nullptr;
        return from_cuda(e);
    }
    am->err_host[0] = am->err_host[1] = 0;
    return OSMPS_OK;
}

// Own-solver mode: waits for slot sl's measurement and writes its results.
osmps_status finish_own_slot(AsyncMeas *am, int sl) {
    if (!am->busy[sl]) return OSMPS_OK;
    osmps_status st = from_cuda(cudaEventSynchronize(am->done[sl]));
    if (st == OSMPS_OK && am->err_host[sl] != 0) st = OSMPS_ETIMEOUT;
    if (st == OSMPS_OK) {
        const AsyncJob &j = am->job[sl];
        if (j.lambda_host) std::memcpy(j.lambda_host, am->host[sl], sizeof(double) * j.n);
        if (j.S_host) *j.S_host = am->host[sl][j.n];
    }
    std::lock_guard<std::mutex> lock(am->mu);
    am->busy[sl] = false;
    if (st != OSMPS_OK && am->err == OSMPS_OK) am->err = st;
    return st;
}

osmps_status create_async(Handle *h, AsyncMeas **out) {
    AsyncMeas *am = new (std::nothrow) AsyncMeas();
    if (am == nullptr) return OSMPS_ENOMEM;
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithPriority(&am->ss[i], cudaStreamNonBlocking, least);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&am->ready[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&am->done[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        destroy_async(am);
        return from_cuda(e);
    }
    try {
        for (int i = 0; i < 2; ++i) am->worker[i] = std::thread(async_worker, h, am, i);
    } catch (...) {
        destroy_async(am);
        return OSMPS_ENOMEM;
    }
    *out = am;
    return OSMPS_OK;
}

// Device (or pinned host) buffer of at least `bytes`, not counted in the handle's bytes.
osmps_status grow_untracked(void **p, size_t *cap, size_t bytes, bool pinned_host) {
    if (bytes <= *cap) return OSMPS_OK;
    if (*p) {
        if (pinned_host)
            cudaFreeHost(*p);
        else
            cudaFree(*p);
    }
    *p = nullptr;
    *cap = 0;
    const cudaError_t e = pinned_host ? cudaMallocHost(p, bytes) : cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return from_cuda(e);
    }
    *cap = bytes;
    return OSMPS_OK;
}

osmps_status entropy_async_own(Handle *h, AsyncMeas *am, const void *psi, int cut, int n, double *S,
                               double *lambda) {
    const int sl = am->next_slot;
    CKS(finish_own_slot(am, sl));  // the slot's previous measurement (host wait)
    const int G = trd_ctas(n, h->prec, am->own_G, h->device);
    if (G == 0) return OSMPS_EUNSUPPORTED;
    CKS(grow_untracked(&am->rho[sl], &am->rho_bytes[sl], (size_t)n * n * h->esize, false));
    CKS(grow_untracked((void **)&am->lam[sl], &am->lam_bytes[sl], sizeof(double) * (n + 1), false));
    CKS(grow_untracked((void **)&am->host[sl], &am->host_bytes[sl], sizeof(double) * (n + 1), true));
    CKS(grow_untracked(&am->tws[sl], &am->tws_bytes[sl], trd_workspace_bytes(n, h->prec, G), false));
    int nn = 0;
    {
        const cudaError_t ge = launch_gram(h, psi, cut, am->rho[sl], &nn);
        if (ge == cudaErrorNotSupported) {
            cudaGetLastError();
            return OSMPS_EUNSUPPORTED;
        }
        CK(ge);
    }
    cudaStream_t st = am->ss[sl];
    CK(cudaEventRecord(am->ready[sl], h->stream));
    CK(cudaStreamWaitEvent(st, am->ready[sl], 0));
    CK(cudaMemsetAsync(am->err_dev + sl, 0, sizeof(int), st));
    TrdRun run{h->prec, h->device, st, G, am->tws[sl], am->tws_bytes[sl], am->err_dev + sl, &h->launches};
    double *w = nullptr;
    {
        const cudaError_t te = trd_eigvals(run, am->rho[sl], nn, &w);
        if (te == cudaErrorNotSupported) {
            cudaGetLastError();
            return OSMPS_EUNSUPPORTED;
        }
        CK(te);
    }
    CK(launch_entropy(st, w, nn, am->lam[sl], am->lam[sl] + nn));
    h->launches += 1;
    CK(cudaMemcpyAsync(am->host[sl], am->lam[sl], sizeof(double) * (nn + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(am->err_host + sl, am->err_dev + sl, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(am->done[sl], st));
    {
        std::lock_guard<std::mutex> lock(am->mu);
        am->busy[sl] = true;
        am->job[sl] = AsyncJob{sl, nn, S, lambda};
        am->next_slot = sl ^ 1;
    }
    return OSMPS_OK;
}

}  // namespace

namespace osmps {

cudaError_t launch_hpsi_timed(Handle *h, const HpsiArgs &a, int *nparts_out) {
    if (!h->timing) return launch_hpsi(h, a, nparts_out);
    if (h->tev_used == h->tev_cap) {
        // flush recorded pairs when the pool is full, then reuse it
        if (h->tev_cap >= 4096) {
            if (timing_flush(h) != OSMPS_OK) return cudaErrorUnknown;
        } else {
            const int ncap = h->tev_cap ? 2 * h->tev_cap : 256;
            cudaEvent_t *nev = new (std::nothrow) cudaEvent_t[2 * ncap];
            if (nev == nullptr) return cudaErrorMemoryAllocation;
            for (int i = 0; i < 2 * h->tev_cap; ++i) nev[i] = h->tev[i];
            for (int i = 2 * h->tev_cap; i < 2 * ncap; ++i) {
                cudaError_t e = cudaEventCreate(&nev[i]);
                if (e != cudaSuccess) return e;
            }
            delete[] h->tev;
            h->tev = nev;
            h->tev_cap = ncap;
        }
    }
    const int i = h->tev_used++;
    cudaError_t e = cudaEventRecord(h->tev[2 * i], h->stream);
    if (e != cudaSuccess) return e;
    e = launch_hpsi(h, a, nparts_out);
    if (e != cudaSuccess) return e;
    return cudaEventRecord(h->tev[2 * i + 1], h->stream);
}

}  // namespace osmps

extern "C" {

osmps_status osmps_ed_launch_count(const osmps_ed_t *ed, int64_t *count) {
    if (ed == nullptr || count == nullptr) return OSMPS_EINVAL;
    *count = ed->h.launches;
    return OSMPS_OK;
}

osmps_status osmps_ed_probe_wait(osmps_ed_t *ed, double seconds, int complete) {
    if (ed == nullptr || !(seconds > 0.0) || seconds > 2.0 || (complete != 0 && complete != 1)) return OSMPS_EINVAL;
    Handle *h = &ed->h;
    probe_wait_kernel<<<1, 32, 0, h->stream>>>(h->ctl, (unsigned long long)(seconds * 1e9), complete);
    h->launches += 1;
    CK(cudaGetLastError());
    return OSMPS_OK;
}

osmps_status osmps_ed_timing_enable(osmps_ed_t *ed, int enable) {
    if (ed == nullptr) return OSMPS_EINVAL;
    ed->h.timing = enable ? 1 : 0;
    return OSMPS_OK;
}

osmps_status osmps_ed_timing_read(osmps_ed_t *ed, double *hpsi_ms, int64_t *hpsi_calls, int reset) {
    if (ed == nullptr) return OSMPS_EINVAL;
    CKS(timing_flush(&ed->h));
    CKS(sync_and_check(&ed->h));
    if (hpsi_ms) *hpsi_ms = ed->h.t_ms;
    if (hpsi_calls) *hpsi_calls = ed->h.t_calls;
    if (reset) {
        ed->h.t_ms = 0.0;
        ed->h.t_calls = 0;
    }
    return OSMPS_OK;
}

const char *osmps_ed_strerror(osmps_status s) {
    switch (s) {
        case OSMPS_OK: return "success";
        case OSMPS_EINVAL: return "invalid argument";
        case OSMPS_ENOMEM: return "out of memory";
        case OSMPS_ECUDA: return "CUDA error";
        case OSMPS_ENOCONV: return "no convergence within max_iter";
        case OSMPS_ETIMEOUT: return "bounded device wait timed out";
        case OSMPS_EUNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

osmps_status osmps_ed_create(int L, const double *couplings, double J, double alpha, double h, int prec,
                             void *cuda_stream, osmps_ed_t **out) {
    if (out == nullptr) return OSMPS_EINVAL;
    *out = nullptr;
    if (L < 1 || L > OSMPS_MAX_L) return OSMPS_EINVAL;
    if (prec != OSMPS_FP64 && prec != OSMPS_MIXED) return OSMPS_EINVAL;
    if (!std::isfinite(h)) return OSMPS_EINVAL;
    double Jr[kMaxL + 1] = {0};
    if (couplings != nullptr) {
        for (int r = 1; r < L; ++r) {
            if (!std::isfinite(couplings[r - 1])) return OSMPS_EINVAL;
            Jr[r] = couplings[r - 1];
        }
    } else {
        if (!std::isfinite(J) || std::isnan(alpha)) return OSMPS_EINVAL;
        const bool nn = (alpha < 0.0) || std::isinf(alpha);
        for (int r = 1; r < L; ++r) Jr[r] = nn ? (r == 1 ? J : 0.0) : J / std::pow((double)r, alpha);
    }
    osmps_ed_t *ed = new (std::nothrow) osmps_ed_t();
    if (ed == nullptr) return OSMPS_ENOMEM;
    std::memset(&ed->h, 0, sizeof(Handle));
    ed->reorth_set = false;
    Handle *hd = &ed->h;
    hd->L = L;
    hd->prec = prec;
    hd->D = 1ull << L;
    hd->esize = (prec == OSMPS_FP64) ? 16 : 8;
    hd->stream = (cudaStream_t)cuda_stream;
    for (int r = 0; r <= kMaxL; ++r) hd->Jr[r] = Jr[r];
    for (int b = 0; b < L; ++b) hd->hbit[b] = h;
    hd->reorth = 0;
    hd->entropy_method = ENT_AUTO;
    hd->flip_fixed = 1;
    hd->pass_threads = 512;
    hd->fold_ctl = 1;
    hd->prefetch = (prec == OSMPS_FP64) ? 0 : 1;  // FP64 passes are bound by the FP64 pipe, not by latency
    cudaError_t err = cudaGetDevice(&hd->device);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&hd->nsm, cudaDevAttrMultiProcessorCount, hd->device);
    if (err != cudaSuccess) {
        cudaGetLastError();
        delete ed;
        return from_cuda(err);
    }
    hd->plan = make_plan(L, prec);
    osmps_status st = OSMPS_OK;
    do {
        err = build_tables(hd);
        if (err != cudaSuccess) break;
        // per-CTA partials: 4 doubles per CTA for every streaming kernel; the
        // multi-dot of the Gram-Schmidt pass needs 2 per vector per CTA
        const size_t g = (size_t)hd->nsm * 8;
        // H.psi writes 4 doubles per consumer warp of each persistent CTA
        const size_t gh = (size_t)hd->nsm * 2 * hpsi_partials_per_cta();
        hd->partials_cap = (gh > g ? gh : g) * 4;
        hd->partials = (double *)dev_alloc(hd, sizeof(double) * hd->partials_cap, &err);
        if (err != cudaSuccess) break;
        hd->partials_upd = (double *)dev_alloc(hd, sizeof(double) * g * 4, &err);
        if (err != cudaSuccess) break;
        const size_t zneed = (g + 1) * ((size_t)(L * L + L + 1) + 4096);
        const size_t dneed = g * 2 * (kMaxLanczos + 1);
        hd->partials2_cap = zneed > dneed ? zneed : dneed;
        hd->partials2 = (double *)dev_alloc(hd, sizeof(double) * hd->partials2_cap, &err);
        if (err != cudaSuccess) break;
        hd->dscratch_cap = (size_t)L * L + L + 64;
        hd->dscratch = (double *)dev_alloc(hd, sizeof(double) * hd->dscratch_cap, &err);
        if (err != cudaSuccess) break;
        hd->ctl = (KrylovCtl *)dev_alloc(hd, sizeof(KrylovCtl), &err);
        if (err != cudaSuccess) break;
        err = cudaMallocHost(&hd->ctl_host, sizeof(KrylovCtl));
        if (err != cudaSuccess) break;
        err = cudaMemsetAsync(hd->ctl, 0, sizeof(KrylovCtl), hd->stream);
        if (err != cudaSuccess) break;
        if (hd->plan.npass > 1) {
            hd->tmp = dev_alloc(hd, vec_bytes(hd), &err);
            if (err != cudaSuccess) break;
        }
        err = cudaStreamSynchronize(hd->stream);
    } while (0);
    if (err != cudaSuccess) st = from_cuda(err);
    if (st != OSMPS_OK) {
        destroy_handle(hd);
        delete ed;
        return st;
    }
    *out = ed;
    return OSMPS_OK;
}

osmps_status osmps_ed_destroy(osmps_ed_t *ed) {
    if (ed == nullptr) return OSMPS_OK;
    destroy_async(ed->am);
    ed->am = nullptr;
    destroy_handle(&ed->h);
    delete ed;
    return OSMPS_OK;
}

osmps_status osmps_ed_set_stream(osmps_ed_t *ed, void *cuda_stream) {
    if (ed == nullptr) return OSMPS_EINVAL;
    ed->h.stream = (cudaStream_t)cuda_stream;
    return OSMPS_OK;
}

osmps_status osmps_ed_set_field(osmps_ed_t *ed, double h) {
    if (ed == nullptr || !std::isfinite(h)) return OSMPS_EINVAL;
    for (int b = 0; b < ed->h.L; ++b) ed->h.hbit[b] = h;
    return OSMPS_OK;
}

osmps_status osmps_ed_set_site_fields(osmps_ed_t *ed, const double *h_sites) {
    if (ed == nullptr || h_sites == nullptr) return OSMPS_EINVAL;
    const int L = ed->h.L;
    for (int k = 0; k < L; ++k)
        if (!std::isfinite(h_sites[k])) return OSMPS_EINVAL;
    for (int k = 1; k <= L; ++k) ed->h.hbit[L - k] = h_sites[k - 1];
    return OSMPS_OK;
}

osmps_status osmps_ed_set_reorth(osmps_ed_t *ed, int mode) {
    if (ed == nullptr || (mode != 0 && mode != 1)) return OSMPS_EINVAL;
    ed->h.reorth = mode;
    ed->reorth_set = true;
    return OSMPS_OK;
}

osmps_status osmps_ed_set_sm_count(osmps_ed_t *ed, int nsm) {
    if (ed == nullptr) return OSMPS_EINVAL;
    int dev_sm = 0;
    CK(cudaDeviceGetAttribute(&dev_sm, cudaDevAttrMultiProcessorCount, ed->h.device));
    if (nsm < 0 || nsm > dev_sm) return OSMPS_EINVAL;
    ed->h.nsm = nsm == 0 ? dev_sm : nsm;
    return OSMPS_OK;
}

osmps_status osmps_ed_set_entropy_method(osmps_ed_t *ed, int method) {
    if (ed == nullptr || method < ENT_GRAM || method > ENT_SUBSPACE) return OSMPS_EINVAL;
    ed->h.entropy_method = method;
    return OSMPS_OK;
}

osmps_status osmps_ed_set_flip_sums(osmps_ed_t *ed, int mode) {
    if (ed == nullptr || mode < 0 || mode > kMaxL) return OSMPS_EINVAL;
    ed->h.flip_fixed = mode;
    return OSMPS_OK;
}

osmps_status osmps_ed_set_lanczos_fold(osmps_ed_t *ed, int on) {
    if (ed == nullptr || (on != 0 && on != 1)) return OSMPS_EINVAL;
    ed->h.fold_ctl = on;
    return OSMPS_OK;
}

osmps_status osmps_ed_set_pass_threads(osmps_ed_t *ed, int threads) {
    if (ed == nullptr || (threads != 256 && threads != 512)) return OSMPS_EINVAL;
    ed->h.pass_threads = threads;
    return OSMPS_OK;
}

osmps_status osmps_ed_set_prefetch(osmps_ed_t *ed, int tiles) {
    if (ed == nullptr || tiles < 0 || tiles > 4) return OSMPS_EINVAL;
    ed->h.prefetch = tiles;
    return OSMPS_OK;
}

osmps_status osmps_ed_set_gram_mode(osmps_ed_t *ed, int mode) {
    if (ed == nullptr || mode < 0 || mode > 2) return OSMPS_EINVAL;
    ed->h.gram_mode = mode;
    return OSMPS_OK;
}

osmps_status osmps_ed_dim(const osmps_ed_t *ed, uint64_t *D) {
    if (ed == nullptr || D == nullptr) return OSMPS_EINVAL;
    *D = ed->h.D;
    return OSMPS_OK;
}

osmps_status osmps_ed_device_bytes(const osmps_ed_t *ed, uint64_t *bytes) {
    if (ed == nullptr || bytes == nullptr) return OSMPS_EINVAL;
    *bytes = ed->h.owned_bytes;
    return OSMPS_OK;
}

osmps_status osmps_ed_init_basis_state(osmps_ed_t *ed, void *psi, uint64_t b) {
    if (ed == nullptr) return OSMPS_EINVAL;
    CKS(check_state_ptr(&ed->h, psi));
    if (b >= ed->h.D) return OSMPS_EINVAL;
    CK(launch_fill_basis(&ed->h, psi, b));
    return OSMPS_OK;
}

osmps_status osmps_ed_upload(osmps_ed_t *ed, void *dst_device, const void *src_host) {
    if (ed == nullptr || src_host == nullptr) return OSMPS_EINVAL;
    CKS(check_state_ptr(&ed->h, dst_device));
    CK(cudaMemcpyAsync(dst_device, src_host, vec_bytes(&ed->h), cudaMemcpyHostToDevice, ed->h.stream));
    return OSMPS_OK;
}

osmps_status osmps_ed_download(osmps_ed_t *ed, void *dst_host, const void *src_device) {
    if (ed == nullptr || dst_host == nullptr) return OSMPS_EINVAL;
    CKS(check_state_ptr(&ed->h, src_device));
    CK(cudaMemcpyAsync(dst_host, src_device, vec_bytes(&ed->h), cudaMemcpyDeviceToHost, ed->h.stream));
    CK(cudaStreamSynchronize(ed->h.stream));
    return OSMPS_OK;
}

osmps_status osmps_ed_apply_H(osmps_ed_t *ed, const void *psi, void *out) {
    if (ed == nullptr) return OSMPS_EINVAL;
    Handle *h = &ed->h;
    CKS(check_state_ptr(h, psi));
    CKS(check_state_ptr(h, out));
    if (psi == out) return OSMPS_EINVAL;
    HpsiArgs a{};
    a.u = psi;
    a.out = out;
    a.tmp = h->tmp;
    a.epilogue = EPI_PLAIN;
    CK(launch_hpsi_timed(h, a, nullptr));
    return OSMPS_OK;
}

osmps_status osmps_ed_energy(osmps_ed_t *ed, const void *psi, double *e_num, double *norm2) {
    if (ed == nullptr) return OSMPS_EINVAL;
    Handle *h = &ed->h;
    CKS(check_state_ptr(h, psi));
    CKS(ensure_vec(h, &h->xbuf));
    int np = 0;
    HpsiArgs a{};
    a.u = psi;
    a.out = h->xbuf;
    a.tmp = h->tmp;
    a.partials = h->partials;
    a.epilogue = EPI_ENERGY;
    CK(launch_hpsi_timed(h, a, &np));
    ctl_finish_energy_kernel<<<1, 32, 0, h->stream>>>(h->ctl, h->partials, np);
    h->launches += 1;
    CK(cudaGetLastError());
    CKS(read_scalars(h, CTL_OFF(work) + 3 * sizeof(double), 2 * sizeof(double)));
    CKS(sync_and_check(h));
    if (e_num) *e_num = h->ctl_host->work[3];
    if (norm2) *norm2 = h->ctl_host->work[4];
    return OSMPS_OK;
}

osmps_status osmps_ed_krylov_evolve(osmps_ed_t *ed, void *psi, double dt, int nsteps, int m, double tol,
                                    double *err_estimate) {
    if (ed == nullptr) return OSMPS_EINVAL;
    Handle *h = &ed->h;
    CKS(check_state_ptr(h, psi));
    if (!std::isfinite(dt) || nsteps < 0 || m < 1 || m > kMaxKrylov || std::isnan(tol)) return OSMPS_EINVAL;
    if (nsteps == 0) {
        if (err_estimate) *err_estimate = 0.0;
        return OSMPS_OK;
    }
    CKS(ensure_basis(h, m));
    CKS(upload_basis_table(h, psi, m));
    ctl_init_kernel<<<1, 1, 0, h->stream>>>(h->ctl, tol > 0.0 ? tol : 1e-12);
    h->launches += 1;
    CK(cudaGetLastError());
    int np = 0;
    CK(launch_norm2(h, psi, h->partials, &np));
    CK(launch_ctl_after_norm(h, h->ctl, h->partials, np, m));
    for (int s = 0; s < nsteps; ++s) {
        for (int j = 0; j < m; ++j) CKS(lanczos_iteration(h, j, h->reorth, true));
        CKS(lanczos_finish(h, m, h->reorth));
        CK(launch_tridiag_exp(h, h->ctl, m, dt));
        CK(launch_combine(h, h->V_dev, m, psi, h->ctl, h->partials, &np));
        CK(launch_ctl_after_norm(h, h->ctl, h->partials, np, m));
    }
    CKS(read_scalars(h, CTL_OFF(err_sum), sizeof(double)));
    CKS(sync_and_check(h));
    if (err_estimate) *err_estimate = h->ctl_host->err_sum;
    return OSMPS_OK;
}

osmps_status osmps_ed_lanczos_ground(osmps_ed_t *ed, void *psi, double tol, int max_iter, double *energy,
                                     double *residual, int *iters) {
    if (ed == nullptr) return OSMPS_EINVAL;
    Handle *h = &ed->h;
    CKS(check_state_ptr(h, psi));
    if (!(tol > 0.0) || !std::isfinite(tol) || max_iter < 1 || max_iter > kMaxLanczos) return OSMPS_EINVAL;
    const int reorth = ed->reorth_set ? h->reorth : 1;
    CKS(ensure_basis(h, max_iter));
    CKS(ensure_vec(h, &h->xbuf));
    void *rbuf = h->V[max_iter];  // scratch for the residual vector (last slot)
    CKS(upload_basis_table(h, psi, max_iter));
    ctl_init_kernel<<<1, 1, 0, h->stream>>>(h->ctl, 1e-14);
    h->launches += 1;
    CK(cudaGetLastError());
    int np = 0;
    CK(launch_norm2(h, psi, h->partials, &np));
    CK(launch_ctl_after_norm(h, h->ctl, h->partials, np, max_iter));
    double best_res = INFINITY, best_e = NAN;
    int done_iters = 0;
    osmps_status result = OSMPS_ENOCONV;
    for (int j = 0; j < max_iter - 1; ++j) {
        CKS(lanczos_iteration(h, j, reorth, false));  // T is read after every step
        done_iters = j + 1;
        CK(launch_tridiag_ground(h, h->ctl, j + 1));
        CKS(read_scalars(h, CTL_OFF(theta), CTL_OFF(m_eff) + sizeof(int) - CTL_OFF(theta)));
        const bool breakdown = h->ctl_host->m_eff <= j + 1;
        const bool last = (j == max_iter - 2);
        if (!(h->ctl_host->est <= tol) && !breakdown && !last) continue;
        // Ritz vector x = sum y_i v_i (into xbuf), normalised; explicit residual
        CK(launch_combine(h, h->V_dev, j + 1, h->xbuf, h->ctl, h->partials, &np));
        ctl_prepare_residual_kernel<<<1, 32, 0, h->stream>>>(h->ctl, h->partials, np);
    h->launches += 1;
        CK(cudaGetLastError());
        CK(launch_scale(h, h->xbuf, &h->ctl->work[0]));
        HpsiArgs a{};
        a.u = h->xbuf;
        a.out = rbuf;
        a.tmp = h->tmp;
        a.epi = h->ctl->epi2;
        a.partials = h->partials;
        a.epilogue = EPI_KRYLOV;
        CK(launch_hpsi_timed(h, a, &np));
        ctl_finish_residual_kernel<<<1, 32, 0, h->stream>>>(h->ctl, h->partials, np);
    h->launches += 1;
        CK(cudaGetLastError());
        CKS(read_scalars(h, CTL_OFF(work), 3 * sizeof(double)));
        const double res = h->ctl_host->work[1];
        const double e = h->ctl_host->work[2];
        if (res < best_res) {
            best_res = res;
            best_e = e;
            CK(cudaMemcpyAsync(psi, h->xbuf, vec_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
        }
        if (res <= tol) {
            result = OSMPS_OK;
            break;
        }
        if (breakdown) break;
    }
    CKS(sync_and_check(h));
    if (energy) *energy = best_e;
    if (residual) *residual = best_res;
    if (iters) *iters = done_iters;
    return result;
}

osmps_status osmps_ed_measure_local(osmps_ed_t *ed, const void *psi, double *sz) {
    if (ed == nullptr || sz == nullptr) return OSMPS_EINVAL;
    Handle *h = &ed->h;
    CKS(check_state_ptr(h, psi));
    CK(launch_zstats(h, psi, h->dscratch));
    CK(cudaMemcpyAsync(sz, h->dscratch, sizeof(double) * h->L, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return OSMPS_OK;
}

osmps_status osmps_ed_measure_corr(osmps_ed_t *ed, const void *psi, double *szsz) {
    if (ed == nullptr || szsz == nullptr) return OSMPS_EINVAL;
    Handle *h = &ed->h;
    CKS(check_state_ptr(h, psi));
    CK(launch_zstats(h, psi, h->dscratch));
    CK(cudaMemcpyAsync(szsz, h->dscratch + h->L, sizeof(double) * h->L * h->L, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return OSMPS_OK;
}

osmps_status osmps_ed_measure_zz(osmps_ed_t *ed, const void *psi, double *sz, double *szsz) {
    if (ed == nullptr) return OSMPS_EINVAL;
    Handle *h = &ed->h;
    CKS(check_state_ptr(h, psi));
    CK(launch_zstats(h, psi, h->dscratch));
    if (sz) CK(cudaMemcpyAsync(sz, h->dscratch, sizeof(double) * h->L, cudaMemcpyDeviceToHost, h->stream));
    if (szsz)
        CK(cudaMemcpyAsync(szsz, h->dscratch + h->L, sizeof(double) * h->L * h->L, cudaMemcpyDeviceToHost,
                           h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return OSMPS_OK;
}

osmps_status osmps_ed_schmidt_entropy(osmps_ed_t *ed, const void *psi, int cut, double *lambda, double *S) {
    if (ed == nullptr) return OSMPS_EINVAL;
    Handle *h = &ed->h;
    CKS(check_state_ptr(h, psi));
    const int L = h->L;
    if (cut == -1) cut = L / 2;
    if (L < 2 || cut < 1 || cut > L - 1) return OSMPS_EINVAL;
    const int ls = cut < L - cut ? cut : L - cut;
    const int n = 1 << ls;
    const size_t gbytes = (size_t)n * n * h->esize;
    int method = h->entropy_method;
    if (method == ENT_AUTO) {
        if (subspace_applicable(h, cut))
            method = ENT_SUBSPACE;
        else if (h->prec == OSMPS_FP64)
            method = ENT_GRAM;
        else
            method = rayleigh_applicable(h, cut) ? ENT_RAYLEIGH : (n <= 8192 ? ENT_SVD : ENT_GRAM);
    }
    if (method == ENT_SUBSPACE && !subspace_applicable(h, cut)) return OSMPS_EUNSUPPORTED;
    if (method == ENT_SUBSPACE) {
        if ((size_t)n + 1 > h->lam_cap) {
            dev_free(h, h->lam_dev, h->lam_cap * sizeof(double));
            h->lam_dev = nullptr;
            h->lam_cap = 0;
            cudaError_t err;
            h->lam_dev = (double *)dev_alloc(h, sizeof(double) * (n + 1), &err);
            if (err != cudaSuccess) return from_cuda(err);
            h->lam_cap = n + 1;
        }
        const osmps_status rs = schmidt_subspace(h, psi, cut, h->lam_dev, h->lam_dev + n);
        if (rs == OSMPS_OK) {  // S was read back (and is finite) inside
            double Sv = 0.0;
            CK(cudaMemcpyAsync(&Sv, h->lam_dev + n, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            if (lambda) CK(cudaMemcpyAsync(lambda, h->lam_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            if (S) *S = Sv;
            return OSMPS_OK;
        }
        if (rs != OSMPS_ENOCONV && rs != OSMPS_EUNSUPPORTED) return rs;
        // the full route
        method = h->prec == OSMPS_FP64 ? ENT_GRAM : (rayleigh_applicable(h, cut) ? ENT_RAYLEIGH : ENT_SVD);
    }
    if (method == ENT_RAYLEIGH && !rayleigh_applicable(h, cut)) return OSMPS_EUNSUPPORTED;
    if (method == ENT_RAYLEIGH) {
        if (gbytes > h->gram_bytes) {
            dev_free(h, h->gram, h->gram_bytes);
            h->gram = nullptr;
            h->gram_bytes = 0;
            cudaError_t err;
            h->gram = dev_alloc(h, gbytes, &err);
            if (err != cudaSuccess) return from_cuda(err);
            h->gram_bytes = gbytes;
        }
        if ((size_t)n + 1 > h->lam_cap) {
            dev_free(h, h->lam_dev, h->lam_cap * sizeof(double));
            h->lam_dev = nullptr;
            h->lam_cap = 0;
            cudaError_t err;
            h->lam_dev = (double *)dev_alloc(h, sizeof(double) * (n + 1), &err);
            if (err != cudaSuccess) return from_cuda(err);
            h->lam_cap = n + 1;
        }
        const osmps_status rs = schmidt_rayleigh(h, psi, cut, h->gram, h->lam_dev, h->lam_dev + n);
        if (rs == OSMPS_ENOCONV) {
            method = ENT_SVD;  // the library eigen-solver failed: singular values of M instead
        } else if (rs != OSMPS_OK) {
            return rs;
        } else {
            double Sv = 0.0;
            CK(cudaMemcpyAsync(&Sv, h->lam_dev + n, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            if (std::isfinite(Sv)) {
                if (lambda) {
                    CK(cudaMemcpyAsync(lambda, h->lam_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
                    CK(cudaStreamSynchronize(h->stream));
                }
                if (S) *S = Sv;
                return OSMPS_OK;
            }
            method = ENT_SVD;  // non-finite eigenvectors from the library: singular values of M instead
        }
    }
    if (method == ENT_SVD) {
        // singular values of M: no Gram product
        if ((size_t)n + 1 > h->lam_cap) {
            dev_free(h, h->lam_dev, h->lam_cap * sizeof(double));
            h->lam_dev = nullptr;
            h->lam_cap = 0;
            cudaError_t err;
            h->lam_dev = (double *)dev_alloc(h, sizeof(double) * (n + 1), &err);
            if (err != cudaSuccess) return from_cuda(err);
            h->lam_cap = n + 1;
        }
        CKS(schmidt_svd(h, psi, cut, h->lam_dev, h->lam_dev + n));
        if (lambda) CK(cudaMemcpyAsync(lambda, h->lam_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
        double Sv = 0.0;
        CK(cudaMemcpyAsync(&Sv, h->lam_dev + n, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (S) *S = Sv;
        return OSMPS_OK;
    }
    if (gbytes > h->gram_bytes) {
        dev_free(h, h->gram, h->gram_bytes);
        h->gram = nullptr;
        h->gram_bytes = 0;
        cudaError_t err;
        h->gram = dev_alloc(h, gbytes, &err);
        if (err != cudaSuccess) return from_cuda(err);
        h->gram_bytes = gbytes;
    }
    if ((size_t)n + 1 > h->lam_cap) {
        dev_free(h, h->lam_dev, h->lam_cap * sizeof(double));
        h->lam_dev = nullptr;
        h->lam_cap = 0;
        cudaError_t err;
        h->lam_dev = (double *)dev_alloc(h, sizeof(double) * (n + 1), &err);
        if (err != cudaSuccess) return from_cuda(err);
        h->lam_cap = n + 1;
    }
    int nn = 0;
    {
        const cudaError_t ge = launch_gram(h, psi, cut, h->gram, &nn);
        if (ge == cudaErrorNotSupported) {
            cudaGetLastError();
            return OSMPS_EUNSUPPORTED;
        }
        CK(ge);
    }
    CKS(schmidt_eig(h, h->gram, nn, h->lam_dev, h->lam_dev + nn));
    if (lambda) CK(cudaMemcpyAsync(lambda, h->lam_dev, sizeof(double) * nn, cudaMemcpyDeviceToHost, h->stream));
    double Sv = 0.0;
    CK(cudaMemcpyAsync(&Sv, h->lam_dev + nn, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (S) *S = Sv;
    return OSMPS_OK;
}

osmps_status osmps_ed_schmidt_entropy_async(osmps_ed_t *ed, const void *psi, int cut, double *S, double *lambda) {
    if (ed == nullptr) return OSMPS_EINVAL;
    Handle *h = &ed->h;
    CKS(check_state_ptr(h, psi));
    const int L = h->L;
    if (cut == -1) cut = L / 2;
    if (L < 2 || cut < 1 || cut > L - 1) return OSMPS_EINVAL;
    const int ls = cut < L - cut ? cut : L - cut;
    const int n = 1 << ls;
    // the asynchronous call takes the Gram route (the automatic choice included)
    if (h->entropy_method != ENT_GRAM && h->entropy_method != ENT_AUTO) return OSMPS_EUNSUPPORTED;
    if (ed->am == nullptr) CKS(create_async(h, &ed->am));
    AsyncMeas *am = ed->am;
    if (am->own_G > 0) return entropy_async_own(h, am, psi, cut, n, S, lambda);
    int sl;
    {
        // wait (host) until the next slot's previous job has finished
        std::unique_lock<std::mutex> lock(am->mu);
        sl = am->next_slot;
        am->cv.wait(lock, [am, sl] { return !am->busy[sl]; });
    }
    CKS(grow_untracked(&am->rho[sl], &am->rho_bytes[sl], (size_t)n * n * h->esize, false));
    CKS(grow_untracked((void **)&am->lam[sl], &am->lam_bytes[sl], sizeof(double) * (n + 1), false));
    CKS(grow_untracked((void **)&am->host[sl], &am->host_bytes[sl], sizeof(double) * (n + 1), true));
    int nn = 0;
    {
        const cudaError_t ge = launch_gram(h, psi, cut, am->rho[sl], &nn);
        if (ge == cudaErrorNotSupported) {
            cudaGetLastError();
            return OSMPS_EUNSUPPORTED;
        }
        CK(ge);
    }
    CK(cudaEventRecord(am->ready[sl], h->stream));
    {
        std::lock_guard<std::mutex> lock(am->mu);
        am->busy[sl] = true;
        am->queued[sl] = true;
        am->job[sl] = AsyncJob{sl, nn, S, lambda};
        am->next_slot = sl ^ 1;
    }
    am->cv.notify_all();
    return OSMPS_OK;
}

osmps_status osmps_ed_set_async_eigensolver(osmps_ed_t *ed, int ctas) {
    if (ed == nullptr || ctas < 0) return OSMPS_EINVAL;
    if (ed->am == nullptr) CKS(create_async(&ed->h, &ed->am));
    CKS(osmps_ed_measure_wait(ed));  // no outstanding measurement changes mode
    if (ctas > 0) CKS(ensure_own_mode(ed->am));
    ed->am->own_G = ctas;
    return OSMPS_OK;
}

osmps_status osmps_ed_measure_wait(osmps_ed_t *ed) {
    if (ed == nullptr) return OSMPS_EINVAL;
    AsyncMeas *am = ed->am;
    if (am == nullptr) return OSMPS_OK;
    if (am->own_G > 0) {
        // oldest slot first (results land in the order the calls were made)
        const int first = am->next_slot;
        finish_own_slot(am, first);
        finish_own_slot(am, first ^ 1);
    }
    std::unique_lock<std::mutex> lock(am->mu);
    am->cv.wait(lock, [am] { return !am->busy[0] && !am->busy[1]; });
    ed->h.launches += am->launches;
    am->launches = 0;
    const osmps_status st = am->err;
    am->err = OSMPS_OK;
    return st;
}

// ---------------------------------------------------------------------------
// Adjoint gradient of a final energy (see include/osmps_ed.h)
// ---------------------------------------------------------------------------
static osmps_status adjoint_grad_impl(osmps_ed_t *ed, const void *psi0, int nsteps, double dt, const double *h_steps,
                                   int m, double h_target, int stride, int nquad, double *loss, double *grad_h,
                                   double *grad_scale) {
    if (ed == nullptr || h_steps == nullptr || loss == nullptr) return OSMPS_EINVAL;
    Handle *h = &ed->h;
    CKS(check_state_ptr(h, psi0));
    if (nsteps < 1 || !std::isfinite(dt) || m < 1 || m > kMaxKrylov || !std::isfinite(h_target) || stride < 1 ||
        nquad < 1 || nquad > 32)
        return OSMPS_EINVAL;
    for (int k = 0; k < nsteps; ++k)
        if (!std::isfinite(h_steps[k])) return OSMPS_EINVAL;
    const bool want_grad = grad_h != nullptr || grad_scale != nullptr;
    double hb_save[kMaxL + 1];
    std::memcpy(hb_save, h->hbit, sizeof(hb_save));
    const size_t vb = vec_bytes(h);
    const int ncp = (nsteps + stride - 1) / stride + 1;  // checkpoints psi_0, psi_stride, ...
    // device buffers of this call: checkpoints, one segment of states, lambda, two node states, two products, dots
    std::vector<void *> bufs;
    osmps_status st = OSMPS_OK;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (st == OSMPS_OK && cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            st = OSMPS_ENOMEM;
            return nullptr;
        }
        bufs.push_back(p);
        return p;
    };
    std::vector<void *> cp(ncp), seg(stride);
    for (int i = 0; i < ncp; ++i) cp[i] = alloc(vb);
    void *x = alloc(vb);
    void *lam = nullptr, *ps = nullptr, *ls = nullptr, *w1 = nullptr, *w0 = nullptr;
    double *zd = nullptr;
    if (want_grad) {
        for (int i = 0; i < stride; ++i) seg[i] = alloc(vb);
        lam = alloc(vb);
        ps = alloc(vb);
        ls = alloc(vb);
        w1 = alloc(vb);
        w0 = alloc(vb);
        // <ls|X ps> and <ls|H_zz ps> of every node of every step, read back once at the end
        zd = static_cast<double *>(alloc(sizeof(double) * 4 * (size_t)nquad * nsteps));
    }
    // Krylov bases of the segment's forward steps (the backward step k needs the basis of
    // psi_{k-1} under H(h_k), which recomputing psi_k builds): kept when they fit in a quarter
    // of the free device memory, else rebuilt in the backward sweep (same arithmetic, same bits)
    std::vector<void *> bstore;
    char *cstash = nullptr;
    const size_t o_alpha = CTL_OFF(alpha), o_beta = CTL_OFF(beta), o_scale = CTL_OFF(scale), o_sc = CTL_OFF(nrm);
    const size_t n_sc = CTL_OFF(m_eff) + sizeof(int) - o_sc;
    const size_t cslot = sizeof(double) * (3 * (size_t)m + 2) + n_sc;  // alpha[m], beta[m+1], scale[m+1], scalars
    if (want_grad && stride > 1 && st == OSMPS_OK) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            fr = 0;
        }
        if ((size_t)(stride - 1) * m * vb <= fr / 4) {
            bstore.assign((size_t)(stride - 1) * m, nullptr);
            for (auto &b : bstore) b = alloc(vb);
            cstash = static_cast<char *>(alloc(cslot * (size_t)(stride - 1)));
            if (st != OSMPS_OK) {  // not enough after all: rebuild the bases instead
                st = OSMPS_OK;
                bstore.clear();
                cstash = nullptr;
            }
        }
    }
    osmps_ed_t *sib = nullptr;  // second handle: Krylov basis of the adjoint state
    osmps_ed_t *xop = nullptr;  // third handle: X = sum_k sigma^x_k alone (no couplings, unit field)
    auto cleanup = [&]() {
        cudaStreamSynchronize(h->stream);
        for (void *p : bufs)
            if (p != nullptr) cudaFree(p);
        if (sib != nullptr) osmps_ed_destroy(sib);
        if (xop != nullptr) osmps_ed_destroy(xop);
        std::memcpy(h->hbit, hb_save, sizeof(hb_save));
    };
    auto fail = [&](osmps_status e) {
        cleanup();
        return e;
    };
    if (st != OSMPS_OK) return fail(st);
#define CKA(expr)                              \
    do {                                       \
        osmps_status _s = (expr);              \
        if (_s != OSMPS_OK) return fail(_s);   \
    } while (0)
#define CKAC(expr)                                   \
    do {                                             \
        cudaError_t _e = (expr);                     \
        if (_e != cudaSuccess) return fail(from_cuda(_e)); \
    } while (0)
    auto set_h = [&](Handle *hh, double v) {
        for (int b = 0; b < hh->L; ++b) hh->hbit[b] = v;
    };
    // one Krylov step of the forward propagation: v <- exp(-i dt H(h_k)) v
    auto step = [&](void *v, double hk) -> osmps_status {
        set_h(h, hk);
        return osmps_ed_krylov_evolve(ed, v, dt, 1, m, 0.0, nullptr);
    };

    // ---- forward sweep with checkpoints ----
    CKAC(cudaMemcpyAsync(x, psi0, vb, cudaMemcpyDeviceToDevice, h->stream));
    CKAC(cudaMemcpyAsync(cp[0], psi0, vb, cudaMemcpyDeviceToDevice, h->stream));
    for (int k = 1; k <= nsteps; ++k) {
        CKA(step(x, h_steps[k - 1]));
        if (k % stride == 0) CKAC(cudaMemcpyAsync(cp[k / stride], x, vb, cudaMemcpyDeviceToDevice, h->stream));
    }
    // loss and the direct coupling-scale term: <psi_N| H_target |psi_N>, <psi_N| H_zz |psi_N>
    double e_num = 0.0, nrm2 = 0.0, ezz = 0.0;
    set_h(h, h_target);
    CKA(osmps_ed_energy(ed, x, &e_num, &nrm2));
    *loss = e_num;
    if (!want_grad) {
        cleanup();
        return OSMPS_OK;
    }
    set_h(h, 0.0);
    CKA(osmps_ed_energy(ed, x, &ezz, &nrm2));

    // ---- backward sweep ----
    {
        double Jr1[kMaxL];
        for (int r = 1; r < h->L; ++r) Jr1[r - 1] = h->Jr[r];
        CKA(osmps_ed_create(h->L, h->L > 1 ? Jr1 : nullptr, 0.0, -1.0, 0.0, h->prec, h->stream, &sib));
        sib->h.reorth = h->reorth;
        double J0[kMaxL] = {0.0};
        CKA(osmps_ed_create(h->L, h->L > 1 ? J0 : nullptr, 0.0, -1.0, 1.0, h->prec, h->stream, &xop));
        xop->h.nsm = h->nsm;
    }
    Handle *hb = &sib->h;
    std::vector<double> xs(nquad), ws(nquad), gh(nsteps, 0.0);
    gauss_legendre01(nquad, xs.data(), ws.data());
    double gs = ezz;  // d/ds of <H_target> through its own coupling term
    // lambda_N = H_target psi_N
    set_h(h, h_target);
    {
        int np = 0;
        HpsiArgs a{};
        a.u = x;
        a.out = lam;
        a.tmp = h->tmp;
        a.partials = h->partials;
        a.epilogue = EPI_PLAIN;
        CKAC(launch_hpsi(h, a, &np));
    }
    std::vector<double> zh(4 * (size_t)nquad * nsteps);
    const int nseg = (nsteps + stride - 1) / stride;
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
        const int k0 = sgi * stride, k1 = std::min(nsteps, k0 + stride);
        // psi_{k0} .. psi_{k1-1} of this segment, recomputed from its checkpoint
        CKAC(cudaMemcpyAsync(seg[0], cp[sgi], vb, cudaMemcpyDeviceToDevice, h->stream));
        const bool keep = !bstore.empty();
        for (int k = k0 + 1; k < k1; ++k) {
            CKAC(cudaMemcpyAsync(seg[k - k0], seg[k - k0 - 1], vb, cudaMemcpyDeviceToDevice, h->stream));
            if (!keep) {
                CKA(step(seg[k - k0], h_steps[k - 1]));
            } else {
                // the same step as its two halves (the kernels of osmps_ed_krylov_evolve in the
                // same order), keeping the basis of psi_{k-1} and its scalars between them
                set_h(h, h_steps[k - 1]);
                CKA(krylov_basis(h, seg[k - k0], m));
                const size_t slot = (size_t)(k - k0 - 1);
                for (int i = 1; i <= m; ++i)
                    CKAC(cudaMemcpyAsync(bstore[slot * m + i - 1], h->V[i], vb, cudaMemcpyDeviceToDevice, h->stream));
                char *cs = cstash + slot * cslot;
                char *cb = reinterpret_cast<char *>(h->ctl);
                CKAC(cudaMemcpyAsync(cs, cb + o_alpha, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->stream));
                CKAC(cudaMemcpyAsync(cs + sizeof(double) * m, cb + o_beta, sizeof(double) * (m + 1),
                                     cudaMemcpyDeviceToDevice, h->stream));
                CKAC(cudaMemcpyAsync(cs + sizeof(double) * (2 * m + 1), cb + o_scale, sizeof(double) * (m + 1),
                                     cudaMemcpyDeviceToDevice, h->stream));
                CKAC(cudaMemcpyAsync(cs + sizeof(double) * (3 * m + 2), cb + o_sc, n_sc, cudaMemcpyDeviceToDevice,
                                     h->stream));
                CKA(krylov_combine(h, m, dt, seg[k - k0]));
            }
        }
        for (int k = k1; k > k0; --k) {
            const double hk = h_steps[k - 1];
            void *psi_prev = seg[k - 1 - k0];
            // Krylov bases of psi_{k-1} (handle h) and lambda_k (handle hb) under H(h_k)
            set_h(h, hk);
            set_h(hb, hk);
            if (keep && k < k1) {
                // the basis kept from the recomputation of this segment
                const size_t slot = (size_t)(k - k0 - 1);
                CKA(ensure_basis(h, m));
                for (int i = 1; i <= m; ++i)
                    CKAC(cudaMemcpyAsync(h->V[i], bstore[slot * m + i - 1], vb, cudaMemcpyDeviceToDevice, h->stream));
                CKA(upload_basis_table(h, psi_prev, m));
                const char *cs = cstash + slot * cslot;
                char *cb = reinterpret_cast<char *>(h->ctl);
                CKAC(cudaMemcpyAsync(cb + o_alpha, cs, sizeof(double) * m, cudaMemcpyDeviceToDevice, h->stream));
                CKAC(cudaMemcpyAsync(cb + o_beta, cs + sizeof(double) * m, sizeof(double) * (m + 1),
                                     cudaMemcpyDeviceToDevice, h->stream));
                CKAC(cudaMemcpyAsync(cb + o_scale, cs + sizeof(double) * (2 * m + 1), sizeof(double) * (m + 1),
                                     cudaMemcpyDeviceToDevice, h->stream));
                CKAC(cudaMemcpyAsync(cb + o_sc, cs + sizeof(double) * (3 * m + 2), n_sc, cudaMemcpyDeviceToDevice,
                                     h->stream));
            } else {
                CKA(krylov_basis(h, psi_prev, m));
            }
            CKA(krylov_basis(hb, lam, m));
            // Frechet derivative of exp(-i dt H) along X and along H_zz, by Gauss-Legendre in s:
            //   <lambda_k| L(A, E) psi_{k-1}> = int_0^1 <e^{i s dt H} lambda_k| E |e^{-i (1-s) dt H} psi_{k-1}> ds
            double *zk = zd + 4 * (size_t)nquad * (k - 1);
            for (int q = 0; q < nquad; ++q) {
                CKA(krylov_combine(h, m, (1.0 - xs[q]) * dt, ps));
                CKA(krylov_combine(hb, m, -xs[q] * dt, ls));
                int np = 0;
                HpsiArgs a{};
                a.u = ps;
                a.epilogue = EPI_PLAIN;
                a.partials = xop->h.partials;
                a.tmp = xop->h.tmp;
                a.out = w1;
                CKAC(launch_hpsi(&xop->h, a, &np));  // X ps
                set_h(h, 0.0);
                a.partials = h->partials;
                a.tmp = h->tmp;
                a.out = w0;
                CKAC(launch_hpsi(h, a, &np));  // H_zz ps
                CKAC(launch_cdot(h, ls, w1, zk + 4 * q));
                CKAC(launch_cdot(h, ls, w0, zk + 4 * q + 2));
            }
            // lambda_{k-1} = exp(+i dt H(h_k)) lambda_k
            CKA(krylov_combine(hb, m, -dt, lam));
        }
    }
    CKAC(cudaMemcpyAsync(zh.data(), zd, sizeof(double) * zh.size(), cudaMemcpyDeviceToHost, h->stream));
    CKA(sync_and_check(h));
    CKA(sync_and_check(hb));
    CKA(sync_and_check(&xop->h));
    for (int k = 1; k <= nsteps; ++k) {
        const double *zk = zh.data() + 4 * (size_t)nquad * (k - 1);
        double gk = 0.0;
        for (int q = 0; q < nquad; ++q) {
            // d/dh_k: E = -i dt X, 2 Re(-i dt z) = 2 dt Im z with z = <ls| X ps>
            gk += ws[q] * 2.0 * dt * zk[4 * q + 1];
            // d/ds: E = -i dt H_zz
            gs += ws[q] * 2.0 * dt * zk[4 * q + 3];
        }
        gh[k - 1] = gk;
    }
    if (grad_h != nullptr)
        for (int k = 0; k < nsteps; ++k) grad_h[k] = gh[k];
    if (grad_scale != nullptr) *grad_scale = gs;
#undef CKA
#undef CKAC
    cleanup();
    return OSMPS_OK;
}

// ---------------------------------------------------------------------------
// Two-site gates and Trotter evolution (see include/osmps_ed.h)
// ---------------------------------------------------------------------------
static osmps_status apply_gates_impl(osmps_ed_t *ed, void *psi, int ngates, const int *site, const double *U) {
    if (ed == nullptr || ngates < 0 || (ngates > 0 && (site == nullptr || U == nullptr))) return OSMPS_EINVAL;
    Handle *h = &ed->h;
    CKS(check_state_ptr(h, psi));
    const int L = h->L;
    if (L < 4) return OSMPS_EUNSUPPORTED;
    std::vector<char> used(L + 2, 0);
    std::vector<int> lo(ngates);
    for (int i = 0; i < ngates; ++i) {
        const int s = site[i];
        if (s < 1 || s > L - 1 || used[s] || used[s + 1]) return OSMPS_EINVAL;  // bonds must be disjoint
        used[s] = used[s + 1] = 1;
        for (int e = 0; e < 32; ++e)
            if (!std::isfinite(U[32 * i + e])) return OSMPS_EINVAL;
        lo[i] = L - s - 1;
    }
    if (ngates == 0) return OSMPS_OK;
    CK(gates::launch_gate_layer(h, psi, ngates, lo.data(), U));
    return OSMPS_OK;
}

static osmps_status trotter_evolve_impl(osmps_ed_t *ed, void *psi, double dt, int nsteps, int order) {
    if (ed == nullptr) return OSMPS_EINVAL;
    Handle *h = &ed->h;
    CKS(check_state_ptr(h, psi));
    if (!std::isfinite(dt) || nsteps < 0 || (order != 1 && order != 2 && order != 4)) return OSMPS_EINVAL;
    if (h->L < 4) return OSMPS_EUNSUPPORTED;
    for (int r = 2; r < h->L; ++r)
        if (h->Jr[r] != 0.0) return OSMPS_EUNSUPPORTED;  // nearest-neighbour chains only
    if (nsteps == 0) return OSMPS_OK;
    auto E = [&](double tau) { return gates::trotter_layer(h, psi, 0, tau); };
    auto O = [&](double tau) { return gates::trotter_layer(h, psi, 1, tau); };
    if (order == 1) {  // Eq. trotter1: exp(-i dt H_o) exp(-i dt H_e)
        for (int k = 0; k < nsteps; ++k) {
            CK(E(dt));
            CK(O(dt));
        }
    } else if (order == 2) {  // Eq. trotter2, the half steps of neighbouring steps merged
        CK(E(0.5 * dt));
        for (int k = 0; k < nsteps; ++k) {
            CK(O(dt));
            CK(E(k + 1 < nsteps ? dt : 0.5 * dt));
        }
    } else {  // Eqs. trotter4, trotter4c
        const double t3 = 1.0 / (2.0 * (4.0 - std::cbrt(4.0)));
        const double t1 = 1.0 - 8.0 * t3, t2 = 0.5 * (1.0 - 6.0 * t3), t4 = 2.0 * t3;
        const double seq[11] = {t3, t4, t4, t4, t2, t1, t2, t4, t4, t4, t3};  // E, O, E, ... from the right
        for (int k = 0; k < nsteps; ++k)
            for (int f = 0; f < 11; ++f) CK((f & 1) ? O(seq[f] * dt) : E(seq[f] * dt));
    }
    return OSMPS_OK;
}

// ---------------------------------------------------------------------------
// Reduced density matrices of all pairs and the bond-entropy sweep
// ---------------------------------------------------------------------------
static osmps_status rdm_pairs_impl(osmps_ed_t *ed, const void *psi, double *rdm2, double *rdm1) {
    if (ed == nullptr) return OSMPS_EINVAL;
    Handle *h = &ed->h;
    CKS(check_state_ptr(h, psi));
    const int L = h->L;
    if (L < 2) return OSMPS_EINVAL;
    const int npairs = L * (L - 1) / 2;
    double *scr = nullptr;
    const size_t nd = pair_rdm_scratch_doubles(L);
    if (cudaMalloc(&scr, sizeof(double) * nd) != cudaSuccess) {
        cudaGetLastError();
        return OSMPS_ENOMEM;
    }
    double *out_dev = scr + (nd - (size_t)npairs * 16);
    std::vector<double> vals((size_t)npairs * 16);
    cudaError_t err = launch_pair_rdm(h, psi, scr, out_dev);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(vals.data(), out_dev, sizeof(double) * vals.size(), cudaMemcpyDeviceToHost, h->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
    cudaFree(scr);
    CK(err);
    // assemble the Hermitian 4 x 4 matrices, (re, im) row-major
    std::vector<double> R((size_t)npairs * 32, 0.0);
    for (int p = 0; p < npairs; ++p) {
        const double *v = &vals[(size_t)p * 16];
        double *M = &R[(size_t)p * 32];
        for (int d = 0; d < 4; ++d) M[(d * 4 + d) * 2] = v[d];
        int q = 4;
        for (int v1 = 0; v1 < 4; ++v1)
            for (int v2 = v1 + 1; v2 < 4; ++v2) {
                M[(v1 * 4 + v2) * 2] = v[q];
                M[(v1 * 4 + v2) * 2 + 1] = v[q + 1];
                M[(v2 * 4 + v1) * 2] = v[q];
                M[(v2 * 4 + v1) * 2 + 1] = -v[q + 1];
                q += 2;
            }
    }
    if (rdm2 != nullptr) std::memcpy(rdm2, R.data(), sizeof(double) * R.size());
    if (rdm1 != nullptr) {
        // rho_i = Tr_j rho_ij with the pair (i, i+1) (the last site from (L-1, L))
        auto pidx = [&](int i, int j) { return (i - 1) * L - (i - 1) * i / 2 + (j - i - 1); };
        for (int i = 1; i <= L; ++i) {
            const bool first = i < L;
            const double *M = &R[(size_t)(first ? pidx(i, i + 1) : pidx(L - 1, L)) * 32];
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    double re = 0.0, im = 0.0;
                    for (int t = 0; t < 2; ++t) {
                        const int r = first ? 2 * a + t : 2 * t + a, c = first ? 2 * b + t : 2 * t + b;
                        re += M[(r * 4 + c) * 2];
                        im += M[(r * 4 + c) * 2 + 1];
                    }
                    rdm1[(size_t)(i - 1) * 8 + (a * 2 + b) * 2] = re;
                    rdm1[(size_t)(i - 1) * 8 + (a * 2 + b) * 2 + 1] = im;
                }
        }
    }
    return OSMPS_OK;
}

osmps_status osmps_ed_entropy_sweep(osmps_ed_t *ed, const void *psi, double *S) {
    if (ed == nullptr || S == nullptr) return OSMPS_EINVAL;
    if (ed->h.L < 2) return OSMPS_EINVAL;
    // largest blocks first, so the Gram and solver workspaces are sized once
    const int L = ed->h.L;
    for (int ls = L / 2; ls >= 1; --ls) {
        CKS(osmps_ed_schmidt_entropy(ed, psi, ls, nullptr, &S[ls - 1]));
        if (L - ls != ls) CKS(osmps_ed_schmidt_entropy(ed, psi, L - ls, nullptr, &S[L - ls - 1]));
    }
    return OSMPS_OK;
}

// Host-side allocations of these calls (small vectors sized by the arguments)
// must not throw across the C boundary.
osmps_status osmps_ed_adjoint_grad(osmps_ed_t *ed, const void *psi0, int nsteps, double dt, const double *h_steps,
                                   int m, double h_target, int stride, int nquad, double *loss, double *grad_h,
                                   double *grad_scale) {
    try {
        return adjoint_grad_impl(ed, psi0, nsteps, dt, h_steps, m, h_target, stride, nquad, loss, grad_h, grad_scale);
    } catch (...) {
        return OSMPS_ENOMEM;
    }
}

osmps_status osmps_ed_apply_gates(osmps_ed_t *ed, void *psi, int ngates, const int *site, const double *U) {
    try {
        return apply_gates_impl(ed, psi, ngates, site, U);
    } catch (...) {
        return OSMPS_ENOMEM;
    }
}

osmps_status osmps_ed_trotter_evolve(osmps_ed_t *ed, void *psi, double dt, int nsteps, int order) {
    try {
        return trotter_evolve_impl(ed, psi, dt, nsteps, order);
    } catch (...) {
        return OSMPS_ENOMEM;
    }
}

osmps_status osmps_ed_rdm_pairs(osmps_ed_t *ed, const void *psi, double *rdm2, double *rdm1) {
    try {
        return rdm_pairs_impl(ed, psi, rdm2, rdm1);
    } catch (...) {
        return OSMPS_ENOMEM;
    }
}

}  // extern "C"
