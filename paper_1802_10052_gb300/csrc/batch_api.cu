// C ABI of the batched ground-state solver (osmps_ed_batch_* in
// include/osmps_ed.h): argument checks, the packed state layout, the buffers
// of one solve, the work-queue order and the optional CUDA graph of a solve.
// The solve itself is one persistent kernel (batch_kernels.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "ed_internal.h"

using namespace osmps;

struct osmps_ed_batch {
    BatchHandle b;
};

namespace {

osmps_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return OSMPS_OK;
    if (e == cudaErrorMemoryAllocation) return OSMPS_ENOMEM;
    return OSMPS_ECUDA;
}

void *balloc(BatchHandle *b, size_t bytes, cudaError_t *err) {
    void *p = nullptr;
    *err = cudaMalloc(&p, bytes);
    if (*err != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    b->owned_bytes += bytes;
    return p;
}

void release(BatchHandle *b) {
    if (b->graph != nullptr) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    void *bufs[] = {b->d_inst, b->d_order, b->R[0], b->R[1], b->R[2], b->X, b->scratch, b->counter};
    for (void *p : bufs)
        if (p != nullptr) cudaFree(p);
    delete[] b->offsets;
    b->offsets = nullptr;
    delete[] b->L;
    b->L = nullptr;
}

// The launch of one solve (memset of the queue head + one kernel) captured
// into a CUDA graph on a private stream; the graph is then launched on the
// handle's stream.
cudaError_t capture(BatchHandle *b, void *psi, double tol, double *energy, double *residual, int *iters,
                    int *status) {
    cudaStream_t cap = nullptr;
    cudaError_t err = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (err != cudaSuccess) return err;
    cudaStream_t user = b->stream;
    const uint64_t launches = b->launches;
    b->stream = cap;
    cudaGraph_t g = nullptr;
    err = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
        cudaError_t e1 = batch::launch_batch(b, psi, tol, energy, residual, iters, status);
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        err = e1 != cudaSuccess ? e1 : e2;
    }
    b->stream = user;
    b->launches = launches;
    if (err == cudaSuccess) {
        if (b->graph != nullptr) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        err = cudaGraphInstantiate(&b->graph, g, 0);
    }
    if (g != nullptr) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (err == cudaSuccess) {
        b->g_psi = psi;
        b->g_tol = tol;
        b->g_energy = energy;
        b->g_residual = residual;
        b->g_iters = iters;
        b->g_status = status;
    }
    return err;
}

}  // namespace

extern "C" {

static osmps_status batch_create_impl(int n, const int *L, const double *J, const double *alpha, const double *h,
                                      int prec, int max_iter, void *cuda_stream, osmps_ed_batch_t **out) {
    if (out == nullptr) return OSMPS_EINVAL;
    *out = nullptr;
    if (n < 1 || n > (1 << 24) || L == nullptr || J == nullptr || alpha == nullptr || h == nullptr)
        return OSMPS_EINVAL;
    if (prec != OSMPS_FP64 && prec != OSMPS_MIXED) return OSMPS_EINVAL;
    if (max_iter < 1 || max_iter > kMaxLanczos) return OSMPS_EINVAL;
    const int lmin = batch::batch_tile_bits(prec);
    bool unsupported = false;
    for (int k = 0; k < n; ++k) {
        if (L[k] < 1 || L[k] > kMaxL) return OSMPS_EINVAL;
        if (!std::isfinite(J[k]) || std::isnan(alpha[k]) || !std::isfinite(h[k])) return OSMPS_EINVAL;
        if (L[k] < lmin || L[k] > kBatchMaxL) unsupported = true;
    }
    if (unsupported) return OSMPS_EUNSUPPORTED;

    osmps_ed_batch *ob = new (std::nothrow) osmps_ed_batch();
    if (ob == nullptr) return OSMPS_ENOMEM;
    BatchHandle *b = &ob->b;
    std::memset(b, 0, sizeof(*b));
    b->n = n;
    b->prec = prec;
    b->max_iter = max_iter;
    b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaError_t err = cudaGetDevice(&b->device);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
    if (err != cudaSuccess) {
        delete ob;
        return from_cuda(err);
    }
    if (err == cudaSuccess) err = batch::batch_prepare(prec);
    if (err != cudaSuccess) {
        delete ob;
        return from_cuda(err);
    }
    b->grid = std::min(n, b->nsm);
    b->csize = 1;
    b->lsplit = kBatchMaxL + 1;
    b->nbig = 0;

    b->offsets = new (std::nothrow) long long[n + 1];
    if (b->offsets == nullptr) {
        delete ob;
        return OSMPS_ENOMEM;
    }
    b->L = new (std::nothrow) int[n];
    if (b->L == nullptr) {
        delete[] b->offsets;
        delete ob;
        return OSMPS_ENOMEM;
    }
    std::copy(L, L + n, b->L);
    std::vector<BatchInst> inst(n);
    b->offsets[0] = 0;
    for (int k = 0; k < n; ++k) {
        BatchInst &in = inst[k];
        std::memset(&in, 0, sizeof(in));
        in.off = b->offsets[k];
        in.L = L[k];
        in.h = h[k];
        const bool nn = alpha[k] < 0.0 || std::isinf(alpha[k]);
        for (int r = 1; r < L[k]; ++r) in.J[r] = nn ? (r == 1 ? J[k] : 0.0) : J[k] / std::pow((double)r, alpha[k]);
        b->offsets[k + 1] = b->offsets[k] + (1ll << L[k]);
    }
    b->total = b->offsets[n];
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return L[x] > L[y]; });

    const size_t esize = prec == OSMPS_FP64 ? 16 : 8;
    const size_t vbytes = esize * (size_t)b->total;
    b->d_inst = static_cast<BatchInst *>(balloc(b, sizeof(BatchInst) * n, &err));
    if (err == cudaSuccess) b->d_order = static_cast<int *>(balloc(b, sizeof(int) * n, &err));
    for (int i = 0; i < 3 && err == cudaSuccess; ++i) b->R[i] = balloc(b, vbytes, &err);
    if (err == cudaSuccess) b->X = balloc(b, vbytes, &err);
    if (err == cudaSuccess)
        b->scratch = static_cast<double *>(balloc(b, sizeof(double) * (size_t)b->nsm * (8 * (size_t)max_iter + 8 + kBatchEllScratch),
                                                        &err));
    if (err == cudaSuccess) b->counter = static_cast<int *>(balloc(b, 3 * sizeof(int), &err));
    if (err == cudaSuccess) {
        b->err = b->counter + 2;
        err = cudaMemcpyAsync(b->d_inst, inst.data(), sizeof(BatchInst) * n, cudaMemcpyHostToDevice, b->stream);
    }
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(b->d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, b->stream);
    if (err == cudaSuccess) err = cudaMemsetAsync(b->counter, 0, 3 * sizeof(int), b->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(b->stream);
    if (err != cudaSuccess) {
        release(b);
        delete ob;
        return from_cuda(err);
    }
    *out = ob;
    return OSMPS_OK;
}

osmps_status osmps_ed_batch_destroy(osmps_ed_batch_t *ob) {
    if (ob == nullptr) return OSMPS_EINVAL;
    cudaStreamSynchronize(ob->b.stream);
    release(&ob->b);
    delete ob;
    return OSMPS_OK;
}

osmps_status osmps_ed_batch_offsets(const osmps_ed_batch_t *ob, uint64_t *offsets) {
    if (ob == nullptr || offsets == nullptr) return OSMPS_EINVAL;
    for (int k = 0; k <= ob->b.n; ++k) offsets[k] = (uint64_t)ob->b.offsets[k];
    return OSMPS_OK;
}

osmps_status osmps_ed_batch_device_bytes(const osmps_ed_batch_t *ob, uint64_t *bytes) {
    if (ob == nullptr || bytes == nullptr) return OSMPS_EINVAL;
    *bytes = ob->b.owned_bytes;
    return OSMPS_OK;
}

osmps_status osmps_ed_batch_set_graph(osmps_ed_batch_t *ob, int enable) {
    if (ob == nullptr || (enable != 0 && enable != 1)) return OSMPS_EINVAL;
    ob->b.use_graph = enable;
    return OSMPS_OK;
}

osmps_status osmps_ed_batch_set_split(osmps_ed_batch_t *ob, int csize, int lsplit) {
    if (ob == nullptr) return OSMPS_EINVAL;
    BatchHandle *b = &ob->b;
    if (csize != 1 && csize != 2 && csize != 4 && csize != 8) return OSMPS_EINVAL;
    int log2c = 0;
    while ((1 << log2c) < csize) ++log2c;
    // a cluster CTA's range of a streaming pass must hold a multiple of 1024 vectors
    const int lmin = 11 + (b->prec == OSMPS_FP64 ? 0 : 1) + log2c;
    if (csize > 1 && (lsplit < lmin || lsplit > kBatchMaxL)) return OSMPS_EINVAL;
    int nbig = 0, grid = std::min(b->n, b->nsm);
    if (csize > 1) {
        for (int k = 0; k < b->n; ++k)
            if (b->L[k] >= lsplit) ++nbig;
        int ncl = 0;
        cudaError_t err = batch::batch_max_clusters(b->prec, csize, b->nsm, &ncl);
        if (err != cudaSuccess) return from_cuda(err);
        if (ncl < 1) return OSMPS_EUNSUPPORTED;
        grid = csize * std::min(ncl, b->nsm / csize);
    }
    if (b->graph != nullptr && (grid != b->grid || csize != b->csize || nbig != b->nbig)) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->csize = csize;
    b->lsplit = csize > 1 ? lsplit : kBatchMaxL + 1;
    b->nbig = nbig;
    b->grid = grid;
    return OSMPS_OK;
}

osmps_status osmps_ed_batch_get_split(const osmps_ed_batch_t *ob, int *csize, int *lsplit, int *grid) {
    if (ob == nullptr || csize == nullptr || lsplit == nullptr || grid == nullptr) return OSMPS_EINVAL;
    *csize = ob->b.csize;
    *lsplit = ob->b.lsplit;
    *grid = ob->b.grid;
    return OSMPS_OK;
}

static osmps_status batch_autotune_impl(osmps_ed_batch_t *ob, void *psi, double tol, double *best_ms) {
    if (ob == nullptr || psi == nullptr || !(tol >= 0.0) || !std::isfinite(tol)) return OSMPS_EINVAL;
    if ((reinterpret_cast<uintptr_t>(psi) & 15u) != 0) return OSMPS_EINVAL;
    BatchHandle *b = &ob->b;
    const size_t esize = b->prec == OSMPS_FP64 ? 16 : 8;
    const size_t vbytes = esize * (size_t)b->total;
    int lmax = 0;
    for (int k = 0; k < b->n; ++k) lmax = std::max(lmax, b->L[k]);
    // candidates: no clusters, and clusters of 2, 4, 8 CTAs for the chains with
    // L >= lmax - 2, lmax - 1 or lmax
    std::vector<std::pair<int, int>> cand;
    cand.push_back({1, kBatchMaxL + 1});
    for (int cs : {2, 4, 8})
        for (int ls = lmax - 2; ls <= lmax; ++ls) cand.push_back({cs, ls});
    void *save = nullptr;
    double *outs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaMalloc(&save, vbytes);
    if (err == cudaSuccess) err = cudaMalloc(&outs, (size_t)b->n * 4 * sizeof(double));
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) err = cudaMemcpyAsync(save, psi, vbytes, cudaMemcpyDeviceToDevice, b->stream);
    const int keep_graph = b->use_graph;
    b->use_graph = 0;
    float best = 1e30f;
    std::pair<int, int> best_c = {b->csize, b->lsplit};
    osmps_status st = OSMPS_OK;
    for (size_t i = 0; i < cand.size() && err == cudaSuccess && st == OSMPS_OK; ++i) {
        if (osmps_ed_batch_set_split(ob, cand[i].first, cand[i].second) != OSMPS_OK) continue;
        if (cand[i].first > 1 && b->nbig == 0) continue;
        err = cudaMemcpyAsync(psi, save, vbytes, cudaMemcpyDeviceToDevice, b->stream);
        if (err == cudaSuccess) err = cudaEventRecord(e0, b->stream);
        if (err == cudaSuccess)
            err = batch::launch_batch(b, psi, tol, outs, outs + b->n, reinterpret_cast<int *>(outs + 2 * b->n),
                                      reinterpret_cast<int *>(outs + 3 * b->n));
        if (err == cudaSuccess) err = cudaEventRecord(e1, b->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) break;
        st = osmps_ed_batch_check(ob);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_c = cand[i];
        }
    }
    if (err == cudaSuccess) err = cudaMemcpyAsync(psi, save, vbytes, cudaMemcpyDeviceToDevice, b->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(b->stream);
    b->use_graph = keep_graph;
    if (e0 != nullptr) cudaEventDestroy(e0);
    if (e1 != nullptr) cudaEventDestroy(e1);
    cudaFree(save);
    cudaFree(outs);
    if (err != cudaSuccess) return from_cuda(err);
    if (st != OSMPS_OK) return st;
    osmps_status s2 = osmps_ed_batch_set_split(ob, best_c.first, best_c.second);
    if (s2 == OSMPS_OK && best_ms != nullptr) *best_ms = (double)best;
    return s2;
}

osmps_status osmps_ed_batch_lanczos_ground(osmps_ed_batch_t *ob, void *psi, double tol, double *energy,
                                           double *residual, int *iters, int *status) {
    if (ob == nullptr || psi == nullptr || energy == nullptr || residual == nullptr || iters == nullptr ||
        status == nullptr)
        return OSMPS_EINVAL;
    if (!(tol >= 0.0) || !std::isfinite(tol)) return OSMPS_EINVAL;
    if ((reinterpret_cast<uintptr_t>(psi) & 15u) != 0) return OSMPS_EINVAL;
    BatchHandle *b = &ob->b;
    if (!b->use_graph) return from_cuda(batch::launch_batch(b, psi, tol, energy, residual, iters, status));
    if (b->graph == nullptr || b->g_psi != psi || b->g_tol != tol || b->g_energy != energy ||
        b->g_residual != residual || b->g_iters != iters || b->g_status != status) {
        cudaError_t err = capture(b, psi, tol, energy, residual, iters, status);
        if (err != cudaSuccess) return from_cuda(err);
    }
    cudaError_t err = cudaGraphLaunch(b->graph, b->stream);
    if (err != cudaSuccess) return from_cuda(err);
    b->launches++;
    return OSMPS_OK;
}

osmps_status osmps_ed_batch_check(osmps_ed_batch_t *ob) {
    if (ob == nullptr) return OSMPS_EINVAL;
    BatchHandle *b = &ob->b;
    cudaError_t err = cudaStreamSynchronize(b->stream);
    if (err != cudaSuccess) return from_cuda(err);
    int flag = 0;
    err = cudaMemcpy(&flag, b->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) return from_cuda(err);
    if (flag != 0) {
        cudaMemset(b->err, 0, sizeof(int));
        return OSMPS_ETIMEOUT;
    }
    return OSMPS_OK;
}

osmps_status osmps_ed_batch_launch_count(const osmps_ed_batch_t *ob, int64_t *count) {
    if (ob == nullptr || count == nullptr) return OSMPS_EINVAL;
    *count = (int64_t)ob->b.launches;
    return OSMPS_OK;
}

// Host-side allocations of these calls (vectors sized by the arguments) must
// not throw across the C boundary.
osmps_status osmps_ed_batch_create(int n, const int *L, const double *J, const double *alpha, const double *h,
                                   int prec, int max_iter, void *cuda_stream, osmps_ed_batch_t **out) {
    try {
        return batch_create_impl(n, L, J, alpha, h, prec, max_iter, cuda_stream, out);
    } catch (...) {
        return OSMPS_ENOMEM;
    }
}

osmps_status osmps_ed_batch_autotune(osmps_ed_batch_t *ob, void *psi, double tol, double *best_ms) {
    try {
        return batch_autotune_impl(ob, psi, tol, best_ms);
    } catch (...) {
        return OSMPS_ENOMEM;
    }
}

}  // extern "C"
