// Internal declarations shared by the translation units of libosmps_ed.
// Not part of the public ABI (include/osmps_ed.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/osmps_ed.h"

namespace osmps {

// ---------------------------------------------------------------------------
// Limits and tiling constants
// ---------------------------------------------------------------------------
constexpr int kMaxL = OSMPS_MAX_L;
constexpr int kMaxKrylov = 64;       // vectors per Krylov step
constexpr int kMaxLanczos = 1000;    // Lanczos vectors
constexpr int kPassThreads = 256;    // consumer threads per CTA of the H.psi passes
constexpr int kVecThreads = 256;     // threads per CTA of the streaming vector kernels
constexpr int kTileBytesLog2 = 16;   // 64 KiB shared-memory tile per H.psi CTA
constexpr int kChunkBytesLog2 = 7;   // 128-byte contiguous chunks in the strided passes
constexpr int kMaxPasses = 4;

// Scalars the device-side Krylov/Lanczos control kernels keep between launches.
struct KrylovCtl {
    double alpha[kMaxLanczos];        // T diagonal
    double beta[kMaxLanczos + 1];     // T off-diagonal, beta[j] couples j-1 and j
    double scale[kMaxLanczos + 1];    // v_j = scale[j] * u_j (stored vectors unnormalised)
    double coef_re[kMaxLanczos];      // combination coefficients (already times scale)
    double coef_im[kMaxLanczos];
    double nrm;                       // ||psi|| at the start of the step
    double err;                       // a-posteriori error estimate of the step
    double err_sum;                   // summed over steps
    double theta;                     // lowest Ritz value (ground state)
    double est;                       // beta_{j+1} |y_j| (ground state)
    double epi[3];                    // epilogue scalars of the next H.psi: sv, a, b
    double epi2[3];                   // epilogue scalars of the ground-state residual pass
    double bd_tol;                    // relative breakdown threshold
    int m_eff;                        // vectors in the basis (< m after breakdown)
    int error;                        // raised by a kernel whose bounded wait gave up
    double work[7 * kMaxLanczos];     // scratch of the single-thread tridiagonal solves
};

// One pass of the multi-pass H.psi (see hpsi_kernels.cu for the scheme).
struct PassDesc {
    int c;        // contiguous chunk bits carried but not flipped
    int o;        // first global bit of the flipped group
    int g;        // number of flipped bits
    int first;    // computes the diagonal and writes (no accumulate input)
    long long ntiles;
};

struct PassPlan {
    int npass;
    int a1;       // bits of the first (contiguous) pass
    int ta;       // split of a1 for the per-tile diagonal tables
    PassDesc p[kMaxPasses];
};

// Epilogue of the last pass.
enum Epilogue : int {
    EPI_PLAIN = 0,   // out = H u
    EPI_KRYLOV = 1,  // out = sv*H u - a*sv*u - b*uprev; partials <sv u, out>, |out|^2
    EPI_ENERGY = 2   // no write; partials <u, H u>, |u|^2
};

struct HpsiArgs {
    const void *u;
    const void *uprev;
    void *out;
    void *tmp;                 // partial-sum vector between passes
    const double *epi;         // device epilogue scalars (sv, a, b) or nullptr (=1,0,0)
    double *partials;          // per-CTA partial sums, 4 doubles per CTA
    const int *m_eff;          // skip the launch when *m_eff <= stop_index
    int stop_index;
    int epilogue;
    // Lanczos step stop_index >= 1 without a control kernel before it: the first
    // pass forms beta, scale and the epilogue scalars of this step from the
    // update's partial |u|^2 (fixed order, every CTA alike; CTA 0 writes them)
    KrylovCtl *fold_ctl;
    const double *fold_parts;
    int fold_nparts;
};

struct Handle;

// hpsi_kernels.cu
PassPlan make_plan(int L, int prec);
cudaError_t build_tables(Handle *h);
cudaError_t launch_hpsi(Handle *h, const HpsiArgs &a, int *nparts_out);
cudaError_t launch_hpsi_timed(Handle *h, const HpsiArgs &a, int *nparts_out);
int hpsi_grid(Handle *h, int pass);
int hpsi_partials_per_cta();

// vec_kernels.cu
cudaError_t launch_fill_basis(Handle *h, void *psi, uint64_t b);
cudaError_t launch_norm2(Handle *h, const void *x, double *partials, int *nparts);
// <a, b> = sum conj(a) b into out_dev[0..1] (re, im); uses partials2
cudaError_t launch_cdot(Handle *h, const void *a, const void *b, double *out_dev);
cudaError_t launch_ctl_after_norm(Handle *h, KrylovCtl *ctl, const double *partials, int nparts, int j);
cudaError_t launch_ctl_after_hpsi(Handle *h, KrylovCtl *ctl, const double *partials, int nparts, int j);
// alpha_j from the product's partials inside the update (no control kernel):
// hp/hnp = the H.psi epilogue partials; alpha_j written by CTA 0
cudaError_t launch_update_folded(Handle *h, void *w, const void *u, KrylovCtl *ctl, int j, const double *hp,
                                 int hnp, double *partials, int *nparts);
cudaError_t launch_update(Handle *h, void *w, const void *u, KrylovCtl *ctl, int j, double *partials,
                          int *nparts);
cudaError_t launch_ctl_after_update(Handle *h, KrylovCtl *ctl, const double *partials, int nparts, int j,
                                    int mode);
cudaError_t launch_multidot(Handle *h, void *const *V, int nvec, const void *w, KrylovCtl *ctl, int j,
                            double *partials, int *nparts);   // 2*nvec doubles per CTA
cudaError_t launch_reorth_update(Handle *h, void *const *V, int nvec, void *w, KrylovCtl *ctl, int j,
                                 const double *dots, int ndots_parts, double *partials, int *nparts);
cudaError_t launch_tridiag_exp(Handle *h, KrylovCtl *ctl, int m, double dt);
cudaError_t launch_tridiag_ground(Handle *h, KrylovCtl *ctl, int m);
cudaError_t launch_combine(Handle *h, void *const *V, int nvec, void *out, KrylovCtl *ctl, double *partials,
                           int *nparts);
cudaError_t launch_scale(Handle *h, void *x, const double *s_dev);
int vec_grid(Handle *h);

// measure_kernels.cu
cudaError_t launch_zstats(Handle *h, const void *psi, double *out_dev);
cudaError_t launch_gram(Handle *h, const void *psi, int cut, void *rho, int *n_out);

// gram_tc.cu (tensor-core Gram product, complex64 only)
bool gram_tc_supported(int n, long long K);
cudaError_t gram_tc_launch(Handle *h, const void *psi, int n, long long K, void *rho, float *planes, float *G);
osmps_status schmidt_eig(Handle *h, void *rho, int n, double *lambda_dev, double *S_dev);
// Schmidt values of the cut as squared singular values of the block matrix M of psi
// (no Gram product); lambda_dev: 2^min(cut, L-cut) values, descending, then S
osmps_status schmidt_svd(Handle *h, const void *psi, int cut, double *lambda_dev, double *S_dev);
// Schmidt values as Rayleigh quotients |u_i^H A|^2 of the eigenvectors of rho = A A^H
// (complex64; rescaled to the FP64 norm): rho is the n x n Gram buffer;
// OSMPS_ENOCONV when the library eigen-solver failed (callers then take schmidt_svd)
bool rayleigh_applicable(const Handle *h, int cut);
osmps_status schmidt_rayleigh(Handle *h, const void *psi, int cut, void *rho, double *lambda_dev, double *S_dev);
// Schmidt values from the dominant subspace (512 <= n <= 8192): OK, or ENOCONV when
// the weight outside an affordable subspace stays above 1e-9 (complex64) or
// 2e-12 (complex128) of the trace or a value is not finite (the caller then takes
// the full route)
bool subspace_applicable(const Handle *h, int cut);
osmps_status schmidt_subspace(Handle *h, const void *psi, int cut, double *lambda_dev, double *S_dev);
bool rayleigh_tc_supported(int n, long long K);
size_t rayleigh_tc_plane_floats(int n, long long K);
cudaError_t rayleigh_tc_launch(Handle *h, const void *R, const void *psi, int n, long long K, long long sx,
                               long long sk, float *planes, double *part_re, double *part_im);
// how osmps_ed_schmidt_entropy obtains the Schmidt values
enum EntropyMethod : int {
    ENT_GRAM = 0,      // eigenvalues of the Gram product
    ENT_SVD = 1,       // squared singular values of M
    ENT_RAYLEIGH = 2,  // Rayleigh quotients of the Gram product's eigenvectors (complex64)
    ENT_AUTO = 3,      // subspace where it applies; else complex64: Rayleigh where it applies, else
                       // singular values up to 2^13 rows, else Gram; complex128: Gram
    ENT_SUBSPACE = 4   // squared singular values on the dominant subspace, full route as fallback
};
// S and the descending spectrum from ascending FP64 eigenvalues w (n values) on a stream
cudaError_t launch_entropy(cudaStream_t stream, const double *w, int n, double *lambda_dev, double *S_dev);

// eig_kernels.cu: eigenvalues of the Hermitian rho (the Gram product's row-major
// upper triangle read as a column-major lower triangle; overwritten) by blocked
// Householder tridiagonalization on G cooperative CTAs and Sturm multisection.
struct TrdRun {
    int prec;
    int device;
    cudaStream_t stream;
    int G;                      // CTAs of the cooperative panel kernel (all resident)
    void *ws;                   // workspace of trd_workspace_bytes(n, prec, G) bytes
    size_t ws_bytes;
    int *error;                 // device int set to 1 when a bounded wait gave up
    int64_t *launches;          // incremented by the kernels launched (may be null)
};
int trd_ctas(int n, int prec, int want, int device);
size_t trd_workspace_bytes(int n, int prec, int G);
// ascending FP64 eigenvalues in the workspace (*w points to them)
cudaError_t trd_eigvals(const TrdRun &run, void *rho, int n, double **w);

// the same on a given stream and workspace (tracked: the workspace counts in the handle's owned bytes)
// solver: a handle from solver_handle_new, or null for the process-wide one (serialised)
osmps_status schmidt_eig_on(Handle *h, cudaStream_t stream, void *solver, void **ws, size_t *ws_bytes, bool tracked,
                            int64_t *launches, void *rho, int n, double *lambda_dev, double *S_dev);
void *solver_handle_new();        // null if the library solver cannot be loaded
void solver_handle_free(void *solver);

// Device memory owned by a handle.
struct Handle {
    int L;
    int prec;                   // OSMPS_FP64 / OSMPS_MIXED
    uint64_t D;
    size_t esize;               // bytes per amplitude (16 or 8)
    cudaStream_t stream;
    int device;
    int nsm;
    double Jr[kMaxL + 1];       // J(r), index r (J[0] unused)
    double hbit[kMaxL + 1];     // field on bit b (site L-b)
    int reorth;
    PassPlan plan;

    // tables for the diagonal energy
    void *Ell;                  // 2^a1 entries (T)
    void *Fhh;                  // 2^(L-a1) x (a1+1) entries (T)
    void *Tab;                  // 2^(L-a1) x 192 entries (T): per-tile TA, TB

    // scratch
    double *partials;           // per-CTA partial sums
    double *partials_upd;       // the folded Lanczos update's partial |u|^2 (read by the next product)
    int fold_ctl;               // fold the Lanczos control kernels into the update and the next product
    size_t partials_cap;        // doubles
    double *partials2;
    size_t partials2_cap;
    double *dscratch;           // small FP64 device scratch (outputs before D2H)
    size_t dscratch_cap;
    KrylovCtl *ctl;             // device control block
    KrylovCtl *ctl_host;        // pinned host mirror (scalars read back)
    void *tmp;                  // pass-to-pass partial vector (D elements)
    void *xbuf;                 // Ritz vector of the ground state (D elements)
    void **V;                   // host array of Krylov vector pointers (V[0] = caller psi)
    void **V_dev;               // device copy of the pointer table
    int Vcap;                   // allocated vectors (excluding V[0])
    void *gram;                 // Gram matrix buffer
    size_t gram_bytes;
    void *gram_aux;             // tensor-core Gram: TF32 hi/lo planes and G
    size_t gram_aux_bytes;
    int gram_mode;              // 0 automatic, 1 CUDA cores, 2 tensor cores
    int prefetch;               // L2 prefetch distance of the H.psi passes (tiles)
    int pass_threads;           // H.psi CTA shape: 256 (16 vectors per thread) or 512 (8)
    int flip_fixed;             // complex128: fewest flipped bits of a uniform-field pass summed in fixed point (0 = none)
    int entropy_method;         // EntropyMethod
    void *solver_ws;            // cuSOLVER workspace
    size_t solver_ws_bytes;
    void *sub_ws;               // dominant-subspace entropy: Y/Q, B, W, Z, a copy of M, partials, solver work
    size_t sub_ws_bytes;
    int sub_hint;               // its starting dimension (from the values above 1e-12 last time; 0 = default)
    int sub_skip;               // calls left that take the full route directly
    double *lam_dev;
    size_t lam_cap;
    uint64_t owned_bytes;
    // optional event timing of the H.psi products
    int timing;
    cudaEvent_t *tev;           // pairs (start, stop)
    int tev_cap;                // pairs allocated
    int tev_used;               // pairs recorded since the last read
    double t_ms;                // accumulated at read time
    int64_t t_calls;
    int64_t launches;           // kernels this handle has launched
};

void *dev_alloc(Handle *h, size_t bytes, cudaError_t *err);
void dev_free(Handle *h, void *p, size_t bytes);

// reduced density matrices of all pairs (rdm_kernels.cu): 16 reals per pair into out_dev
cudaError_t launch_pair_rdm(Handle *h, const void *psi, double *scratch_dev, double *out_dev);
size_t pair_rdm_scratch_doubles(int L);  // scratch plus the npairs x 16 output at its end

// two-site gates (gate_kernels.cu)
namespace gates {
// gate i on bits (lo[i] + 1, lo[i]): U[32 i ..] 4 x 4 complex, row-major, basis 2 bit_hi + bit_lo
cudaError_t launch_gate_layer(Handle *h, void *psi, int ng, const int *lo, const double *U);
// exp(-i tau H_p) psi, p = 1: bonds (s, s+1) with s odd (H_o), p = 0: s even (H_e)
cudaError_t trotter_layer(Handle *h, void *psi, int parity, double tau);
}  // namespace gates

// ---------------------------------------------------------------------------
// Batched ground states (batch_kernels.cu, batch_api.cu)
// ---------------------------------------------------------------------------
constexpr int kBatchMaxL = 22;          // gathered pass-B segments stay >= 64 bytes
constexpr int kBatchEllScratch = 4096;  // doubles per CTA for the E_ll table of the 64 KiB tile

// One chain of a batch as the kernel sees it.
struct BatchInst {
    long long off;                      // amplitude offset of its state in the packed buffers
    int L;
    int pad;
    double h;                           // uniform transverse field
    double J[kMaxL + 1];                // J(r), r = 1..L-1 (J[0] = 0)
};

struct BatchHandle {
    int device;
    int nsm;
    int n;
    int prec;
    int max_iter;
    int grid;                           // CTAs of the persistent launch
    int csize;                          // CTAs per cluster (1: no clusters)
    int lsplit;                         // chains with L >= lsplit are solved by whole clusters
    int nbig;                           // number of such chains (first in the work order)
    cudaStream_t stream;
    long long total;                    // packed state length (amplitudes)
    long long *offsets;                 // host, n + 1
    int *L;                             // host, chain lengths
    BatchInst *d_inst;
    int *d_order;                       // chain order of the work queue (largest first)
    void *R[3];                         // recurrence vectors (packed like the states)
    void *X;                            // Ritz vector accumulator
    double *scratch;                    // per CTA: alpha, beta, y, tridiagonal work
    int *counter;                       // work-queue heads: [0] large chains, [1] the others
    int *err;                           // raised when a bounded wait gives up
    uint64_t owned_bytes;
    uint64_t launches;
    // CUDA graph of one solve, captured on first use with a given argument set
    int use_graph;
    cudaGraphExec_t graph;
    void *g_psi;
    double g_tol;
    double *g_energy, *g_residual;
    int *g_iters, *g_status;
};

namespace batch {
size_t batch_smem_bytes(int prec);
int batch_tile_bits(int prec);
cudaError_t batch_prepare(int prec);
cudaError_t batch_max_clusters(int prec, int csize, int nsm, int *out);
cudaError_t launch_batch(BatchHandle *b, void *psi, double tol, double *energy, double *residual, int *iters,
                         int *status);
}  // namespace batch

}  // namespace osmps
