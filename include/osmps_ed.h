/*
 * osmps_ed.h -- C ABI of the GB300 exact-diagonalization hot path.
 *
 * Matrix-free Hamiltonian-times-state product for spin-1/2 chains, used inside
 * Lanczos ground-state search and Krylov real-time evolution, followed by the
 * measurements <sz_k>, <sz_i sz_j> and the half-chain Schmidt spectrum.
 * Everything runs on one CUDA device; all vector work is done by the kernels of
 * this library.
 *
 * Model (arXiv:1802.10052, Eq. genericH with one site rule sigma^x and one
 * distance-only infinite-function rule sigma^z sigma^z; the nearest-neighbour
 * quantum Ising model Eq. HQI and the long-range H_LRQI of Sec. VII are special
 * cases):
 *
 *     H = sum_{i<j} J(j-i) sz_i sz_j + sum_k h_k sx_k        (signed inputs)
 *
 * The paper's conventions are reached with J(r) = -1 (r = 1 only), h -> -h
 * (Eq. HQI) or J(r) = -cos(phi)/r^alpha, h = -sin(phi) (H_LRQI).
 *
 * State layout (the rank-L tensor of Sec. IV in row-major order): a state is
 * D = 2^L interleaved complex numbers (re, im) in device memory, complex128
 * (double2) for OSMPS_FP64 and complex64 (float2) for OSMPS_MIXED.  Basis index
 * b in [0, D); site k (1-based) is bit L-k, so site 1 is the most significant
 * bit; bit value 0 is spin up (sz = +1).  All-up is b = 0.
 *
 * Ownership: the caller owns every state buffer (device pointers, 16-byte
 * aligned, D elements, no aliasing between an input and an output of the same
 * call unless stated).  The handle owns its tables and its Krylov workspace,
 * allocated at create or on first use and released by osmps_ed_destroy.
 *
 * Ordering: work is enqueued on the handle's CUDA stream.  Calls that return
 * host scalars synchronise that stream before returning; osmps_ed_apply_H and
 * osmps_ed_init_basis_state return without synchronising.  One handle must
 * not be used from two host threads at once.
 *
 * Errors: every call returns an osmps_status, never aborts.  After an error
 * other than OSMPS_ECUDA the handle stays valid and the contents of output
 * buffers are unspecified.  After OSMPS_ECUDA the CUDA context may be
 * unusable; destroy the handle.
 */
#ifndef OSMPS_ED_H
#define OSMPS_ED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct osmps_ed osmps_ed_t;

typedef enum {
    OSMPS_OK = 0,
    OSMPS_EINVAL = 1,       /* bad argument (range, NULL, non-finite, alignment) */
    OSMPS_ENOMEM = 2,       /* device or host allocation failed */
    OSMPS_ECUDA = 3,        /* a CUDA runtime or library call failed */
    OSMPS_ENOCONV = 4,      /* Lanczos did not reach the tolerance in max_iter */
    OSMPS_ETIMEOUT = 5,     /* a bounded device wait gave up */
    OSMPS_EUNSUPPORTED = 6  /* valid request the library does not support here */
} osmps_status;

typedef enum {
    OSMPS_FP64 = 0,  /* complex128 states, FP64 arithmetic throughout */
    OSMPS_MIXED = 1  /* complex64 states and H.psi in FP32; inner products,
                        norms, Krylov coefficients and the small tridiagonal
                        problem in FP64 */
} osmps_prec;

/* Largest chain length accepted (2^30 amplitudes). */
#define OSMPS_MAX_L 30

/*
 * Create a handle for a chain of L sites (1 <= L <= OSMPS_MAX_L).
 * Paper: Eq. genericH (site rule + infinite-function rule, coupling depending
 * only on the distance, c_{k',k} = c(k'-k)); Eq. HQI; H_LRQI (Sec. VII).
 *   couplings  host array J(r) for r = 1..L-1 (index r-1), or NULL.  When NULL,
 *              J(r) = J / r^alpha; alpha < 0 (or +inf) keeps only J(1) = J
 *              (nearest neighbours).
 *   h          uniform transverse field (see osmps_ed_set_site_fields).
 *   prec       OSMPS_FP64 or OSMPS_MIXED; fixes the element type of all states.
 *   cuda_stream  cudaStream_t to enqueue work on (NULL = legacy default stream).
 *   out        receives the handle.
 * Errors: EINVAL (L out of range, non-finite input, out == NULL), ENOMEM, ECUDA.
 */
osmps_status osmps_ed_create(int L, const double *couplings, double J, double alpha, double h,
                             int prec, void *cuda_stream, osmps_ed_t **out);

/* Release the handle and everything it owns (synchronises its stream). NULL is OK. */
osmps_status osmps_ed_destroy(osmps_ed_t *ed);

/* Replace the stream used by later calls. */
osmps_status osmps_ed_set_stream(osmps_ed_t *ed, void *cuda_stream);

/* Uniform transverse field h (piecewise-constant h(t) is set between calls;
 * the caller evaluates it at mid-step t + dt/2, Sec. III.A). */
osmps_status osmps_ed_set_field(osmps_ed_t *ed, double h);

/* Site-dependent fields h_k, host array of L values in site order k = 1..L
 * (site rule with spatially dependent coupling c_k, Eq. genericH). */
osmps_status osmps_ed_set_site_fields(osmps_ed_t *ed, const double *h_sites);

/* Reorthogonalisation of Lanczos/Krylov vectors: 0 = three-term recurrence
 * only, 1 = additionally one classical Gram-Schmidt pass against all stored
 * vectors ("orthogonalized against all previous", Sec. III.D).  Default:
 * 1 for osmps_ed_lanczos_ground, the handle's value for krylov_evolve
 * (initially 0). */
osmps_status osmps_ed_set_reorth(osmps_ed_t *ed, int mode);

/* Gram product of osmps_ed_schmidt_entropy: 0 = automatic (tensor cores,
 * tcgen05 with a 3xTF32 split, for OSMPS_MIXED states whose left block has
 * at least 128 rows and at most as many rows as columns; CUDA cores
 * otherwise), 1 = CUDA cores, 2 = tensor cores (EUNSUPPORTED where they do
 * not apply).  Not from the paper (implementation choice). */
osmps_status osmps_ed_set_gram_mode(osmps_ed_t *ed, int mode);

/* Number of SMs the handle's kernels size their grids for (persistent
 * kernels launch one CTA per SM of this count): 1..device SMs, 0 = all.
 * A smaller count leaves SMs free for work on other streams, e.g. the
 * eigen-solves of osmps_ed_schmidt_entropy_async.  Not from the paper
 * (scheduling). */
osmps_status osmps_ed_set_sm_count(osmps_ed_t *ed, int nsm);

/* How osmps_ed_schmidt_entropy obtains the Schmidt values (Sec. IV bond
 * entropy).  Not from the paper (numerics).
 *   0  Gram product rho_A = M M^dag (tensor cores for complex64) and its
 *      eigenvalues.  Every Schmidt value then carries an absolute error of
 *      order the working precision; in complex64 that noise reaches ~2e-5 in S
 *      of a weakly entangled L = 24 state.
 *   1  squared singular values of the block matrix M itself (library SVD on a
 *      copy of M, no Gram product): accurate (~2e-7 in S in complex64) at ~5x
 *      the cost of 0.  The copy (2^L amplitudes) and the library workspace stay
 *      with the handle after the call and are counted by osmps_ed_device_bytes;
 *      ENOMEM when they do not fit.
 *   2  Rayleigh quotients (complex64 only; 128 <= 2^min(cut, L-cut) <= 8192):
 *      the eigenvectors u_i of the Gram product (library solver), then
 *      Lambda_i = |u_i^dag M|^2 from M itself on the tensor cores, all
 *      rescaled to sum to <psi|psi> (FP64).  No value is formed by squaring M
 *      in FP32, so S keeps ~1e-7 in complex64 at ~1.1x the cost of 0; values
 *      of nearly equal size (closer than ~1e-7) come out as averages of each
 *      other, which moves S only at second order.  Scratch (4 n^2 + 2 n K complex-sized floats) is kept by the handle.
 *      Falls back to 1 when the library eigen-solver fails or its eigenvectors
 *      give a non-finite value (seen for nearly product states whose rho has
 *      FP32-subnormal entries).  EUNSUPPORTED where it does not apply.
 *   3  automatic (the default): 4 where it applies; else complex128 takes 0
 *      (FP64 Gram and eigenvalues meet 1e-10) and complex64 takes 2 where it
 *      applies, else 1 for blocks up to 8192 rows, else 0.
 *   4  dominant subspace (512 <= 2^min(cut, L-cut) <= 8192): Y = M G for a
 *      seeded random K x p block G, Q = orth(Y) (library Householder QR),
 *      B = Q^dag M (library GEMMs in the handle's precision), and the Schmidt
 *      values as the eigenvalues of C = B B^dag formed and diagonalised in FP64
 *      (the squared singular values of B), rescaled with the residual weight to
 *      the FP64 norm.  The weight outside the subspace, |M - Q B|_F^2, is
 *      measured directly and must stay at or below 1e-9 (complex64) or 2e-12
 *      (complex128) of the trace, its share of S then below the precision's
 *      tolerance; otherwise p doubles up to min(n/2, 768), beyond which (or on a
 *      non-finite value) the call takes the full route (complex64: method 2,
 *      then 1; complex128: method 0) and skips the subspace for four calls.  p
 *      starts from the number of values above 1e-12 at the handle's previous
 *      call plus a quarter and 64 (128 the first time).  The spectrum has p
 *      values and zeros after them.  Scratch (n p + 2 p K complex, up to
 *      16 p^2 FP64 complex partials, a copy of M, solver work) is kept by the
 *      handle.  The cost follows p: weakly entangled states (p ~ 100) need a
 *      small fraction of the full eigen-solve.
 * osmps_ed_schmidt_entropy_async takes method 0 (also when 3 is set) and
 * returns EUNSUPPORTED for 1, 2 and 4. */
osmps_status osmps_ed_set_entropy_method(osmps_ed_t *ed, int method);

/* L2 prefetch distance of the H.psi passes: each CTA asks L2 (TMA prefetch)
 * for the tiles it will stage `tiles` steps after the ones its shared-memory
 * stages hold; 0 = off.  Default 1 for OSMPS_MIXED, 0 for OSMPS_FP64.
 * 0 <= tiles <= 4.  Not from the paper (memory scheduling). */
osmps_status osmps_ed_set_prefetch(osmps_ed_t *ed, int tiles);

/* Launches of a Krylov Lanczos step without the Gram-Schmidt pass (not from
 * the paper; scheduling).  1 (default): alpha_j is summed inside the update
 * kernel and beta_{j+1} inside the next product's first pass (three launches
 * per step); 0: separate single-warp control kernels (five).  The scalars are
 * the same fixed-order sums either way, so results are bit-identical.  The
 * ground-state search always uses the separate kernels (it reads T after every
 * step). */
osmps_status osmps_ed_set_lanczos_fold(osmps_ed_t *ed, int on);

/* CTA shape of the H.psi passes (not from the paper; scheduling): 256 threads
 * holding 16 vectors of a 64 KiB tile each, or 512 threads holding 8 (twice the
 * warps per SM to hide latency, one more bit flipped through shared memory).
 * Defaults: 256 for OSMPS_MIXED (its passes are issue-bound and the 128-register
 * cap of the larger CTA adds instructions), 512 for OSMPS_FP64 (latency-bound,
 * 3 % faster).  Results agree to rounding (the order of the flip terms
 * differs).  Takes effect at the next product. */
osmps_status osmps_ed_set_pass_threads(osmps_ed_t *ed, int threads);

/* Arithmetic of the sigma^x flip sums of complex128 H.psi (not from the paper;
 * numerics).  mode >= 1 (default 1): in every pass that flips at least `mode`
 * bits sharing one field value, the tile's amplitudes are put on one 64-bit
 * fixed-point grid (unit 2^-57 of the tile's largest magnitude or finer;
 * truncation toward zero, by integer operations), the flipped partners are
 * summed exactly in integers and the sum is rounded back to FP64 and multiplied
 * by the field.  Each sum is thus within (number of flipped bits) units of the
 * exact one: relative to the largest amplitude of the tile, not to the partners'
 * own magnitudes.  A non-finite amplitude makes its tile's sums NaN.  Passes with
 * site-dependent fields, and every pass with mode 0, use FP64 multiply-adds.
 * 0 <= mode <= 30.  No effect on complex64 handles.  Takes effect at the next
 * product. */
osmps_status osmps_ed_set_flip_sums(osmps_ed_t *ed, int mode);

/* D = 2^L. */
osmps_status osmps_ed_dim(const osmps_ed_t *ed, uint64_t *D);

/* Bytes of device memory the handle currently owns. */
osmps_status osmps_ed_device_bytes(const osmps_ed_t *ed, uint64_t *bytes);

/* psi <- |b> (product state; all-up b = 0).  Device buffer, no sync. */
osmps_status osmps_ed_init_basis_state(osmps_ed_t *ed, void *psi, uint64_t b);

/* Stream-ordered copies of one state between host and device memory
 * (D elements of the handle's type).  Pinned host memory gives async copies. */
osmps_status osmps_ed_upload(osmps_ed_t *ed, void *dst_device, const void *src_host);
osmps_status osmps_ed_download(osmps_ed_t *ed, void *dst_host, const void *src_device);

/*
 * out <- H psi, matrix-free (Sec. III.D, rule set times psi; Eq. OKrylov).
 * psi, out: device buffers of D elements, must not alias.  No sync.  The
 * kernels' internal waits are bounded; if one gives up, the next call of this
 * handle that synchronises (energy, Lanczos, Krylov, timing_read) returns
 * OSMPS_ETIMEOUT.
 */
osmps_status osmps_ed_apply_H(osmps_ed_t *ed, const void *psi, void *out);

/* <psi|H|psi> and <psi|psi> (energy measurement, Sec. IV); host outputs,
 * either may be NULL.  Synchronises. */
osmps_status osmps_ed_energy(osmps_ed_t *ed, const void *psi, double *e_num, double *norm2);

/*
 * Lowest eigenpair by Lanczos (statics, Sec. II; eigsh replaced by Lanczos
 * with full reorthogonalisation unless osmps_ed_set_reorth(ed, 0) was called
 * after the last create).
 *   psi       in: start vector (any nonzero norm); out: normalised ground state.
 *   tol       stop when ||H x - E x|| <= tol for the normalised Ritz vector x
 *             (checked explicitly once beta_{j+1}|y_j| <= tol).
 *   max_iter  Lanczos vectors stored at most (1 <= max_iter <= 1000).
 *   energy, residual, iters: host outputs (may be NULL).
 * Returns ENOCONV (with the best vector in psi) if tol was not reached.
 */
osmps_status osmps_ed_lanczos_ground(osmps_ed_t *ed, void *psi, double tol, int max_iter,
                                     double *energy, double *residual, int *iters);

/*
 * psi <- exp(-i H dt)^nsteps psi by the Krylov approximation (Sec. III.D):
 * each step builds m Lanczos vectors v_1 = psi/||psi||, v_{i+1} from H v_i,
 * and sets psi <- ||psi|| sum_i [exp(-i dt T_m)]_{i,1} v_i with the m x m
 * tridiagonal T_m diagonalised in FP64 on the device.
 *   m         Krylov vectors per step (1 <= m <= 64).
 *   tol       relative breakdown threshold: a new vector whose norm beta_{j+1}
 *             is below tol*(|alpha_j| + beta_j) ends the step's basis early
 *             (the subspace is then invariant and the step exact);
 *             tol <= 0 selects 1e-12.
 *   err_estimate  host output (may be NULL): sum over steps of the a-posteriori
 *             estimate beta_{m+1} |[exp(-i dt T_m) e_1]_m| ||psi||.
 * The norm of psi is not renormalised between steps.
 */
osmps_status osmps_ed_krylov_evolve(osmps_ed_t *ed, void *psi, double dt, int nsteps, int m,
                                    double tol, double *err_estimate);

/*
 * Gradient of a final energy under a piecewise-constant field (the paper has
 * no gradients; this is the adjoint of its Krylov time evolution, Sec. III.D).
 * With H(h) = H_zz + h X (H_zz the handle's couplings, X = sum_k sigma^x_k),
 *     psi_k = exp(-i dt H(h_k)) psi_{k-1},  k = 1..nsteps,  psi_0 = psi0,
 *     loss  = <psi_N| H(h_target) |psi_N>,
 * returns loss and, unless both pointers are NULL, d loss / d h_k for every
 * step and d loss / d s, s the overall scale of the couplings (J(r) -> s J(r)
 * at s = 1, in H(h_k) and in the target; for J(r) = J / r^alpha this is
 * J d loss / d J).  The forward steps are Krylov steps of dimension m as in
 * osmps_ed_krylov_evolve.  Backward sweep: lambda_N = H(h_target) psi_N,
 * lambda_{k-1} = exp(+i dt H(h_k)) lambda_k, and
 *     d loss / d h_k = 2 Re <lambda_k| L(A_k, -i dt X) psi_{k-1}>,
 * with L(A, E) = int_0^1 e^{sA} E e^{(1-s)A} ds the Frechet derivative of the
 * exponential at A_k = -i dt H(h_k), evaluated by nquad-point Gauss-Legendre
 * quadrature in s on Krylov representations of psi_{k-1} and lambda_k
 * (likewise with E = -i dt H_zz for the coupling scale).  Forward states are
 * checkpointed every `stride` steps and recomputed segment by segment.
 *   psi0        device state (not modified).
 *   h_steps     host array of nsteps fields.
 *   grad_h      host array of nsteps (may be NULL); grad_scale host (may be NULL).
 *   nquad       1..32 (8 resolves dt |H| up to ~3 to 1e-14).
 * Allocates (1 + nsteps/stride + stride + 5) state vectors, two more handles
 * (a second Krylov workspace for the adjoint state, and the operator X alone),
 * and, when they fit in a quarter of the free device memory, (stride - 1) * m
 * more vectors that keep the Krylov bases built while a segment is recomputed
 * (the backward sweep then does not rebuild them; same arithmetic, same
 * results).  Everything is freed before returning; the handle's fields are
 * left as they were.  Synchronises.
 */
osmps_status osmps_ed_adjoint_grad(osmps_ed_t *ed, const void *psi0, int nsteps, double dt,
                                   const double *h_steps, int m, double h_target, int stride,
                                   int nquad, double *loss, double *grad_h, double *grad_scale);

/*
 * <sz_k> for k = 1..L (Sec. IV, Tr(sz rho_k) from the single-site reduced
 * density matrix).  sz: host array of L doubles.  Unnormalised: for a state of
 * norm n the values scale with n^2.  Synchronises.
 */
osmps_status osmps_ed_measure_local(osmps_ed_t *ed, const void *psi, double *sz);

/*
 * <sz_i sz_j> for all i, j (Sec. IV, Tr((sz x sz) rho_ij) from the two-site
 * reduced density matrices).  szsz: host array of L*L doubles, row-major,
 * symmetric, diagonal = <psi|psi>.  Synchronises.
 */
osmps_status osmps_ed_measure_corr(osmps_ed_t *ed, const void *psi, double *szsz);

/* Both of the above from one pass over the state (either output may be NULL). */
osmps_status osmps_ed_measure_zz(osmps_ed_t *ed, const void *psi, double *sz, double *szsz);

/*
 * <sz_k> and <sz_i sz_j> like osmps_ed_measure_zz, but without a handle and
 * without allocating any memory.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory at run time,
 * e.g. code whose device memory is owned by another allocator or budget (a
 * framework's caching pool), or a latency-critical loop that cannot afford
 * cudaMalloc/cudaFree and the device-wide synchronisation they imply.
 *   L         1 <= L <= OSMPS_MAX_L (30); larger chains return OSMPS_EINVAL.
 *   prec      OSMPS_FP64 (psi is complex128) or OSMPS_MIXED (complex64).
 *   psi       device state, 2^L elements, 16-byte aligned.
 *   out_dev   device array of L + L*L doubles: <sz_k> for k = 1..L, then
 *             <sz_i sz_j> row-major (site order, diagonal = <psi|psi>).
 *   cuda_stream  stream the kernels are enqueued on; the call does not
 *             synchronise.
 * Scratch: a file-scope device array of 3.75 MiB (3,932,160 bytes) that every
 * GPU loading this library holds until the process exits.  All calls share it
 * and it keeps the last call's contents; every entry a call reads was written
 * earlier in the same call, so nothing needs clearing.  Calls that overlap on
 * the GPU (different streams, or different host threads) race on the scratch:
 * order them.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  No cudaMalloc, cudaFree or allocating
 * library routine is called.
 */
osmps_status osmps_ed_measure_zz_noalloc(int L, int prec, const void *psi, double *out_dev, void *cuda_stream);

/*
 * Schmidt spectrum and entanglement entropy of the bipartition sites 1..cut |
 * cut+1..L (Sec. IV, bond entropy: rho = M M^dagger with M the state reshaped
 * to (2^cut, 2^(L-cut)); S = -sum_j Lambda_j ln Lambda_j, Sec. V).
 *   cut      1 <= cut <= L-1, or -1 for floor(L/2).
 *   lambda   host array of 2^min(cut, L-cut) doubles (descending), or NULL.
 *   S        host output (may be NULL); eigenvalues <= 0 contribute 0.
 * How the Schmidt values are obtained is set by osmps_ed_set_entropy_method
 * (default: the most accurate route that applies).  The products run on this
 * library's kernels; the Hermitian eigen-solve and the SVD are cuSOLVER's,
 * loaded at first use.  Returns EUNSUPPORTED if cuSOLVER cannot be loaded.
 * Synchronises.
 */
osmps_status osmps_ed_schmidt_entropy(osmps_ed_t *ed, const void *psi, int cut, double *lambda,
                                      double *S);

/*
 * The same measurement without blocking the caller (Sec. IV, entanglement
 * measures taken along a time evolution).  The Gram product rho =
 * psi_A psi_A^dag is enqueued on the handle's stream, so psi may be changed
 * by work enqueued after this call; the eigen-solve and the entropy then run
 * on the lowest-priority non-blocking stream of one of two result slots of
 * the handle; with the library solver each slot also has its own solver
 * handle and worker thread (the solver blocks its host thread).  Results go
 * to the host pointers S (one double) and lambda (2^min(cut, L-cut) doubles,
 * or NULL), which the caller keeps valid and does not read until
 * osmps_ed_measure_wait returns.  Two measurements may be outstanding; a
 * third call blocks the caller until the older one has finished.  Buffers of
 * the asynchronous path are not counted by osmps_ed_device_bytes.  Errors of
 * the argument checks and of the Gram product return here; errors of the
 * eigen-solve are returned by the next osmps_ed_measure_wait.  Not from the
 * paper (scheduling).
 */
osmps_status osmps_ed_schmidt_entropy_async(osmps_ed_t *ed, const void *psi, int cut, double *S,
                                            double *lambda);

/*
 * Eigen-solver of osmps_ed_schmidt_entropy_async.  ctas = 0: the library
 * routine (cuSOLVER heevd) on the handle's worker thread.  ctas > 0: this
 * library's kernels, enqueued by the calling thread on one lowest-priority
 * stream per result slot: blocked Householder reduction of rho to real
 * tridiagonal form (panels of 32 columns, one cooperative launch of at least
 * `ctas` CTAs per panel, more when the CTAs' row slices would not fit in
 * shared memory) with a trailing rank-64 update per panel, then every
 * eigenvalue by Sturm-count multisection in the working precision, so that
 * two measurements can run beside the caller's work on a few SMs each.
 * Waits for outstanding measurements first.  EUNSUPPORTED (at the entropy
 * call) when no CTA count up to the device's SMs fits.  Not from the paper
 * (eigen-solver and scheduling).
 */
osmps_status osmps_ed_set_async_eigensolver(osmps_ed_t *ed, int ctas);

/* Blocks until every osmps_ed_schmidt_entropy_async of this handle has
 * written its results; returns the first error among them (then clears it).
 * Call it before osmps_ed_destroy when measurements are outstanding. */
osmps_status osmps_ed_measure_wait(osmps_ed_t *ed);

/*
 * Check of the failure path of the bounded device waits (not from the paper;
 * failure detection).  Enqueues one kernel that waits, with the same bounded
 * mbarrier wait the H.psi and Gram kernels use, for a barrier phase that
 * nothing completes (complete = 0) or that the kernel completes itself first
 * (complete = 1).  The wait gives up after `seconds` (0 < seconds <= 2; the
 * library's own kernels give up after 2 s), raises the handle's error word and
 * returns; the next synchronising call of the handle (energy, Lanczos, Krylov)
 * then returns OSMPS_ETIMEOUT and clears the word, and the handle stays usable.
 * No fault, trap or hang is involved.  Enqueues only.
 */
osmps_status osmps_ed_probe_wait(osmps_ed_t *ed, double seconds, int complete);

/*
 * Timing of the H.psi products with CUDA events recorded on the handle's
 * stream around every product (all passes), for roofline measurements.
 * Not from the paper (instrumentation).  enable = 0 stops recording.
 * osmps_ed_timing_read synchronises the stream and returns the summed device
 * time in milliseconds and the number of products since the last reset;
 * reset != 0 clears the counters.
 */
osmps_status osmps_ed_timing_enable(osmps_ed_t *ed, int enable);
osmps_status osmps_ed_timing_read(osmps_ed_t *ed, double *hpsi_ms, int64_t *hpsi_calls, int reset);

/* Number of kernels this handle has launched so far (its own kernels; the
 * cuSOLVER eigenvalue routine is not counted; those of the asynchronous
 * entropy are added at osmps_ed_measure_wait).  Not from the paper. */
osmps_status osmps_ed_launch_count(const osmps_ed_t *ed, int64_t *count);

/*
 * Batched ground states: the lowest eigenpair of many independent chains in
 * one persistent launch (statics, Sec. II, for a set of Hamiltonians of
 * Eq. genericH).  Each CTA of the launch takes one chain at a time from a work
 * queue (largest first) and runs that chain's Lanczos iteration by itself, so
 * chains converge independently; no Krylov basis is stored (a second sweep
 * regenerates the vectors to form the Ritz vector).  Vectors are complex64
 * (OSMPS_MIXED) or complex128 (OSMPS_FP64); alpha, beta, all reductions and
 * the tridiagonal problem are FP64.
 *
 * osmps_ed_batch_create: n chains; chain k has L[k] sites with
 *   J(r) = J[k] / r^alpha[k] (alpha[k] < 0 or +inf: nearest neighbour only,
 *   J(1) = J[k]) and uniform field h[k].  L[k] must lie in [13, 22] for
 *   OSMPS_MIXED and [12, 22] for OSMPS_FP64 (one 64 KiB tile of low bits).
 *   max_iter (1..1000) bounds the Lanczos steps per chain.  Allocates every
 *   buffer the solve needs (four packed vectors and per-CTA scratch).
 * osmps_ed_batch_offsets: host array of n + 1 amplitude offsets; chain k's
 *   state occupies [offsets[k], offsets[k+1]) of the packed state buffer
 *   (each offset a multiple of 32 amplitudes; offsets[n] is the total).
 * osmps_ed_batch_lanczos_ground: psi (device, packed, offsets as above) holds
 *   the start vectors on entry (any non-zero vectors) and the normalised
 *   ground states on return.  energy, residual (doubles), iters and status
 *   (ints) are DEVICE arrays of n entries: the lowest Ritz value, the true
 *   residual |H x - theta x| of the returned state, the Lanczos steps taken,
 *   and the chain's osmps_status (OSMPS_ENOCONV when max_iter steps did not
 *   bring beta_{j+1} |y_j| below tol; the best Ritz pair is still returned).
 *   The call only enqueues work on the handle's stream (a memset and one
 *   kernel launch; with osmps_ed_batch_set_graph(b, 1) one CUDA graph launch)
 *   and allocates nothing, so it may itself be captured into a CUDA graph.
 * osmps_ed_batch_check: synchronises the stream; OSMPS_ETIMEOUT if a bounded
 *   device wait of the last solve gave up (chains then carry OSMPS_ETIMEOUT).
 */
typedef struct osmps_ed_batch osmps_ed_batch_t;
osmps_status osmps_ed_batch_create(int n, const int *L, const double *J, const double *alpha, const double *h,
                                   int prec, int max_iter, void *cuda_stream, osmps_ed_batch_t **out);
osmps_status osmps_ed_batch_destroy(osmps_ed_batch_t *b);
osmps_status osmps_ed_batch_offsets(const osmps_ed_batch_t *b, uint64_t *offsets);
osmps_status osmps_ed_batch_device_bytes(const osmps_ed_batch_t *b, uint64_t *bytes);
osmps_status osmps_ed_batch_set_graph(osmps_ed_batch_t *b, int enable);
/*
 * Work split (a tuning knob, not from the paper).  csize = 1 (the default):
 * every CTA solves one chain at a time.  csize = 2, 4 or 8: the launch uses
 * thread-block clusters of csize CTAs; the chains with L >= lsplit are solved
 * first, each by a whole cluster (tiles and vector ranges split over its CTAs,
 * reductions through distributed shared memory), then the others one per CTA,
 * so that a few long chains do not leave one SM working alone at the end.
 * lsplit must satisfy lsplit >= 11 + log2(csize) (+1 for OSMPS_MIXED) and
 * lsplit <= 22.  EUNSUPPORTED if no cluster of that size fits.
 * osmps_ed_batch_autotune times one solve per candidate (csize 1; csize 2, 4,
 * 8 with lsplit = Lmax-2 .. Lmax) on the given start vectors, keeps the
 * fastest split and restores psi to the start vectors; best_ms (may be NULL)
 * receives its device time.  It allocates a copy of psi and synchronises.
 */
osmps_status osmps_ed_batch_set_split(osmps_ed_batch_t *b, int csize, int lsplit);
osmps_status osmps_ed_batch_get_split(const osmps_ed_batch_t *b, int *csize, int *lsplit, int *grid);
osmps_status osmps_ed_batch_autotune(osmps_ed_batch_t *b, void *psi, double tol, double *best_ms);
osmps_status osmps_ed_batch_lanczos_ground(osmps_ed_batch_t *b, void *psi, double tol, double *energy,
                                           double *residual, int *iters, int *status);
osmps_status osmps_ed_batch_check(osmps_ed_batch_t *b);
osmps_status osmps_ed_batch_launch_count(const osmps_ed_batch_t *b, int64_t *count);

/*
 * Two-site gates (quantum cellular automata and gates, App. C): applies the
 * ngates 4 x 4 complex matrices U[32 i .. 32 i + 31] (row-major, (re, im)
 * interleaved, basis index 2 sigma_s + sigma_{s+1} with sigma = 0 for up) to
 * the bonds (site[i], site[i] + 1), 1 <= site[i] <= L-1, in place.  The bonds
 * must be pairwise disjoint (one layer; the gates then commute).  Gates need
 * not be unitary.  Requires L >= 4 (EUNSUPPORTED otherwise).  Enqueues only.
 */
osmps_status osmps_ed_apply_gates(osmps_ed_t *ed, void *psi, int ngates, const int *site, const double *U);

/*
 * psi <- (Trotter product)^nsteps psi for a nearest-neighbour chain (Sec.
 * III.C): H = H_o + H_e, the bonds (s, s+1) with s odd and with s even, each
 * site field weighted 1/2 in each layer (the first and last site 1, open
 * chain); the layer exponentials are exact two-site propagators.
 *   order 1  Eq. trotter1: exp(-i dt H_o) exp(-i dt H_e)
 *   order 2  Eq. trotter2: exp(-i dt/2 H_e) exp(-i dt H_o) exp(-i dt/2 H_e)
 *   order 4  Eqs. trotter4, trotter4c (eleven layers per step).
 * EUNSUPPORTED for couplings beyond the nearest neighbour or L < 4.
 * Enqueues only.
 */
osmps_status osmps_ed_trotter_evolve(osmps_ed_t *ed, void *psi, double dt, int nsteps, int order);

/*
 * Reduced density matrices of every pair of sites (Sec. IV: trace out the
 * other L-2 indices of the rank-L tensor), i.e. all two-point Pauli
 * correlators <s^a_i s^b_j> = Tr(s^a (x) s^b rho_ij):
 *     rho_ij[v'][v] = sum_rest psi(v', rest) conj(psi(v, rest)),  v = 2 sigma_i + sigma_j
 * (sigma = 0 for up).  rdm2: host, L(L-1)/2 matrices of 4 x 4 complex ((re, im),
 * row-major), pairs ordered (1,2), (1,3), ..., (1,L), (2,3), ..., (L-1,L); or NULL.
 * rdm1: host, L matrices of 2 x 2 complex (the one-site RDMs, partial traces of
 * the pair RDMs); or NULL.  L >= 2.  FP64 reductions.  Allocates its scratch
 * for the call.  Synchronises.
 */
osmps_status osmps_ed_rdm_pairs(osmps_ed_t *ed, const void *psi, double *rdm2, double *rdm1);

/*
 * Bond entropy of every cut: S[l-1] = S(sites 1..l | l+1..L) for l = 1..L-1
 * (Sec. IV bond entropy, Sec. V), each as osmps_ed_schmidt_entropy.  Synchronises.
 */
osmps_status osmps_ed_entropy_sweep(osmps_ed_t *ed, const void *psi, double *S);

/* Static description of a status code. */
const char *osmps_ed_strerror(osmps_status status);

#ifdef __cplusplus
}
#endif

#endif /* OSMPS_ED_H */
