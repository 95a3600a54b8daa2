/*
 * cvsadc.h -- C ABI of libcvsadc, a GB300 (sm_103a) implementation of the
 * hot path of Cholesky-decomposed two-component CVS-ADC(2) for L-edge core
 * excitations over complex spinors (arXiv 2604.27451).
 *
 * Problem statement (section "Implementation and Computational Details"
 * and section "Core-Valence Separation (CVS)"): spinor energies, complex
 * Cholesky vectors B^P_pq, the core / valence / virtual partition and the
 * dipole matrices go in; the lowest CVS-ADC(2) excitation energies
 * (Eq. 11, M X = X Omega), their eigenvectors and oscillator strengths
 * (f = 2/3 omega |T|^2, section "Properties in ISR formulation") come out.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Spinor order: [core | valence | virtual], n = ncore + nval + nvirt.
 *   Frozen core is already removed: every occupied spinor is correlated.
 * Complex numbers: interleaved (re, im) double pairs, i.e. C99 double
 *   complex / numpy complex128 layout.
 * eps : [n] double, canonical spinor energies (Fock matrix = diag(eps)).
 * B   : [naux][n][n] complex, row-major, B[P][p][q] = B^P_pq; every B^P
 *   must be Hermitian (B^P_pq = conj(B^P_qp)); two-electron integrals are
 *   (pq|rs) = sum_P B^P_pq B^P_rs and <pq||rs> = (pr|qs) - (ps|qr).
 * dip : [3][n][n] complex, each Hermitian; d_pq = <p|mu_x|q>.
 * CVS packed vectors (length N = N1 + N2):
 *   singles s = I*nvirt + a                              (N1 = ncore*nvirt)
 *   doubles N1 + (I*nval + j)*npair + pair(a,b), a < b  (npair = nvirt(nvirt-1)/2,
 *     pair(a,b) = a*(2*nvirt-a-1)/2 + (b-a-1),          N2 = ncore*nval*npair)
 *   basis vectors a_a^+ a_I |Phi0> and a_a^+ a_b^+ a_I a_j |Phi0>, the
 *   operator order of the CVS section.
 * Ownership: the caller owns every buffer it passes; the library copies or
 *   reads inputs and writes outputs, and never keeps a caller pointer after
 *   a call returns.  The context owns its device workspaces.
 * Memory space: pointers are host memory unless CVSADC_FLAG_DEVICE_PTRS is
 *   set in params->flags, in which case every array argument of that call
 *   is device memory on the context's device.
 * Errors: every int-returning function returns CVSADC_OK (0) on success, a
 *   negative code on failure (nothing is written to outputs except where
 *   stated), or CVSADC_ENOTCONV (> 0) when the eigen-solver hit max_iter
 *   (outputs then hold the best estimate).  No exception crosses the ABI.
 * Threads/streams: one context per host thread; all work is issued on the
 *   context's stream and every call returns after that stream is synchronised.
 *   Device inputs are read on the context's stream with no wait on any other
 *   stream: the caller makes them ready first (a non-blocking context stream
 *   is not ordered after work still running on another stream).
 * Units: Hartree.
 */
#ifndef CVSADC_H
#define CVSADC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define CVSADC_OK 0
#define CVSADC_EINVAL (-1)     /* bad sizes, partition or argument */
#define CVSADC_ENONHERM (-2)   /* B^P or a dipole matrix not Hermitian */
#define CVSADC_ENOMEM (-3)     /* device allocation failed */
#define CVSADC_ECUDA (-4)      /* CUDA runtime/driver error */
#define CVSADC_ETIMEOUT (-5)   /* a bounded device wait gave up */
#define CVSADC_ESTATE (-6)     /* call order: no prepared problem */
#define CVSADC_ENOTCONV 1      /* max_iter reached, best estimate returned */

/* ----------------------------------------------------------- precision */
#define CVSADC_FP64 0          /* complex128 throughout, FP64 FMA GEMMs */
#define CVSADC_MIXED_BF16X3 1  /* Davidson sigma GEMMs on tcgen05 tensor
                                  cores: each real value split into bf16
                                  hi + lo, three products kept, FP32
                                  accumulation in tensor memory; the
                                  accumulation limits the error to ~1e-5
                                  relative at K ~ 10^3-10^4, so the problem
                                  itself (t2, M11, couplings, moments) is
                                  built with the FP64-class 7-slice product */
#define CVSADC_MIXED_SLICE4 2  /* tensor-core GEMMs on exact integer slices:
                                  per-row/column power-of-two scales, four
                                  7-bit slices per value (10 slice products),
                                  exact FP32 runs of <= 1024 products drained
                                  to float-float accumulators: error ~2^-28
                                  of (row max x column max) */
#define CVSADC_FP64_SLICE7 3   /* as SLICE4 with seven slices (28 products):
                                  FP64-class accuracy on the tensor cores.
                                  In every precision the denominators, the
                                  subspace eigensolve and the final residual
                                  correction run in FP64; the Davidson inner
                                  products, Gram-Schmidt and norms run in
                                  FP64 for CVSADC_FP64 and FP64_SLICE7 and in
                                  double-float on the FP32 pipes for the two
                                  mixed modes (products within ~2^-46 of
                                  |a||b|, tiles summed in FP64) */

/* ---------------------------------------------------------------- flags */
#define CVSADC_FLAG_DEVICE_PTRS 1  /* array arguments are device pointers */
#define CVSADC_FLAG_RETURN_X 2     /* write eigenvectors to X */
#define CVSADC_FLAG_NO_REFINE 4    /* mixed path: skip the FP64 residual
                                      correction sweep */
#define CVSADC_FLAG_FOLDED 16      /* the doubles-folded solver (singles-
                                      space vectors only; see cvsadc_solve);
                                      chosen without this flag when the
                                      full-space subspace would not fit */
#define CVSADC_FLAG_DIAG_PRECOND 8 /* Davidson with the diagonal
                                      preconditioner only (no Schur
                                      complement) */

typedef struct {
  int32_t ncore, nval, nvirt, naux;
  int32_t nroots;         /* lowest nroots eigenvalues of the CVS-ADC(2) matrix */
  int32_t precision;      /* CVSADC_FP64, _MIXED_BF16X3, _MIXED_SLICE4,
                             _FP64_SLICE7 */
  double fns_threshold;   /* tau for frozen natural spinors; <= 0 keeps all virtuals */
  double conv_residual;   /* Davidson convergence, 2-norm of M x - w x; default 1e-6 */
  int32_t max_iter;       /* default 400: roots dominated by strongly coupled
                             doubles can take a few hundred iterations */
  int32_t max_subspace;   /* default max(8 nroots, 48) */
  int32_t flags;          /* CVSADC_FLAG_* */
  int32_t refine_sweeps;  /* mixed precision: FP64 residual-correction
                             iterations after the mixed Davidson (which stops
                             at max(conv_residual, 3e-4) for BF16X3 and
                             max(conv_residual, 1e-6) for SLICE4); each
                             costs one FP64-class sigma per unconverged
                             root; default 20 (stops when converged) */
} cvsadc_params;

typedef struct {
  int32_t iterations;      /* Davidson iterations */
  int32_t sigma_vectors;   /* single-vector sigma builds done */
  int32_t nvirt_kept;      /* virtuals after FNS truncation */
  int32_t converged;       /* number of converged roots */
  double emp2;             /* MP2 correlation energy (final basis) */
  double max_residual;     /* max over roots of ||M x - w x|| */
  double t_prepare_ms;     /* t2 + FNS + M11 + transition moments */
  double t_davidson_ms;    /* Davidson iterations */
  double t_refine_ms;      /* FP64 residual correction */
  double t_total_ms;
  double t_sigma_ms;       /* device time of the sigma builds (CUDA events) */
  double t_schur_ms;       /* building the Schur-complement preconditioner */
  double schur_theta;      /* its trial energy theta0 (0: not used) */
  int32_t coupling_vectors;/* one-sided coupling products M21 x1 or M12 x2
                              done by the preconditioner (two make one
                              sigma's worth of work) */
  int32_t schur_builds;    /* S(theta) evaluations of the theta0 search */
} cvsadc_info;

typedef struct cvsadc_ctx cvsadc_ctx;

/* Create a context on CUDA device `device`.  `cuda_stream` is a
 * cudaStream_t (NULL: the context creates its own non-blocking stream).
 * Returns CVSADC_EINVAL for a bad device, CVSADC_ECUDA on runtime errors. */
int cvsadc_create(cvsadc_ctx** ctx, int device, void* cuda_stream);

/* Release every device buffer and the context.  NULL is accepted. */
void cvsadc_destroy(cvsadc_ctx* ctx);

/* Human-readable text for a status code (static storage). */
const char* cvsadc_strerror(int status);

/* Text of the last error recorded on ctx (static per context). */
const char* cvsadc_last_error(cvsadc_ctx* ctx);

/* --------------------------------------------------------------------
 * cvsadc_solve -- the whole path in one call.
 * Section "Implementation and Computational Details": MP2 amplitudes from
 * the Cholesky vectors, optional frozen-natural-spinor truncation (Eqs.
 * 15, 17-20) with rotation of B^P, the CVS-ADC(2) matrix (Eqs. 11-12 under
 * the CVS restriction), a Davidson eigensolver, and transition moments
 * through first order with oscillator strengths.  The Davidson solver is
 * preconditioned with the Schur complement S(theta0) of the diagonal M22
 * block (see cvsadc_get_schur; info->schur_theta reports theta0) when the
 * singles space has at most 4096 elements and the lowest root lies below
 * every M22 entry; CVSADC_FLAG_DIAG_PRECOND selects the diagonal
 * preconditioner instead.  The preconditioner changes the iteration, not
 * the converged roots.  When the full-space Davidson subspace would not fit
 * on the device, or with CVSADC_FLAG_FOLDED, the doubles-folded solver runs
 * instead: a Rayleigh-Ritz of M over singles vectors lifted with
 * (w - M22)^-1 M21 (exact because M22 is diagonal, Eqs. 11-12), which
 * stores no doubles vector; above 4096 singles its preconditioner is the
 * lowest 64 eigenpairs of S(theta0).  The full eigenvectors (X) and the
 * oscillator strengths are rebuilt from the converged singles.
 *   omega : [nroots] out, ascending excitation energies (Eh)
 *   X     : [nroots][N] complex out (CVS packed, in the final basis) or NULL;
 *           written only with CVSADC_FLAG_RETURN_X.  The largest-modulus
 *           component of each vector is made real and positive.
 *   osc   : [nroots] out or NULL (requires dip)
 *   dip   : may be NULL (no oscillator strengths)
 *   info  : may be NULL
 * Errors: EINVAL (sizes, nroots > N, NULL required pointer), ENONHERM
 * (B or dip not Hermitian to 1e-12 of its largest entry), ENOMEM, ECUDA.
 */
int cvsadc_solve(cvsadc_ctx* ctx, const cvsadc_params* params,
                 const double* eps, const void* B, const void* dip,
                 double* omega, void* X, double* osc, cvsadc_info* info);

/* --------------------------------------------------------------------
 * cvsadc_grad -- gradient of E = sum of the selected lowest roots.
 * Because M is Hermitian and the eigenvectors are normalised, dE/dtheta =
 * sum_n x_n^H (dM/dtheta) x_n (Hellmann-Feynman); the library builds the
 * problem in FP64 (no dipoles, no FNS: tau must be <= 0), finds the roots
 * with the sigma of params->precision (the tensor-core precisions followed
 * by the FP64-class refinement, as in cvsadc_solve), then runs an FP64
 * adjoint pass through every contraction of M -- the M11 pieces, the MP2
 * amplitudes t2 (with their energy denominators, from the stored <ab||ij>)
 * and the B^P couplings.
 *   root_mask : [nroots] 0/1 (NULL: all roots) -- which roots are summed
 *   omega     : [nroots] out, the roots
 *   grad_eps  : [n] out, dE/deps
 *   grad_B    : [naux][n][n] complex out, dE/dRe B + i dE/dIm B, projected on
 *               Hermitian matrices (each B^P is constrained Hermitian); for a
 *               Hermitian perturbation dB, dE = Re sum conj(grad_B) dB.
 * Memory space per params->flags.  Errors: EINVAL (tau > 0, bad mask),
 * ENOTCONV (Davidson did not converge to conv_residual, default 1e-8),
 * ENOMEM, ECUDA. */
int cvsadc_grad(cvsadc_ctx* ctx, const cvsadc_params* params,
                const double* eps, const void* B, const int32_t* root_mask,
                double* omega, double* grad_eps, void* grad_B);

/* --------------------------------------------------------------------
 * cvsadc_solve_batched -- many independent problems of uneven size.
 * Each instance i is what cvsadc_solve(params[i], eps[i], B[i], dip[i],
 * omega[i], X[i], osc[i], &info[i]) computes (the paper solves one
 * molecule at a time; batching is this library's addition).  The
 * instances run on `lanes` worker contexts (0: 4), each with its own
 * non-blocking stream and host thread, created on ctx's device at the
 * first call and kept by ctx.  Instances are taken largest first and one is
 * started when its estimated footprint (cvsadc_estimate_bytes) fits next to
 * the running ones within 90 % of the device memory free at the call, or
 * when nothing else runs; one that runs out of memory beside others is
 * retried alone.  Which lane runs an instance, and when, does not change
 * its result.
 *   dip, X, osc, info, status : may be NULL (as a whole); entries of dip, X
 *                               and osc may be NULL as in cvsadc_solve
 *   status : [ninst] out, each instance's cvsadc_solve status
 * Device inputs must be ready before the call (the lanes' streams wait on
 * nothing).  Returns OK, ENOTCONV if any instance did not converge, or the
 * first instance's negative error (cvsadc_last_error names it); every
 * instance is attempted either way. */
int cvsadc_solve_batched(cvsadc_ctx* ctx, int32_t ninst,
                         const cvsadc_params* params, const double* const* eps,
                         const void* const* B, const void* const* dip,
                         double* const* omega, void* const* X,
                         double* const* osc, cvsadc_info* info, int32_t* status,
                         int32_t lanes);

/* Upper estimate of the device bytes one cvsadc_solve of `params` holds at
 * its peak (inputs, the t2 / <ab||ij> band buffers, M11, the eigensolver's
 * vectors, the sigma intermediates of the largest group, the
 * preconditioner, the tensor-core workspace and the kept operand packs),
 * computed on the host without a GPU.  Without CVSADC_FLAG_FOLDED it prices
 * the full-space Davidson subspace; the solve itself switches to the
 * doubles-folded solver when that subspace does not fit on the device, and
 * with the flag set the estimate prices that solver.  Errors: EINVAL for
 * invalid params. */
int cvsadc_estimate_bytes(const cvsadc_params* params, int64_t* bytes);

/* Device bytes the buffers of ctx hold now (they persist between calls and
 * are reused; the worker contexts of cvsadc_solve_batched are not counted).
 * Errors: EINVAL for NULL arguments. */
int cvsadc_device_bytes(cvsadc_ctx* ctx, int64_t* bytes);

/* --------------------------------------------------------------------
 * Stage entry points.  cvsadc_prepare runs everything before the
 * eigen-solver and keeps the result in ctx; the calls below it then use
 * that prepared problem (CVSADC_ESTATE if there is none).
 */

/* MP2 amplitudes, MP2 energy and (if tau > 0) the FNS truncation with the
 * rotation of B^P, then the M11 block and the transition moments.  The
 * dipole pointer may be NULL.  Section "Implementation and Computational
 * Details", Eqs. 15 and 17-20. */
int cvsadc_prepare(cvsadc_ctx* ctx, const cvsadc_params* params,
                   const double* eps, const void* B, const void* dip,
                   cvsadc_info* info);

/* Sizes of the prepared problem: nvirt after truncation, N1, N2. */
int cvsadc_prepared_sizes(cvsadc_ctx* ctx, int32_t* nvirt, int64_t* N1,
                          int64_t* N2);

/* MP2 amplitudes of the prepared problem, t[i][j][a][b] = t^{ab}_{ij} =
 * <ab||ij>/(e_i+e_j-e_a-e_b), [o][o][v][v] complex (o = ncore+nval, v =
 * nvirt after truncation), and E_MP2 = 1/4 sum <ij||ab> t^{ab}_{ij}.
 * t2 may be NULL.  Memory space per `flags` (CVSADC_FLAG_DEVICE_PTRS). */
int cvsadc_get_t2(cvsadc_ctx* ctx, int32_t flags, void* t2, double* emp2);

/* The explicit core-singles block M11 [N1][N1] complex (row-major). */
int cvsadc_get_m11(cvsadc_ctx* ctx, int32_t flags, void* m11);

/* FNS results of the prepared problem: occupations [nvirt_in] (descending)
 * and U [nvirt_in][nvirt_kept] complex; either may be NULL.  Only valid
 * when the problem was prepared with tau > 0. */
int cvsadc_get_fns(cvsadc_ctx* ctx, int32_t flags, double* occ, void* U);

/* The singles block with the doubles folded in at a trial energy theta,
 * S(theta) = M11 + M12 (theta - M22)^-1 M21, [N1][N1] complex (row-major),
 * computed in FP64 from the prepared problem.  Exact because M22 is
 * diagonal: an eigenvalue w of M below every M22 entry is an eigenvalue of
 * S(w).  The Davidson solver uses S(theta0) as its preconditioner (see
 * cvsadc_info.schur_theta); this call exposes it for inspection and tests.
 * theta must differ from every M22 entry.  Memory space per `flags`. */
int cvsadc_get_schur(cvsadc_ctx* ctx, double theta, int32_t flags, void* S);

/* Modified transition moments F [3][N] complex, through first order. */
int cvsadc_get_moments(cvsadc_ctx* ctx, int32_t flags, void* F);

/* sigma = M x for nvec CVS-packed vectors x [nvec][N] complex, written to
 * sigma [nvec][N].  precision: any CVSADC_FP64 / CVSADC_MIXED_* (the
 * couplings M12 and M21 are contracted through B^P; M22 is applied on the
 * fly; M11 x1 is a dense product).  With the tensor-core precisions the
 * packed slices of the products' operands that are fixed views of B^P are
 * kept in ctx after the first call (at most min(35 % of the free device
 * memory, 64 GB)); preparing another problem releases them. */
int cvsadc_sigma(cvsadc_ctx* ctx, int32_t precision, int32_t flags,
                 const void* x, void* sigma, int32_t nvec);

/* Plain complex GEMM with the library's engines: C = A B for row-major
 * complex matrices A [M][lda], B [K][ldb], C [M][ldc] (interleaved
 * complex128).  precision CVSADC_FP64 runs the FP64 FMA kernel;
 * the mixed modes the tcgen05 kernels (see the precision constants) when
 * the product is large enough to pay for its operand packing, else the
 * FP64 kernel.  Memory space per `flags`.  Errors:
 * EINVAL (sizes, leading dimensions), ETIMEOUT (a bounded device wait of
 * the tensor-core kernel expired), ENOMEM, ECUDA. */
int cvsadc_zgemm(cvsadc_ctx* ctx, int32_t precision, int32_t flags,
                 int32_t M, int32_t N, int32_t K, const void* A, int64_t lda,
                 const void* B, int64_t ldb, void* C, int64_t ldc);

/* Number of CUDA kernels this library has launched in this process (all
 * contexts); a counter for launch accounting, never reset. */
int64_t cvsadc_launch_count(void);

/* Kernel timing for measurement: when enabled, every launch of the main
 * GEMM kernels is bracketed by CUDA events on its stream.  kernel: 0 =
 * tcgen05 BF16X3 GEMM, 1 = tcgen05 exact-slice GEMM, 2 = FP64 FMA GEMM.
 * cvsadc_kernel_stats returns the launches, summed device milliseconds and
 * summed algorithmic flops (8 M N K per complex GEMM) recorded since the
 * last reset (synchronising the recorded events).  Process-wide. */
void cvsadc_kernel_timing(int32_t enable);
int cvsadc_kernel_stats(int32_t kernel, int64_t* launches, double* ms,
                        double* flops);
void cvsadc_kernel_stats_reset(void);

/* The error path of the bounded device waits, on demand (the paper has no
 * counterpart: a service for failure handling).  Every wait inside the
 * library's kernels (mbarrier phases of the tensor-core pipelines) gives up
 * after 4 s of the GPU's global timer, records a code and lets its kernel
 * return, so that a stuck pipeline surfaces as CVSADC_ETIMEOUT instead of a
 * hang.  This call runs one such wait on an mbarrier that nothing arrives
 * on, with limit_ns (clamped to [1 ms, 4 s]), on the context's stream.
 * Returns CVSADC_ETIMEOUT (the wait expired, the context stays usable and
 * its error flag is cleared), CVSADC_EINVAL for a NULL context, or
 * CVSADC_ECUDA. */
int cvsadc_wait_probe(cvsadc_ctx* ctx, int64_t limit_ns);

/* --------------------------------------------------------------------
 * Allocation-free small-output GEMM.  The paper has no counterpart: this
 * is a service for callers that must not let a library allocate device
 * memory -- a process whose device memory is already reserved by another
 * allocator (a framework's caching allocator, a pre-sized pool), where an
 * extra cudaMalloc fails or fragments that pool, or a latency-sensitive
 * loop that cannot take the implicit synchronisation of cudaMalloc and
 * cudaFree.
 *
 * C = A B, complex128, row-major, all three device pointers on the current
 * device: A [M][lda], B [K][ldb], C [M][ldc], with M * N <= 4096 and
 * M + N <= 384 (e.g. an ncore x nvirt block contracted over a long K).
 * Computed by the FP64 FMA kernels of cvsadc_zgemm (FP64 precision) on
 * cuda_stream (NULL: the legacy default stream); returns after that stream
 * is synchronised.
 *
 * No allocation: the split-K partial products live in a fixed 8 MiB device
 * array compiled into the library (every GPU that loads the library holds
 * it until the process exits).  The first call on a device looks up that
 * array's device address for the current device (cudaGetSymbolAddress) and
 * sets a kernel attribute, so make that first call on each device before
 * any stream capture begins; no call makes a cudaMalloc, cudaFree or
 * allocating library routine.  All calls on a device share the array, so calls that
 * overlap on the GPU (other streams or host threads) race on it: serialise
 * them.  Each call writes every partial it reads, so nothing carries over.
 * Errors: CVSADC_EINVAL for NULL pointers, non-positive sizes, a product
 * beyond the limits above, or a leading dimension smaller than its row
 * length (lda < K, ldb < N or ldc < N); CVSADC_ECUDA for a CUDA error. */
#define CVSADC_NOALLOC_MAX_MN 4096
#define CVSADC_NOALLOC_MAX_M_PLUS_N 384
int cvsadc_zgemm_small_noalloc(void* cuda_stream, int32_t M, int32_t N,
                               int32_t K, const void* A, int64_t lda,
                               const void* B, int64_t ldb, void* C,
                               int64_t ldc);

/* Broadened spectrum (sections "Computational Details" and "Results and
 * Discussion": computed spectra are sums of Lorentzian lines of a given
 * FWHM, 0.3 eV in most figures, moved by one uniform energy shift to align
 * an edge with experiment):
 *   out[g] = sum_n osc[n] L(E_g - (omega[n] * 27.211386245988 + shift_ev)),
 *   E_g = e0_ev + g de_ev (g < npts),
 *   L(x) = (h / pi) / (x^2 + h^2), h = fwhm_ev / 2 (unit area).
 * omega [nroots] in Hartree (as cvsadc_solve returns them), osc [nroots],
 * out [npts]; host pointers unless flags has CVSADC_FLAG_DEVICE_PTRS.
 * Computed on the context's stream.  Errors: CVSADC_EINVAL for NULL arrays
 * with positive sizes, negative sizes or fwhm_ev <= 0; CVSADC_ECUDA. */
int cvsadc_spectrum(cvsadc_ctx* ctx, int32_t flags, int32_t nroots, const double* omega,
                    const double* osc, double e0_ev, double de_ev, int32_t npts,
                    double fwhm_ev, double shift_ev, double* out);

/* Block inner products out[i][j] = sum_n conj(A[i][n]) B[j][n] (i < ma,
 * j < mb; out host [ma][mb] complex128) of device vectors A [ma][N] and
 * B [mb][N] (complex128, on the context's device), in the arithmetic the
 * Davidson solver uses for `precision`: plain FP64 for CVSADC_FP64 and
 * CVSADC_FP64_SLICE7 (Gram matrices, Gram-Schmidt, Ritz combinations);
 * double-float on the FP32 pipes for the mixed precisions (float hi/lo
 * pairs, ~48-bit significand and the float exponent range, tiles of 16
 * terms summed in FP64).  The section "Implementation and Computational
 * Details" names Davidson; this exposes its inner product so that callers
 * can check the arithmetic.  Errors: CVSADC_EINVAL for NULL pointers or
 * non-positive sizes; CVSADC_ECUDA. */
int cvsadc_block_dot(cvsadc_ctx* ctx, int32_t precision, const void* A,
                     int32_t ma, const void* B, int32_t mb, int64_t N, void* out);

/* Davidson on the prepared problem (see cvsadc_solve for outputs). */
int cvsadc_davidson(cvsadc_ctx* ctx, const cvsadc_params* params,
                    double* omega, void* X, double* osc, cvsadc_info* info);

#ifdef __cplusplus
}
#endif
#endif /* CVSADC_H */
