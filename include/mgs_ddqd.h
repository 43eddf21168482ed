/*
 * mgs_ddqd.h -- C ABI of the GB300 (sm_103a) complex double-double / quad-double
 * modified Gram-Schmidt least-squares library.
 *
 * Method: Verschelde & Yoffe, "Orthogonalization on a General Purpose Graphics Processing
 * Unit with Double Double and Quad Double Arithmetic".
 *
 * Number format.  A real number is L float64 limbs (L = 1: double, L = 2: double-double,
 * L = 4: quad-double) whose exact sum is its value, largest limb first.  A complex element is
 * 2L consecutive doubles {re_0..re_{L-1}, im_0..im_{L-1}} (32 bytes for DD, 64 for QD).
 * Matrices are column-major BY ELEMENT: element (i, j) of a matrix with leading
 * dimension ld starts at base + (j * ld + i) * 2L doubles.  Vectors are contiguous.
 *
 * Memory.  Every pointer is a DEVICE pointer into memory the caller owns (for example
 * a PyTorch float64 CUDA tensor) and must be 16-byte aligned.  The library allocates
 * nothing: scratch memory is the caller's `workspace` of at least
 * mgs_workspace_bytes(...) bytes, valid for the duration of the call on `stream`.
 *
 * Execution.  Calls are stream-ordered and asynchronous: they enqueue work on `stream`
 * (a cudaStream_t; NULL = the legacy default stream) and return without synchronising.
 * The return value reports only what the host can detect (bad arguments, a CUDA launch
 * failure).  What is found while the solve runs is written to *dev_status (one int32 in
 * device memory, reset to MGS_OK by the call): MGS_ERANK, MGS_ENONFINITE or
 * MGS_ETIMEOUT.  The first error recorded wins.  Outputs are unspecified when the
 * status is not MGS_OK.  No exception crosses the ABI.
 *
 * Concurrency.  A single-system call occupies the whole GPU with one persistent launch
 * of at most one CTA per SM whose CTAs wait for one another (a cooperative launch, or a
 * launch of thread-block clusters whose residency the library checks first); calls on
 * the same stream run one after another.  Issue single-system calls on one stream at a
 * time: a launch that finds SMs occupied by another call's kernel waits for them when it
 * is cooperative, and a cluster launch captured into a CUDA graph (which cannot carry the
 * cooperative attribute) would find its waits running out and report MGS_ETIMEOUT rather
 * than hang.  A workspace must not be shared by calls that may run at the same time.  The first call for a given size and device queries the
 * device (occupancy); make it before capturing calls into a CUDA graph.
 */
#ifndef MGS_DDQD_H
#define MGS_DDQD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes (host return values and the device status word). */
#define MGS_OK 0         /* success */
#define MGS_EINVAL 1     /* host: invalid argument (null or misaligned pointer, m < n, n < 1, ld < m, ...) */
#define MGS_ERANK 2      /* device: some r_kk is zero or not finite -- the method does not pivot (Section 4) */
#define MGS_ENONFINITE 3 /* device: an input limb is Inf or NaN */
#define MGS_ETIMEOUT 4   /* device: a wait between CTAs ran out of time; the kernel returned early */
#define MGS_ECUDA 5      /* host: a CUDA call failed; mgs_last_cuda_error() returns its cudaError_t */
#define MGS_ENOSPACE 6   /* host: workspace too small, or the problem exceeds what one GPU solve holds */

/* Library version (major * 10000 + minor * 100 + patch).  0.2.0 (200): mgs_tune gained the
 * `chunks` field; callers built against 0.1 must be rebuilt. */
int mgs_version(void);

/* Human-readable name of a status code. */
const char* mgs_status_string(int code);

/* cudaError_t of the last call that returned MGS_ECUDA on this host thread. */
int mgs_last_cuda_error(void);

/*
 * Bytes of workspace a call needs on the current device.
 *   limbs    1 (complex double), 2 (DD) or 4 (QD)
 *   m, n     matrix size (m >= n >= 1)
 *   with_rhs 1 for ls_solve_* (augmented [A b]), 0 for mgs_qr_*
 * Returns 0 for unsupported arguments or sizes.
 */
size_t mgs_workspace_bytes(int limbs, int m, int n, int with_rhs);

/*
 * How a single-system call of these sizes is laid out on the current device (no
 * counterpart in the paper; for tests and tuning).  `out` has room for 5 ints.
 *   out[0] Br  row blocks (CTAs per column group), out[1] Bc  column groups,
 *   out[2] h   rows per row block, out[3] kernel:
 *     0  grid-barrier kernel: one grid-wide barrier per elimination step;
 *     1  cluster schedule on hardware thread-block clusters (the Br CTAs of a column
 *        group form one cluster and exchange Gram partials through distributed shared
 *        memory; Br <= 8);
 *     2  the same schedule on software groups (the Br CTAs meet at a counter in global
 *        memory and exchange partials through L2; every SM usable).
 *   The default is 1 for limbs 1 and 2 where the clusters fill at least 90 % of the SMs
 *   a plain grid would use (else 0), and 0 for limbs 4: measured on GB300, the cluster
 *   schedule hides the per-step latency that dominates the cheaper arithmetic, while quad
 *   double, and layouts where clusters leave SMs idle, are bound by FP64 throughput.
 *   The environment variable MGS_KERNEL = grid | cluster | group, read at each call,
 *   forces a kernel (cluster falls back to grid where clusters cannot be formed);
 *   out[4] threads per CTA: 128, or 256 where a CTA owns 16 or more columns (two warps
 *          per SM sub-partition hide each other's FP64 latency in the long loops).
 *   MGS_ROWS = h overrides the rows per row block (default 64); MGS_CTA_THREADS = 128 |
 *   256 the threads per CTA; MGS_CTAS_PER_SM = 1 | 2 how many CTAs of the solve share an
 *   SM (default 1: each has the SM's FP64 unit to itself; 2 doubles the column groups).
 * Returns MGS_OK, MGS_EINVAL or MGS_ENOSPACE (no layout fits shared memory).
 */
int mgs_plan_query(int limbs, int m, int n, int with_rhs, int* out);

/*
 * QR decomposition A = Q R by modified Gram-Schmidt (Section 3, Figure 1): for
 * k = 1..n, r_kk = sqrt(a_k^H a_k), q_k = a_k / r_kk, and for j > k
 * r_kj = q_k^H a_j, a_j = a_j - r_kj q_k, with x^H y = sum_l conj(x_l) y_l.
 *   A        in: m x n matrix (lda >= m); out: Q (Q^H Q = I), overwriting A (Figure 2)
 *   R        out: n x n upper triangle (ldr >= n), diagonal real and positive; the
 *            strictly lower triangle is not written
 *   workspace, workspace_bytes   caller-owned device scratch (see mgs_workspace_bytes)
 *   dev_status  device int32, reset then set as described above
 *   stream   cudaStream_t
 * Host returns: MGS_OK, MGS_EINVAL, MGS_ENOSPACE or MGS_ECUDA.
 */
int mgs_qr_dd(double* A, int lda, double* R, int ldr, int m, int n, void* workspace, size_t workspace_bytes,
              int32_t* dev_status, void* stream);
int mgs_qr_qd(double* A, int lda, double* R, int ldr, int m, int n, void* workspace, size_t workspace_bytes,
              int32_t* dev_status, void* stream);

/*
 * Complex double (L = 1: one FP64 number per real part, element = {re, im}) versions of
 * mgs_qr_* and ls_solve_*: the paper's "complex double" runs (Sections 4 and 8, Tables 2-4),
 * same method, plain IEEE double arithmetic.  Arguments as for the DD versions.
 */
int mgs_qr_d(double* A, int lda, double* R, int ldr, int m, int n, void* workspace, size_t workspace_bytes,
             int32_t* dev_status, void* stream);
int ls_solve_d(double* A, int lda, double* b, double* x, double* R, int ldr, double* z, int m, int n, void* workspace,
               size_t workspace_bytes, int32_t* dev_status, void* stream);

/*
 * Least squares: x minimising ||b - A x||_2 (Section 3): modified Gram-Schmidt on the
 * augmented matrix [A b] = [Q q_{n+1}] [[R y], [0 z]] (Eq. 1), so y = Q^H b and
 * ||b - A x||^2 = ||R x - y||^2 + z^2, followed by the back substitution R x = y of
 * Section 6, Figure 3 (x_k = y_k / r_kk, then y_j -= r_jk x_k for j < k).
 *   A    in: m x n (lda >= m); out: Q
 *   b    in: m-vector; out: the residual b - A x (the reduced last column of Eq. 1)
 *   x    out: n-vector
 *   R    out (optional, may be NULL): n x n upper triangle, ldr >= n when R != NULL
 *   z    out (optional, may be NULL): L doubles, the residual norm z of Eq. 1 (real)
 *   other arguments as for mgs_qr_*.
 * Host returns: MGS_OK, MGS_EINVAL, MGS_ENOSPACE or MGS_ECUDA.
 */
int ls_solve_dd(double* A, int lda, double* b, double* x, double* R, int ldr, double* z, int m, int n,
                void* workspace, size_t workspace_bytes, int32_t* dev_status, void* stream);
int ls_solve_qd(double* A, int lda, double* b, double* x, double* R, int ldr, double* z, int m, int n,
                void* workspace, size_t workspace_bytes, int32_t* dev_status, void* stream);

/*
 * Batched least squares: `batch` independent systems of different sizes in one launch
 * (many paths tracked at once; the paper solves one system at a time, Section 2, and
 * its related work [ASK12] studies many small independent QR factorisations).  Each
 * system is the ls_solve_* of Section 3 (Figure 1, Eq. 1) and Section 6 (Figure 3).
 *   A_pool, b_pool, x_pool   element pools (device); system i uses
 *       A_pool + a_off[i]*2L  (m[i] x n[i], column-major, leading dimension m[i]; Q on exit)
 *       b_pool + b_off[i]*2L  (m[i] elements; the residual on exit)
 *       x_pool + x_off[i]*2L  (n[i] elements, output)
 *   a_off, b_off, x_off  device int64 arrays of element offsets (8-byte aligned)
 *   m, n                 device int32 arrays of sizes (1 <= n[i] <= m[i] <= max_m, n[i] <= max_n)
 *   order                optional device int32 permutation: the order in which systems are
 *                        handed out (largest first balances the work); NULL = 0, 1, 2, ...
 *   dev_status           device int32 array of `batch` words: per-system status
 *                        (MGS_OK, MGS_EINVAL for a bad size, MGS_ERANK, MGS_ENONFINITE)
 *   tune                 optional launch shape (NULL or zero fields = defaults)
 * Workspace: mgs_batched_workspace_bytes(limbs, batch, max_m, max_n, tune).
 * One CTA (or one cluster of `split` CTAs, see mgs_tune) solves one system at a time; no
 * CTA waits for a CTA outside its own cluster.
 */
typedef struct {
  int threads;     /* threads per CTA: 128 or 256 (0 = 256) */
  int ctas_per_sm; /* resident CTAs per SM, 1..4 (0 = 1) */
  int split;       /* CTAs per system, 1, 2 or 4 (0 = automatic: 2 or 4 when the batch is
                      smaller than half or a quarter of the resident CTAs and every slice
                      keeps 32 rows); the CTAs of a system form a thread-block cluster, each
                      holds a slice of the rows, the slices' Gram partials are summed
                      through distributed shared memory */
  int chunks;      /* most lanes that share one (column, part) of a system's Gram row in a
                      step, i.e. rows per lane = ceil(slice rows / chunks): 0 = as many as
                      the threads allow (fewest rows per lane, deepest reduction trees);
                      1..threads caps it (more columns per pass, shallower trees) */
} mgs_tune;

size_t mgs_batched_workspace_bytes(int limbs, int batch, int max_m, int max_n, const mgs_tune* tune);
/* R_pool (optional, may be NULL): packed upper triangle of R of system i at
 * R_pool + r_off[i]*2L, element (k, j), k <= j, at index j(j+1)/2 + k (n(n+1)/2 elements). */
int ls_solve_d_batched(double* A_pool, double* b_pool, double* x_pool, double* R_pool, const int64_t* a_off,
                       const int64_t* b_off, const int64_t* x_off, const int64_t* r_off, const int32_t* m,
                       const int32_t* n, const int32_t* order, int batch, int max_m, int max_n, void* workspace,
                       size_t workspace_bytes, int32_t* dev_status, const mgs_tune* tune, void* stream);
int ls_solve_dd_batched(double* A_pool, double* b_pool, double* x_pool, double* R_pool, const int64_t* a_off,
                        const int64_t* b_off, const int64_t* x_off, const int64_t* r_off, const int32_t* m,
                        const int32_t* n, const int32_t* order, int batch, int max_m, int max_n, void* workspace,
                        size_t workspace_bytes, int32_t* dev_status, const mgs_tune* tune, void* stream);
int ls_solve_qd_batched(double* A_pool, double* b_pool, double* x_pool, double* R_pool, const int64_t* a_off,
                        const int64_t* b_off, const int64_t* x_off, const int64_t* r_off, const int32_t* m,
                        const int32_t* n, const int32_t* order, int batch, int max_m, int max_n, void* workspace,
                        size_t workspace_bytes, int32_t* dev_status, const mgs_tune* tune, void* stream);

/*
 * Adjoint (backward) of the batched least squares: for a real loss with gradient
 * G = dL/dRe(x) + i dL/dIm(x) (PyTorch's convention for complex tensors), the gradients
 * with respect to A and b.  The paper has no backward pass; this differentiates the
 * solve of Section 3 (Eq. 1) and Section 6 through the normal equations A^H A x = A^H b:
 *     u = R^{-H} G,  w = R^{-1} u,  grad_b = A w = Q u,  grad_A = r w^H - grad_b x^H,
 * with Q, R, x and the residual r = b - A x of the forward solve (two triangular solves,
 * one matrix-vector product, one rank-2 update per system; one CTA per system).
 *   Q_pool, x_pool, r_pool  the forward's outputs (A_pool, x_pool and b_pool after the solve)
 *   R_pool, r_off           the forward's packed R (ls_solve_*_batched with R_pool)
 *   G_pool                  gradient of x, laid out like x_pool
 *   gA_pool, gb_pool        outputs, laid out like A_pool and b_pool
 *   workspace               at least 256 bytes (a work-queue counter)
 *   dev_status              per-system status (MGS_ERANK for a zero r_kk)
 */
int ls_adjoint_dd_batched(const double* Q_pool, const double* R_pool, const double* x_pool, const double* r_pool,
                          const double* G_pool, double* gA_pool, double* gb_pool, const int64_t* a_off,
                          const int64_t* r_off, const int64_t* b_off, const int64_t* x_off, const int32_t* m,
                          const int32_t* n, const int32_t* order, int batch, int max_m, int max_n, void* workspace,
                          size_t workspace_bytes, int32_t* dev_status, const mgs_tune* tune, void* stream);
int ls_adjoint_qd_batched(const double* Q_pool, const double* R_pool, const double* x_pool, const double* r_pool,
                          const double* G_pool, double* gA_pool, double* gb_pool, const int64_t* a_off,
                          const int64_t* r_off, const int64_t* b_off, const int64_t* x_off, const int32_t* m,
                          const int32_t* n, const int32_t* order, int batch, int max_m, int max_n, void* workspace,
                          size_t workspace_bytes, int32_t* dev_status, const mgs_tune* tune, void* stream);

/*
 * ls_solve_dd without a caller workspace, for callers that cannot allocate device memory
 * (a host whose device memory is all owned by another allocator, or an application that
 * must not allocate after start-up).  The paper has no counterpart: it is a packaging of
 * ls_solve_dd.  Arguments and results are those of ls_solve_dd minus the workspace, and
 * the results are bit for bit those of ls_solve_dd on the same inputs.
 *   Scratch: a fixed device array of MGS_NOALLOC_WORKSPACE_BYTES inside the library.  With
 *   lazy module loading (the CUDA default) it is reserved on a device when the first call
 *   on that device and context loads the library's module, and it stays until the context
 *   is destroyed (normally at process exit).  No allocation routine is called by this
 *   entry point; make the first call on each device at start-up, before the host's
 *   allocator takes the rest of device memory (or set CUDA_MODULE_LOADING=EAGER), else
 *   that first call can fail with MGS_ECUDA (out of memory).
 *   Sizes whose workspace (mgs_workspace_bytes(2, m, n, 1)) exceeds the array are rejected
 *   with MGS_ENOSPACE before any work (on GB300, m = n <= 346 fits, 347 does not, with the
 *   default kernel choice).
 *   The first call on a device and context looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and caches it for that context; a
 *   device reset or a new context makes the next call look it up again.  Make the first
 *   call before any stream capture.
 *   Every call shares the array: calls that may overlap on the GPU race and must not be
 *   issued.  Each call clears what must start at zero itself.
 */
#define MGS_NOALLOC_WORKSPACE_BYTES (4u * 1024u * 1024u)
int ls_solve_dd_noalloc(double* A, int lda, double* b, double* x, double* R, int ldr, double* z, int m, int n,
                        int32_t* dev_status, void* stream);

/*
 * Newton corrector on the device (Section 7: Newton's method is the corrector of path
 * tracking; the Jacobian and the system stay on the GPU, only solutions go back).  The
 * caller evaluates F(x) and its Jacobian J = F'(x) on the device; this library does not
 * evaluate functions.  One step:
 *   f_norm[i] = ||F||_inf; solve min ||F - J s|| by MGS on [J F] and back substitution
 *   (as ls_solve_*); x <- x - s; dx_norm[i] = ||s||_inf, x_norm[i] = ||x||_inf,
 *   z[i] = ||F - J s||; done = 1 when dx_norm[i] <= tol * x_norm[i].
 * Norms are taken on the leading limbs (|v| = hypot(re_0, im_0)).
 * While done != 0 at the start of a step, the step does nothing (the gate is read on the
 * device), so a whole run of steps can be enqueued, or captured in a CUDA graph, and the
 * host reads the state once at the end.  A solve that reports an error (MGS_ERANK, ...)
 * sets done = 2 and status to that code and leaves x unchanged.
 */
#define MGS_NEWTON_HISTORY 64
typedef struct {
  int32_t done;       /* 0 running, 1 converged, 2 stopped by a solve status */
  int32_t iterations; /* steps taken */
  int32_t status;     /* the solve status that stopped the run (done == 2) */
  int32_t reserved;
  double f_norm[MGS_NEWTON_HISTORY];  /* ||F(x_i)||_inf, as passed to step i */
  double dx_norm[MGS_NEWTON_HISTORY]; /* ||x_{i+1} - x_i||_inf */
  double x_norm[MGS_NEWTON_HISTORY];  /* ||x_{i+1}||_inf */
  double z[MGS_NEWTON_HISTORY];       /* residual of the linearised problem of step i */
} mgs_newton_state;

/* Workspace bytes of newton_step_* (the solve's workspace plus the step s); 0 when
 * unsupported. */
size_t newton_workspace_bytes(int limbs, int m, int n);

/*
 * One gated Newton step (see above).
 *   J          in: m x n Jacobian (ldj >= m), layout of A in ls_solve_*; out: overwritten (Q)
 *   F          in: F(x), m elements; out: overwritten (the linearised residual)
 *   x          in/out: n elements, 16-byte aligned
 *   tol        relative stopping tolerance on the step (>= 0)
 *   dev_state  device mgs_newton_state, 16-byte aligned, zeroed by the caller before the
 *              first step of a run
 *   workspace  newton_workspace_bytes(limbs, m, n) bytes of device memory
 *   dev_status device int32: the status of this step's solve (reset by each step)
 * Host returns: MGS_OK, MGS_EINVAL, MGS_ENOSPACE or MGS_ECUDA.
 */
int newton_step_d(double* J, int ldj, double* F, double* x, int m, int n, double tol, mgs_newton_state* dev_state,
                  void* workspace, size_t workspace_bytes, int32_t* dev_status, void* stream);
int newton_step_dd(double* J, int ldj, double* F, double* x, int m, int n, double tol, mgs_newton_state* dev_state,
                   void* workspace, size_t workspace_bytes, int32_t* dev_status, void* stream);
int newton_step_qd(double* J, int ldj, double* F, double* x, int m, int n, double tol, mgs_newton_state* dev_state,
                   void* workspace, size_t workspace_bytes, int32_t* dev_status, void* stream);

/* ======================================================================================
 * Diagnostics.  Not part of the solve: a measurement hook (the FP64 rate the roofline is
 * quoted against) and a failure-detection hook (a bounded wait run out on purpose).
 * ====================================================================================== */

/*
 * FP64 throughput probe (no counterpart in the paper): launches `blocks` x `threads`
 * threads, each running 8 independent chains of `iters` fused multiply-adds, and writes
 * one double per thread to dev_out (blocks * threads doubles).  The caller times the
 * stream: blocks * threads * iters * 8 FMA lane-operations per launch.  This measures the
 * rate the roofline of the FP64-bound solve is quoted against.
 * Host returns: MGS_OK, MGS_EINVAL or MGS_ECUDA.
 */
int mgs_fp64_probe(double* dev_out, int blocks, int threads, int iters, void* stream);

/* Failure-detection probe (no counterpart in the paper): runs one of the solver kernels'
 * bounded waits on a condition that never comes true, so that it runs out of time and
 * takes the same exit a solve takes when a CTA goes missing.
 *   kind 0: the pivot-ready flag wait, on a flag nothing sets (one CTA);
 *   kind 1: the grid barrier, with one of two CTAs never arriving.
 * dev_words: 4 caller-owned, caller-zeroed device words (4-byte aligned):
 *   [0] arrival counter, [1] abort flag, [2] status, [3] the flag of kind 0.
 * After the kernel: [2] = MGS_ETIMEOUT and [1] = 1 once timeout_ns nanoseconds have
 * passed.  A caller that sets [1] = 1 before the call (an abort raised earlier) sees the
 * wait fall through within 64 polls (tens of microseconds), [2] unchanged.  The GPU
 * context stays usable either way.
 * Stream-ordered, asynchronous.  Host returns: MGS_OK, MGS_EINVAL (null or misaligned
 * words, kind not 0 or 1, timeout_ns outside [1, 1e10]) or MGS_ECUDA.
 */
int mgs_wait_probe(unsigned* dev_words, int kind, long long timeout_ns, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MGS_DDQD_H */
