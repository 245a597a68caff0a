/*
 * ekcg.h - C ABI of the GB300 s-step enlarged Krylov subspace CG library.
 *
 * Method: Moufawad, "Numerical Stability of s-step Enlarged Krylov Subspace Conjugate
 * Gradient methods" (arXiv:1804.10629).
 *   - s-step SRE-CG (Algorithm 4), s-step SRE-CG2 (Algorithm 3), s-step MSDO-CG (Algorithm 6)
 *   - their communication-avoiding forms built with CA-Arnoldi (Algorithm 5) or the
 *     stable modified CA-Arnoldi (Algorithm 7), Section 3 and Section 4
 *   - A-orthonormalisation by CGS2 against previous vectors, then A-CholQR or Pre-CholQR
 *     against itself (Section 3.1, Section 4)
 *
 * Conventions shared by every entry point:
 *   - Status: 0 = EKCG_OK; EKCG_MAXIT (> 0) is a warning, outputs are valid; negative values
 *     are errors (see ekcg_strerror).  A failing call leaves caller buffers in an unspecified
 *     state only where the description says so; it never frees caller memory.
 *   - Ownership: the caller owns every pointer it passes and keeps it alive for the call.
 *     The context owns its device copies of the matrix and all workspace, released by
 *     ekcg_destroy.  No entry point keeps a caller pointer after it returns.
 *   - Memory spaces: "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory on the context's device (for example torch tensor data_ptr()).
 *   - Row order: ekcg_solve takes and returns vectors in the caller's (natural) order.  The
 *     kernel-level entry points (ekcg_split_T, ekcg_spmm, ekcg_permute) work in the
 *     context's permuted order, where the t domains are contiguous.
 *   - Layout of an n x w block of vectors: row-major, element (i, c) at [i*w + c].
 *   - Work is enqueued on the context's stream; calls that return results to the host
 *     synchronise that stream before returning.
 *   - Not thread-safe per context: one host thread drives one context at a time.
 */
#ifndef EKCG_H
#define EKCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define EKCG_OK 0
#define EKCG_MAXIT 1          /* maxit reached before the tolerance: outputs are valid     */
#define EKCG_EINVAL (-1)      /* bad argument: shapes, CSR structure, partition, NaN/Inf   */
#define EKCG_ENOMEM (-2)      /* device memory or stored-basis capacity exhausted          */
#define EKCG_EBREAKDOWN (-3)  /* Cholesky pivot failed the breakdown rule                  */
#define EKCG_ETIMEOUT (-4)    /* reserved: a bounded device wait ran out                   */
#define EKCG_ECUDA (-5)       /* a CUDA runtime call failed (see ekcg_last_error)          */

/* ---- solver options ------------------------------------------------------------- */
#define EKCG_SRE 0    /* s-step SRE-CG  (Algorithm 4): orthonormalise against 2 blocks  */
#define EKCG_SRE2 1   /* s-step SRE-CG2 (Algorithm 3): against all previous blocks       */
#define EKCG_MSDO 2   /* s-step MSDO-CG (Algorithm 6): T(r_{k-1}) starts every iteration  */

#define EKCG_SSTEP 0  /* basis built t vectors at a time (Algorithms 3, 4, 6)             */
#define EKCG_CA5 1    /* CA-Arnoldi A-orthonormalisation (Algorithm 5, monomial, unstable) */
#define EKCG_CA7 2    /* modified CA-Arnoldi A-orthonormalisation (Algorithm 7)           */
#define EKCG_RESTRUCT 3 /* restructured SRE-CG / SRE-CG2 (Algorithms 2, 1): the s-step basis,
                         * then s sequential updates, one per block (SRE and SRE2 only)    */

#define EKCG_ACHOLQR 0    /* A-CholQR: G = W^T A W = R^T R, W <- W R^{-1}                 */
#define EKCG_PRECHOLQR 1  /* Euclidean CholQR2 first, then A-CholQR                       */

#define EKCG_FP64 0       /* all vectors and arithmetic in float64                       */
#define EKCG_FP32_IR 1    /* float32 inner solve in a float64 iterative-refinement loop   */

/* Arithmetic of the float64 tall-skinny contractions (CGS update W - Q C):               */
#define EKCG_CONTRACT_FP64 0   /* float64 fused multiply-adds                             */
#define EKCG_CONTRACT_SPLIT 1  /* float64-accurate split products on the bf16 tensor cores:
                                * eight 7-bit slices per value (56-bit fixed point against
                                * the row / column binade), the 36 slice pairs with
                                * a + b <= 9 summed exactly in fp32 tensor memory, groups
                                * combined in 64-bit integers; error per term about 2^-52 of
                                * max|row| max|column|.  Shapes it does not take (more than
                                * 64 contracted columns per launch, widths other than 16 or
                                * 32) use float64 FMAs.                                     */

typedef struct ekcg_ctx ekcg_ctx;

typedef struct {
    int variant;          /* EKCG_SRE / EKCG_SRE2 / EKCG_MSDO                            */
    int basis;            /* EKCG_SSTEP / EKCG_CA5 / EKCG_CA7 / EKCG_RESTRUCT            */
    int orth;             /* EKCG_ACHOLQR / EKCG_PRECHOLQR                                */
    int precision;        /* EKCG_FP64 / EKCG_FP32_IR                                     */
    int max_s;            /* largest s any solve on this context uses (workspace size)     */
    int max_blocks;       /* stored t-blocks for full-history forms (SRE2, MSDO, CA SRE2);
                             0 = as many as fit in max_basis_bytes                          */
    int64_t max_basis_bytes; /* device bytes for stored basis vectors; 0 = 40% of free    */
    double breakdown_tol; /* Cholesky pivot d_i <= breakdown_tol*|G_ii| stops the solve   */
    double inner_tol;     /* FP32_IR: relative residual reduction of each inner solve      */
    int max_refine;       /* FP32_IR: maximum outer refinement steps                       */
    int profile;          /* 1: time every kernel class with CUDA events (ekcg_profile)   */
    int contraction;      /* EKCG_CONTRACT_FP64 / EKCG_CONTRACT_SPLIT (float64 path)      */
    int deflate;          /* 1: rank-revealing A-CholQR.  A Cholesky pivot that fails the
                             breakdown rule drops its column from the block (zero in W and
                             A W, no update from it) and the solve continues with fewer
                             directions, as enlarged CG deflates dependent search directions
                             (Section 2); only a block whose columns all drop (or a non-finite
                             pivot) is a breakdown.  A-CholQR only; 0 (default): stop.      */
} ekcg_opts;

/* Fill *opts with the defaults: SRE, SSTEP, ACHOLQR, FP64, max_s 8, max_blocks 0,
 * max_basis_bytes 0, breakdown_tol 1e-14, inner_tol 1e-4, max_refine 30, profile 0,
 * contraction EKCG_CONTRACT_SPLIT, deflate 0.                                             */
void ekcg_default_opts(ekcg_opts* opts);

/* Build a solver context for the SPD matrix A (Section 2) and its t-way partition.
 *   n, rowptr[n+1] (int64), colind[nnz] (int32, sorted and unique per row), val[nnz]:
 *     host CSR arrays of A, copied; A must be structurally and numerically symmetric with a
 *     positive diagonal (checked: structure and positive diagonal; values are not).
 *   t (>= 1), part[n]: host array, part[i] in [0, t) is the domain of row i; every domain
 *     must be non-empty.  Rows are stably sorted by domain (Section 4 reordering) and the
 *     matrix is permuted symmetrically on the device.
 *   opts: may be NULL for defaults.  stream: a cudaStream_t (NULL = legacy default stream).
 *   *out receives the context.  Errors: EKCG_EINVAL (bad CSR / partition / options),
 *   EKCG_ENOMEM, EKCG_ECUDA.  Device memory for the workspace is allocated here.          */
int ekcg_setup(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
               int t, const int32_t* part, const ekcg_opts* opts, void* stream,
               ekcg_ctx** out);

/* Solve A x = b (Algorithms 3, 4, 6 and their CA forms, per the context's options).
 *   b, x0, x: device float64 arrays of length n in natural order; x0 may be NULL (x0 = 0)
 *     and may alias x.
 *   s (1 <= s <= opts.max_s), tol (> 0), maxit (>= 0): the loop runs while
 *     ||r_k||_2 > tol*||r_0||_2 and fewer than maxit s-step iterations were done, with r_k
 *     the recursively updated residual.
 *   *iters: s-step iterations performed (FP32_IR: inner s-step iterations, summed).
 *   res_hist: host array of hist_cap doubles (may be NULL) receiving ||r_0||, ||r_1||, ...
 *     (FP32_IR: the float64 residual norm after each refinement step); *hist_len the count.
 *   Returns EKCG_OK, EKCG_MAXIT, EKCG_EBREAKDOWN (x holds the last complete iterate),
 *   EKCG_ENOMEM (stored-basis capacity exceeded; x holds the last iterate), EKCG_EINVAL
 *   (bad sizes, non-finite b), EKCG_ECUDA.                                                 */
int ekcg_solve(ekcg_ctx* ctx, const double* b, const double* x0, int s, double tol,
               int maxit, double* x, int* iters, double* res_hist, int hist_cap,
               int* hist_len);

/* ekcg_solve with host arrays b, x0 (nullable) and x: the host-to-device copy of b (and x0)
 * and the device-to-host copy of x are part of the call.                                 */
int ekcg_solve_host(ekcg_ctx* ctx, const double* b_host, const double* x0_host, int s,
                    double tol, int maxit, double* x_host, int* iters, double* res_hist,
                    int hist_cap, int* hist_len);

/* Release the context and all device memory it owns.  NULL is accepted.                  */
void ekcg_destroy(ekcg_ctx* ctx);

/* Static string for a status code.                                                        */
const char* ekcg_strerror(int status);

/* Text of the last EKCG_ECUDA / EKCG_EINVAL cause seen by the calling thread.            */
const char* ekcg_last_error(void);

/* ---- inspection ------------------------------------------------------------------- */
/* n, t and nnz of the context.                                                            */
int ekcg_shape(const ekcg_ctx* ctx, int64_t* n, int* t, int64_t* nnz);

/* perm[i] = natural row index placed at permuted position i (host array of n int64):
 * the stable sort of rows by domain id (Section 4).                                      */
int ekcg_get_perm(const ekcg_ctx* ctx, int64_t* perm);

/* Kernel launches and sparse products of the last solve.                                 */
int ekcg_last_stats(const ekcg_ctx* ctx, int64_t* kernel_launches, int64_t* spmm_calls);

/* Block Jacobi split preconditioner M = L L^T of Section 5 (Algorithms 8-10) for later
 * solves: L is block diagonal over the blocks of bpart (host array of n block ids in
 * [0, nblocks), natural row order, copied), each diagonal block factored by incomplete
 * Cholesky with zero fill-in, computed on the host in the library's row order (within a
 * block the natural order).  Every block must lie inside one of the t domains (the paper's
 * blocks are subdomains of the t domains).  The solves then build the first block as
 * L^{-T} T(L^{-1} r) and every later candidate as M^{-1} A W_{j-1}; in the CA bases every
 * power M^{-1} A W_{j+i-1} as well.  bpart = NULL removes the preconditioner.  Float64
 * precision; the s-step or a CA basis (EKCG_SSTEP, EKCG_CA5, EKCG_CA7).
 * Errors: EKCG_EINVAL (ids out of range, a block across two domains, IC(0) breakdown,
 * other precision or basis), EKCG_ENOMEM, EKCG_ECUDA.                                    */
int ekcg_set_block_jacobi(ekcg_ctx* ctx, const int32_t* bpart, int nblocks);

/* Host-only inspection of the preconditioner setup (no device work, no context): for the
 * CSR matrix (n, rowptr, colind sorted per row, val) and block ids bpart[n] in [0, nblocks)
 * with the rows in the given order, the IC(0) factor of every diagonal block and the solve
 * levels, as computed by ekcg_set_block_jacobi.  lval[nnz] (caller-owned) receives L_ik for
 * every stored (i, k) with k < i in the same block, L_ii on the diagonal and 0 elsewhere;
 * fwd_level[n] / bwd_level[n] the level of each row in the L and L^T solves.
 * Errors: EKCG_EINVAL (bad CSR, ids out of range, IC(0) breakdown).                       */
int ekcg_block_ic0_host(int64_t n, const int64_t* rowptr, const int32_t* colind,
                        const double* val, const int32_t* bpart, int nblocks, double* lval,
                        int32_t* fwd_level, int32_t* bwd_level);

/* Diagnostic, no counterpart in the paper: runs the bounded mbarrier wait of the
 * bulk-copy-staged kernels on a stage that never completes (16 bytes expected, no copy
 * issued), with a limit of limit_cycles SM cycles (1 .. 2^32), on `stream` (NULL = default
 * stream).  Returns EKCG_ETIMEOUT when the wait ran out and reported it, as the staged
 * kernels do; EKCG_EINVAL for a limit out of range; EKCG_ENOMEM / EKCG_ECUDA.  The device
 * stays usable afterwards.  Allocates and frees one int.                                 */
int ekcg_wait_selftest(long long limit_cycles, void* stream);

/* Measurement, no counterpart in the paper: the float64 FMA rate of the current device
 * (every thread of 8 CTAs per SM x 256 threads runs 16 independent fused multiply-add
 * chains; timed with CUDA events on `stream`, after a warm-up launch).  *num_sms receives
 * the device's SM count, *tflops 2 x FMAs per second / 1e12: the roofline peak of the
 * float64-FMA kernels.  Allocates and frees one double.  Errors: EKCG_EINVAL (NULL
 * outputs), EKCG_ENOMEM, EKCG_ECUDA.                                                      */
int ekcg_fp64_fma_rate(void* stream, int* num_sms, double* tflops);

/* Columns dropped by the rank-revealing A-CholQR (opts.deflate) in the last solve.
 * Errors: EKCG_EINVAL (NULL arguments).                                                  */
int ekcg_deflation_stats(const ekcg_ctx* ctx, int64_t* columns);

/* Device-side convergence test (the `while` line of Algorithms 3 and 4) for later solves of
 * s-step or restructured SRE-CG in float64 (on != 0, the default) or the host-side test
 * (on = 0).  On the device, once the basis window is full, the iterations run as a CUDA
 * graph of conditional iterations: a one-thread kernel after each iteration compares
 * ||r_k|| with tol ||r_0||, checks k against maxit and the breakdown / timeout status word,
 * appends ||r_k|| to a device history and enables the next iteration; the host
 * synchronises once per graph launch (a batch of B iterations, B a multiple of the period
 * of the basis ring slots and at least 8) and copies the history at the end.
 * The kernels, their order and their arguments are those of the host-driven loop, so
 * results are bitwise the same.  Per-launch profiling (ekcg_set_profile) and the other
 * variants, bases and precisions use the host loop.  Errors: EKCG_EINVAL (NULL ctx).       */
int ekcg_set_device_loop(ekcg_ctx* ctx, int on);

/* Iterations of the last solve that ran in the device loop (0: the host loop ran all).
 * Errors: EKCG_EINVAL (NULL arguments).                                                  */
int ekcg_device_loop_stats(const ekcg_ctx* ctx, int64_t* device_iters);

/* Turn the per-launch CUDA-event timing of later solves on (on != 0) or off, whatever
 * opts.profile was at setup.  Errors: EKCG_EINVAL (NULL ctx).                            */
int ekcg_set_profile(ekcg_ctx* ctx, int on);

/* Per-kernel-class accounting of the last solve: for class i < *count, names[i] (static
 * strings), launches[i], flops[i] and bytes[i] (algorithmic: the arithmetic the method needs
 * and the compulsory DRAM traffic of each launch, summed), and ms[i], the total device time
 * measured with CUDA events around each launch when opts.profile = 1 (0 otherwise).  Any
 * output array may be NULL; each holds cap entries.                                       */
int ekcg_profile(const ekcg_ctx* ctx, int cap, const char** names, double* ms,
                 int64_t* launches, double* flops, double* bytes, int* count);

/* ---- kernel-level entry points (device pointers, permuted order) ------------------ */
/* T(r) of Section 2: T[i*t + d] = r[i] if row i lies in domain d, else 0.  r: n doubles,
 * T: n*t doubles.                                                                         */
int ekcg_split_T(ekcg_ctx* ctx, const double* r, double* T);

/* C = X^T Y (the block inner products of Section 3.1: CGS coefficients, Gram matrices,
 * alpha = V^T r): X n x p and Y n x q row-major device doubles, C p x q row-major device
 * doubles (1 <= p, q <= 256; EKCG_EINVAL if the output tiles exceed the workspace sized
 * for max_s*t columns).  Two-stage deterministic reduction through the context's
 * workspace.                                                                             */
int ekcg_gram(ekcg_ctx* ctx, const double* X, int p, const double* Y, int q, double* C);

/* OUT = Y - X C, the CGS update of Section 3.1 (W <- W - Q C): X n x p, Y and OUT n x q,
 * C p x q, all row-major device doubles (OUT may be Y; X must not overlap OUT).
 * contraction: EKCG_CONTRACT_FP64 (float64 FMAs, any 1 <= p <= 256, 1 <= q <= 256) or
 * EKCG_CONTRACT_SPLIT (tensor-core split products; p a multiple of 16 up to 64 and
 * q = 16 or 32, 16-byte aligned buffers; other shapes return EKCG_EINVAL).  Enqueued on
 * the context's stream; returns EKCG_ETIMEOUT if a bounded device wait ran out.           */
int ekcg_sub_xc(ekcg_ctx* ctx, const double* X, int p, const double* C, const double* Y,
                int q, double* OUT, int contraction);

/* ekcg_gram with an explicit contraction: EKCG_CONTRACT_FP64 (any 1 <= p, q <= 256) or
 * EKCG_CONTRACT_SPLIT (tensor-core split products over tiles of 128 rows, each column
 * scaled by its binade over the tile; p a multiple of 16 up to 64 and q = 16 or 32, other
 * shapes return EKCG_EINVAL).  Synchronises the context's stream; EKCG_ETIMEOUT if a
 * bounded device wait ran out.                                                           */
int ekcg_gram_with(ekcg_ctx* ctx, const double* X, int p, const double* Y, int q, double* C,
                   int contraction);

/* Allocation-free C = X^T Y.  The paper has no counterpart: this serves callers that cannot
 * allocate device memory, such as code running while a stream is captured into a CUDA graph
 * (an allocation there breaks or is refused by the capture) or programs whose device memory
 * belongs to another allocator or is fixed at start-up.  Needs no context.
 *   n rows; X n x p and Y n x q row-major device doubles; C p x q row-major device doubles;
 *   1 <= p, q <= 64, else EKCG_EINVAL.  stream: a cudaStream_t (NULL = legacy default).
 *   The work is enqueued on the stream and the call returns without waiting.
 * Scratch: a fixed 2 MiB device array inside the library (64 CTAs x one 64 x 64 tile of
 * doubles), present on every GPU that loads the library until the process exits; no call
 * allocates or frees memory.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call before any
 * stream capture.  The address is kept per device for the life of the process and does not
 * survive a device reset: make no call on a device after cudaDeviceReset.  Every call shares the array and each call overwrites every entry it later
 * reads, so nothing has to be cleared between calls; calls that overlap on the GPU (other
 * streams, other host threads) race on the array and must be serialised by the caller.
 * Errors: EKCG_EINVAL (sizes, null pointers), EKCG_ECUDA (lookup or launch failure).     */
int ekcg_gram_noalloc(int64_t n, const double* X, int p, const double* Y, int q, double* C,
                      void* stream);

/* U = A W for the permuted matrix, W and U n x w row-major doubles (1 <= w <= 256).      */
int ekcg_spmm(ekcg_ctx* ctx, const double* W, double* U, int w);

/* ---- differentiation (adjoint solve support) --------------------------------------- */
/* Replace the matrix values, keeping the sparsity pattern given to ekcg_setup: val is a
 * device array of nnz doubles in the caller's CSR order.  A must stay SPD.               */
int ekcg_update_values(ekcg_ctx* ctx, const double* val);

/* Gradient of a loss L(x), x = A^{-1} b, with respect to the stored values of A:
 * dval[k] = -lambda_i x_j for the k-th nonzero (i, j) in the caller's CSR order, where
 * lambda = A^{-1} dL/dx is the adjoint solution (A is SPD, so the adjoint solve is another
 * ekcg_solve).  lam, x: device arrays of n doubles (natural order); dval: nnz doubles.   */
int ekcg_grad_A(ekcg_ctx* ctx, const double* lam, const double* x, double* dval);

/* 2D diffusion model A(kappa) (5-point edge form, harmonic-mean edge weights times the axis
 * factors ax, ay, Dirichlet faces a*kappa_p, node p = i + nx*j): write the values of
 * A(exp(log_kappa)) in natural CSR order with sorted columns into val (device, nnz
 * doubles).  The context's pattern must be that stencil on an nx x ny grid.              */
int ekcg_diffusion2d_values(ekcg_ctx* ctx, int nx, int ny, double ax, double ay,
                            const double* log_kappa, double* val);

/* Chain rule of the same model: grad[p] = dL/dlog(kappa_p) from the adjoint lambda and the
 * solution x (device arrays of n doubles, natural order).                               */
int ekcg_diffusion2d_grad_logkappa(ekcg_ctx* ctx, int nx, int ny, double ax, double ay,
                                   const double* log_kappa, const double* lam, const double* x,
                                   double* grad);

/* y[i] = x[perm[i]] (direction 0: natural -> permuted) or y[perm[i]] = x[i] (direction 1).*/
int ekcg_permute(ekcg_ctx* ctx, const double* x, double* y, int direction);

/* ---- batched solves: many independent systems in one persistent launch ----------- */
/* Not in the paper: the s-step SRE-CG of Algorithm 4 (A-CholQR, fresh-product CGS2) run on
 * nsys independent SPD systems at once.  A group of CTAs -- one CTA, or a thread-block
 * cluster of 2, 4 or 8 CTAs that split the system's rows and reduce their block inner
 * products through distributed shared memory -- solves one system at a time, taking
 * systems from a device queue, largest first; the gather, the solve and the scatter are one
 * captured CUDA graph replayed per call.  Results are deterministic for a given launch
 * shape; different cluster sizes sum the inner products in different orders.             */
typedef struct ekcg_batch ekcg_batch;

/* n[nsys]: system sizes.  rowptr: the nsys local row-pointer arrays (n_k + 1 entries each,
 * starting at 0) concatenated; colind (local column indices) and val: the nsys nonzero
 * arrays concatenated; part: the nsys partitions (local domain ids in [0, t)) concatenated.
 * All host arrays, copied.  t <= 16; opts: variant SRE, basis SSTEP, orth ACHOLQR, max_s <= 4,
 * precision FP64 or FP32_IR (inner_tol, max_refine, breakdown_tol apply).
 * Errors: EKCG_EINVAL, EKCG_ENOMEM, EKCG_ECUDA.                                           */
int ekcg_batched_setup(int nsys, const int64_t* n, const int64_t* rowptr, const int32_t* colind,
                       const double* val, int t, const int32_t* part, const ekcg_opts* opts,
                       void* stream, ekcg_batch** out);

/* Solve all systems with x0 = 0: b and x are device arrays of sum(n) doubles (the systems'
 * vectors concatenated, natural order).  iters[nsys] and status[nsys] (host, nullable)
 * receive each system's s-step iteration count (FP32_IR: inner iterations) and status
 * (EKCG_OK, EKCG_MAXIT, EKCG_EBREAKDOWN, EKCG_EINVAL for a non-finite right-hand side).
 * The call returns EKCG_OK when the launch ran; per-system outcomes are in status.        */
int ekcg_batched_solve(ekcg_batch* batch, const double* b, int s, double tol, int maxit,
                       double* x, int* iters, int* status);

/* Time seven launch shapes (threads per CTA x CTAs per SM x CTAs per system) with one solve
 * each on right-hand side b (device array, as in ekcg_batched_solve; a small maxit keeps
 * this short) and keep the fastest for later solves.  Errors: EKCG_EINVAL, EKCG_ECUDA.    */
int ekcg_batched_tune(ekcg_batch* batch, const double* b, int s, double tol, int maxit);

/* Set the launch shape: threads per CTA in {256, 512}, CTAs per SM in {1, 2}, CTAs per
 * system (cluster) in {1, 2, 4, 8}; setup chooses 512 x 1 x 4.  The persistent grid holds
 * as many groups as the GPU keeps resident at once.  Errors: EKCG_EINVAL (values outside
 * these sets, or a shape with no resident group), EKCG_ECUDA.                            */
int ekcg_batched_set_shape(ekcg_batch* batch, int threads, int ctas_per_sm, int cluster);

/* Launch shape in use (threads per CTA, CTAs per SM, CTAs per system, groups launched) and
 * device time (ms) of the last captured solve; every pointer nullable.                   */
int ekcg_batched_info(const ekcg_batch* batch, int* threads, int* ctas_per_sm, int* cluster,
                      int* groups, double* last_ms);

/* Mixed (FP32_IR) batched solves: the number of systems of the last solve whose float32
 * refinement stagnated (a refinement step reduced the float64 residual by less than 0.9,
 * as when kappa(A) eps32 approaches 1) and that then continued, on the device, with a
 * float64 s-step solve from the refined iterate in the same workspace.  Synchronises the
 * batch's stream.  Errors: EKCG_EINVAL, EKCG_ECUDA.                                        */
int ekcg_batched_precision_switches(const ekcg_batch* batch, int* count);

/* Release the batch and its device memory (NULL accepted).                               */
void ekcg_batched_destroy(ekcg_batch* batch);

/* Text of the last batched-entry error seen by the calling thread.                        */
const char* ekcg_batched_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* EKCG_H */
