/*
 * gbcg.h -- C ABI of the GB300 (sm_103a) conjugate-gradient library libgbcg.so.
 *
 * The library solves A x = b for a symmetric positive definite matrix A given
 * in Compressed Sparse Row form, with the conjugate gradient method: the case
 * study of the paper's Section IV ("Case Study"), whose experiment runs
 * double-precision CG on a CSR matrix with N = 132651 and NNZ = 3442951 to a
 * tolerance of 1e-10 (Table I).  One CG iteration is one sparse matrix-vector
 * product ("DGEMV(sparse)" in Section IV), two dot products and three axpy
 * updates; Table I's GFLOPS column is 2*NNZ + 10*N flops per iteration.
 *
 * The paper computes the scalars of each iteration on the CPU and the vector
 * operations on the GPU (Section IV), crossing the host/device boundary every
 * iteration.  Here the whole loop, scalars and stop test included, runs on
 * the device in one persistent cooperative kernel launch per solve; the host
 * reads back a 40-byte status once at the end.
 *
 * Conventions shared by every call:
 *   - Every function that can fail returns an int status (CG_OK = 0) and
 *     never aborts the process.  No call frees memory it did not allocate.
 *   - "device pointer": memory of the CUDA device that was current when the
 *     handle was created (for example a torch tensor's data_ptr()).
 *     "host pointer": ordinary or pinned CPU memory.
 *   - Vectors are dense FP64 arrays of length n, contiguous, 8-byte aligned.
 *   - All device work of a handle is ordered on the CUDA stream given to
 *     cg_create.  A handle must not be used from two threads at once, and
 *     two solves on one handle must not overlap (they share its workspace).
 */
#ifndef GBCG_H
#define GBCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define CG_OK 0          /* converged (or nothing to do)                        */
#define CG_EINVAL 1      /* invalid argument or malformed CSR                   */
#define CG_ENOMEM 2      /* device or host allocation failed                    */
#define CG_ECUDA 3       /* a CUDA runtime call or kernel launch failed         */
#define CG_ENOCONV 4     /* maxit iterations done without meeting the tolerance;
                            x holds the last iterate                            */
#define CG_EBREAKDOWN 5  /* p.q <= 0 (A not positive definite), or r.z <= 0 with
                            a preconditioner; x holds the last iterate          */
#define CG_ENAN 6        /* a reduction produced NaN or infinity (e.g. NaN in b) */
#define CG_ETIMEOUT 7    /* a bounded device-side wait (grid barrier or TMA
                            barrier) ran past cg_opts.wait_limit_s; the kernel
                            returned early and x is unspecified                 */

/* ---- where the arrays of a cg_csr live --------------------------------- */
#define CG_MEM_HOST 0
#define CG_MEM_DEVICE 1

/* ---- precision of the inner solve --------------------------------------- */
#define CG_VALUES_FP64 0     /* plain FP64 CG (the paper's double precision)      */
#define CG_VALUES_FP32 1     /* FP32 inner CG on FP32 values + FP64 refinement    */
#define CG_VALUES_BF16 2     /* FP32 inner CG on BF16 values + FP64 refinement    */

/* ---- preconditioners --------------------------------------------------- */
#define CG_PRECOND_NONE 0    /* plain CG, as in Section IV                      */
#define CG_PRECOND_JACOBI 1  /* z = diag(A)^-1 r (Jacobi-preconditioned CG)     */
#define CG_PRECOND_LEARNED 2 /* learned convolutional preconditioner inside
                                flexible CG, Jacobi-PCG as fallback (needs
                                cg_set_learned before the first solve)         */

/*
 * A square sparse matrix in CSR form (Section IV stores the FEM matrix this
 * way).  rowptr has n+1 entries, rowptr[0] = 0, non-decreasing,
 * rowptr[n] = nnz; colidx[k] in [0, n) is the column of vals[k].  Columns of a
 * row need not be sorted; repeated columns add.  Explicitly stored zeros are
 * kept (and streamed by the kernels).  The matrix must be symmetric positive
 * definite for CG to converge; symmetry is not checked.
 */
typedef struct {
    int32_t n;               /* rows = columns, >= 0                             */
    int64_t nnz;             /* stored entries, 0 <= nnz < 2^31                  */
    const int32_t *rowptr;   /* n + 1 entries                                    */
    const int32_t *colidx;   /* nnz entries                                      */
    const double *vals;      /* nnz entries                                      */
    int32_t mem;             /* CG_MEM_HOST or CG_MEM_DEVICE for the three arrays */
} cg_csr;

/* Options fixed at cg_create.  Fill with cg_opts_default, then change fields. */
typedef struct {
    int32_t precond;         /* CG_PRECOND_*; default CG_PRECOND_NONE             */
    int32_t true_residual;   /* 1: after the loop compute ||b - A x||_2/||b||_2
                                (one more SpMV) into cg_info.relres_true; default 1 */
    double wait_limit_s;     /* bound on every device-side spin wait, seconds;
                                default 5.0                                       */
    int32_t grid_ctas;       /* persistent CTAs; 0 = one per SM (capped by the
                                number of row tiles); default 0                   */
    int32_t debug_phantom_arrivals; /* test knob, default 0: grid barriers also
                                wait for this many CTAs that never arrive, so
                                every wait runs out and the solve returns
                                CG_ETIMEOUT without hanging the device            */
    int32_t vectors_in_memory; /* 0 (default): when every thread owns at most 4
                                rows, the solver keeps x, r, z, p, q and 1/diag of
                                those rows in registers for the whole solve;
                                1: always keep every vector in device memory     */
    int32_t inner_values;    /* CG_VALUES_*; default CG_VALUES_FP64.  FP32/BF16
                                turn the solve into iterative refinement: the
                                outer loop keeps x and r = b - A x in FP64 with
                                the FP64 matrix and stops on the true residual;
                                each correction solves A_lo d = r by CG in FP32
                                on a copy of A whose off-diagonals are rounded
                                (nearest-even) to FP32/BF16 and whose FP32
                                diagonal is row-sum compensated (A_lo keeps A's
                                row sums); precond applies to the inner CG     */
    double inner_tol;        /* inner stop: ||r_in|| <= inner_tol ||r||; 0 =
                                1e-3 (FP32) or 1e-2 (BF16)                      */
    int32_t max_outer;       /* refinement steps at most; default 50             */
    int32_t max_inner;       /* inner iterations per step at most; 0 = n         */
} cg_opts;

/* Result of a solve (also returned through the status code). */
typedef struct {
    int32_t iters;           /* products A p inside the loop (x updates applied);
                                with refinement: inner iterations, all steps    */
    int32_t status;          /* same value as the function's return code         */
    double relres;           /* ||r_k||_2 / ||b||_2 of the recursive residual
                                (with refinement: of the FP64 outer residual)   */
    double relres_true;      /* ||b - A x||_2 / ||b||_2 if requested, else -1     */
    double kernel_ms;        /* device time of the solve kernel (CUDA events)     */
    int32_t launches;        /* kernels this call launched                        */
    int32_t outer;           /* refinement steps applied (0 for plain CG)         */
    int32_t reverted_at;     /* CG_PRECOND_LEARNED: iteration at which the solve
                                switched to Jacobi-PCG (0 = before the first
                                step), -1 if it never did; -1 otherwise          */
    int32_t reserved;        /* 0                                                 */
} cg_info;

/* Read-only description of the launch plan of a handle. */
typedef struct {
    int32_t n;
    int64_t nnz;
    int32_t ctas;            /* CTAs of the persistent kernels                    */
    int32_t threads;         /* threads per CTA                                   */
    int32_t tiles;           /* row tiles (each staged through shared memory)     */
    int32_t tile_nnz;        /* largest tile in stored entries                    */
    int32_t stages;          /* TMA stages (shared-memory tile buffers) per CTA   */
    int32_t smem_bytes;      /* dynamic shared memory per CTA                     */
    int32_t lanes_per_row;   /* threads that share one row in the SpMV            */
    int32_t l2_evict_first;  /* 1 when the matrix stream is marked evict-first    */
    int32_t reg_rows;        /* rows per thread held in registers (0: none)       */
    int32_t window_tiles;    /* tiles whose gathers read a staged x-window        */
    int64_t device_bytes;    /* device memory the handle owns                     */
    int32_t slice_solve;     /* FP64 solves run: 1 the SELL-32 kernel with one
                                32-row slice per warp and rows in registers; 2
                                the SELL-32 kernel with the vectors in memory
                                (systems too large for 1 and for register rows
                                in the tiled kernel); 0 the tiled kernel
                                described by the fields above                    */
    int32_t inner_solve;     /* handles with inner_values FP32/BF16: 1 when the
                                refinement runs on SELL-32 copies (one 32-row
                                slice per warp), 0 when it runs on the staged
                                tiles described above; 0 for FP64 handles       */
} cg_plan;

typedef struct cg_handle cg_handle;

/* Version of this ABI (major * 10000 + minor * 100 + patch). */
int cg_version(void);

/* Fills *opts with the defaults listed above.  CG_EINVAL if opts is NULL. */
int cg_opts_default(cg_opts *opts);

/*
 * Validates A, copies it into device memory owned by the new handle, plans
 * the row tiling and allocates the solver workspace (Section IV's "data
 * reading" and "initial configuration" blocks).  The caller may free its
 * arrays as soon as the call returns.  stream is a cudaStream_t (NULL = the
 * legacy default stream); the current CUDA device becomes the handle's device.
 * opts may be NULL for defaults.  On success *out receives the handle; on
 * failure *out is NULL and the return code says why (CG_EINVAL for a
 * malformed matrix: rowptr not starting at 0, decreasing, or not ending at
 * nnz; a column outside [0, n); negative sizes; a non-positive or missing
 * diagonal when CG_PRECOND_JACOBI is asked for).  Synchronous.
 */
int cg_create(const cg_csr *A, const cg_opts *opts, void *stream, cg_handle **out);

/*
 * Runs CG from x (in: x0, out: the last iterate) until
 * ||r_k||_2 <= tol * ||b||_2 (the continue-condition of Section IV; Table I
 * uses tol = 1e-10) or maxit iterations (maxit <= 0 means n: "a 132651 loop",
 * Section IV).  With inner_values FP32/BF16 the stop test is on the true
 * FP64 residual and maxit caps the inner iterations of all steps together.  b and x are device pointers of length n; b must not alias x.
 * b = 0 gives x = 0 after 0 iterations.  Synchronous: returns after the
 * result is on the device and the status is read back.  info may be NULL.
 * Returns CG_OK, CG_ENOCONV, CG_EBREAKDOWN, CG_ENAN, CG_ETIMEOUT, CG_EINVAL
 * (NULL handle or vectors, negative or non-finite tol) or CG_ECUDA.
 */
int cg_solve(cg_handle *h, const double *b, double *x, double tol, int32_t maxit,
             cg_info *info);

/*
 * cg_solve with b and x in host memory: copies b and x0 to the device, solves
 * and copies x back, all on the handle's stream (pinned host memory makes the
 * copies asynchronous DMA).  Same results and return codes as cg_solve.
 */
int cg_solve_host(cg_handle *h, const double *b, double *x, double tol, int32_t maxit,
                  cg_info *info);

/*
 * y = A x (the SpMV of Section IV alone), x and y device pointers of length n,
 * not aliased.  Asynchronous: enqueued on the handle's stream, returns after
 * the launch.  Returns CG_OK, CG_EINVAL or CG_ECUDA.
 */
int cg_spmv(cg_handle *h, const double *x, double *y);

/*
 * y = A_lo x: the SpMV of the inner CG of iterative refinement alone (the
 * "DGEMV(sparse)" of Section IV on the low-precision copy of A), for a handle
 * created with inner_values FP32 or BF16.  A_lo is the matrix the inner solve
 * uses: off-diagonals rounded (nearest-even) to FP32 or BF16, diagonal the
 * FP32 row-sum compensated value (see cg_opts.inner_values).  x and y are
 * device arrays of n floats; products and sums are FP32, each row's
 * off-diagonal sum first, then y_i = fmaf(diag_i, x_i, sum), through the same
 * device routine and launch layout as the handle's refinement kernel
 * (cg_plan.inner_solve).  x is copied into the handle's workspace first, so
 * this call must not overlap a solve on the same handle.  Synchronous.
 * Returns CG_OK, CG_EINVAL (NULL handle or vectors, an FP64 handle),
 * CG_ECUDA, or CG_ETIMEOUT if a bounded copy wait ran out.
 */
int cg_spmv_inner(cg_handle *h, const float *x, float *y);

/* Fills *plan with the handle's launch plan.  CG_EINVAL on NULL arguments. */
int cg_get_plan(const cg_handle *h, cg_plan *plan);

/* Frees everything the handle owns (after synchronizing its stream).
 * cg_destroy(NULL) is a no-op; a handle must not be destroyed twice. */
void cg_destroy(cg_handle *h);

/* Static description of a status code ("unknown status" for other values). */
const char *cg_strerror(int code);

/*
 * Index faults seen by a library built with -DGBCG_BOUNDS_CHECK (the
 * bounds-check build, libgbcg_check.so): its kernels test every column index
 * they gather through and every staged row range they walk, skip a bad one
 * (an empty range, or index 0) and count it here, for the whole process and
 * every device.  *count receives the count, or -1 for a normal build (which
 * checks nothing).  Synchronous.  CG_EINVAL for a NULL count.
 */
int cg_bounds_faults(int64_t *count);

/*
 * Measurement helper, not part of the method: the FP64 FMA throughput of the
 * current device, the denominator of the FP64 roofline the solve kernels are
 * reported against (one CG iteration is 2 NNZ + 10 N flops, Table I).  One
 * kernel of 4 x SMs CTAs x 512 threads, each thread `iters` steps of 8
 * independent FP64 FMA chains, timed with CUDA events on `stream` after a
 * shorter warm-up launch.  *flops receives the flops of the timed launch
 * (2 per FMA) and *ms its device time.  Writes no memory, allocates none.
 * Synchronous.  CG_EINVAL for iters < 1 or NULL outputs, CG_ECUDA otherwise
 * on failure.
 */
int cg_fp64_peak(void *stream, int32_t iters, double *flops, double *ms);

/* ---- batched solves ---------------------------------------------------- */

/* Result of one (system, right-hand side) pair of a batched solve. */
typedef struct {
    int32_t iters;           /* inner iterations, all refinement steps           */
    int32_t outer;           /* refinement steps applied                         */
    int32_t status;          /* CG_OK, CG_ENOCONV, CG_EBREAKDOWN or CG_ENAN      */
    int32_t reserved;
    double relres;           /* ||b - A x||_2 / ||b||_2 (FP64) at the last check  */
} cg_batch_result;

/* What cg_batch_tune chose (also the argument of cg_batch_set_tuning). */
typedef struct {
    double inner_tol;        /* inner tolerance of the fastest trial             */
    int32_t gather_tiles;    /* 1: tiles gather x from memory instead of staging
                                x-windows                                       */
    int32_t trials;
    double best_ms;          /* device time of the fastest trial                 */
    int32_t lanes_per_row;   /* lanes that share one row in the inner SpMM: 1, 2
                                or 4 (a warp steps through a 32-row tile 32, 16
                                or 8 rows at a time)                              */
    int32_t static_split;    /* 0: the inner loop re-splits the tiles of the
                                systems still active evenly over the CTAs each
                                time a system leaves it; 1: it keeps the
                                creation-time split over all systems (not
                                searched by cg_batch_tune, which reports the
                                handle's setting)                                 */
} cg_batch_tuning;

typedef struct cg_batch cg_batch;

/*
 * Many independent SPD systems (nsys >= 1, each a cg_csr as for cg_create,
 * host or device arrays) solved together: the batched time stepping of an
 * FEM model, each step a new right-hand side (Section IV solves one such
 * system; the paper has no batched form).  The systems are stored as one
 * block-diagonal matrix whose row tiles never cross a system.  Every (system,
 * right-hand side) pair runs the mixed-precision refinement of cg_solve
 * (opts->inner_values FP32 or BF16; FP64 is taken as FP32; precond applies
 * to the inner CG) and all pairs advance in lockstep inside one persistent
 * cooperative kernel; tiles of finished systems are skipped, and the inner
 * loop re-splits the tiles still active evenly over the CTAs (deterministic:
 * results are bitwise reproducible).  A CTA may
 * hold tiles of at most 64 systems (CG_EINVAL otherwise).  Synchronous.
 */
int cg_batch_create(const cg_csr *systems, int32_t nsys, const cg_opts *opts, void *stream,
                    cg_batch **out);

/*
 * Enqueues a batched solve on the handle's stream and returns (no
 * synchronization; only stream-ordered copies, memsets and one cooperative
 * kernel launch).  B and X are device arrays of nrhs (1..4) columns over the
 * concatenated systems: column r of system s starts at
 * r * N + (rows of systems 0..s-1), N the total row count; X holds x0 and
 * receives the solutions.  The stop test per pair is the true FP64 residual
 * ||b - A x|| <= tol ||b|| (squares compared); maxit caps each pair's inner
 * iterations (<= 0: N).  Read the per-pair results with cg_batch_results
 * once the stream has passed this work.
 */
int cg_batch_enqueue(cg_batch *h, const double *B, double *X, int32_t nrhs, double tol, int32_t maxit);

/*
 * Copies the per-pair results of the last enqueued solve to results
 * (nsys x nrhs, system-major; may be NULL) after synchronizing the stream.
 * Returns CG_OK if every pair converged, else the first failing pair's
 * status, or CG_ETIMEOUT if a bounded device wait ran out.
 */
int cg_batch_results(cg_batch *h, cg_batch_result *results);

/* cg_batch_enqueue + cg_batch_results; kernel_ms (may be NULL) receives the
 * device time of the enqueued work (CUDA events). */
int cg_batch_solve(cg_batch *h, const double *B, double *X, int32_t nrhs, double tol, int32_t maxit,
                   cg_batch_result *results, double *kernel_ms);

/*
 * Autotuner: times full solves of B (x0 from X, X left unchanged) for every
 * combination of the inner tolerance in {1e-2, 3e-3, 1e-3, 1e-4} (BF16:
 * >= 1e-3), the tile kind (staged x-windows or gather tiles) and the rows a
 * warp takes per step of the inner SpMM (32, 16 or 8: 1, 2 or 4 lanes per
 * row), keeps the fastest converged choice for later solves and reports it
 * in *choice (may be NULL).  Synchronous.
 */
int cg_batch_tune(cg_batch *h, const double *B, double *X, int32_t nrhs, double tol,
                  cg_batch_tuning *choice);

/*
 * Applies a choice (for example one cg_batch_tune found on a smaller batch
 * of the same kind of systems): inner_tol in (0, 1), gather_tiles 0 or 1,
 * lanes_per_row 1, 2 or 4, static_split 0 or 1; trials and best_ms are
 * ignored.  CG_EINVAL otherwise.  Takes effect at the next enqueue.
 */
int cg_batch_set_tuning(cg_batch *h, const cg_batch_tuning *choice);

/* Frees the batch handle (NULL is a no-op). */
void cg_batch_destroy(cg_batch *h);

/*
 * Largest n that cg_solve_noalloc accepts (its fixed workspace holds three
 * vectors of this length: 6 MiB, held by every GPU that loads the library
 * until the process exits).
 */
#define CG_NOALLOC_MAX_N 262144

/*
 * FP64 CG without any allocation, for callers that cannot allocate device
 * memory: code inside a framework whose caching allocator owns the device
 * memory (a cudaMalloc beside it can fail, and it synchronizes the device),
 * real-time loops with no room for that synchronization, plug-ins with a
 * fixed device-memory budget.  The paper has no counterpart; it computes
 * what cg_solve computes with CG_PRECOND_NONE (same recurrence, stop test
 * and status codes) from the caller's arrays: A must be CG_MEM_DEVICE with
 * rowptr, colidx and vals on the current device, b and x are device vectors
 * (x: in x0, out the last iterate), stream is a cudaStream_t.  Its workspace
 * is one fixed __device__ array shared by all calls: each call clears what
 * must start at zero, but calls whose work overlaps on the GPU (other
 * streams, other host threads) race on it.  The first call on a device looks
 * the array's address up (cudaGetSymbolAddress) and, under lazy module
 * loading, loads the module that holds the array (it is created then); make
 * that first call before any stream capture.  cudaDeviceReset invalidates the
 * looked-up address: do not call this again on a device that was reset.
 * Synchronous: returns once the result and the status are back.  Returns
 * CG_EINVAL for n > CG_NOALLOC_MAX_N, NULL vectors, b == x, any array that is
 * not device or managed memory of the current device (checked on the host
 * with cudaPointerGetAttributes before any launch), and for a malformed
 * matrix found by the kernel (a row range or a column out of bounds; such
 * entries are never read); otherwise as cg_solve.  info->kernel_ms is 0 and
 * relres_true is -1 (no events, no extra SpMV).
 */
int cg_solve_noalloc(const cg_csr *A, const double *b, double *x, double tol, int32_t maxit,
                     void *stream, cg_info *info);

/* ======================================================================
 * Learned preconditioner and flexible CG.
 *
 * The paper (Section IV) runs CG without a preconditioner; these calls add
 * one that it does not have.  For a Q1 matrix on the node grid of an
 * Ex x Ey x Ez box (n = (Ex+1)(Ey+1)(Ez+1), nodes numbered x fastest) the
 * preconditioner is
 *     z = D^-1/2 L^T L D^-1/2 r,   L = C2 diag(g) C1,   D = diag(A),
 * where C1 (1 -> 16 channels) and C2 (16 -> 16) are 3x3x3 correlations over
 * the node grid with zeros outside it, L^T applies C2's and C1's adjoints
 * (flipped taps, swapped channels) and g = sigmoid(Cg(log nu / 8) + bg) are
 * 16 gate channels computed from the log-reluctivity field at the nodes.  It
 * is linear in r, symmetric and positive semi-definite for any parameters.
 * The residual is scaled by 1 / rms(D^-1/2 r) before the network (which the
 * linearity cancels) so that BF16 sees values of order one.  Inference and
 * training run on the tensor cores: BF16 weights and activations, FP32
 * accumulation; the Krylov vectors stay FP64.
 *
 * Parameters: CG_LEARN_PARAMS floats, W1[o][t] (16 x 27), W2[o][c][t]
 * (16 x 16 x 27), Wg[o][t] (16 x 27), bg[o] (16); tap t = 9 (dz+1) +
 * 3 (dy+1) + (dx+1) reads the node at offset (dx, dy, dz).
 * ==================================================================== */
#define CG_LEARN_PARAMS 7792

typedef struct cg_net cg_net;

/* Network on the current device with the given parameters (host array of
 * CG_LEARN_PARAMS floats; used in BF16 by the kernels, kept in FP32 for
 * training).  CG_EINVAL for NULL arguments or non-finite parameters. */
int cg_net_create(const float *params, cg_net **out);

/* Copies the FP32 parameters to a host array of CG_LEARN_PARAMS floats. */
int cg_net_get_params(const cg_net *net, float *params);

/* Replaces the parameters (host array) and resets the optimizer state. */
int cg_net_set_params(cg_net *net, const float *params);

/* Frees the network (NULL is a no-op).  Handles that use it must not solve
 * with CG_PRECOND_LEARNED afterwards. */
void cg_net_destroy(cg_net *net);

/*
 * Attaches the learned preconditioner to a handle created with
 * CG_PRECOND_LEARNED: the box has ex x ey x ez elements with
 * (ex+1)(ey+1)(ez+1) == n, lognu holds log nu at each node (host, n floats,
 * node order), net must stay alive while the handle solves with it (its
 * current parameters are read at each solve).  stall_window (1..128, 0 =
 * 50) and stall_factor (in (0, 1], 0 = 0.9) set the switch to Jacobi-PCG:
 * when no residual norm of the last stall_window iterations is below
 * stall_factor times the smallest one before them.  Allocates the
 * activation buffers (about 200 bytes per node).  CG_EINVAL for a handle
 * without CG_PRECOND_LEARNED, a grid that does not match n or whose padded
 * x-extent exceeds 520 nodes, non-finite lognu or a net on another device.
 *
 * With a learned handle cg_solve runs flexible CG: alpha = rho / p.q,
 * beta = -alpha (z_new . q) / rho, p = z_new + beta p, rho = r.z; a stall or
 * r.z <= 0 restarts it as Jacobi-PCG from the current x for the rest of the
 * solve (cg_info.reverted_at).  Statuses and stop test as for CG.
 */
int cg_set_learned(cg_handle *h, cg_net *net, int32_t ex, int32_t ey, int32_t ez, const float *lognu,
                   int32_t stall_window, double stall_factor);

/* z = M r once with the attached network (device vectors of n doubles, on
 * the handle's stream; synchronous).  r = 0 gives z = 0. */
int cg_precond_apply(cg_handle *h, const double *r, double *z);

/*
 * Training pairs from restarted FP64 CG: starting from x = 0, for
 * s = 0 .. count-1 it records r_s = b - A x and e_s = xstar - x (as floats,
 * row s of the count x n device arrays r_out and e_out) and then runs
 * `segment` plain CG iterations from x (each segment a fresh CG start).
 * xstar must solve A xstar = b (e.g. b built as A xstar), so e_s is the
 * true error of r_s.  Device pointers; synchronous.
 */
int cg_learn_pairs(cg_handle *h, const double *b, const double *xstar, int32_t segment, int32_t count,
                   float *r_out, float *e_out);

/* A set of training pairs over instances that share one grid. */
typedef struct {
    int32_t ninst;             /* instances                                         */
    cg_handle *const *inst;    /* host array of ninst learned handles (cg_set_learned
                                  done, same ex, ey, ez, same device as the net)  */
    int64_t npairs;
    const int32_t *pair_inst;  /* host, npairs: instance of each pair              */
    const float *r;            /* device, npairs x n: residuals                     */
    const float *e;            /* device, npairs x n: their true errors (A e = r)   */
} cg_learn_set;

/*
 * Loss and gradient of the pairs listed in `pairs` (host, count indices into
 * the set), without changing the network: the loss of a pair is
 * (u - e_hat)^T A_hat (u - e_hat) / (2n) with A_hat = D^-1/2 A D^-1/2,
 * s = D^-1/2 r, sigma = rms(s), u the network output for s / sigma before
 * the final D^-1/2 scaling, e_hat = D^1/2 e / sigma; *loss receives the
 * mean over the pairs and grad (host, CG_LEARN_PARAMS floats, may be NULL)
 * its gradient.  Synchronous.
 */
int cg_learn_grad(cg_net *net, const cg_learn_set *set, const int64_t *pairs, int32_t count, double *loss,
                  float *grad);

/*
 * Adam on the mean loss of mini-batches: step k uses the pairs
 * order[k * batch .. k * batch + batch - 1] (host indices into the set),
 * learning rate lr, beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; the
 * optimizer state persists in the net across calls.  losses (host, steps
 * doubles, may be NULL) receives each step's mean loss.  Synchronous.
 */
int cg_learn_train(cg_net *net, const cg_learn_set *set, const int64_t *order, int32_t steps, int32_t batch,
                   float lr, double *losses);

#ifdef __cplusplus
}
#endif

#endif /* GBCG_H */
