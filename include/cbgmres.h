/*
 * cbgmres.h -- C ABI of the GB300 (sm_103a) compressed-basis GMRES library.
 *
 * Method: Aliaga, Anzt, Gruetzmacher, Quintana-Orti, Tomas, "Compressed Basis GMRES on
 * High Performance GPUs" (arXiv 2009.12101).  Restarted, right-preconditioned GMRES(m)
 * (Fig. 1) whose Krylov basis V is stored in a compact format while the arithmetic
 * works at FP64 class accuracy (Section 3: native FP64, or by default double-float
 * FP32 pairs with about 47-bit operations, see cbg_arith); the basis is decompressed on every read and
 * compressed on every store (the memory accessor of Section 4.2); fixed-point formats carry
 * the per-vector scale sigma_j = (||v_j||_inf / ||v_j||_2) / max_intxx (Section 4.2);
 * convergence ||b - A x||_2 <= tau ||b||_2 is confirmed by an explicit residual each
 * time the recurrence residual says so (Section 5.2).
 *
 * Conventions for every entry point
 *   - Plain pointers and sizes; no library types cross the boundary except the opaque
 *     handles and the option/statistics structs below.
 *   - "device" pointers are CUDA device addresses of the current device; "host"
 *     pointers are ordinary CPU memory.  Vectors are dense FP64 arrays of length n.
 *   - All work is enqueued on options.stream (a cudaStream_t, NULL = legacy default
 *     stream); calls that return results to the host synchronise that stream.
 *   - Every function returns an int status (CBG_OK = 0).  Positive values are
 *     non-fatal (x still holds the best iterate); negative values are errors and leave
 *     outputs unspecified.  Nothing throws across the ABI.  Where an entry point lists no
 *     errors of its own: CBG_ERR_ARG for a null handle or pointer or a size out of range,
 *     CBG_ERR_CUDA when a CUDA call fails (cbgmres_last_error names it).
 *   - Ownership: the library never keeps or frees caller memory; buffers passed in are
 *     read or written during the call (or, for asynchronous calls, until the stream
 *     reaches that work).  A handle owns its device allocations until its destroy call.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef CBGMRES_H
#define CBGMRES_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- storage formats of the Krylov basis (Section 4.2; bf16/e4m3 are additions) ---- */
typedef enum {
    CBG_F64 = 0,   /* IEEE double                                                   */
    CBG_F32 = 1,   /* IEEE single, round-to-nearest cast                           */
    CBG_F16 = 2,   /* IEEE half, one round-to-nearest-even of the FP64 value       */
    CBG_BF16 = 3,  /* bfloat16 of v / 2^e, per-vector power-of-two scale 2^e       */
    CBG_E4M3 = 4,  /* OCP FP8 E4M3 of v / 2^e, saturating, power-of-two scale 2^e  */
    CBG_I32 = 5,   /* fixed point, code = rint(v / sigma), sigma = max|v| / (2^31-1) */
    CBG_I16 = 6    /* fixed point, code = rint(v / sigma), sigma = max|v| / (2^15-1) */
} cbg_format;

/* Right preconditioners M^{-1} (Fig. 1: w = A M^{-1} v, x += M^{-1} V y).
 * JACOBI: diagonal scaling, folded into the stored values A D^{-1} (Section 5.1).
 * SPAI:   z = P v with P on A's pattern (cbgmres_set_spai; the learned preconditioner).
 * BJ4:    block-Jacobi with diagonal blocks of 4 consecutive rows (the last block may be
 *         smaller), each inverted in FP64 with partial pivoting at create (Section 5.5,
 *         block size 4); applied as z = D^{-1} v before the SpMV.  A singular block makes
 *         cbgmres_create fail with CBG_ERR_ARG. */
typedef enum { CBG_PC_NONE = 0, CBG_PC_JACOBI = 1, CBG_PC_SPAI = 2, CBG_PC_BJ4 = 3 } cbg_precond;
/* Re-orthogonalisation (Fig. 1's second Gram-Schmidt pass).
 * ALWAYS (default): every step runs both passes (CGS2).
 * CONDITIONAL: as Fig. 1 prints it, the second pass runs only when the first left
 *   ||w|| < eta * omega (omega = ||A M^{-1} v_j||).  The decision is taken on the device
 *   by the first pass's last block; the second pass's kernels skip themselves otherwise.
 *   eta in (0, 1] (else CBG_ERR_ARG); CGS only (with MGS: CBG_ERR_UNSUPPORTED).
 * NEVER: one pass. */
typedef enum { CBG_REORTH_ALWAYS = 0, CBG_REORTH_CONDITIONAL = 1, CBG_REORTH_NEVER = 2 } cbg_reorth;

/* Orthogonalisation (Fig. 1 prints classical Gram-Schmidt; Section 2 names modified
 * Gram-Schmidt as the alternative and prefers CGS for its BLAS-2 efficiency).
 * CBG_ORTHO_CGS: one basis dot and one basis axpy per pass over all j+1 columns (default).
 * CBG_ORTHO_MGS: column by column, each coefficient from w as the previous columns have
 *   reduced it: 2(j+1) dependent one-column launches per pass.  Same passes (reorth),
 *   arithmetic and Hessenberg output.  Single-system solver only. */
typedef enum { CBG_ORTHO_CGS = 0, CBG_ORTHO_MGS = 1 } cbg_ortho;

/* Arithmetic of the basis products (the CGS projection, its re-orthogonalisation and
 * the solution update of Fig. 1) and of the per-step SpMV.
 * CBG_ARITH_DF32: products and partial sums in double-float (pairs of FP32 with
 *   error-free transformations), cross-thread and cross-block combination in FP64.
 *   Accuracy: each product and sum is carried to about 2^-46 relative (FP64: 2^-53), so
 *   the error bounds of the basis products and of the SpMV rows are those of FP64 with
 *   the unit roundoff 2^-46 in place of 2^-53: 2^6 - 2^8 looser than the same sums in
 *   native FP64, 2^20 tighter than FP32.  The basis dot sums each thread's chain of
 *   about n / 38,912 products in double-float and the chains in FP64, so its bound,
 *   about (n / 38,912) 2^-46 sum |v_i w_i|, stays below FP64's recursive-summation
 *   bound n 2^-53 sum |v_i w_i| for every n >= 128.  The per-step SpMV forms each
 *   product val * x exactly as an FP32 pair from the values split once into FP32 hi / lo
 *   planes (a relative 2^-48 perturbation of A) and delivers w as such planes.  The
 *   per-step operator (A, or A D^{-1} under Jacobi) is normalised by a power of two so
 *   that its largest |value| lies in [1, 2) and the FP32 pairs stay far from underflow
 *   and overflow at any matrix scale; the Hessenberg columns are scaled back exactly.
 *   An operator whose smallest nonzero |value| is below 2^-64 of its largest keeps FP64
 *   products in that SpMV.  GB300's
 *   FP64 pipe issues about 1/70 of its FP32 rate, so this is the mode that streams the
 *   basis at HBM speed.
 * CBG_ARITH_FP64: every product and sum is a native FP64 operation, as the paper
 *   prescribes; on GB300 the basis products then run at FP64-pipe speed.
 * With CBG_ARITH_DF32 the norms of the Arnoldi step (omega = ||A v_j|| in the SpMV,
 * ||w|| in the last CGS pass) are also summed in double-float per thread and combined
 * in FP64.  The residual SpMV (b - Ax, which decides convergence), ||r||, the Givens
 * rotations, the least-squares solve and the solution update are FP64 in both modes. */
typedef enum { CBG_ARITH_DF32 = 0, CBG_ARITH_FP64 = 1 } cbg_arith;

/* status codes */
#define CBG_OK                 0
#define CBG_NOT_CONVERGED      1   /* maxit Arnoldi steps done, tau not reached        */
#define CBG_STAGNATED          2   /* stop_on_stagnation: a restart did not lower the
                                      explicit residual                               */
#define CBG_ERR_ARG          (-1)  /* invalid argument                                 */
#define CBG_ERR_NONFINITE    (-2)  /* NaN/Inf in the data or produced by the iteration */
#define CBG_ERR_OOM          (-3)  /* device allocation failed                         */
#define CBG_ERR_CUDA         (-4)  /* a CUDA call failed                               */
#define CBG_ERR_TIMEOUT      (-5)  /* a bounded device-side wait ran out               */
#define CBG_ERR_UNSUPPORTED  (-6)  /* combination not implemented                      */

/* Sparse matrix in CSR form: row_ptr[n+1] (int32, row_ptr[0] = 0), col[nnz] (int32,
 * 0-based), val[nnz] (FP64).  on_device != 0: the three arrays are device pointers,
 * otherwise host pointers.  cbgmres_create deep-copies them; the caller keeps
 * ownership and may free them once create returns. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int32_t* row_ptr;
    const int32_t* col;
    const double* val;
    int32_t on_device;
    int32_t pad0;
} cbg_csr;

typedef struct {
    int32_t reorth;          /* cbg_reorth, default CBG_REORTH_ALWAYS (CGS + 1 pass)   */
    int32_t precond;         /* cbg_precond, default CBG_PC_NONE                       */
    int32_t arith;           /* cbg_arith, default CBG_ARITH_DF32                      */
    int32_t spmv_group;      /* lanes per CSR row: 0 = automatic, else 1..32 (pow2),   *
                              * or -1 = the per-step SpMV on a sliced-ELL copy        *
                              * (DF32 arithmetic; padding <= nnz/4, else              *
                              * CBG_ERR_UNSUPPORTED).  Automatic times 1, 2, .., 32    *
                              * lanes and the sliced-ELL copy at create on matrices   *
                              * of >= 65536 rows (shortest of 5 launches each, L2    *
                              * flushed before each) and keeps the fastest, the copy  *
                              * only when 10 % faster than every CSR schedule (else   *
                              * it is freed); below 65536 rows it picks by nonzeros   *
                              * per row                                               */
    double eta;              /* conditional re-orthogonalisation threshold (1/sqrt 2)  */
    double breakdown_eps;    /* breakdown when !(h_{j+1,j} > eps * omega) (2^-46)      */
    void* stream;            /* cudaStream_t for all work (NULL: default stream)        */
    int32_t check_every;     /* host polls the convergence flag every k steps (4)      */
    int32_t use_graph;       /* reserved, must be 0                                     */
    int32_t profile;         /* 1: time every kernel launch with CUDA events recorded on
                                options.stream (read with cbgmres_profile)              */
    int32_t stop_on_stagnation; /* 1: stop with CBG_STAGNATED when the explicit residual
                                   at a restart is not below the previous one (0)      */
    int32_t adapt;           /* 1: adaptive basis format (no counterpart in the paper, which
                                fixes one format per solve; Section 5.3 shows the 16-bit
                                formats losing iterations).  At every restart after the first,
                                if the explicit residual exceeds adapt_gap times the
                                recurrence residual the previous cycle ended with, the basis
                                moves one step up the ladder e4m3 -> bf16 -> f32 -> f64,
                                f16 -> f32, i16 -> i32 -> f64 for the following cycles.  The
                                basis is then allocated for 8-byte codes.  Default 0.      */
    int32_t pad1;
    double adapt_gap;        /* promotion threshold of adapt (default 4)                */
    int32_t ortho;           /* cbg_ortho, default CBG_ORTHO_CGS                        */
    int32_t pad2;
} cbg_options;

typedef struct {
    int64_t iters;           /* Arnoldi steps (sparse products of Fig. 1)         */
    int64_t restarts;        /* restart cycles started                                 */
    int64_t reorths;         /* re-orthogonalisation passes                            */
    double true_relres;      /* ||b - A x||_2 / ||b||_2 at exit (FP64, explicit)       */
    double est_relres;       /* last recurrence residual |g_{j+1}| / ||b||_2           */
    double ms_total;         /* wall time of the solve on the stream (CUDA events)     */
    double bytes_model;      /* model HBM bytes: SpMV + 4 basis passes per step         */
    int32_t status;          /* same value as the function's return                    */
    int32_t fmt_final;       /* basis format of the last cycle (differs from the handle's
                                only with options.adapt)                                */
    double* history;         /* optional host buffer: recurrence residual per step     */
    int64_t history_cap;     /* its capacity (0: none)                                  */
    int64_t history_len;     /* entries written                                         */
    int64_t kernel_launches; /* library kernels launched by this call                   */
    int64_t promotions;      /* basis format promotions of options.adapt in this solve  */
} cbg_stats;

/* Per-kernel-class timing gathered while options.profile == 1 (accumulated over
 * solves until cbgmres_profile(..., reset = 1)).  Classes: 0 basis dot (V^T w),
 * 1 basis axpy (w - V h), 2 SpMV (Arnoldi and residual), 3 store/finalize, 4 other.
 * ms: summed CUDA-event durations; bytes: algorithmic HBM bytes (basis codes read for
 * classes 0-1: columns * n * bytes(fmt); CSR + vectors for class 2; codes written plus
 * w read for class 3); launches: count. */
typedef struct {
    double ms[5];
    double bytes[5];
    int64_t launches[5];
} cbg_profile;

typedef struct cbg_handle cbg_handle;
typedef struct cbg_batch cbg_batch;

/* Fill *opt with the defaults listed above. */
void cbgmres_options_default(cbg_options* opt);

/* Human-readable text of a status code (static storage). */
const char* cbgmres_status_string(int status);

/* Text of the last CUDA error the library saw on the calling thread (after an entry
 * point returned CBG_ERR_CUDA); static storage. */
const char* cbgmres_last_error(void);

/* Bytes per stored basis element of `fmt` (8, 4, 2 or 1), 0 for an invalid format. */
int cbgmres_format_bytes(int fmt);

/* Create a solver for A with restart length `restart` (basis dimension m, Fig. 1) and
 * basis format `fmt`.  Copies A to library-owned device memory and allocates the basis
 * V ((m+1) columns of n codes, each column padded to a multiple of 4096 elements), the
 * per-vector scales, the Hessenberg and the work vectors once; every solve reuses them.
 * Errors: CBG_ERR_ARG (n < 1, restart < 1 or > 319, bad format, bad CSR bounds when the
 * CSR is on the host), CBG_ERR_OOM, CBG_ERR_CUDA.  *out is NULL on error. */
int cbgmres_create(const cbg_csr* A, int restart, int fmt, const cbg_options* opt,
                   cbg_handle** out);

/* Right preconditioner z = P v with P on A's sparsity pattern (learned sparse
 * approximate inverse); pvals[nnz] in A's CSR order, FP64, device (on_device != 0) or
 * host.  Takes effect when options.precond == CBG_PC_SPAI.  Errors: CBG_ERR_ARG. */
int cbgmres_set_spai(cbg_handle* h, const double* pvals, int on_device);

/* Solve A x = b.  b, x: device pointers (length n).  x holds x0 on entry and the
 * final iterate on exit.  Stops when ||b - A x|| <= tol ||b|| (explicit residual,
 * Section 5.2) or after maxit Arnoldi steps (CBG_NOT_CONVERGED).  stats may be NULL.
 * Synchronises options.stream once per restart (to read the explicit residual).
 * Errors: CBG_ERR_ARG (null pointers, CBG_PC_SPAI without cbgmres_set_spai),
 * CBG_ERR_NONFINITE (NaN/Inf in b, x0 or produced by the iteration), CBG_ERR_TIMEOUT (a
 * bounded device wait ran out; the handle stays usable), CBG_ERR_CUDA. */
int cbgmres_solve(cbg_handle* h, const double* b, double* x, double tol, int64_t maxit,
                  cbg_stats* stats);

/* As cbgmres_solve with host b and x: copies b and x0 to the device on the stream,
 * solves, copies x back.  For callers without device buffers. */
int cbgmres_solve_host(cbg_handle* h, const double* b_host, double* x_host, double tol,
                       int64_t maxit, cbg_stats* stats);

/* Run k Arnoldi steps of the first restart cycle from x0 (device b, x0) and copy the
 * raw (k+1) x k Hessenberg (before Givens rotations, column-major, leading dimension
 * k+1) to H_host.  *k_done receives the number of columns produced (< k on breakdown).
 * Used to check parity of the orthogonalisation (the Arnoldi step of Fig. 1). */
int cbgmres_arnoldi(cbg_handle* h, const double* b, const double* x0, int k,
                    double* H_host, int* k_done);

/* Decoded basis column `col` of the last run (FP64, device out[n]).  Test access to
 * what the accessor returns (Section 4.2). */
int cbgmres_basis_column(cbg_handle* h, int col, double* out);

void cbgmres_destroy(cbg_handle* h);

/* ---- codec kernels (Section 4.2 accessor), exposed for bit-exact parity checks ----
 * Encode a normalised FP64 vector v (device, length n) whose largest magnitude is vmax
 * into codes (device, n elements of cbgmres_format_bytes(fmt) bytes); *scale_out gets
 * the decode scale (sigma, 2^e, or 1).  Decode multiplies back into FP64 out (device).
 * Synchronises `stream`. */
int cbg_encode(int fmt, int64_t n, const double* v, double vmax, void* codes,
               double* scale_out, void* stream);
int cbg_decode(int fmt, int64_t n, const void* codes, double scale, double* out,
               void* stream);

/* ---- basis products, exposed for parity checks (CGS and re-orthogonalisation, Fig. 1) ---
 * V: device codes, ncols columns of leading dimension ld elements; scales[ncols] host.
 * cbg_basis_dot:  h[k] = sum_i dec(V[i,k]) w[i]      (h: host, w: device)
 * cbg_basis_axpy: w[i] -= sum_k dec(V[i,k]) h[k]     (h: host, w: device, in place)
 * arith: cbg_arith.  Synchronise `stream`. */
int cbg_basis_dot(int fmt, int arith, int64_t n, int ncols, const void* V, int64_t ld,
                  const double* scales, const double* w, double* h, void* stream);
int cbg_basis_axpy(int fmt, int arith, int64_t n, int ncols, const void* V, int64_t ld,
                   const double* scales, const double* h, double* w, void* stream);

/* ---- multi-RHS basis product: H = V^T W for k <= 64 vectors sharing one basis ------
 * No counterpart in the paper (its GMRES has one right-hand side); the building block of
 * block Krylov orthogonalisation.  Vectors are taken in groups of 8 (the last may be
 * smaller); each group reads V once for all its vectors (one split-K product in
 * double-float arithmetic, like cbg_basis_dot with arith = CBG_ARITH_DF32).
 *   V: device codes of format fmt, ncols (<= 320) columns of leading dimension ld
 *      elements (ld >= n, ld % 4096 == 0, rows n..ld-1 zero);
 *   scales[ncols]: device decode factors;  W: device, n x k column-major, leading
 *      dimension ldw >= n (only rows < n are read);
 *   H: device, ncols x k row-major: H[c*k + r] = sum_i dec(V[i,c]) W[i,r];
 *   workspace: device scratch of at least cbg_basis_dot_multi_workspace(ld, ncols, k)
 *      bytes, owned by the caller, not shared between concurrent calls.
 * Asynchronous on `stream` (no allocation, no synchronisation).  Errors: CBG_ERR_ARG
 * (sizes, null pointers, workspace too small), CBG_ERR_CUDA. */
size_t cbg_basis_dot_multi_workspace(int64_t ld, int ncols, int k);
int cbg_basis_dot_multi(int fmt, int64_t n, int ncols, const void* V, int64_t ld, const double* scales, int k,
                        const double* W, int64_t ldw, double* H, void* workspace, size_t ws_bytes,
                        void* stream);
/* The same product with the implementation chosen by `path`: 0 automatic (what
 * cbg_basis_dot_multi does), 1 CUDA cores (double-float, every format), 2 tensor cores
 * (tcgen05, f16 basis with ncols <= 128, else CBG_ERR_UNSUPPORTED).  The tensor-core
 * path cuts codes and vectors into small pieces whose FP16 products and FP32 sums are
 * exact; W is truncated once, 54 bits below the largest |W| of each 512-row block, so
 * H matches the double-float path to FP64-level accuracy.  It covers codes with
 * |code| <= 1 (the range of normalised basis vectors) and finite W: any other input
 * makes every entry of H NaN. */
int cbg_basis_dot_multi_path(int fmt, int64_t n, int ncols, const void* V, int64_t ld, const double* scales,
                             int k, const double* W, int64_t ldw, double* H, void* workspace, size_t ws_bytes,
                             void* stream, int path);

/* Debug build only (libcbgmres_debug.so, compiled with -DCBG_DEBUG): every device
 * allocation of the single-system solver carries a 4 KiB guard tail of 0xA5 bytes, and
 * cbgmres_solve checks every live guard after the solve (CBG_ERR_CUDA, with
 * cbgmres_last_error naming the overrun, if one was overwritten); the SpMV kernels check
 * every column index against n and skip one that is out of range, and the next solver
 * synchronisation returns CBG_ERR_ARG.  This entry point checks the guards now; poke != 0
 * first overwrites one guard byte of h's basis (a test of the check).  The release build
 * returns CBG_ERR_UNSUPPORTED. */
int cbgmres_debug_guard_check(cbg_handle* h, int poke);

/* Lanes per CSR row of the handle's SpMV (the tuned or given schedule); 0 when the
 * create-time timing chose the sliced-ELL copy of the double-float values (chunks of 32
 * rows, one coalesced load per warp and entry) for the per-step SpMV; or CBG_ERR_ARG. */
int cbgmres_spmv_group(const cbg_handle* h);

/* Test of the failure path (no counterpart in the paper).  The next `dots` launches of
 * the pipelined basis dot (DF32 arithmetic) made by solves on h withhold their first
 * bulk-copy stage -- no arrival, no copies -- and give up their waits after
 * wait_cycles clock cycles instead of about a second.  Every wait on that stage runs
 * out, the kernel records the timeout and returns, and the solve returns
 * CBG_ERR_TIMEOUT at its next synchronisation; no copy is left in flight and the
 * context stays usable, so the next solve on h runs normally.  Errors: CBG_ERR_ARG
 * (dots < 0, wait_cycles < 1), CBG_ERR_UNSUPPORTED (the handle uses FP64 arithmetic,
 * which has no pipelined dot). */
int cbgmres_test_stall(cbg_handle* h, int dots, long long wait_cycles);

/* Copy the accumulated per-kernel profile of a handle (options.profile == 1) into
 * *out; reset != 0 clears it afterwards.  Errors: CBG_ERR_ARG. */
int cbgmres_profile(cbg_handle* h, cbg_profile* out, int reset);

/* Same computation and arguments as cbg_basis_dot, without allocating device memory.
 * No counterpart in the paper.  cbg_basis_dot obtains its scratch (per-block partial
 * sums, a completion counter, device copies of scales and result) from cudaMalloc and
 * returns it with cudaFree on every call; callers whose device memory is owned by
 * another allocator (a framework's caching allocator, a fixed pool) cannot count on a
 * private cudaMalloc succeeding, and callers in latency-critical loops cannot accept the
 * device-wide synchronisation of cudaFree.  This variant keeps its scratch in one
 * file-scope device array of about 765 KiB that every GPU loading the library holds
 * until the process exits; it calls no cudaMalloc, cudaFree or allocating routine.
 * Limits: ncols <= 320 (larger: CBG_ERR_ARG); the kernel uses at most 304 thread blocks.
 * Every call looks up the array's address on the current device, copies `scales` from
 * the host, reads h back to the host and synchronises `stream`: it must not be called
 * while that stream is being captured into a CUDA graph.  All calls share the one
 * array, which keeps the last call's contents (the call clears what must start at
 * zero), so calls whose work overlaps on the GPU (other streams, other host threads)
 * race and must be serialised by the caller. */
int cbg_basis_dot_noalloc(int fmt, int arith, int64_t n, int ncols, const void* V, int64_t ld,
                          const double* scales, const double* w, double* h, void* stream);

/* y = A x with the library's SpMV (device x, y).  For parity checks. */
int cbgmres_spmv(cbg_handle* h, const double* x, double* y);

/* ---- batched solve (many independent systems, one persistent launch) ---------------
 * nsys systems As[s] (host or device CSR per on_device), all with restart length
 * `restart` (<= 64) and basis format `fmt`; options.precond NONE or JACOBI, reorth ALWAYS,
 * arith DF32, ortho CGS.  One persistent kernel with thread-block clusters runs every GMRES(m)
 * solve on the device (Fig. 1 with the explicit-residual recheck of Section 5.2): a
 * device work queue hands out systems in decreasing size; systems with at least
 * `split_rows` rows are solved by a whole cluster (rows split across its blocks, sums
 * through distributed shared memory), smaller ones by single blocks.  With
 * options.use_graph the launch is replayed from a CUDA graph.  Each system's per-step
 * operator is normalised and its SpMV runs in double-float under the rules cbg_arith
 * describes (f64 bases keep FP64 products in that SpMV).
 * Vectors are packed: system s occupies entries [off_s, off_s + n_s) with off_s the sum
 * of the sizes of systems 0..s-1 (the order of As).  Errors: CBG_ERR_ARG (bad CSR,
 * restart > 64), CBG_ERR_UNSUPPORTED (other options), CBG_ERR_OOM, CBG_ERR_CUDA. */
int cbgmres_create_batched(int nsys, const cbg_csr* As, int restart, int fmt,
                           const cbg_options* opt, cbg_batch** out);
/* Solve every system: b, x device arrays (packed, total rows); x holds x0 on entry.
 * per_sys (host, nsys entries, may be NULL) receives iterations, restarts, the explicit
 * relative residual and the status of each system; ms_total is the batch time.  Returns
 * the worst status (negative first, then CBG_NOT_CONVERGED).  Synchronises the stream. */
int cbgmres_solve_batched(cbg_batch* bt, const double* b, double* x, double tol, int64_t maxit,
                          cbg_stats* per_sys);
/* Autotuner: time every feasible schedule (cluster size 1..16, split threshold) on this
 * problem (x restored to x0 before each trial) with a thread per SpMV row, then the
 * SpMV's lanes per row (2, 4, 8: the lanes of a row split its nonzeros) for the best of
 * them, and keep the fastest; cache_path (may be NULL) is a JSON-lines file consulted
 * first and appended to, keyed by GPU, format, restart length, system count and total
 * rows.  The chosen cluster size and split threshold are returned
 * (cbgmres_batched_spmv_lanes(bt, 0) reports the lanes). */
int cbgmres_tune_batched(cbg_batch* bt, const double* b, double* x, double tol, int64_t maxit,
                         const char* cache_path, int* cluster_out, int* split_rows_out);
/* Set the schedule explicitly (cluster size a power of two <= 16). */
int cbgmres_batched_schedule(cbg_batch* bt, int cluster, int split_rows);
/* SpMV lanes per row of the batched kernel: lanes = 1 (a thread per row, four rows in
 * flight), 2, 4 or 8 sets it; lanes = 0 only queries.  Returns the lanes in use, or
 * CBG_ERR_ARG. */
int cbgmres_batched_spmv_lanes(cbg_batch* bt, int lanes);
void cbgmres_destroy_batched(cbg_batch* bt);

/* Try the handles in order (e.g. learned SPAI, Jacobi, none -- all for the same A),
 * each continuing from the current x, until one reaches ||b - A x|| <= tol ||b||: the
 * FP64 explicit residual decides.  A handle whose solve ends non-converged or
 * stagnated hands over its x; one that produces non-finite values hands over the x it
 * started from.  maxit caps the total Arnoldi steps.  *used = index of the handle that
 * converged (or the last one tried).  stats accumulates over the attempts. */
int cbgmres_solve_fallback(cbg_handle* const* hs, int nh, const double* b, double* x, double tol,
                           int64_t maxit, cbg_stats* stats, int* used);

/* ---- learned sparse approximate inverse (no counterpart in the paper) ---------------
 * A per-row MLP (inputs: the row's 7-point stencil coefficients divided by a_ii, in the
 * order -z,-y,-x,centre,+x,+y,+z with 0 for a missing neighbour; layers 7 -> 64 -> 64 -> 7
 * with ReLU) emits P on A's pattern, P_{i,nb(i,k)} = out_k(i) / a_ii, for use as the right
 * preconditioner (CBG_PC_SPAI).  The network runs on the tensor cores (tcgen05): weights,
 * features, activations and output gradients enter as BF16, every product sum
 * accumulates in FP32; biases, ReLU and the loss are FP32; gradients are summed over
 * CTAs in FP64.  One training step is one fused pass over the rows (forward, loss,
 * backward, weight gradients) and an Adam update of FP32 master weights.
 * Training minimises mean over pairs of ||P r - e||^2 / ||e||^2 on pairs (r = A e,
 * e = x* - x_k); each pair is folded into per-row statistics on arrival.
 * create: A must be a 3D 7-point pattern with line stride sx and plane stride sxy (host
 * or device CSR); weights start at a deterministic initialisation equal to Jacobi.
 * add_pair: xstar, xk device vectors of length n.  train: `steps` Adam steps (rate lr)
 * on all pairs so far; losses before and after.  values: P (device, nnz, A's CSR order).
 * params: get (set = 0) or set (set = 1) the FP32 master weights (host,
 * cbg_spai_num_params() floats: W1[64x7], b1[64], W2[64x64], b2[64], W3[7x64], b3[7]). */
typedef struct cbg_spai cbg_spai;
int cbg_spai_create(const cbg_csr* A, int64_t sx, int64_t sxy, const cbg_options* opt, cbg_spai** out);
int cbg_spai_add_pair(cbg_spai* s, const double* xstar, const double* xk);
int cbg_spai_train(cbg_spai* s, int steps, double lr, double* loss_first, double* loss_last);
int cbg_spai_loss(cbg_spai* s, double* loss);
int cbg_spai_values(cbg_spai* s, double* pvals);
int cbg_spai_params(cbg_spai* s, float* params, int set);
int cbg_spai_num_params(void);
void cbg_spai_destroy(cbg_spai* s);
/* One forward / backward of the MLP with given FP32 parameters (host; rounded to BF16),
 * on the same tensor-core kernel as training: feat (device, rows x 7 FP32, 16-byte
 * aligned) -> out (device, rows x 7); gout (device, rows x 7, 16-byte aligned) -> grad
 * (host, cbg_spai_num_params() FP64, summed over rows).  For gradient checks.  Errors:
 * CBG_ERR_ARG (sizes, null or misaligned pointers), CBG_ERR_TIMEOUT (a tensor-core wait
 * ran out), CBG_ERR_CUDA. */
int cbg_mlp_forward(int64_t rows, const float* feat, const float* params, float* out, void* stream);
int cbg_mlp_backward(int64_t rows, const float* feat, const float* params, const float* gout,
                     double* grad, void* stream);

#ifdef __cplusplus
}
#endif
#endif
