/*
 * mpk.h -- C ABI of the GB300 (sm_103a) library for mixed-precision ILU(0)-preconditioned
 * multi-component Krylov solvers (Kouya, arXiv 2504.14498).
 *
 * Problem (Sec. 3, Eq. 1): solve A x = b with A an n x n nonsingular real or complex sparse
 * matrix in CSR ("CRS") storage with binary64 entries (Sec. 3, last paragraph: the matrices
 * are binary64, the vectors multi-component).
 *
 * Conventions shared by every entry point
 *   - Pointers named *_dev are DEVICE pointers (e.g. torch CUDA tensors), owned by the caller,
 *     16-byte aligned, and must stay valid until the stream work that uses them completes.
 *     Vectors and complex matrix values are accessed 16 bytes at a time: a misaligned vector
 *     pointer, or a misaligned val of a complex matrix, is refused with MPK_INVALID_ARG
 *     before any work is queued.
 *     Pointers named *_host are host pointers.  `stream` is a cudaStream_t (NULL = default
 *     stream); every call is ordered on it.
 *   - Multi-component numbers: w = 1 (D), 2 (DD), 3 (TD), 4 (QD) binary64 components,
 *     leading component first (Sec. 2).  A real entry is w doubles, a complex entry 2w doubles
 *     (real part then imaginary part).  A vector of n entries is n*c*w contiguous doubles,
 *     c = 1 (real) or 2 (complex).
 *   - CSR: row_ptr int32[n+1] (row_ptr[0] = 0, nondecreasing), col_idx int32[nnz] strictly
 *     ascending within each row, val double[nnz] (real) or double[2*nnz] interleaved (re, im)
 *     (complex).  The diagonal must be stored for ILU(0).
 *   - Return value: an mpk_status.  On failure mpk_last_error() returns a message (per host
 *     thread).  Arguments are validated on the host before any launch: invalid pointers,
 *     sizes or enum values give MPK_INVALID_ARG and launch nothing.
 *   - Errors found on the device (zero pivot, a bounded device wait that ran out) are reported
 *     through the status returned by the call that waits for them (mpk_ilu0_factor,
 *     mpk_krylov_solve); device waits are bounded (about one second each) and never hang.
 *
 * Arithmetic: see paper_2504_14498_gb300/csrc/mp.cuh (DD: Joldes-Muller-Popescu double-word
 * algorithms; TD/QD: renormalisation of the exact terms, relative error about 2^(-53 w));
 * mpk_mp_op exposes each operation.
 *
 * Environment variables (none changes a result; all choose how the same operations run):
 *   MPK_SUBST_SCHEDULE=static|owner|cluster8|cluster16  substitution schedule (mpk_ilu0_schedule);
 *                                                        read at every call; default: tuned.
 *   MPK_SUBST_POLL=lane0|all|allsleep                    dependency polling of the substitutions
 *                                                        (lane 0 polls a chunk's latest dependency
 *                                                        first, or every lane its own, spinning
 *                                                        or sleeping between rounds;
 *                                                        mpk_ilu0_polling); read at every call;
 *                                                        default: tuned.
 *   MPK_SUBST_POLL_SLEEP_NS=16..4096                     the sleep of the sleeping polling mode;
 *                                                        read at every call; default 256.
 *   MPK_ILU_SCHEDULE=levels|dataflow                     ILU(0) schedule (mpk_ilu0_factor); read
 *                                                        at every factorisation; default: by the
 *                                                        width of the levels.
 *   MPK_RESIDENT_WARPS=k                                 warps per SM of the dependency-driven
 *                                                        kernels (default 32); read once.
 *   MPK_NO_GRAPH=1                                       run a solve's iterations as plain
 *                                                        launches instead of replays of one
 *                                                        captured CUDA graph; read once.
 */
#ifndef MPK_H
#define MPK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MPK_OK = 0,
  MPK_MAXIT = 1,          /* iteration limit reached without convergence                   */
  MPK_BREAKDOWN = 2,      /* an exactly zero denominator (rho, <r~,v>, LS determinant, ...)  */
  MPK_ZERO_PIVOT = 3,     /* ILU(0): U_kk = 0 (Algorithm 1 tests U_kk != 0); fail_row = k    */
  MPK_MISSING_DIAG = 4,   /* ILU(0): a row without a stored diagonal; fail_row = that row     */
  MPK_NAN = 5,            /* a residual norm became NaN (e.g. NaN in b)                      */
  MPK_INVALID_ARG = 6,    /* bad pointer / size / enum / unsorted columns                    */
  MPK_CUDA_ERROR = 7,     /* a CUDA runtime call failed                                      */
  MPK_TIMEOUT = 8,        /* a bounded device wait ran out (never expected)                  */
  MPK_NOT_IMPLEMENTED = 9
} mpk_status;

/* Precision of the ILU(0) factor and of the substitutions (Sec. 3; Sec. 4 "_d" variants). */
typedef enum {
  MPK_ILU_NONE = -1, /* no preconditioner, M = I                                            */
  MPK_ILU_FP64 = 0,  /* binary64 factor; substitutions multiply binary64 factor entries with
                        the multi-component vector and accumulate in it (paper's "_d")      */
  MPK_ILU_FP32 = 1,  /* A rounded to binary32, factor and substitutions in binary32: the
                        right-hand side is scaled by 2^-e (e = exponent of its largest entry),
                        rounded to binary32, solved, widened and scaled back                 */
  MPK_ILU_BF16 = 2,  /* binary32 factorisation, factor stored as bfloat16 (round to nearest
                        even); substitutions as MPK_ILU_FP32                                 */
  MPK_ILU_MP = 3     /* factor entries in the solve's w-component arithmetic (the paper's rows
                        without "_d"): factorisation, products and divisions of the
                        substitutions all in w components; made by mpk_ilu0_factor_mp       */
} mpk_ilu_prec;

/* Product-type Krylov methods (Sec. 3): BiCG is Algorithm 3; CGS, BiCGSTAB and GPBiCG are the
 * standard right-preconditioned forms in which r is the residual b - A x of the original
 * system (the paper names them without a listing). */
typedef enum { MPK_BICG = 0, MPK_CGS = 1, MPK_BICGSTAB = 2, MPK_GPBICG = 3 } mpk_method;

typedef struct {
  int32_t n;               /* rows = columns, n >= 1                                          */
  int32_t nnz;             /* row_ptr[n]                                                       */
  const int32_t* row_ptr;  /* device, n+1                                                      */
  const int32_t* col_idx;  /* device, nnz                                                      */
  const double* val;       /* device, nnz (real) or 2*nnz (complex, interleaved re,im)         */
  int32_t is_complex;      /* 0 real, 1 complex                                                */
} mpk_csr;

/* Opaque ILU(0) handle: factor values on A's pattern, a copy of the pattern, the conjugate
 * transposed factor (built on first use by BiCG's M^H solve) and the flags of the
 * dependency-driven substitutions.  One solve at a time per handle. */
typedef struct mpk_ilu mpk_ilu;

/* mpk_opts.flags bits. */
#define MPK_FLAG_ETA0 1      /* GPBiCG with eta forced to 0 (it then reduces to BiCGSTAB)            */
#define MPK_FLAG_MP_MATRIX 2 /* every SpMV (A x, A^H p~, the final b - A x) promotes the binary64
                                entry a to the w-component number (a, 0, ..., 0) -- the same value --
                                and multiplies in full w-component arithmetic, matrix entry first:
                                the SpMV of the paper's rows without "_d" (Sec. 4); default (0) is
                                the mixed-precision SpMV of the "_d" rows                           */

typedef struct {
  double tol_rel;          /* eps_r of the stopping rule ||r|| < eps_r ||r0|| + eps_a (Alg. 3) */
  double tol_abs;          /* eps_a                                                            */
  int32_t maxit;           /* iteration limit (Sec. 4 uses 3n)                                  */
  int32_t check_every;     /* iterations queued between host checks of the device "done" flag */
  int32_t flags;           /* MPK_FLAG_* bits                                                   */
  int32_t true_res_period; /* P > 0: residual replacement.  After the stopping test of iteration
                              k, whenever k is a multiple of P or the recursive ||r_k|| passed the
                              test, the true residual b - A x_k is formed in the vector format
                              (the SpMV of r0) and its norm taken; above 10 (eps_r ||r0|| + eps_a)
                              it replaces r and a passed test is withdrawn (the iteration goes
                              on), else a passed test stands.  0: the test reads the recursive r
                              alone and b - A x is formed once, after the last iteration        */
  double* hist_dev;        /* nullable device array of maxit+1 doubles: leading component of
                              ||r_k||_2, k = 0..iters                                            */
  double* hist_true_dev;   /* nullable device array of maxit+1 doubles: leading component of
                              ||b - A x_k||_2 at every iteration k checked by the replacement
                              rule (entries of unchecked iterations are left as they were)      */
} mpk_opts;

typedef struct {
  int32_t status;          /* mpk_status of the solve                                           */
  int32_t iters;           /* iterations performed                                              */
  int32_t fail_row;        /* ILU failures: the row; otherwise -1                               */
  int32_t graph;           /* 1: the iterations ran as replays of one captured CUDA graph         */
  double res0;             /* ||b - A x0|| (leading component)                                  */
  double relres_rec;       /* ||r_k|| / ||r0|| of the recursively updated residual               */
  double relres_true;      /* ||b - A x_k|| / ||r0|| recomputed at the end in the vector format */
  float ms_solve;          /* device time of the solve (CUDA events on `stream`)                */
  int32_t hermitian;       /* BiCG: 1 if A was found equal to A^H (entries compared as numbers),
                              so that q~ = A^H p~ used A's own rows and no transpose was built     */
  int32_t replacements;    /* residual replacements performed (see true_res_period)              */
} mpk_info;

/* Library version (major*10000 + minor*100 + patch). */
int mpk_version(void);

/* Message of the last failing call on this host thread ("" if none). */
const char* mpk_last_error(void);

/* Number of CUDA kernels this library has launched in this process so far (all threads).
 * Lets a caller count the library's launches inside a timed region. */
uint64_t mpk_kernel_launches(void);

/* y = A x (Sec. 3 "mixed-precision SpMV": binary64 A, w-component vectors).  Row i is
 * accumulated in CSR order from 0: y_i = (((0 + a_i,j1 x_j1) + a_i,j2 x_j2) + ...), each
 * product and sum in w-component arithmetic (real D: one fused multiply-add per entry).  x_dev, y_dev: n*c*w doubles (c from A), must
 * not overlap. */
int mpk_spmv_mp(const mpk_csr* A, int w, const double* x_dev, double* y_dev, void* stream);

/* y = A x with A held in the vectors' w-component type (the SpMV of the paper's rows without
 * "_d", Sec. 4): each binary64 entry a is promoted to (a, 0, ..., 0) -- the same value -- and
 * multiplied as a full w-component number, matrix entry first; accumulation as mpk_spmv_mp.
 * For w = 1, 3, 4 the result equals mpk_spmv_mp's (exactly rounded products and sums); for
 * w = 2 the double-word product of two double words differs from the double word times binary64
 * product in rounding.  Arguments and errors as mpk_spmv_mp. */
int mpk_spmv_mp_matrix(const mpk_csr* A, int w, const double* x_dev, double* y_dev, void* stream);

/* out_dev[0 .. c*w) = <a, b> = sum_i conj(a_i) b_i in w-component arithmetic (Alg. 3 inner
 * products), reduced in a fixed order (deterministic for a given n). */
int mpk_dot(int n, int is_complex, int w, const double* a_dev, const double* b_dev, double* out_dev,
            void* stream);

/* The same inner product as mpk_dot, for callers that must not let the library allocate device
 * memory (the paper has no counterpart: this is a property of the library, not of the method).
 * Examples: a host that gives the library a fixed device-memory budget, a latency-critical loop
 * in which an allocation could synchronise the device, a plugin whose allocator owns all device
 * memory.  No cudaMalloc / cudaFree / pool allocation happens: the reduction scratch is a fixed
 * device array inside the library (256 KiB, kept by every GPU that loads the library until the
 * process exits).
 *   - n must not exceed MPK_DOT_NOALLOC_MAX_N; larger n returns MPK_INVALID_ARG (use mpk_dot).
 *   - The first call on each device looks up the scratch's device address (cudaGetSymbolAddress)
 *     and caches it; make that first call before any stream capture on that device.
 *   - All calls share the one scratch array, which keeps the last call's contents (the call
 *     clears the part that must start at zero).  Calls that overlap on the GPU -- on different
 *     streams, or on host threads without ordering -- race on it: serialise them.
 * Result, layout and summation order are those of mpk_dot (bit-identical results). */
#define MPK_DOT_NOALLOC_MAX_N 16777216
int mpk_dot_noalloc(int n, int is_complex, int w, const double* a_dev, const double* b_dev, double* out_dev,
                    void* stream);

/* Elementwise real w-component arithmetic on device arrays: out_i = a_i op b_i for i < n, each
 * entry w doubles (leading component first).  These are the operations every kernel of the
 * library performs on the formats of Sec. 2 (binary64 with w components): w = 1 plain binary64,
 * w = 2 the double-word algorithms of Joldes, Muller and Popescu (TOMS 2017), w = 3, 4 a
 * magnitude sort, an exact TwoSum chain and a top-down renormalisation to w components
 * (relative error at most about 2^(-53 w) of the exact result).  They are exported so that
 * callers and tests can check the arithmetic on its own against exact values.
 *   op: MPK_OP_ADD, MPK_OP_SUB, MPK_OP_MUL (a * b), MPK_OP_MUL_FP (a times the binary64 b_i[0]),
 *       MPK_OP_DIV (a / b), MPK_OP_DIV_FP (a / b_i[0]), MPK_OP_SQRT (square root of a; b unused,
 *       may be NULL).
 * a_dev, b_dev, out_dev: n*w doubles; out_dev may alias neither input.  n = 0 does nothing. */
#define MPK_OP_ADD 0
#define MPK_OP_SUB 1
#define MPK_OP_MUL 2
#define MPK_OP_MUL_FP 3
#define MPK_OP_DIV 4
#define MPK_OP_DIV_FP 5
#define MPK_OP_SQRT 6
int mpk_mp_op(int op, int w, int n, const double* a_dev, const double* b_dev, double* out_dev, void* stream);

/* Measurement aid: the one-way latency of a cross-SM notification on this GPU -- a strong relaxed
 * store by one SM seen by a strong relaxed polling load on another -- from `rounds` (1..10^6)
 * round trips of a counter between block 0 and block `partner` (1 .. SMs-1) of a cooperative
 * grid with one block per SM, timed with the device's global timer.  It is the synchronisation
 * cost that the level-scheduled substitutions and ILU(0) pay per level.  *one_way_ns (host)
 * receives the mean one-way time; sm_pair (host, nullable) the two blocks' SM ids.  Waits are
 * bounded; MPK_TIMEOUT if one ran out.  Synchronises `stream`. */
int mpk_probe_notify_ns(int rounds, int partner, double* one_way_ns, int* sm_pair, void* stream);

/* ILU(0) of A (Algorithm 1; the "!= 0" tests read as membership in A's stored pattern; the
 * update A_ij -= L_ik U_kj is one fused multiply-add; a zero pivot is an error instead of
 * being skipped).  Rows are factored in the level order of the lower triangle, either level by
 * level (a cooperative grid with a grid barrier between levels; taken when the levels are
 * narrow) or as a dataflow over chunk flags (wide levels); the environment variable
 * MPK_ILU_SCHEDULE=levels|dataflow forces one.  Either way the result equals the sequential KIJ
 * order bit for bit.  On success *out receives a new handle (free with
 * mpk_ilu0_destroy); on failure *out is NULL and *fail_row (if not NULL) the failing row.
 * The call synchronises `stream` to read the device status. */
int mpk_ilu0_factor(const mpk_csr* A, int prec, mpk_ilu** out, int* fail_row, void* stream);

/* ILU(0) of A in w-component arithmetic (w = 1..4; Algorithm 1 with every step in the
 * multi-component format of Sec. 2, the factor of the paper's rows without "_d").  Entry
 * values start as A's binary64 values (lower components 0); the KIJ updates
 * L_ik := A_ik / U_kk and A_ij := A_ij - L_ik * U_kj are the format's division, product (L_ik
 * first) and subtraction, each rounded to w components, in the sequential order.  The zero
 * pivot test reads the leading components.  The handle (prec MPK_ILU_MP) serves solves and
 * mpk_precond_apply with the same w only (MPK_INVALID_ARG otherwise); it holds nnz*c*w
 * doubles of factor.  Status, ownership and synchronisation as mpk_ilu0_factor. */
int mpk_ilu0_factor_mp(const mpk_csr* A, int w, mpk_ilu** out, int* fail_row, void* stream);

/* Copy the factor values (nnz*c doubles on A's pattern: strict lower part = L~ without its
 * unit diagonal, upper part with diagonal = U~; binary32/bfloat16 values widened) to
 * out_dev.  A MPK_ILU_MP handle copies nnz*c*w doubles (entry p: its w real components, then
 * its w imaginary components). */
int mpk_ilu0_values(const mpk_ilu* M, double* out_dev, void* stream);

/* Precision the handle was built with (mpk_ilu_prec), or -2 for a NULL handle. */
int mpk_ilu0_prec(const mpk_ilu* M);

/* Components per factor value: w for a MPK_ILU_MP handle, 1 otherwise; -2 for NULL. */
int mpk_ilu0_width(const mpk_ilu* M);

/* Substitution schedule the handle last used or was tuned to: 0 = static chunk schedule (every
 * level's chunks dealt over all SMs), 1 = owner-block schedule (contiguous row blocks per SM,
 * levels separated by block barriers, shared-memory values for dependencies inside a block),
 * 2 / 3 = owner-block schedule per thread-block cluster of 8 / 16 SMs (distributed shared
 * memory); *wpb_out (if not NULL): warps per SM.  -2 for NULL.  All give identical results.  A
 * solve times schedules 0 and 1 once per matrix pattern and keeps the faster; the environment
 * variable MPK_SUBST_SCHEDULE=static|owner|cluster8|cluster16 selects one instead. */
int mpk_ilu0_schedule(const mpk_ilu* M, int* wpb_out);

/* Dependency polling the substitutions last used or were tuned to (with the schedule, or forced by
 * MPK_SUBST_POLL): 0 = lane 0 polls each 32-row chunk's latest dependency, then every lane loads
 * its own; 1 = every lane polls its own from the start; 2 = as 1, sleeping a fixed short time
 * between polling rounds.  The results do not depend on it.  -2 for a NULL handle. */
int mpk_ilu0_polling(const mpk_ilu* M);

/* Level structure of the factor's triangles (the substitutions of Algorithm 2 and the ILU(0)
 * kernels run in this order): tri = 0 for L~, 1 for U~.  *nlevels_out (if not NULL) receives the
 * number of levels; depth_dev (if not NULL: n ints of device memory, the caller's) receives the
 * level of every row, 0 for a row with no dependency in that triangle, else 1 + the largest level
 * among the rows it depends on (the columns of its entries left of the diagonal for L~, right of
 * it for U~), ordered on `stream`.  MPK_INVALID_ARG for a NULL handle or another tri. */
int mpk_ilu0_levels(const mpk_ilu* M, int tri, int* nlevels_out, int* depth_dev, void* stream);

/* Testing aid for failure detection: the handle's substitutions leave row `row` unpublished
 * (-1: none, the default), so every row that depends on it waits until its bounded wait runs out
 * (about a second), the kernels leave, and the call returns MPK_TIMEOUT.  Nothing faults or
 * hangs; the error is reported once and the handle serves the next call.  MPK_INVALID_ARG for
 * a NULL handle or a row outside -1..n-1. */
int mpk_ilu0_test_withhold(mpk_ilu* M, int row);

void mpk_ilu0_destroy(mpk_ilu* M);

/* z = M^-1 r (trans = 0) or z = M^-H r (trans = 1) with M = L~U~ (Algorithm 2; the M^H solve
 * of Algorithm 3 is U~^H w = r then L~^H z = w).  r_dev, z_dev: n*c*w doubles, distinct. */
int mpk_precond_apply(const mpk_ilu* M, int w, int trans, const double* r_dev, double* z_dev, void* stream);

/* Solve A x = b with `method` in w-component arithmetic, preconditioned by M (NULL = none).
 * x_dev holds x0 on entry (Alg. 3 starts from a given x0) and the last iterate on return, for
 * every status.  Work vectors are allocated stream-ordered (cudaMallocAsync) and freed before
 * return.  The call synchronises `stream`.  info is filled in every case. */
int mpk_krylov_solve(int method, int w, const mpk_csr* A, const mpk_ilu* M, const double* b_dev, double* x_dev,
                     const mpk_opts* opts, mpk_info* info, void* stream);

/* Batched solve of nsys independent systems (the paper solves one system at a time).  A is
 * block-diagonal: system s owns rows and columns sys_rows[s] .. sys_rows[s+1]-1, and every
 * stored column of a row lies in its system's block
 * (checked; MPK_INVALID_ARG otherwise, nothing solved).  All systems advance together, each step
 * of every system in the same kernel launches; each system follows exactly the operation
 * sequence mpk_krylov_solve would perform on it alone (identical results), with its own scalars,
 * stopping test, breakdown test and iteration count, and a finished system keeps its iterate and
 * residual while the others go on.
 *   M: ILU(0) handle of the whole block-diagonal matrix (it equals the block-diagonal of the
 *      systems' ILU(0)s), or NULL.  With a binary32 / bfloat16 factor each system's right-hand
 *      side is scaled by its own power of two.
 *   sys_rows_host, sys_rows_dev: the same nsys+1 increasing row offsets (0 .. n) on host and device.
 *   b_dev, x_dev: n*c*w doubles (x0 in, iterates out).  infos: HOST array of nsys records.
 *   opts->hist_dev, opts->hist_true_dev (nullable): nsys*(maxit+1) doubles each, system s's
 *   history at s*(maxit+1).  The replacement rule (true_res_period) applies per system.
 * Returns MPK_OK when every system converged, else the first non-OK system status (or an error
 * code of the call itself).  The call synchronises `stream`. */
int mpk_krylov_solve_batched(int method, int w, const mpk_csr* A, int nsys, const int32_t* sys_rows_host,
                             const int32_t* sys_rows_dev, const mpk_ilu* M, const double* b_dev, double* x_dev,
                             const mpk_opts* opts, mpk_info* infos, void* stream);

/* ---- Learned correction of the ILU(0) factor (a learned preconditioner;
 * the paper has no counterpart) -----------------------------------------------------------------
 * A graph network on A's pattern (3 message-passing layers, hidden width 32, binary32 weights,
 * bfloat16-stored activations; the exact network is documented in csrc/gnn.cu) predicts one value
 * o_p per stored entry p; the corrected factor is f'_p = f_p (1 + 0.5 tanh o_p), so o = 0 is the
 * plain ILU(0) factor.  Real matrices only.  Parameters: MPK_GNN_NPARAMS binary32 values in one
 * device array.  work_dev: caller-owned device scratch of at least mpk_gnn_workspace_bytes(n, nnz,
 * nprobe, nsys) bytes; mpk_gnn_forward leaves in it the activations that mpk_gnn_backward reads,
 * so the three calls of a training step share one workspace and one (A, M). */
#define MPK_GNN_NPARAMS 12193
int mpk_gnn_nparams(void);
size_t mpk_gnn_workspace_bytes(int n, int nnz, int nprobe, int nsys);
/* o_dev[nnz] = network output for A and the factor M (its features read A's values and M's). */
int mpk_gnn_forward(const mpk_csr* A, const mpk_ilu* M, const float* params_dev, float* o_dev, void* work_dev,
                    size_t work_bytes, void* stream);
/* Training loss of the corrected factor and its gradient with respect to o:
 *   loss = mean over systems s of  sum_{i in s} ||((L'U' - A) W)_i||^2 / sum_{i in s} ||(A W)_i||^2
 * W: nprobe (1..16) probe vectors, n x nprobe row-major binary32 (device); L' unit lower, U' upper,
 * both from f'.  nsys > 1: A is a block-diagonal batch with row offsets sys_rows_dev[nsys+1].
 * loss_dev: one float; g_o_dev: nnz floats. */
int mpk_gnn_loss(const mpk_csr* A, const mpk_ilu* M, const float* o_dev, int nprobe, const float* probes_dev,
                 int nsys, const int32_t* sys_rows_dev, float* loss_dev, float* g_o_dev, void* work_dev,
                 size_t work_bytes, void* stream);
/* Training loss of the preconditioned operator and its gradient with respect to o:
 *   loss = mean over systems s of  sum_{i in s} ||(M'^-1 A W - W)_i||^2 / sum_{i in s} ||W_i||^2
 * with M' = L'U' from f' (binary32 arithmetic; four level-scheduled triangular solves per call,
 * two of them with the transposed factors).  nprobe 1..4; the pattern must be structurally
 * symmetric (MPK_INVALID_ARG otherwise).  Other arguments as mpk_gnn_loss. */
int mpk_gnn_loss_precond(const mpk_csr* A, const mpk_ilu* M, const float* o_dev, int nprobe,
                         const float* probes_dev, int nsys, const int32_t* sys_rows_dev, float* loss_dev,
                         float* g_o_dev, void* work_dev, size_t work_bytes, void* stream);
/* g_params_dev = d loss / d params by back-propagating g_o_dev through the network (after
 * mpk_gnn_forward with the same A, M, params and workspace). */
int mpk_gnn_backward(const mpk_csr* A, const mpk_ilu* M, const float* params_dev, const float* g_o_dev,
                     float* g_params_dev, void* work_dev, size_t work_bytes, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; step counts from 1). */
int mpk_gnn_adam(int nparams, float* params_dev, const float* grad_dev, float* m_dev, float* v_dev, float lr,
                 int step, void* stream);
/* Replace M's factor by f' = f (1 + 0.5 tanh o) in M's precision (repacks the triangles; the
 * conjugate transpose is rebuilt on its next use).  MPK_ILU_MP handles: MPK_INVALID_ARG (the
 * network reads binary64, binary32 and bfloat16 factors). */
int mpk_ilu0_correct(mpk_ilu* M, const float* o_dev, void* stream);

/* End-to-end convenience: host CSR, host b and x (x0 in, solution out).  Copies A and b to
 * the device, builds ILU(0) in `prec` (MPK_ILU_NONE: none; MPK_ILU_MP: in w components),
 * solves, copies x back and frees everything.  info->ms_solve covers the whole call. */
int mpk_solve_host(int method, int w, int prec, int32_t n, int32_t is_complex, const int32_t* row_ptr_host,
                   const int32_t* col_idx_host, const double* val_host, const double* b_host, double* x_host,
                   const mpk_opts* opts, mpk_info* info);

#ifdef __cplusplus
}
#endif
#endif /* MPK_H */
