/*
 * ozk2.h - C ABI of an FP64 matrix-multiplication emulation on FP8 tensor cores
 * (Ozaki-II scheme with FP8 E4M3 digits; Uchino, Ozaki, Imamura, arXiv:2603.10634),
 * built for NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every entry point
 *   - Matrices are row-major.  A is m x k with leading dimension lda >= max(1, k);
 *     B is k x n with ldb >= max(1, n); C is m x n with ldc >= max(1, n).
 *     Leading dimensions are counted in elements.
 *   - Pointers named A, B, C, D and every array argument are DEVICE pointers on the
 *     current CUDA device, owned by the caller.  Work is enqueued on `stream`
 *     (a cudaStream_t; NULL is the legacy default stream) and the call returns
 *     after enqueueing: results are valid once the stream has reached that point.
 *   - num_moduli is the paper's N, 1 <= N <= 20, taking the first N moduli of the
 *     hybrid list (Sec. III-D).  N = 12 reaches P/2 > 2^110 (Sec. III-D) and is the
 *     usual FP64-level choice; each further modulus adds about 4.5 bits.
 *   - Argument errors are detected on the host, return OZK2_ERR_INVALID_VALUE and
 *     touch no memory.  Errors of enqueued work (a CUDA launch failure) return
 *     OZK2_ERR_CUDA.  Conditions found by the kernels themselves (non-finite input,
 *     a bounded device wait that gave up) are recorded in a device flag word and
 *     reported by ozk2_device_status().
 *   - Not thread-safe: serialise calls that use the library-owned workspace.
 */
#ifndef OZK2_H
#define OZK2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ozk2_stream_t; /* identical to cudaStream_t */

typedef enum {
  OZK2_OK = 0,
  OZK2_ERR_INVALID_VALUE = 1, /* bad size, leading dimension, pointer or N      */
  OZK2_ERR_UNSUPPORTED = 2,   /* no sm_103a-class device, or a shape outside the
                                 supported range                               */
  OZK2_ERR_ALLOC = 3,         /* workspace allocation failed                     */
  OZK2_ERR_CUDA = 4,          /* a CUDA runtime / driver call failed             */
  OZK2_ERR_INTERNAL = 5,      /* inconsistent internal state                     */
  OZK2_ERR_TIMEOUT = 6,       /* a device-side wait exceeded its bound (kernel
                                 returned early; results are invalid)            */
  OZK2_ERR_NONFINITE = 7,     /* informational: NaN/Inf inputs were seen; the
                                 affected rows/columns of C are NaN              */
  OZK2_ERR_RANGE = 8          /* a scaled input exceeded the supported exponent
                                 range (results are invalid)                     */
} ozk2_status;

/*
 * ozk2_dgemm - C := A * B in emulated FP64.
 *
 * The operation of Sec. II (C ~ AB via A' = trunc(diag(mu) A), B' = trunc(B diag(nu)),
 * residues modulo p_1..p_N, CRT, inverse scaling) with the FP8 construction of
 * Sec. III: hybrid moduli (Sec. III-D), square moduli by Eq. 3matmult-notKaratsuba,
 * the rest by the Karatsuba split (Sec. III-B), accurate-mode scaling by an FP8
 * bound product (Sec. III-E).  3N + 1 FP8 products run on the tensor cores.
 *
 * m, n, k >= 0.  If m == 0 or n == 0 nothing is written; if k == 0, C is set to 0.
 * k is unrestricted: reductions longer than 2^16 are split into exact blocks.
 * C must not overlap A or B.  Uses a workspace owned by the library (one per
 * device, grown on demand with cudaMalloc, which synchronises the device when it
 * grows; see ozk2_workspace_size for its size).  Each output entry is the
 * correctly rounded value of the CRT result times 2^-(e_i + f_j).  Rows of A or
 * columns of B holding NaN/Inf give NaN rows/columns of C.
 */
ozk2_status ozk2_dgemm(int64_t m, int64_t n, int64_t k,
                       const double *A, int64_t lda,
                       const double *B, int64_t ldb,
                       double *C, int64_t ldc,
                       int num_moduli, ozk2_stream_t stream);

/*
 * ozk2_workspace_size - bytes of device workspace one call with these sizes needs:
 * the FP8 bound operands, M_N digit planes per operand (Sec. IV-B Eq. M), N int16
 * residue-product matrices and the scale vectors.  Returns 0 on invalid arguments.
 */
size_t ozk2_workspace_size(int64_t m, int64_t n, int64_t k, int num_moduli);

/*
 * ozk2_dgemm_ws - ozk2_dgemm with a caller-owned workspace (device memory of the current
 * device, at least ozk2_workspace_size bytes, 256-byte aligned).  The workspace is in use
 * until the stream passes this call.  OZK2_ERR_INVALID_VALUE, touching no memory, if it
 * is too small, misaligned, or not device memory of the current device (host, managed or
 * another GPU's memory, as cudaPointerGetAttributes reports it): the FP8 product kernels
 * read the workspace through TMA tensor maps, which this library builds only over the
 * calling GPU's own memory.  The same check applies to every caller workspace below.
 */
ozk2_status ozk2_dgemm_ws(int64_t m, int64_t n, int64_t k,
                          const double *A, int64_t lda,
                          const double *B, int64_t ldb,
                          double *C, int64_t ldc,
                          int num_moduli, void *workspace, size_t workspace_bytes,
                          ozk2_stream_t stream);

/*
 * ozk2_dgemm_noalloc - ozk2_dgemm for callers that may not allocate device memory
 * (their GPU memory is owned by a host application or framework, or they cannot
 * afford the device-wide synchronisation that cudaMalloc / cudaFree may cause).  It
 * allocates nothing: its workspace is a static device array of this library, of
 * OZK2_NOALLOC_MAX_BYTES bytes, which every GPU that loads it keeps until the process
 * exits.  The paper has no counterpart; this is an interface convenience.
 *
 * Same arguments and result as ozk2_dgemm: argument errors, m or n = 0 (nothing written)
 * and k = 0 (C = 0) behave exactly as there.  Returns OZK2_ERR_UNSUPPORTED, touching no
 * memory, when ozk2_workspace_size(m, n, k, num_moduli) exceeds OZK2_NOALLOC_MAX_BYTES
 * (for N = 12 that is square sizes up to 1664).  The first call on a device looks
 * the array up (cudaGetSymbolAddress, which loads this part of the library on that
 * device and so reserves the array there); make that first call before any stream
 * capture.  On a device without room for the array that first call fails with
 * OZK2_ERR_CUDA.  With eager module loading (CUDA_MODULE_LOADING=EAGER) the array is
 * reserved on every device the process initialises, for every user of the library,
 * whether or not this entry point is ever called.  All calls on a device share the
 * array and each call overwrites it (clearing what must start at zero), so calls whose
 * work overlaps on the GPU (other streams, other threads) race; serialise them.
 * Device-side conditions of the last call are read by ozk2_noalloc_device_status, not by
 * ozk2_device_status (which reads the library-owned workspace of ozk2_dgemm and reports
 * nothing about these calls); non-finite inputs give NaN rows/columns either way.
 */
#define OZK2_NOALLOC_MAX_BYTES (256u * 1024u * 1024u)
ozk2_status ozk2_dgemm_noalloc(int64_t m, int64_t n, int64_t k,
                               const double *A, int64_t lda,
                               const double *B, int64_t ldb,
                               double *C, int64_t ldc,
                               int num_moduli, ozk2_stream_t stream);

/* ozk2_noalloc_device_status - ozk2_device_status for the static workspace of
 * ozk2_dgemm_noalloc on the current device: synchronises `stream`, then reads and clears
 * the flag word of the last ozk2_dgemm_noalloc call (OZK2_OK if none has run on this
 * device).  Allocates nothing. */
ozk2_status ozk2_noalloc_device_status(ozk2_stream_t stream);

/* Operand form and scaling mode of ozk2_dgemm_ex. */
typedef enum { OZK2_OP_N = 0, OZK2_OP_T = 1 } ozk2_op;
typedef enum {
  OZK2_MODE_ACCURATE = 0, /* bound from an FP8 product of |A| and |B| (Sec. III-E); 3N + 1
                             FP8 products                                              */
  OZK2_MODE_FAST = 1      /* Cauchy-Schwarz bound from row / column norms (Sec. III-E,
                             "fast mode"); 3N FP8 products, a few bits less accuracy     */
} ozk2_mode;

/*
 * ozk2_dgemm_ex - C := op(A) * op(B) with the choices ozk2_dgemm fixes left open.
 *
 * op(A) is m x k: A itself (transa = OZK2_OP_N, A is m x k, lda >= max(1, k)) or A^T
 * (OZK2_OP_T, A is stored k x m, lda >= max(1, m)); op(B) is k x n: B (OZK2_OP_N, ldb >=
 * max(1, n)) or B^T (OZK2_OP_T, B stored n x k, ldb >= max(1, k)).  Row-major storage.
 * mode selects the scaling of Sec. III-E (accurate or fast).  block_m, block_n > 0 run the
 * product as independent emulations of block_m x block_n blocks of C with k unblocked
 * (the m/n blocking of Sec. IV-C), each with its own scaling, so the workspace is that of
 * one block; 0 means no blocking.  workspace (device, 256-byte aligned, at least
 * ozk2_workspace_size_ex bytes) or NULL for the library-owned workspace.
 */
ozk2_status ozk2_dgemm_ex(ozk2_op transa, ozk2_op transb,
                          int64_t m, int64_t n, int64_t k,
                          const double *A, int64_t lda,
                          const double *B, int64_t ldb,
                          double *C, int64_t ldc,
                          int num_moduli, ozk2_mode mode,
                          int64_t block_m, int64_t block_n,
                          void *workspace, size_t workspace_bytes,
                          ozk2_stream_t stream);

/* ozk2_workspace_size_ex - workspace bytes of one ozk2_dgemm_ex call with these sizes,
 * mode and blocking (the transposes do not change it); 0 on invalid arguments. */
size_t ozk2_workspace_size_ex(int64_t m, int64_t n, int64_t k, int num_moduli,
                              ozk2_mode mode, int64_t block_m, int64_t block_n);

/*
 * ozk2_dgemm_host - C := op(A) * op(B) with A, B and C in HOST memory (same shapes,
 * leading dimensions and ops as ozk2_dgemm_ex, no blocking).
 *
 * The library copies B and then A (in four line chunks) to the device on its own copy
 * stream while the scaling, bound product and residues of what has arrived run on
 * `stream`; the residue products and the CRT then run in output row blocks and each
 * block is copied back (on a second copy stream) while the next one is computed.  The
 * device arithmetic is that of ozk2_dgemm_ex, so C is bit-identical to the
 * device-buffer call.
 *   A, B, C    host pointers.  Page-locked (pinned) memory lets the copies overlap the
 *              kernels; pageable memory works, with less overlap.  They must stay valid
 *              and A, B unchanged until `stream` reaches the end of the call.
 *   workspace  device, 256-byte aligned, >= ozk2_workspace_size_host bytes (it also
 *              holds the device copies of A, B and C), or NULL for the library-owned
 *              workspace.
 * Asynchronous: returns after enqueueing; C is complete when `stream` is.  k = 0
 * synchronises `stream` and zero-fills C on the host.
 */
ozk2_status ozk2_dgemm_host(ozk2_op transa, ozk2_op transb,
                            int64_t m, int64_t n, int64_t k,
                            const double *A, int64_t lda,
                            const double *B, int64_t ldb,
                            double *C, int64_t ldc,
                            int num_moduli, ozk2_mode mode,
                            void *workspace, size_t workspace_bytes,
                            ozk2_stream_t stream);

/*
 * ozk2_dgemm_host_ex - ozk2_dgemm_host with flags (0: exactly ozk2_dgemm_host).
 *
 *   OZK2_HOST_INPUTS_READY  A and B are complete in host memory when the call is made
 *              (no earlier work on `stream` writes them).  Then, with the library-owned
 *              workspace (workspace = NULL) and when the previous call that used that
 *              workspace was a host-buffer call of the same sizes, the upload of A and B
 *              starts as soon as that call's kernels have read its own staged inputs for
 *              the last time, instead of after all earlier work on `stream`: back-to-back
 *              calls then overlap each upload with the previous call's residue products.
 *              Every kernel of the call still runs after earlier work on `stream`, and C
 *              is complete when `stream` reaches the end of the call, as without the flag.
 * Other flag bits: OZK2_ERR_INVALID_VALUE.
 */
#define OZK2_HOST_INPUTS_READY 1u

ozk2_status ozk2_dgemm_host_ex(ozk2_op transa, ozk2_op transb,
                               int64_t m, int64_t n, int64_t k,
                               const double *A, int64_t lda,
                               const double *B, int64_t ldb,
                               double *C, int64_t ldc,
                               int num_moduli, ozk2_mode mode, unsigned flags,
                               void *workspace, size_t workspace_bytes,
                               ozk2_stream_t stream);

/* ozk2_workspace_size_host - workspace bytes of one ozk2_dgemm_host call; 0 on
 * invalid arguments. */
size_t ozk2_workspace_size_host(int64_t m, int64_t n, int64_t k, int num_moduli, ozk2_mode mode);

/*
 * Batches of independent products C_i := A_i * B_i (row-major, as ozk2_dgemm), all with
 * the same N and mode, of any mix of shapes.  Each phase of the method runs as ONE
 * launch over the whole batch: the scaling, exponent, residue and CRT kernels map their
 * blocks to problems through a descriptor table, and the two FP8 product kernels are
 * persistent grouped GEMMs over the tiles of every problem (longest reductions first),
 * with each problem's operand tensor maps in device memory.  Every C_i is bit-identical
 * to ozk2_dgemm on the same inputs.  Problems with m or n = 0 are skipped; k = 0 gives
 * C_i = 0.  This is the batching the paper's small-size results call for (Sec. V).
 *
 * m, n, k, A, lda, B, ldb, C, ldc are HOST arrays of `count` entries; A[i], B[i], C[i]
 * are device pointers.
 */
typedef struct ozk2_batch_plan_st *ozk2_batch_plan;

/* ozk2_workspace_size_batched - workspace bytes of a batch plan; 0 on invalid sizes. */
size_t ozk2_workspace_size_batched(int count, const int64_t *m, const int64_t *n, const int64_t *k,
                                   int num_moduli, ozk2_mode mode);

/*
 * ozk2_batch_plan_create - validates the batch, lays out its workspace, encodes every
 * problem's descriptors on the host and enqueues their upload on `stream`.
 *   workspace  device, 256-byte aligned, >= ozk2_workspace_size_batched bytes, reserved
 *              for the plan until it is destroyed; NULL: the plan allocates its own.
 * The plan records the operand pointers: executing it reads A_i, B_i and writes C_i at
 * those addresses.  Not capturable (it copies from host memory); execute is.
 */
ozk2_status ozk2_batch_plan_create(ozk2_batch_plan *plan, int count,
                                   const int64_t *m, const int64_t *n, const int64_t *k,
                                   const double *const *A, const int64_t *lda,
                                   const double *const *B, const int64_t *ldb,
                                   double *const *C, const int64_t *ldc,
                                   int num_moduli, ozk2_mode mode,
                                   void *workspace, size_t workspace_bytes,
                                   ozk2_stream_t stream);

/* ozk2_batch_plan_execute - enqueues the whole batch on `stream` (device work only: a
 * few memsets and one launch per phase; capturable into a CUDA graph).  B's scaling and
 * residue kernels run on a second stream that the plan owns, forked from `stream` and
 * joined back to it by events, so the execution is complete when `stream` reaches its
 * end, and a graph captured from `stream` holds both branches.  Must be called on the
 * device the plan was created on; executions of one plan must not overlap. */
ozk2_status ozk2_batch_plan_execute(ozk2_batch_plan plan, ozk2_stream_t stream);

/* ozk2_batch_plan_workspace - the plan's device workspace (for ozk2_device_status). */
void *ozk2_batch_plan_workspace(ozk2_batch_plan plan);

/* ozk2_batch_plan_destroy - waits for the descriptor upload, frees what the plan
 * allocated.  Work already enqueued by execute must be complete if the plan owns its
 * workspace. */
void ozk2_batch_plan_destroy(ozk2_batch_plan plan);

/* ozk2_dgemm_batched - create (on the library-owned workspace when `workspace` is
 * NULL), execute and destroy a plan in one call. */
ozk2_status ozk2_dgemm_batched(int count,
                               const int64_t *m, const int64_t *n, const int64_t *k,
                               const double *const *A, const int64_t *lda,
                               const double *const *B, const int64_t *ldb,
                               double *const *C, const int64_t *ldc,
                               int num_moduli, ozk2_mode mode,
                               void *workspace, size_t workspace_bytes,
                               ozk2_stream_t stream);

/* ozk2_status_string - a static, human-readable name for a status code. */
const char *ozk2_status_string(ozk2_status status);

/*
 * ozk2_device_status - synchronises `stream`, then reads and clears the device flag
 * word of the given workspace (NULL: the library-owned workspace of the current
 * device).  Returns OZK2_OK, OZK2_ERR_INTERNAL (only in a library built with
 * -DOZK2_DEBUG: a kernel's range check failed, e.g. a digit beyond |d| <= 16 or a residue
 * outside its symmetric range), OZK2_ERR_TIMEOUT, OZK2_ERR_RANGE or OZK2_ERR_NONFINITE
 * (most severe first), or OZK2_ERR_CUDA if the synchronisation fails.
 */
ozk2_status ozk2_device_status(void *workspace, ozk2_stream_t stream);

/*
 * ozk2_moduli - writes the first N moduli of the hybrid list (Sec. III-D) to
 * p_out (host memory, N entries).  Returns N, or -1 if N is outside 1..20.
 */
int ozk2_moduli(int num_moduli, int32_t *p_out);

/*
 * ozk2_set_timing / ozk2_get_timing - per-phase timing of the next ozk2_dgemm calls
 * with CUDA events recorded on the call's stream (enable = 1 turns it on).
 * ozk2_get_timing waits for the last timed call and writes up to `max` phase times
 * in milliseconds, in the order: 0 scaling pass, 1 bound product, 2 exponents,
 * 3 residues and digits, 4 residue products, 5 CRT and inverse scaling
 * (the quant / gemms / requant / dequant split of Sec. V-C with requant fused into
 * phase 4).  Returns the number of phases written, or -1 if nothing was timed.
 */
void ozk2_set_timing(int enable);
int ozk2_get_timing(float *ms, int max);

/* ozk2_last_launch_count - kernels launched by the last ozk2_dgemm / ozk2_dgemm_ws
 * call on this thread (host-side count). */
int ozk2_last_launch_count(void);

/*
 * ozk2_set_wait_limit - the bound, in nanoseconds, of every device-side wait of the FP8
 * product kernels launched after this call (a wait on a TMA copy, a tensor-core product
 * or the epilogue).  0 restores the default of 4 s.  A wait that reaches the bound makes
 * the kernel stop issuing work, let the copies and products it has in flight complete,
 * free its tensor memory and return; the call's results are then invalid and
 * ozk2_device_status reports OZK2_ERR_TIMEOUT.  Returns the previous setting.
 * Process-wide; not a feature of the paper (failure detection of this library).
 */
uint64_t ozk2_set_wait_limit(uint64_t ns);

/*
 * ozk2_set_tile_n - the output tile width of the FP8 tensor-core products launched after
 * this call (and of batch plans created after it): 256 (128 x 256 tiles), 128 (128 x 128
 * tiles, for narrow or ragged products), or 0, the default: the library chooses 128 where
 * a 256-wide tile would pad the product's columns by a quarter or more, else 256 (a batch
 * plan applies that rule to each problem's residue products, which then run in up to two
 * grouped launches, one per width, and to the batch's total padded work for its bound
 * products).  Results are bit-identical for either width.  Returns the previous setting,
 * or -1 (unchanged) for other values.  Process-wide; a tuning knob (the moduli-and-tile
 * tuner measures the settings).
 */
int ozk2_set_tile_n(int tile_n);

/* ozk2_batch_plan_tile_n - the tile width a batch plan runs its residue products with:
 * 256 or 128, 0 when its problems use both widths, -1 for NULL. */
int ozk2_batch_plan_tile_n(ozk2_batch_plan plan);

/*
 * ozk2_set_square_split - the residue products of a square modulus p = s^2 (Eq.
 * 3matmult-notKaratsuba: X = A1 B2 + A2 B1, Z = A2 B2, C' = mod(s X + Z, p)) run as one
 * pass over both tensor-memory accumulators, or, for reductions of at most kmax terms, as
 * two single-slot passes (X, whose residue is kept, then Z), which lets the epilogue of
 * one pass overlap the next when k is short.  Applies to calls and batch plans made
 * after it; results are bit-identical either way.  Default 0 (never split: measured
 * neutral or slower on this GPU); a negative kmax only queries.  Returns the previous (or
 * current) setting.
 */
int64_t ozk2_set_square_split(int64_t kmax);

/*
 * ozk2_debug_inject_fault - host-side fault injection for tests of the error paths.
 * Arms one fault that fires once, at the next point where it applies, then disarms:
 *   OZK2_FAULT_ALLOC   the next workspace allocation of the library (the library-owned
 *                      workspace, a batch plan's private workspace or its pinned
 *                      descriptor staging) reports failure without allocating: the call
 *                      returns OZK2_ERR_ALLOC and touches no caller memory.
 *   OZK2_FAULT_LAUNCH  the next launch of an FP8 product kernel is not made and the call
 *                      returns OZK2_ERR_CUDA (C is not written: the CRT comes later).
 *   OZK2_FAULT_STALL   the next FP8 product kernel waits first on a barrier that nothing
 *                      signals; the wait runs out after the wait limit
 *                      (ozk2_set_wait_limit), the kernel returns early and
 *                      ozk2_device_status reports OZK2_ERR_TIMEOUT.
 * OZK2_FAULT_NONE disarms.  A negative kind only queries.  Returns the kind armed before
 * the call, or -1 (nothing changed) for an unknown kind.  The environment variable
 * OZK2_FAULT=alloc|launch|stall arms one fault when the library first needs the setting.
 * No fault is made on the GPU: every injected failure is a host-side decision or a
 * bounded wait.
 */
typedef enum {
  OZK2_FAULT_NONE = 0,
  OZK2_FAULT_ALLOC = 1,
  OZK2_FAULT_LAUNCH = 2,
  OZK2_FAULT_STALL = 3
} ozk2_fault;
int ozk2_debug_inject_fault(int kind);

/* ozk2_debug_timeline - of the last timed call: milliseconds from its start to the end
 * of each of the six phases (as ozk2_get_timing orders them).  Returns the number of
 * values written (6), or -1 if there is no timed call or max < 6. */
int ozk2_debug_timeline(float *ms, int max);

/*
 * ozk2_dgemm_backward - the gradients dA = dC B^T (m x k) and dB = A^T dC (k x n) of
 * C = A B (row-major, as ozk2_dgemm) by the same emulation, reusing the forward call's
 * scaling exponents e, f and digit planes of A' = trunc(diag(2^e) A), B' = trunc(B diag(2^f))
 * (Eqs. def:A', def:B').  The paper treats the product only; the construction is its own:
 *   dA: G'_ij = trunc(2^(g_i - f_j) dC_ij) with B' fixed, dA_ih = 2^-g_i (G' B'^T)_ih;
 *   dB: H'_ij = trunc(2^(h_j - e_i) dC_ij) with A' fixed, dB_hj = 2^-h_j (A'^T H')_hj;
 * g and h take the whole budget of P (Eq. condition: 2 sum |G'||B'| < P) from FP8 bound
 * products of |dC| with |B| and of |A| with |dC| (as accurate mode, Sec. III-E), so
 * 3N + 1 FP8 products run per gradient, as in a fresh emulation, but A and B are not
 * converted again (their planes are transposed), and one kernel converts dC for both.
 *   forward_workspace  device memory of the current device, the workspace of the
 *                      ozk2_dgemm_ws / ozk2_dgemm_ex call (accurate mode, no blocking,
 *                      same m, n, k, num_moduli) that computed C = A B, unchanged since
 *                      (at least ozk2_workspace_size bytes).  Read only.
 *   A, B, dC           device, row-major: A m x k (lda), B k x n (ldb), dC m x n (lddc).
 *   dA, dB             device outputs (ldda >= k, lddb >= n); either may be NULL (not
 *                      computed), not both.
 *   workspace          device, >= ozk2_workspace_size_backward bytes, 256-byte aligned,
 *                      or NULL for the library-owned workspace.
 * Each output entry is the correctly rounded value of its integer result; rows of dC and
 * of B holding NaN/Inf give NaN rows / columns of dA, columns of dC and of A NaN columns /
 * rows of dB.  m, n or k = 0: the outputs with an empty reduction are set to 0.
 */
ozk2_status ozk2_dgemm_backward(int64_t m, int64_t n, int64_t k,
                                const double *A, int64_t lda,
                                const double *B, int64_t ldb,
                                const double *dC, int64_t lddc,
                                double *dA, int64_t ldda,
                                double *dB, int64_t lddb,
                                int num_moduli, const void *forward_workspace,
                                size_t forward_workspace_bytes,
                                void *workspace, size_t workspace_bytes,
                                ozk2_stream_t stream);

/* ozk2_workspace_size_backward - bytes of one ozk2_dgemm_backward call's own workspace
 * (bound operands, the digit planes of dC's two integer matrices and of the transposed
 * A', B', the residue products of both gradients); 0 on invalid arguments. */
size_t ozk2_workspace_size_backward(int64_t m, int64_t n, int64_t k, int num_moduli);

/* ---------------------------------------------------------------------------
 * Parity hooks.  Each runs one step (or a prefix) of the method on its own so the
 * CPU oracle can check it.  Same conventions as above; all arrays are device
 * memory, and kp denotes the padded FP8 row length, kp = 32 * ceil(k / 32).
 * ------------------------------------------------------------------------- */

/*
 * ozk2_debug_fp8_gemm - D = A8 * B8^T with FP8 E4M3 operands and FP32 accumulation
 * on the tcgen05 tensor cores (the product used throughout Sec. III).  A8 is m x k
 * bytes with row stride lda8, B8 is n x k bytes with row stride ldb8 (both K-major);
 * lda8 and ldb8 must be multiples of 16 and the pointers 16-byte aligned.  D is
 * m x n float, row stride ldd.  Any k >= 1 is accepted; bytes past column k of a
 * row are never read.  The products are exact for integer-valued operands with
 * k * max|a| * max|b| <= 2^24 (Sec. III-B, Eq. error-free-FP8-matmult).
 */
ozk2_status ozk2_debug_fp8_gemm(int64_t m, int64_t n, int64_t k,
                                const uint8_t *A8, int64_t lda8,
                                const uint8_t *B8, int64_t ldb8,
                                float *D, int64_t ldd, ozk2_stream_t stream);

/*
 * ozk2_debug_scales - the accurate-mode scaling of Sec. III-E (workflow steps 1-3
 * of Sec. IV-B): e'_i, f'_j (Eq. def:mu'nu'), the E4M3 bound operands
 * Abar (m x kp) and Bbar^T (n x kp), the row / column maxima R_i, S_j of
 * Cbar = RU((1 + k 2^-24) Abar Bbar) (Eq. barCupper), and the exponents e_i, f_j of
 * Eqs. mu-computation / nu-computation.  Any output pointer may be NULL.
 */
ozk2_status ozk2_debug_scales(int64_t m, int64_t n, int64_t k,
                              const double *A, int64_t lda,
                              const double *B, int64_t ldb, int num_moduli,
                              int32_t *e, int32_t *f, int32_t *eprime, int32_t *fprime,
                              float *R, float *S, uint8_t *Abar, uint8_t *BbarT,
                              ozk2_stream_t stream);

/*
 * ozk2_debug_scales_ex - ozk2_debug_scales for op(A), op(B) and either scaling mode.
 * In fast mode R and S receive the round-up sums of squares of the scaled rows of op(A)
 * and columns of op(B) (the Cauchy-Schwarz bound that replaces the row / column maxima
 * of Cbar), and Abar, BbarT are not produced.
 */
ozk2_status ozk2_debug_scales_ex(ozk2_op transa, ozk2_op transb,
                                 int64_t m, int64_t n, int64_t k,
                                 const double *A, int64_t lda,
                                 const double *B, int64_t ldb, int num_moduli, ozk2_mode mode,
                                 int32_t *e, int32_t *f, int32_t *eprime, int32_t *fprime,
                                 float *R, float *S, uint8_t *Abar, uint8_t *BbarT,
                                 ozk2_stream_t stream);

/*
 * ozk2_debug_residue_planes - FP8 digit planes of A' = trunc(diag(2^e) A) and
 * B' = trunc(B diag(2^f)) for the given exponents (Eqs. def:A', def:B'; digit splits
 * of Sec. III-B and III-D).  planesA: M_N x m x kp bytes, planesB: M_N x n x kp bytes
 * (B transposed, K-major).  Square modulus l < 6 owns planes 2l, 2l+1 (d1, d2);
 * Karatsuba modulus l >= 6 owns planes 12 + 3(l-6) + {0,1,2} (d1, d2, d3).
 */
ozk2_status ozk2_debug_residue_planes(int64_t m, int64_t n, int64_t k,
                                      const double *A, int64_t lda,
                                      const double *B, int64_t ldb, int num_moduli,
                                      const int32_t *e, const int32_t *f,
                                      uint8_t *planesA, uint8_t *planesB,
                                      ozk2_stream_t stream);

/*
 * ozk2_debug_residue_products - C'_l = mod(A'_l B'_l, p_l), l = 1..N (Eq. CRTmatmul),
 * from the three FP8 digit products per modulus (Eqs. 3matmult-notKaratsuba and
 * C'-Karatsuba) for the given exponents.  Cres: N x m x n int16, contiguous,
 * symmetric residues in [-floor(p/2), p - 1 - floor(p/2)].
 */
ozk2_status ozk2_debug_residue_products(int64_t m, int64_t n, int64_t k,
                                        const double *A, int64_t lda,
                                        const double *B, int64_t ldb, int num_moduli,
                                        const int32_t *e, const int32_t *f,
                                        int16_t *Cres, ozk2_stream_t stream);

/*
 * ozk2_debug_backward_exponents - the exponents g (m, dC's rows) and h (n, dC's columns)
 * that the last ozk2_dgemm_backward call with these sizes used, read from its workspace
 * (NULL: the library-owned workspace).  Either output may be NULL.
 */
ozk2_status ozk2_debug_backward_exponents(int64_t m, int64_t n, int64_t k, int num_moduli,
                                          const void *workspace, int32_t *g, int32_t *h,
                                          ozk2_stream_t stream);

/*
 * ozk2_debug_crt - C = diag(2^-e) mod(sum_l q_l P/p_l C'_l, P) diag(2^-f)
 * (Eqs. CRT_finalreduction, inversescaling) from given residue products
 * Cres (N x m x n int16, contiguous) and exponents; each entry correctly rounded.
 */
ozk2_status ozk2_debug_crt(int64_t m, int64_t n, int num_moduli,
                           const int16_t *Cres, const int32_t *e, const int32_t *f,
                           double *C, int64_t ldc, ozk2_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* OZK2_H */
