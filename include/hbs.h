/*
 * hbs.h -- C ABI of the GB300 library for black-box randomized compression of HBS matrices
 * (Levitt & Martinsson, "Linear-Complexity Black-Box Randomized Compression of
 * Rank-Structured Matrices").
 *
 * The problem (Section 1): an N x N matrix A is reachable only through products X -> A X and
 * X -> A^* X. Draw Gaussian test matrices Omega, Psi (N x s), form the samples Y = A Omega and
 * Z = A^* Psi, and recover from {Y, Omega, Z, Psi} the telescoping factorization of Section
 * 3.3 (bases U_tau, V_tau and discrepancy blocks D_tau on the tree of Section 3.1) by the
 * level-by-level sweep of Algorithm 2. The factorization is applied by Algorithm 1.
 *
 * Conventions for every call below:
 *  - Real matrices only; "*" is the transpose (Section 2.1).
 *  - Every matrix argument is ROW-MAJOR with the leading dimension stated. Unless a call says
 *    otherwise, array pointers are DEVICE pointers on the current CUDA device.
 *  - The caller owns every input and output buffer and keeps it alive until the work queued on
 *    `cuda_stream` (a cudaStream_t; NULL = legacy default stream) has finished.
 *  - Calls are asynchronous on `cuda_stream` unless stated. Argument and shape errors are
 *    detected on the host before anything is queued or allocated and are returned at once.
 *  - Numerical failures found on the device (a zero or non-finite pivot of a triangular
 *    factor) and bounded device-side waits that gave up are recorded in a status word (one per
 *    handle for the sweep, one per device for the tensor-core sampling), read and cleared by
 *    hbs_sync_status() / hbs_sample_sync(). A wait that gives up also ends the other waits of
 *    the same run at once; the next run starts with that abort cleared, so a timeout never
 *    cuts a later run short (its report stays until it is read).
 *  - A handle belongs to the CUDA device that was current at hbs_plan; calls on it with
 *    another device current return HBS_ERR_ARG.
 *  - Every non-OK return leaves a message for hbs_last_error() (per calling thread).
 *  - The tree is the one of Section 3.1: root I = [0, N); the left child of a node of n
 *    indices receives the first ceil(n/2); nodes are split while larger than leaf_max, all
 *    leaves sit on level L; node ids follow Fig. 1 (root 1, children 2t and 2t+1).
 */
#ifndef HBS_H
#define HBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HBS_OK = 0,
  HBS_ERR_ARG = -1,         /* NULL pointer, non-positive size, bad enum, item out of range */
  HBS_ERR_SHAPE = -2,       /* (N, r, s, leaf_max) not admissible, see hbs_compress */
  HBS_ERR_NOMEM = -3,       /* device allocation failed */
  HBS_ERR_CUDA = -4,        /* a CUDA runtime call failed (message has the CUDA error) */
  HBS_ERR_NUMERIC = -5,     /* zero or non-finite diagonal of a triangular factor */
  HBS_ERR_TIMEOUT = -6,     /* a bounded device-side wait gave up */
  HBS_ERR_CALLBACK = -7,    /* the black-box operator callback returned non-zero */
  HBS_ERR_UNSUPPORTED = -8  /* valid request outside what this build implements */
} hbs_status;

typedef enum {
  HBS_PREC_FP64 = 0,        /* every step in IEEE binary64 on the FP64 pipe */
  HBS_PREC_MIXED_BF16X3 = 1,/* sampling: FP32 A and FP64 Omega split into 2 bfloat16 slices,
                               3 slice products on the tensor cores, FP32 accumulation over
                               chunks of 2048, chunks summed in FP64 (~16 significant bits) */
  HBS_PREC_MIXED_BF16X6 = 2,/* as above with 3 slices and 6 products (~24 significant bits) */
  HBS_PREC_FP64_TC = 3,     /* sampling: FP64 A and Omega written as 7 exact 8-bit digits per
                               entry (one exponent per 64-wide block; an error-free splitting in
                               the manner of Ozaki et al., Numer. Algorithms 59, 2012), the 28
                               digit-pair products with exactly representable FP32 sums on the
                               tensor cores, double-float accumulation over 2048 indices, FP64
                               beyond: FP64-class products (~55-bit terms). Sweep in FP64 as
                               HBS_PREC_FP64. Needs N <= 2^20 and about 28 N^2 bytes of device
                               scratch (the digit planes of A in both orientations) */
  HBS_PREC_MIXED_COMPENSATED = 4
                            /* sampling: as HBS_PREC_FP64_TC with 5 digits per entry (15
                               digit-pair products) and one exponent per 64 x 64 block of A, its
                               digit planes kept in one orientation (the product with A^* reads
                               them transposed): each entry is kept to ~2^-38 of the largest
                               entry of its block, so a row or column far below the rest of its
                               block loses relative accuracy (the products' normwise error is
                               unaffected); about 10 N^2 bytes of scratch. Sweep: the LQ of each test block
                               (nullspace, pseudo-inverse) and the bases in FP64, the sample
                               rows pushed through the LQ (see hbs_plan), D_tau and the
                               parent blocks in double-float arithmetic (pairs of FP32 numbers,
                               ~48 significant bits, FP32 exponent range: every intermediate
                               of those products must stay within about 1e-30 .. 1e38 in
                               magnitude) on the FP32 pipe */
} hbs_precision;

typedef enum { HBS_F64 = 0, HBS_F32 = 1 } hbs_dtype;

/* ---------------------------------------------------------------------------------------
 * Test matrices (Algorithm 2, first block; Section 2.3, step 2).
 * Fills out[0 .. N*s) (row-major N x s) with i.i.d. standard normals from the counter-based
 * generator Philox4x32-10 (Salmon et al., SC'11) and the Box-Muller transform:
 *   element e = i*s + j belongs to pair p = e / 2; counter = (p mod 2^32, p div 2^32,
 *   stream_id, 0), key = (seed mod 2^32, seed div 2^32); with output words x0..x3,
 *   u1 = (top 52 bits of x0*2^32+x1 + 1/2) 2^-52, u2 likewise from x2, x3,
 *   element 2p = sqrt(-2 ln u1) cos(2 pi u2), element 2p+1 = sqrt(-2 ln u1) sin(2 pi u2).
 * stream_id 0 draws Omega and 1 draws Psi in hbs_sample. out: device, FP64.
 * Errors: HBS_ERR_ARG (out NULL, N < 1 or s < 1), HBS_ERR_CUDA.
 */
int hbs_draw_gaussian(int64_t N, int32_t s, uint32_t stream_id, uint64_t seed, double* out,
                      void* cuda_stream);

/* ---------------------------------------------------------------------------------------
 * The black-box operator (Section 1): either a dense matrix or a callback.
 * Dense: A != NULL, row-major N x N with leading dimension lda >= N, element type `dtype`
 *   (HBS_F64, or HBS_F32 for the mixed precisions), in device memory, or -- HBS_F64 with
 *   HBS_PREC_FP64 only -- in page-locked host memory (cudaHostAlloc / cudaHostRegister): the
 *   products then stream A through the device in row blocks on an internal stream, each
 *   block's copy overlapping the previous block's products; the call stays ordered on
 *   cuda_stream and A must stay valid until the stream has passed it. Pageable host memory
 *   gives HBS_ERR_ARG.
 * Callback: A == NULL and fn != NULL. fn(user, trans, N, ncols, X, Out, cuda_stream) must
 *   queue Out = A X (trans = 0) or Out = A^* X (trans = 1) on cuda_stream, X and Out row-major
 *   N x ncols FP64 device arrays, and return 0 (any other value gives HBS_ERR_CALLBACK).
 */
typedef int (*hbs_matmat_fn)(void* user, int trans, int64_t N, int32_t ncols, const double* X,
                             double* Out, void* cuda_stream);

typedef struct {
  int64_t N;
  int32_t dtype;
  const void* A;
  int64_t lda;
  hbs_matmat_fn fn;
  void* user;
} hbs_operator;

/* Precision of the products (hbs_sample, hbs_sample_products): HBS_PREC_FP64 needs a dense A in
 * HBS_F64 or a callback; HBS_PREC_MIXED_BF16X3/X6 need a dense A in HBS_F32, 16-byte aligned,
 * with lda a multiple of 4 and s <= 256; HBS_PREC_FP64_TC and HBS_PREC_MIXED_COMPENSATED need a
 * dense A in HBS_F64 (any lda >= N), s <= 256 and N <= 2^20. All keep Omega, Psi, Y, Z in FP64. */

/* Randomized samples (Algorithm 2, first block): draws Omega (stream 0) and Psi (stream 1)
 * from `seed` as hbs_draw_gaussian does, then Y = A Omega and Z = A^* Psi.
 * Omega, Psi, Y, Z: device, FP64, row-major N x s (leading dimension s), written.
 * Errors: HBS_ERR_ARG, HBS_ERR_UNSUPPORTED (precision or dtype), HBS_ERR_CALLBACK, HBS_ERR_CUDA.
 */
int hbs_sample(const hbs_operator* op, int32_t s, uint64_t seed, int32_t precision,
               double* Omega, double* Psi, double* Y, double* Z, void* cuda_stream);

/* The products alone, for test matrices the caller already holds (Algorithm 2, "Multiply
 * Y = A Omega and Z = A^* Psi"): Omega, Psi read, Y, Z written; all device FP64 row-major
 * N x s. Same operator rules and errors as hbs_sample. */
int hbs_sample_products(const hbs_operator* op, int32_t s, int32_t precision, const double* Omega,
                        const double* Psi, double* Y, double* Z, void* cuda_stream);

/* Waits for `cuda_stream` and returns the device status of the tensor-core sampling on the
 * current device since the last call: HBS_OK, HBS_ERR_TIMEOUT if a bounded wait inside the
 * kernel gave up, or HBS_ERR_NUMERIC if HBS_PREC_FP64_TC met an Inf or NaN (the products are
 * then invalid). Clears the status. */
int hbs_sample_sync(void* cuda_stream);

/* ---------------------------------------------------------------------------------------
 * One compression problem: test matrices and samples of one N x N matrix.
 * Omega, Psi, Y, Z: device, FP64, row-major N x s, leading dimension s.
 * r: rank parameter r = k + p of Section 4 (block rank plus oversampling).
 */
typedef struct {
  int64_t N;
  int32_t r;
  int32_t s;
  int32_t leaf_max;
  const double* Omega;
  const double* Psi;
  const double* Y;
  const double* Z;
} hbs_problem;

typedef struct hbs_handle hbs_handle;   /* opaque: owns the factors and all workspace */

/* Plan a batch of compressions: validates every problem, builds every tree and allocates the
 * device arena for the factors and workspace. Queues no work. Admissible shapes (Section 4
 * asks for s >= max(r + m, 3r)): with L >= 1, every leaf has between r and s - r rows and
 * s >= 3r; with L = 0 (N <= leaf_max), N <= s. This build also needs s <= 192 and, for every
 * node of n rows, the sweep kernels' shared-memory tiles within 227 KB: the test block,
 * n (s + 1) + 2n doubles; the basis tile, r (n + 1) + n (r + 1) + 10 r doubles (floats with
 * HBS_PREC_MIXED_BF16X3/X6); the reduced-precision D tile below.
 * Sweep precision: HBS_PREC_FP64 and HBS_PREC_FP64_TC keep every step in FP64; every other
 * precision keeps the LQ of each test block (nullspace and pseudo-inverse) in FP64 and pushes
 * the sample rows through it in double-float where a height runs the one-CTA side form (in FP64
 * where it runs the cluster form; a height that falls back to the FP64 finish, below, streams
 * in FP64); HBS_PREC_MIXED_BF16X3/X6 compute the bases, D_tau and the parent
 * blocks in FP32, HBS_PREC_MIXED_COMPENSATED the bases in FP64 and D_tau and the parent blocks
 * in double-float (factors stored in FP64). The D and merge tiles of the reduced finishes take
 * r (n + 1) + 3 n r + n (n + 1) + n^2 values (4-byte floats, or 8-byte pairs); a tree height
 * whose double-float tiles exceed 227 KB (n near 96 and above) runs D_tau and the merges in FP64
 * instead.
 * Errors: HBS_ERR_ARG, HBS_ERR_SHAPE, HBS_ERR_UNSUPPORTED, HBS_ERR_NOMEM, HBS_ERR_CUDA.
 */
int hbs_plan(int32_t batch, const hbs_problem* probs, int32_t precision, hbs_handle** out);

/* Run Algorithm 2 for every problem of a planned handle on `cuda_stream`. `probs` must have
 * the same batch size and shapes as at planning; its pointers may differ. The factors of the
 * previous execution are overwritten.
 * Errors: HBS_ERR_ARG (NULL, shape differs from the plan), HBS_ERR_CUDA.
 */
int hbs_execute(hbs_handle* h, const hbs_problem* probs, void* cuda_stream);

/* hbs_plan followed by hbs_execute. */
int hbs_compress(int32_t batch, const hbs_problem* probs, int32_t precision, hbs_handle** out,
                 void* cuda_stream);

/* Algorithm 2 from the operator on, for a handle planned for one problem: hbs_sample into
 * probs->Omega, Psi, Y, Z (draws from `seed`, products at `precision`), then hbs_execute, with
 * the leaves' test-block factorizations overlapped with the products. The LQ of each leaf's
 * Omega_tau and Psi_tau (Section 2.4) needs only the test matrices -- the remark of Section 1
 * that the test matrices can be drawn, and all work that depends on them alone be done, before
 * the operator is applied once -- so it runs on a second stream owned by the handle (highest
 * stream priority) from the draws on, and `cuda_stream` waits for it before the sweep. The
 * leaf level's side kernel then takes those factorizations instead of computing them: the
 * factors are bit-identical to hbs_sample + hbs_execute. Where the leaf height runs the cluster
 * form of the side kernel (a tree with few leaves), or a reduced sweep precision streams the
 * leaves' sample rows in double-float (there the fused side kernel is faster), nothing is
 * overlapped and the call equals hbs_sample + hbs_execute.
 * probs->Omega, Psi, Y and Z are written (writable device buffers, N x s FP64 row-major).
 * op->N must equal probs->N; the operator rules are hbs_sample's. The handle's second stream
 * and its image buffer (2 leaves (n (s + 1) + 2 n) doubles for leaves of n rows) are made on
 * the first call; a later call must be ordered after the earlier one's sweep (the same stream,
 * or the caller's synchronization). A call made while `cuda_stream` is being captured records
 * the fork and join into the capture.
 * Errors: those of hbs_sample and hbs_execute; HBS_ERR_ARG when the handle holds more than one
 * problem; HBS_ERR_NOMEM.
 */
int hbs_sample_execute(hbs_handle* h, const hbs_operator* op, uint64_t seed, int32_t precision,
                       const hbs_problem* probs, void* cuda_stream);

/* Algorithm 1: Out = A~ X (trans = 0) or A~^* X (trans = 1) for the compressed form of problem
 * `item` of the handle. X, Out: device, FP64, row-major N x ncols, leading dimension ncols,
 * must not overlap. The handle keeps a workspace of 2 (2^(L+1) - 2) r ncols doubles, grown
 * (by cudaMalloc, on the first call that needs more) and reused.
 * Errors: HBS_ERR_ARG, HBS_ERR_NOMEM, HBS_ERR_CUDA.
 */
int hbs_apply(hbs_handle* h, int32_t item, int trans, int32_t ncols, const double* X,
              double* Out, void* cuda_stream);

/* Algorithm 1 for every problem of the handle at once: Out[i] = A~_i X[i] (or A~_i^* X[i]),
 * X[i], Out[i] device FP64 row-major N_i x ncols[i] (leading dimension ncols[i]); X, Out and
 * ncols are host arrays with one entry per problem. The upward pass runs one launch per tree
 * height and the downward pass one per depth across all problems (2 max L + 1 launches). The
 * handle keeps a workspace (sum over problems of 2 (2^(L+1) - 2) r ncols doubles), grown by
 * cudaMalloc on the first call that needs more. Errors: HBS_ERR_ARG, HBS_ERR_NOMEM, HBS_ERR_CUDA.
 */
int hbs_apply_batch(hbs_handle* h, int trans, const double* const* X, double* const* Out,
                    const int32_t* ncols, void* cuda_stream);

/* Overwrites every factor of the handle from `src` (host or device), in the order of
 * hbs_copy_factors: per problem, per node id 1 .. 2^(L+1) - 1, U (n x r) and V (n x r) for nodes
 * on levels 1..L, then D (n x n; n = 2r at the root, or N when L = 0), all row-major FP64.
 * This turns any telescoping factorization of Section 3.3 (for instance a known HBS operator to
 * be used as a black box) into a handle that hbs_apply can apply. Asynchronous on cuda_stream.
 * Errors: HBS_ERR_ARG, HBS_ERR_CUDA. */
int hbs_load_factors(hbs_handle* h, const void* src, void* cuda_stream);

/* Tuning of the sweep launches (Algorithm 2 runs a side kernel, then the bases, D_tau and merge
 * kernels, per tree height). The side kernel's shape per height is one integer R: R > 0 splits
 * each (node, side) into R row slices, each CTA factoring the test block itself; R = -C (C = 2..8)
 * gives each (node, side) a thread-block cluster of C CTAs that share one factorization (rows
 * owned round-robin, reflectors published through distributed shared memory; C = 1 is that
 * form on one CTA, the sample rows updated with the factorization); 0 = automatic.
 * Every shape rounds exactly alike, so the factors do not depend on the tuning.
 * hbs_autotune times R = 1, 2, 3, 4, 6, 8, 12, 16 and C = 1, 2, 3, 4, 6, 8 (at most n/8, and C only
 * where the cluster's shared-memory tile fits) on the handle's current inputs -- execute the
 * handle once first -- and keeps the fastest; then, per height, the grids of the finish kernels
 * (the merges' column chunk, 8 .. 32, and for the FP64 finish the D kernels' column blocks per
 * node, 1 .. 8), kept until the next hbs_autotune. It synchronizes cuda_stream and leaves the
 * factors unchanged (every shape rounds alike). hbs_get_tuning returns the number of heights in *heights and copies up to `count`
 * values to R (may be NULL); hbs_set_tuning installs saved ones (values below -8 read as -8).
 * Errors: HBS_ERR_ARG, HBS_ERR_CUDA. */
int hbs_autotune(hbs_handle* h, void* cuda_stream);

/* Measurement of the sweep (Algorithm 2, no counterpart in the paper): runs the handle's sweep
 * once more on cuda_stream with plain launches (no graph) and CUDA events between them, and
 * writes, per tree height t (finest first), the device times in ms of its four phases to
 * ms[4t .. 4t+3]: the side kernel (LQ of the test blocks, sample rows), the bases, D_tau, and
 * the merges into the parent's blocks (at most `count` values; ms may be NULL). *heights gets
 * the number of heights. Execute the handle once first; the factors are recomputed from the
 * same inputs. Synchronizes cuda_stream. Errors: HBS_ERR_ARG, HBS_ERR_CUDA. */
int hbs_profile_sweep(hbs_handle* h, void* cuda_stream, float* ms, int32_t count,
                      int32_t* heights);
int hbs_get_tuning(const hbs_handle* h, int32_t* R, int32_t count, int32_t* heights);
int hbs_set_tuning(hbs_handle* h, const int32_t* R, int32_t count);

/* hbs_execute captures the sweep's launches into a CUDA graph the first time it sees a set of
 * input pointers and replays it afterwards (a stream being captured by the caller gets plain
 * launches instead). enable = 0 turns this off for the handle. Errors: HBS_ERR_ARG. */
int hbs_set_graph(hbs_handle* h, int enable);

/* Waits for the handle's queued work (cudaStreamSynchronize on cuda_stream) and returns the
 * device status of its executions since the last call: HBS_OK, HBS_ERR_TIMEOUT if a bounded
 * wait of the sweep gave up (the factors of that run are then invalid), or HBS_ERR_NUMERIC
 * (zero or non-finite pivot). Clears the status word. */
int hbs_sync_status(hbs_handle* h, void* cuda_stream);

/* For tests of the status handling (not for production use): ORs `bits` (1 = numeric,
 * 2 = timeout) into the status word of handle h -- or, with h == NULL, into the tensor-core
 * sampling status of the current device, where that sampling has run -- exactly as a failing
 * pivot or a device-side wait that gave up would leave it, without running any kernel. A
 * timeout bit also raises the abort flag of the current run. Synchronous.
 * Errors: HBS_ERR_ARG (unknown bits), HBS_ERR_CUDA. */
int hbs_test_inject_status(hbs_handle* h, int32_t bits);

/* Frees the handle and everything it owns (NULL-safe). The caller must make sure no queued
 * work still uses it. */
void hbs_free(hbs_handle* h);

/* Message for the last non-OK status returned to the calling thread ("" if none). */
const char* hbs_last_error(void);

/* ---------------------------------------------------------------------------------------
 * Introspection (for tests and tools; synchronous, not on any hot path).
 */

/* Depth L and, when the arrays are non-NULL, the 0-based offsets and sizes of nodes
 * 1 .. 2^(L+1) - 1 of problem `item` written at indices 0 .. 2^(L+1) - 2 (host arrays of at
 * least 2^(L+1) - 1 entries). */
int hbs_tree(const hbs_handle* h, int32_t item, int32_t* L, int64_t* offsets, int64_t* sizes);

/* Tree of Section 3.1 without a handle: same output as hbs_tree; max_nodes bounds the arrays.
 * Errors: HBS_ERR_ARG (N < 1, leaf_max < 1, arrays too small). */
int hbs_tree_build(int64_t N, int32_t leaf_max, int32_t* L, int64_t* offsets, int64_t* sizes,
                   int64_t max_nodes);

/* Copies the factors of node `node` (Fig. 1 numbering) of problem `item`: U and V (n x r) for
 * nodes on levels 1..L, D (n x n; for the root n = 2r, or N when L = 0). Destination pointers
 * may be host or device (any may be NULL to skip). Waits for the device. Row-major. */
int hbs_get_node(const hbs_handle* h, int32_t item, int64_t node, int32_t* n, double* U,
                 double* V, double* D);

/* Total bytes of all factors of the handle, and an asynchronous copy of them to `dst` (host
 * or device) in the handle's arena order: per item, per node id 1.., U, V then D. */
size_t hbs_factor_bytes(const hbs_handle* h);
int hbs_copy_factors(const hbs_handle* h, void* dst, void* cuda_stream);

/* ---------------------------------------------------------------------------------------
 * Measurement support (no counterpart in the paper): the FP64 (DFMA) and FP32 (FFMA) multiply-
 * add throughput of the current GPU in TFLOP/s, timed with CUDA events around kernels that keep
 * every SM's pipes busy with independent chains (a warm-up launch, then five). These are the
 * denominators of the roofline fractions of the FP64-pipe and double-float kernels.
 * Synchronizes cuda_stream; allocates 16 bytes. Errors: HBS_ERR_ARG, HBS_ERR_NOMEM, HBS_ERR_CUDA.
 */
int hbs_probe_peaks(double* fp64_tflops, double* fp32_tflops, void* cuda_stream);

/* The same for the FP64 tensor instruction (mma.sync m8n8k4 with FP64 operands, 512 flops per
 * warp instruction), in TFLOP/s; this library does not use it (it shares the FP64 units' rate).
 * Synchronizes cuda_stream; allocates 16 bytes. Errors: HBS_ERR_ARG, HBS_ERR_NOMEM, HBS_ERR_CUDA. */
int hbs_probe_dmma(double* tflops, void* cuda_stream);

/* No counterpart in the paper: a probe of the tcgen05 MMA issue rate behind the digit products'
 * bound. On every SM one thread issues back-to-back M = N = 128, K = 16 FP16 MMAs while eight
 * other warps of the CTA are idle (cycles_per_mma[0]), run FP32 TwoSum chains (cycles_per_mma[1])
 * or run them only on the three warp schedulers the issuing warp does not use
 * (cycles_per_mma[2]); each entry is SM clock cycles per MMA, averaged over the SMs. The tensor
 * pipe's own rate is 64 cycles per MMA on GB300. Synchronizes the stream; allocates and frees a
 * few bytes of device memory.
 * Errors: HBS_ERR_ARG (NULL), HBS_ERR_TIMEOUT (the bounded wait for the MMAs gave up),
 * HBS_ERR_CUDA. */
int hbs_probe_mma_issue(double* cycles_per_mma, void* cuda_stream);

/* ---------------------------------------------------------------------------------------
 * Apply without allocating (no counterpart in the paper; a service of this library).
 *
 * hbs_apply grows a device workspace with cudaMalloc the first time it needs more. Some callers
 * must not allocate: cudaMalloc synchronizes the whole device and fails when another allocator
 * (for instance a framework's caching pool) already holds the GPU's memory, which latency-bound
 * services and black-box operator callbacks (hbs_matmat_fn) that apply a compressed matrix in
 * the middle of someone else's stream cannot accept. hbs_apply_static computes exactly what
 * hbs_apply computes (Algorithm 1, same kernel) but keeps its workspace and its work list in
 * fixed arrays inside the library (file-scope device memory, reserved on every GPU that loads
 * the library until the process exits), so it calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 * Limits: the workspace of one call, 2 (2^(L+1) - 2) r ncols doubles, must not exceed
 * HBS_APPLY_STATIC_MAX_DOUBLES, and the work list, 2^(L+2) - 3 node products (2^(L+1) - 1 when
 * L = 0), must not exceed HBS_APPLY_STATIC_MAX_TASKS; larger requests return
 * HBS_ERR_UNSUPPORTED with the limit in the message, before anything is queued.
 *
 * Set-up: the device addresses of the two arrays are looked up (cudaGetSymbolAddress, with the
 * device current, result checked) once per device, by hbs_plan on the device it plans for, or
 * else by the first hbs_apply_static call on a device. That lookup loads the arrays onto the
 * device, which then holds them (about 17.3 MiB) until the process exits, so plan (or make the
 * first call) before another allocator takes the GPU's memory; when the first call does the
 * set-up, make it before any stream capture. A call queues only kernels on cuda_stream: the
 * work list is written into its fixed array by a kernel, with no host-to-device copy.
 * Every call on a device shares the same two arrays and they keep the last call's contents
 * (nothing in them needs to start at zero: every entry a call reads it has written first).
 * Calls whose GPU work overlaps in time -- on different streams, or from several threads --
 * race on the arrays; queue them on one stream or order them yourself.
 * Arguments and errors otherwise as hbs_apply.
 */
#define HBS_APPLY_STATIC_MAX_DOUBLES 2097152   /* 16 MiB of FP64 workspace per device */
#define HBS_APPLY_STATIC_MAX_TASKS 16384      /* 1.25 MiB of work list per device */
int hbs_apply_static(const hbs_handle* h, int32_t item, int trans, int32_t ncols,
                     const double* X, double* Out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* HBS_H */
