// Internal declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace hbs {

// Device status block: two ints. Word 0 collects the report bits below until the host reads
// and clears it. Word 1 is the abort flag of the current run: set together with the timeout bit
// when a bounded wait gives up, so that the other CTAs of that run stop waiting too, and cleared
// by the host at the start of every run (a memset queued before the run's first kernel), so
// that a timeout left by an earlier run never cuts a later run short.
constexpr int kStatusNumeric = 1;   // bit set in the device status word on a bad pivot
constexpr int kStatusTimeout = 2;   // bit set when a bounded device-side wait gave up
constexpr int kAbortWord = 1;       // index of the abort flag in the status block
constexpr int kStatusWords = 2;

// One node of Algorithm 2 for the per-level sweep kernel. All matrices are row-major.
struct NodeTask {
  const double* Om;   // n x s test block Omega_tau   (leading dimension s)
  const double* Ps;   // n x s test block Psi_tau
  const double* Y;    // n x s sample block Y_tau
  const double* Z;    // n x s sample block Z_tau
  double* U;          // n x r output basis U_tau
  double* V;          // n x r output basis V_tau
  double* D;          // n x n output block D_tau
  double* WY;         // n x n workspace: Y_tau Omega_tau^dagger
  double* WZ;         // n x n workspace: Z_tau Psi_tau^dagger
  double* XY;         // n x r workspace: Y_tau P_tau
  double* XZ;         // n x r workspace: Z_tau Q_tau
  double* Om_p;       // this node's r x s rows of the parent's blocks (leading dimension s):
  double* Ps_p;       //   left child rows 0..r-1, right child rows r..2r-1; unused at the root
  double* Y_p;
  double* Z_p;
  int32_t n, r, s;
  int32_t is_root;    // 1: only D = Y_tau Omega_tau^dagger (root step of Algorithm 2)
};

// One small product task of Algorithm 1: C (m x ncols) = op1(A1) B1 [+ op2(A2) B2].
// op(A) = A (A stored m x k, leading dimension lda) or A^T (A stored k x m, leading dim lda).
struct GemmTask {
  const double* A1; const double* B1;
  const double* A2; const double* B2;   // A2 == NULL: single term
  double* C;
  int32_t m, k1, k2;
  int32_t lda1, lda2;
  int32_t ldb1, ldb2, ldc;
  int32_t t1, t2;                       // 1 = transpose
  int32_t ncols;                        // columns of C and B; 0 = the launch's ncols
};

// One node of a compressed problem, for building the work list of Algorithm 1 on the device:
// first row, row count (2r above the leaves; N when the tree has one node) and the arena
// offsets (doubles) of U, V (-1 at the root) and D.
struct ApplyNode {
  int64_t off;
  int64_t oU, oV, oD;
  int32_t n;
  int32_t pad;
};

// Writes Algorithm 1's work list for one problem (depth L, rank r, N rows; nodes indexed by node
// id) into out: the upward pass, levels L .. 1 (2^l node products each), then the downward pass,
// levels 0 .. L (2^l each), 2^(L+2) - 3 tasks in all (1 when L = 0). q-hat and u-hat of node t
// (levels >= 1) live in ws at (t - 2) r c and (2^(L+1) - 2 + t - 2) r c doubles (level-major,
// r x c each). trans swaps U and V and uses D^*.
cudaError_t launch_build_apply_tasks(const ApplyNode* nodes, int L, int r, int64_t N, int trans,
                                     int c, const double* arena, const double* X, double* Out,
                                     double* ws, GemmTask* out, cudaStream_t st);

// Shared memory of the sweep kernels for a node of n rows (sweep.cu).
size_t side_smem_doubles(int n, int s);
// The finish of a sweep (bases, D_tau, merges): FP64, FP32, or double-float (FP32 pairs).
constexpr int kFinishF64 = 0, kFinishF32 = 1, kFinishDF32 = 2;
size_t node_smem_bytes(int n, int r, int s, int finish);   // largest sweep-kernel tile
// The finish a height with nodes of up to n rows runs (the double-float finish falls back to FP64
// where its tiles exceed shared memory).
int effective_finish(int n, int r, int finish);
constexpr size_t kMaxNodeSmemBytes = 227 * 1024;
constexpr int kMaxS = 192;              // register tile of the sample-row streaming
constexpr int kMaxSideCluster = 8;      // CTAs sharing one test-block factorization

// Grids of the finish kernels of one height: merge_chunk = columns per merge CTA (8 .. 32),
// d_blocks = column blocks per node of the FP64 D kernels (1 .. 8); 0 = the automatic choice
// from the node count. Every choice rounds exactly alike.
struct FinishShape {
  int merge_chunk = 0;
  int d_blocks = 0;
};

// One tree height of Algorithm 2: the side kernel (FP64), then the bases, D_tau and merge
// kernels in the given finish precision. With marks (5 events), records them before the side
// kernel and after the side, bases, D and merge launches. With lq (a height whose side shape
// is R > 0), the side kernel takes the test blocks' factorizations from launch_side_lq's output
// instead of computing them.
cudaError_t launch_sweep_level(const NodeTask* d_tasks, int ntasks, int max_n, int max_r,
                               int max_s, int finish, int row_splits, int* d_status,
                               cudaStream_t st, cudaEvent_t* marks = nullptr,
                               FinishShape shape = FinishShape{}, const double* lq = nullptr);
// The side kernel of one height alone (for tuning; idempotent). R > 0: R row slices per
// (node, side), each CTA factoring the test block (or copying it from lq); R < 0: a cluster of
// -R CTAs per (node, side) sharing one factorization. df: the one-CTA form streams the sample
// rows in double-float (the reduced finishes; the cluster form streams in FP64 either way).
cudaError_t launch_side_only(const NodeTask* d_tasks, int ntasks, int max_n, int max_s,
                             int R, int* d_status, cudaStream_t st, const double* lq = nullptr,
                             bool df = false);
// The LQ of every test block of a height (both sides), written to lq: 2 ntasks images of
// side_lq_stride(max_n, max_s) doubles, (node, side) at (2 node + side) * stride.
cudaError_t launch_side_lq(const NodeTask* d_tasks, int ntasks, int max_n, int max_s, double* lq,
                           int* d_status, cudaStream_t st);
int64_t side_lq_stride(int max_n, int max_s);
bool side_cluster_fits(int n, int s, int C);
int side_row_splits(int ntasks, int n, int s);   // the automatic side shape (R as above)
// The side shape a height runs: row_splits when set (tuned), else the automatic one.
int side_shape(int ntasks, int n, int s, int row_splits);
cudaError_t launch_gaussian(int64_t count, uint32_t stream_id, uint64_t seed, double* out,
                            cudaStream_t st);
cudaError_t launch_sample_dense_f64(const double* A, int64_t lda, int64_t N, const double* Om,
                                    const double* Ps, int s, double* Y, double* Z,
                                    cudaStream_t st);
// The same products for A in page-locked host memory, streamed through the device in row
// blocks (a second stream copies block b+1 while block b is multiplied).
cudaError_t launch_sample_host_f64(const double* A, int64_t lda, int64_t N, const double* Om,
                                   const double* Ps, int s, double* Y, double* Z,
                                   cudaStream_t st);
// Tensor-core sampling (sample_tc.cu): A FP32 row-major (lda % 4 == 0), slices = 2 (bf16x3) or
// 3 (bf16x6), s <= 256; kchunk = reduction columns per split (0: chosen to fill the GPU). The
// scratch it grows holds the device status word at its start.
cudaError_t launch_sample_dense_tc(const float* A, int64_t lda, int64_t N, const double* Om,
                                   const double* Ps, int s, double* Y, double* Z, int slices,
                                   int kchunk, cudaStream_t st);
cudaError_t sample_tc_status(int* host_status, bool clear);
// ORs report bits into the status block (a timeout bit also raises the abort flag), as a wait
// that gave up would leave them; for tests of the host-side status handling.
cudaError_t sample_tc_inject(int bits);
// Column tiling shared by the tensor-core products: s <= 128 as one tile of s rounded up to 32,
// wider s as tiles of 128 (sample_tc.cu).
void column_tiles(int s, int* BN, int* BNt);
// FP64-class sampling by exact FP16 digit products on the tensor cores (sample_oz.cu):
// A FP64 row-major (any lda >= N), digits = 7 or 5, s <= 256, N <= 2^20. The scratch it grows
// holds the device status word at its start.
// shared_planes: one exponent per 64 x 64 block of A and its digit planes in one orientation,
// read transposed by the product with A^* (half the split's work and scratch).
cudaError_t launch_sample_dense_oz(const double* A, int64_t lda, int64_t N, const double* Om,
                                   const double* Ps, int s, double* Y, double* Z, int digits,
                                   bool shared_planes, cudaStream_t st);
cudaError_t sample_oz_status(int* host_status, bool clear);
cudaError_t sample_oz_inject(int bits);
// ncols: the column count of every task (1 .. 4 takes the grouped skinny kernel), or 0 when each
// task carries its own.
cudaError_t launch_gemm_tasks_f64(const GemmTask* d_tasks, int ntasks, int ncols, cudaStream_t st);

}  // namespace hbs
