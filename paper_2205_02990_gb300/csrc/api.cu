// C ABI of include/hbs.h: argument checks, the Section 3.1 tree, the device arena, the
// per-level work lists of Algorithm 2 and Algorithm 1, and the launches.
//
// Arena layout (doubles), one allocation per handle:
//   [factors]   per item, per node id 1..2^(L+1)-1: U (n x r), V (n x r) for levels >= 1,
//               then D (n x n; root: 2r x 2r, or N x N when L = 0)
//   [workspace] per item, per node on levels >= 1: Y Omega^+ and Z Psi^+ (n x n each)
//   [blocks]    per item, per node on levels 0..L-1: the node's Omega, Psi, Y, Z blocks
//               (2r x s each), filled by its children (Eq. omega_tau_and_y_tau)
// Work lists: height t = L_i - level groups level L_i - t of every item, so one launch per
// height covers a whole batch of trees of different depths; heights run finest first.
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hbs.h"
#include "hbs_internal.cuh"

using hbs::GemmTask;
using hbs::NodeTask;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(HBS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int ok() {
  g_last_error.clear();
  return HBS_OK;
}

// Section 3.1 tree: depth, offsets and sizes indexed by node id (entry 0 unused).
void build_tree(int64_t N, int64_t leaf_max, int* L, std::vector<int64_t>* off,
                std::vector<int64_t>* size) {
  int depth = 0;
  while (true) {
    const int64_t biggest = (N + (int64_t(1) << depth) - 1) >> depth;   // ceil(N / 2^depth)
    if (biggest <= leaf_max) break;
    ++depth;
  }
  const int64_t count = int64_t(1) << (depth + 1);
  off->assign(count, 0);
  size->assign(count, 0);
  (*size)[1] = N;
  for (int64_t t = 1; t < (int64_t(1) << depth); ++t) {
    const int64_t left = ((*size)[t] + 1) / 2;
    (*off)[2 * t] = (*off)[t];
    (*size)[2 * t] = left;
    (*off)[2 * t + 1] = (*off)[t] + left;
    (*size)[2 * t + 1] = (*size)[t] - left;
  }
  *L = depth;
}

struct Item {
  int64_t N = 0;
  int r = 0, s = 0, leaf_max = 0, L = 0;
  std::vector<int64_t> off, size;
  std::vector<int64_t> oU, oV, oD, oWY, oWZ, oXY, oXZ, oOm, oPs, oY, oZ;   // arena offsets
  const double *Om = nullptr, *Ps = nullptr, *Y = nullptr, *Z = nullptr;
  int64_t node_rows(int64_t t) const { return level_of(t) == L ? size[t] : 2 * r; }
  int level_of(int64_t t) const {
    int l = 0;
    while ((int64_t(2) << l) <= t) ++l;
    return l;
  }
};

struct Height {
  std::vector<NodeTask> tasks;
  NodeTask* d_tasks = nullptr;
  int max_n = 0, max_r = 0, max_s = 0;
  int R = 0;                  // side-kernel row splits (0: automatic, > 0: tuned)
  hbs::FinishShape fs;        // grids of the finish kernels (0: automatic)
};

}  // namespace

struct hbs_handle {
  int precision = 0;
  int device = -1;            // the CUDA device current at hbs_plan; every call must run there
  std::vector<Item> items;
  hbs::ApplyNode* d_nodes = nullptr;   // per item, per node id: Algorithm 1's node table
  std::vector<int64_t> node_base;      // first entry of each item's table in d_nodes
  double* arena = nullptr;
  size_t arena_doubles = 0;
  size_t factor_doubles = 0;
  int* d_status = nullptr;
  std::vector<Height> heights;
  bool tasks_uploaded = false;
  double* apply_ws = nullptr;
  size_t apply_ws_doubles = 0;
  GemmTask* d_gemm = nullptr;
  size_t d_gemm_cap = 0;
  // the work list in d_gemm was built for these arguments (hbs_apply reuses it when they repeat)
  struct ApplyKey {
    int item = -1, trans = 0, ncols = 0;
    const double* X = nullptr;
    double* Out = nullptr;
    double* ws = nullptr;
    cudaStream_t st = nullptr;
    bool operator==(const ApplyKey& o) const {
      return item == o.item && trans == o.trans && ncols == o.ncols && X == o.X && Out == o.Out &&
             ws == o.ws && st == o.st;
    }
  } apply_key;
  // likewise for hbs_apply_batch and d_batch: direction, stream, workspace, then per item
  // (X, Out, columns)
  std::vector<uintptr_t> batch_key;
  std::vector<int> batch_sizes;
  int batch_ncols = 0;
  std::vector<int> tuned_R;   // per height, kept across task rebuilds
  std::vector<hbs::FinishShape> tuned_fs;
  // the sweep's launches captured once per set of inputs and replayed; graph_pre: the same
  // with the leaves' test blocks factored beforehand (hbs_sample_execute)
  bool use_graph = true;
  cudaGraphExec_t graph_exec = nullptr;
  cudaGraphExec_t graph_pre = nullptr;
  cudaStream_t capture_stream = nullptr;
  // hbs_sample_execute: the leaves' LQ images, the stream they are made on (while the products
  // run on the caller's stream) and the events joining the two
  double* lq_buf = nullptr;
  size_t lq_doubles = 0;
  cudaStream_t lq_stream = nullptr;
  cudaEvent_t ev_drawn = nullptr, ev_lq = nullptr;
  // hbs_apply_batch workspace and task list
  double* batch_ws = nullptr;
  size_t batch_ws_doubles = 0;
  GemmTask* d_batch = nullptr;
  size_t d_batch_cap = 0;
};

namespace {

// The finish precision of a sweep planned with `precision`.
int finish_of(int precision) {
  if (precision == HBS_PREC_MIXED_BF16X3 || precision == HBS_PREC_MIXED_BF16X6) return hbs::kFinishF32;
  if (precision == HBS_PREC_MIXED_COMPENSATED) return hbs::kFinishDF32;
  return hbs::kFinishF64;
}

bool known_precision(int precision) {
  return precision == HBS_PREC_FP64 || precision == HBS_PREC_MIXED_BF16X3 ||
         precision == HBS_PREC_MIXED_BF16X6 || precision == HBS_PREC_FP64_TC ||
         precision == HBS_PREC_MIXED_COMPENSATED;
}

int check_problem(const hbs_problem& p, int idx, int finish) {
  if (p.N < 1 || p.r < 1 || p.s < 1 || p.leaf_max < 1)
    return fail(HBS_ERR_ARG, "problem %d: N, r, s, leaf_max must be positive", idx);
  if (!p.Omega || !p.Psi || !p.Y || !p.Z)
    return fail(HBS_ERR_ARG, "problem %d: NULL input pointer", idx);
  int L;
  std::vector<int64_t> off, size;
  build_tree(p.N, p.leaf_max, &L, &off, &size);
  if (L == 0) {
    if (p.N > p.s) return fail(HBS_ERR_SHAPE, "problem %d: single-node tree needs N <= s", idx);
  } else {
    int64_t mn = size[int64_t(1) << L], mx = mn;
    for (int64_t t = int64_t(1) << L; t < (int64_t(2) << L); ++t) {
      mn = std::min(mn, size[t]);
      mx = std::max(mx, size[t]);
    }
    if (mn < p.r) return fail(HBS_ERR_SHAPE, "problem %d: a leaf has %lld < r rows", idx, (long long)mn);
    if (mx + p.r > p.s)
      return fail(HBS_ERR_SHAPE, "problem %d: leaf of %lld rows needs s >= leaf + r", idx, (long long)mx);
    if (p.s < 3 * p.r) return fail(HBS_ERR_SHAPE, "problem %d: s < 3r", idx);
  }
  if (p.s > hbs::kMaxS)
    return fail(HBS_ERR_UNSUPPORTED, "problem %d: s = %d exceeds %d", idx, p.s, hbs::kMaxS);
  const int64_t nmax = (L == 0) ? p.N : std::max<int64_t>(2 * p.r, size[int64_t(1) << L]);
  if (hbs::node_smem_bytes(int(nmax), p.r, p.s, finish) > hbs::kMaxNodeSmemBytes)
    return fail(HBS_ERR_UNSUPPORTED, "problem %d: node tile of %lld x %d exceeds shared memory",
                idx, (long long)nmax, p.s);
  return HBS_OK;
}

void build_tasks(hbs_handle* h) {
  int maxL = 0;
  for (auto& it : h->items) maxL = std::max(maxL, it.L);
  for (auto& H : h->heights) cudaFree(H.d_tasks);
  h->heights.assign(maxL + 1, Height{});
  for (int t = 0; t <= maxL && t < int(h->tuned_R.size()); ++t) h->heights[t].R = h->tuned_R[t];
  for (int t = 0; t <= maxL && t < int(h->tuned_fs.size()); ++t) h->heights[t].fs = h->tuned_fs[t];
  for (auto& it : h->items) {
    const int r = it.r, s = it.s;
    for (int level = it.L; level >= 0; --level) {
      Height& H = h->heights[it.L - level];
      for (int64_t t = int64_t(1) << level; t < (int64_t(2) << level); ++t) {
        NodeTask tk{};
        const int64_t n = (it.L == 0) ? it.N : it.node_rows(t);
        tk.n = int(n);
        tk.r = r;
        tk.s = s;
        if (level == it.L) {
          const int64_t o = it.off[t] * s;
          tk.Om = it.Om + o;
          tk.Ps = it.Ps + o;
          tk.Y = it.Y + o;
          tk.Z = it.Z + o;
        } else {
          tk.Om = h->arena + it.oOm[t];
          tk.Ps = h->arena + it.oPs[t];
          tk.Y = h->arena + it.oY[t];
          tk.Z = h->arena + it.oZ[t];
        }
        tk.D = h->arena + it.oD[t];
        if (level == 0) {
          tk.is_root = 1;
        } else {
          tk.U = h->arena + it.oU[t];
          tk.V = h->arena + it.oV[t];
          tk.WY = h->arena + it.oWY[t];
          tk.WZ = h->arena + it.oWZ[t];
          tk.XY = h->arena + it.oXY[t];
          tk.XZ = h->arena + it.oXZ[t];
          const int64_t p = t / 2, row = (t % 2) * int64_t(r) * s;
          tk.Om_p = h->arena + it.oOm[p] + row;
          tk.Ps_p = h->arena + it.oPs[p] + row;
          tk.Y_p = h->arena + it.oY[p] + row;
          tk.Z_p = h->arena + it.oZ[p] + row;
        }
        H.tasks.push_back(tk);
        H.max_n = std::max(H.max_n, tk.n);
        H.max_r = std::max(H.max_r, r);
        H.max_s = std::max(H.max_s, s);
      }
    }
  }
}

int upload_tasks(hbs_handle* h, cudaStream_t st) {
  for (auto& H : h->heights) {
    if (!H.d_tasks) {
      cudaError_t e = cudaMalloc(&H.d_tasks, H.tasks.size() * sizeof(NodeTask));
      if (e != cudaSuccess) return fail(HBS_ERR_NOMEM, "task list: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaMemcpyAsync(H.d_tasks, H.tasks.data(), H.tasks.size() * sizeof(NodeTask),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "task upload");
  }
  return HBS_OK;
}

void free_handle(hbs_handle* h) {
  if (!h) return;
  for (auto& H : h->heights) cudaFree(H.d_tasks);
  cudaFree(h->arena);
  cudaFree(h->d_status);
  cudaFree(h->d_nodes);
  cudaFree(h->apply_ws);
  cudaFree(h->d_gemm);
  cudaFree(h->batch_ws);
  cudaFree(h->d_batch);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph_pre) cudaGraphExecDestroy(h->graph_pre);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  cudaFree(h->lq_buf);
  if (h->lq_stream) cudaStreamDestroy(h->lq_stream);
  if (h->ev_drawn) cudaEventDestroy(h->ev_drawn);
  if (h->ev_lq) cudaEventDestroy(h->ev_lq);
  delete h;
}

// The captured sweeps are stale once the tasks, the shapes or the graph setting change.
void drop_graphs(hbs_handle* h) {
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph_pre) cudaGraphExecDestroy(h->graph_pre);
  h->graph_exec = nullptr;
  h->graph_pre = nullptr;
}

// The sweep's launches, one launch_sweep_level per height, finest height first; with pre, the
// leaf height's side kernel takes the factorizations in lq_buf.
cudaError_t launch_levels(hbs_handle* h, cudaStream_t st, bool pre = false) {
  const int finish = finish_of(h->precision);
  // a new run: clear the abort flag an earlier run may have left (the report bits stay until
  // hbs_sync_status reads them)
  cudaError_t me = cudaMemsetAsync(h->d_status + hbs::kAbortWord, 0, sizeof(int), st);
  if (me != cudaSuccess) return me;
  for (size_t t = 0; t < h->heights.size(); ++t) {
    const Height& H = h->heights[t];
    cudaError_t e = hbs::launch_sweep_level(H.d_tasks, int(H.tasks.size()), H.max_n, H.max_r,
                                            H.max_s, finish, H.R, h->d_status, st, nullptr, H.fs,
                                            (pre && t == 0) ? h->lq_buf : nullptr);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Runs the sweep on `st`: replays the captured graph when there is one, else captures the
// launches on a private stream (so a caller's own capture of `st` is never disturbed) and
// replays that; launches directly when `st` is itself being captured or capture fails.
int launch_sweep(hbs_handle* h, cudaStream_t st, bool pre = false) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
  if (!h->use_graph || cs != cudaStreamCaptureStatusNone) {
    e = launch_levels(h, st, pre);
    return e == cudaSuccess ? HBS_OK : cuda_fail(e, "sweep kernels");
  }
  cudaGraphExec_t& exec = pre ? h->graph_pre : h->graph_exec;
  if (!exec) {
    if (!h->capture_stream &&
        cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
      h->capture_stream = nullptr;
      h->use_graph = false;
    }
    cudaGraph_t graph = nullptr;
    if (h->use_graph &&
        cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const cudaError_t le = launch_levels(h, h->capture_stream, pre);
      const cudaError_t ce = cudaStreamEndCapture(h->capture_stream, &graph);
      if (le != cudaSuccess || ce != cudaSuccess ||
          cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        exec = nullptr;
        h->use_graph = false;
        cudaGetLastError();                       // clear a sticky launch error from capture
      }
      if (graph) cudaGraphDestroy(graph);
    } else {
      h->use_graph = false;
      cudaGetLastError();
    }
    if (!exec) {
      e = launch_levels(h, st, pre);
      return e == cudaSuccess ? HBS_OK : cuda_fail(e, "sweep kernels");
    }
  }
  e = cudaGraphLaunch(exec, st);
  return e == cudaSuccess ? HBS_OK : cuda_fail(e, "sweep graph launch");
}

}  // namespace

// ---- hbs_apply_static: Algorithm 1 with workspace and work list in fixed device arrays -----

namespace {

// Held on every GPU where this module is loaded (the first cudaGetSymbolAddress below loads it
// there), until the process exits. Host code may not take these names as device addresses: in
// host code they are stand-ins, and the per-device addresses come from cudaGetSymbolAddress.
static __device__ __align__(256) double g_static_apply_ws[HBS_APPLY_STATIC_MAX_DOUBLES];
static __device__ __align__(256) GemmTask g_static_apply_tasks[HBS_APPLY_STATIC_MAX_TASKS];

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
double* g_static_ws_ptr[kMaxDevices] = {};
GemmTask* g_static_task_ptr[kMaxDevices] = {};

// Device addresses of the two arrays on the current device (looked up once per device).
int static_arrays(double** ws, GemmTask** tasks) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "hbs_apply_static: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return fail(HBS_ERR_UNSUPPORTED, "hbs_apply_static: device %d beyond %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ws_ptr[dev]) {
    void* a = nullptr;
    void* b = nullptr;
    e = cudaGetSymbolAddress(&a, g_static_apply_ws);
    if (e != cudaSuccess) return cuda_fail(e, "hbs_apply_static: cudaGetSymbolAddress(workspace)");
    e = cudaGetSymbolAddress(&b, g_static_apply_tasks);
    if (e != cudaSuccess) return cuda_fail(e, "hbs_apply_static: cudaGetSymbolAddress(work list)");
    g_static_task_ptr[dev] = static_cast<GemmTask*>(b);
    g_static_ws_ptr[dev] = static_cast<double*>(a);
  }
  *ws = g_static_ws_ptr[dev];
  *tasks = g_static_task_ptr[dev];
  return HBS_OK;
}

}  // namespace

namespace {

// Doubles of Algorithm 1's workspace for c columns: q-hat and u-hat of every node on levels
// 1..L, r x c each.
size_t apply_ws_doubles(const Item& it, int c) {
  return 2 * ((size_t(2) << it.L) - 2) * size_t(it.r) * size_t(c);
}

// Tasks of Algorithm 1's work list: 2^(L+1) - 2 upward, 2^(L+1) - 1 downward (1 when L = 0).
size_t apply_task_count(const Item& it) { return it.L == 0 ? 1 : (size_t(4) << it.L) - 3; }

// The passes of a work list built by hbs::launch_build_apply_tasks, one launch each: upward
// levels L .. 1, then downward levels 0 .. L (2^l tasks per pass).
int launch_apply_passes(const Item& it, const GemmTask* tasks, int c, cudaStream_t st,
                        const char* who) {
  std::vector<int> sizes;
  if (it.L == 0) {
    sizes.push_back(1);
  } else {
    for (int l = it.L; l >= 1; --l) sizes.push_back(1 << l);
    for (int l = 0; l <= it.L; ++l) sizes.push_back(1 << l);
  }
  size_t at = 0;
  for (int cnt : sizes) {
    cudaError_t e = hbs::launch_gemm_tasks_f64(tasks + at, cnt, c, st);
    if (e != cudaSuccess) return cuda_fail(e, who);
    at += size_t(cnt);
  }
  return HBS_OK;
}

// Every call on a handle must run on the device the handle was planned on.
int check_device(const hbs_handle* h, const char* who) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, who);
  if (dev != h->device)
    return fail(HBS_ERR_ARG, "%s: current device %d, handle planned on device %d", who, dev, h->device);
  return HBS_OK;
}

}  // namespace

extern "C" {

const char* hbs_last_error(void) { return g_last_error.c_str(); }

int hbs_draw_gaussian(int64_t N, int32_t s, uint32_t stream_id, uint64_t seed, double* out,
                      void* cuda_stream) {
  if (!out || N < 1 || s < 1) return fail(HBS_ERR_ARG, "hbs_draw_gaussian: bad arguments");
  cudaError_t e = hbs::launch_gaussian(N * int64_t(s), stream_id, seed, out,
                                       static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(e, "gaussian kernel");
  return ok();
}

// A in page-locked (pinned or registered) host memory; anything else is taken as device memory.
static bool host_resident(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

// Pageable host memory (not registered with CUDA) cannot be read by the kernels or streamed.
static bool pageable_host(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeUnregistered;
}

static int check_operator(const hbs_operator* op, int32_t s, int32_t precision, const void* a,
                          const void* b, const void* c, const void* d, const char* who) {
  if (!op || !a || !b || !c || !d || s < 1 || op->N < 1)
    return fail(HBS_ERR_ARG, "%s: bad arguments", who);
  if (!known_precision(precision))
    return fail(HBS_ERR_ARG, "%s: unknown precision %d", who, precision);
  if (!op->A && !op->fn) return fail(HBS_ERR_ARG, "%s: operator has neither A nor fn", who);
  if (op->A && op->lda < op->N) return fail(HBS_ERR_ARG, "%s: lda < N", who);
  if (op->A && pageable_host(op->A))
    return fail(HBS_ERR_ARG, "%s: A is pageable host memory (pin it or pass device memory)", who);
  if (op->A && precision != HBS_PREC_FP64 && host_resident(op->A))
    return fail(HBS_ERR_UNSUPPORTED, "%s: host-resident A is streamed in FP64 only", who);
  if (precision == HBS_PREC_FP64) {
    if (op->A && op->dtype != HBS_F64)
      return fail(HBS_ERR_UNSUPPORTED, "%s: FP64 products need a FP64 dense A", who);
  } else if (precision == HBS_PREC_FP64_TC || precision == HBS_PREC_MIXED_COMPENSATED) {
    if (!op->A || op->dtype != HBS_F64)
      return fail(HBS_ERR_UNSUPPORTED, "%s: digit products need a dense FP64 A", who);
    if (s > 256 || op->N > (int64_t(1) << 20))
      return fail(HBS_ERR_UNSUPPORTED, "%s: digit products need s <= 256 and N <= 2^20", who);
  } else {
    if (!op->A || op->dtype != HBS_F32)
      return fail(HBS_ERR_UNSUPPORTED, "%s: mixed products need a dense FP32 A", who);
    if (op->lda % 4 != 0 || s > 256 || op->N > (int64_t(1) << 30) ||
        reinterpret_cast<uintptr_t>(op->A) % 16 != 0)
      return fail(HBS_ERR_UNSUPPORTED,
                  "%s: mixed products need a 16-byte aligned A, lda %% 4 == 0 and s <= 256", who);
  }
  return HBS_OK;
}

int hbs_sample_products(const hbs_operator* op, int32_t s, int32_t precision, const double* Omega,
                        const double* Psi, double* Y, double* Z, void* cuda_stream) {
  const int rc = check_operator(op, s, precision, Omega, Psi, Y, Z, "hbs_sample_products");
  if (rc != HBS_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (precision == HBS_PREC_FP64_TC || precision == HBS_PREC_MIXED_COMPENSATED) {
    const int digits = precision == HBS_PREC_FP64_TC ? 7 : 5;   // digits per entry
    // compensated products: one exponent per 64 x 64 block of A, planes in one orientation
    cudaError_t e = hbs::launch_sample_dense_oz(static_cast<const double*>(op->A), op->lda, op->N,
                                                Omega, Psi, s, Y, Z, digits,
                                                precision == HBS_PREC_MIXED_COMPENSATED, st);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core digit sampling");
    return ok();
  }
  if (precision != HBS_PREC_FP64) {
    cudaError_t e = hbs::launch_sample_dense_tc(static_cast<const float*>(op->A), op->lda, op->N,
                                                Omega, Psi, s, Y, Z,
                                                precision == HBS_PREC_MIXED_BF16X3 ? 2 : 3,
                                                0, st);   // reduction split chosen to fill the GPU
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core sampling");
    return ok();
  }
  if (op->A) {
    const bool host = host_resident(op->A);
    cudaError_t e = host ? hbs::launch_sample_host_f64(static_cast<const double*>(op->A), op->lda,
                                                       op->N, Omega, Psi, s, Y, Z, st)
                         : hbs::launch_sample_dense_f64(static_cast<const double*>(op->A), op->lda,
                                                        op->N, Omega, Psi, s, Y, Z, st);
    if (e != cudaSuccess) return cuda_fail(e, host ? "host-streamed sampling" : "sampling kernel");
    return ok();
  }
  if (op->fn(op->user, 0, op->N, s, Omega, Y, cuda_stream) != 0)
    return fail(HBS_ERR_CALLBACK, "callback failed for A");
  if (op->fn(op->user, 1, op->N, s, Psi, Z, cuda_stream) != 0)
    return fail(HBS_ERR_CALLBACK, "callback failed for A^*");
  return ok();
}

int hbs_sample_sync(void* cuda_stream) {
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  int status = 0, oz_status = 0;
  e = hbs::sample_tc_status(&status, true);
  if (e == cudaSuccess) e = hbs::sample_oz_status(&oz_status, true);
  if (e != cudaSuccess) return cuda_fail(e, "sampling status read");
  if ((status | oz_status) & hbs::kStatusTimeout)
    return fail(HBS_ERR_TIMEOUT, "tensor-core sampling: a bounded device wait gave up");
  if (oz_status & hbs::kStatusNumeric)
    return fail(HBS_ERR_NUMERIC, "tensor-core digit sampling: A or a test matrix has an Inf or NaN");
  return ok();
}

int hbs_sample(const hbs_operator* op, int32_t s, uint64_t seed, int32_t precision,
               double* Omega, double* Psi, double* Y, double* Z, void* cuda_stream) {
  const int rc = check_operator(op, s, precision, Omega, Psi, Y, Z, "hbs_sample");
  if (rc != HBS_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int64_t count = op->N * int64_t(s);
  cudaError_t e = hbs::launch_gaussian(count, 0u, seed, Omega, st);
  if (e == cudaSuccess) e = hbs::launch_gaussian(count, 1u, seed, Psi, st);
  if (e != cudaSuccess) return cuda_fail(e, "gaussian kernel");
  return hbs_sample_products(op, s, precision, Omega, Psi, Y, Z, cuda_stream);
}

int hbs_plan(int32_t batch, const hbs_problem* probs, int32_t precision, hbs_handle** out) {
  if (!out || !probs || batch < 1) return fail(HBS_ERR_ARG, "hbs_plan: bad arguments");
  *out = nullptr;
  if (!known_precision(precision))
    return fail(HBS_ERR_UNSUPPORTED, "hbs_plan: unknown precision %d", precision);
  for (int i = 0; i < batch; ++i) {
    const int rc = check_problem(probs[i], i, finish_of(precision));
    if (rc != HBS_OK) return rc;
  }
  auto* h = new hbs_handle();
  h->precision = precision;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return cuda_fail(cudaGetLastError(), "hbs_plan: cudaGetDevice");
  }
  h->items.resize(batch);
  size_t cursor = 0;
  // factors
  for (int i = 0; i < batch; ++i) {
    Item& it = h->items[i];
    const hbs_problem& p = probs[i];
    it.N = p.N;
    it.r = p.r;
    it.s = p.s;
    it.leaf_max = p.leaf_max;
    build_tree(p.N, p.leaf_max, &it.L, &it.off, &it.size);
    const int64_t count = int64_t(2) << it.L;
    for (auto* v : {&it.oU, &it.oV, &it.oD, &it.oWY, &it.oWZ, &it.oXY, &it.oXZ, &it.oOm, &it.oPs,
                    &it.oY, &it.oZ})
      v->assign(count, -1);
    for (int64_t t = 1; t < count; ++t) {
      const int64_t n = (it.L == 0) ? it.N : it.node_rows(t);
      if (t > 1) {
        it.oU[t] = int64_t(cursor);
        cursor += size_t(n) * it.r;
        it.oV[t] = int64_t(cursor);
        cursor += size_t(n) * it.r;
      }
      it.oD[t] = int64_t(cursor);
      cursor += size_t(n) * n;
    }
  }
  h->factor_doubles = cursor;
  // workspace and parent blocks
  for (auto& it : h->items) {
    const int64_t count = int64_t(2) << it.L;
    for (int64_t t = 2; t < count; ++t) {
      const int64_t n = it.node_rows(t);
      it.oWY[t] = int64_t(cursor);
      cursor += size_t(n) * n;
      it.oWZ[t] = int64_t(cursor);
      cursor += size_t(n) * n;
      it.oXY[t] = int64_t(cursor);
      cursor += size_t(n) * it.r;
      it.oXZ[t] = int64_t(cursor);
      cursor += size_t(n) * it.r;
    }
    for (int64_t t = 1; t < (int64_t(1) << it.L); ++t) {
      const size_t blk = size_t(2) * it.r * it.s;
      for (auto* v : {&it.oOm, &it.oPs, &it.oY, &it.oZ}) {
        (*v)[t] = int64_t(cursor);
        cursor += blk;
      }
    }
  }
  h->arena_doubles = cursor;
  cudaError_t e = cudaMalloc(&h->arena, std::max<size_t>(cursor, 1) * sizeof(double));
  if (e != cudaSuccess) {
    free_handle(h);
    return fail(HBS_ERR_NOMEM, "arena of %zu bytes: %s", cursor * sizeof(double), cudaGetErrorString(e));
  }
  e = cudaMalloc(&h->d_status, hbs::kStatusWords * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, hbs::kStatusWords * sizeof(int));
  if (e != cudaSuccess) {
    free_handle(h);
    return fail(HBS_ERR_NOMEM, "status word: %s", cudaGetErrorString(e));
  }
  // Algorithm 1's node table of every item (hbs_apply and hbs_apply_static build their work
  // lists from it on the device)
  std::vector<hbs::ApplyNode> nodes;
  for (auto& it : h->items) {
    h->node_base.push_back(int64_t(nodes.size()));
    const int64_t count = int64_t(2) << it.L;
    for (int64_t t = 0; t < count; ++t) {
      hbs::ApplyNode nd{};
      if (t >= 1) {
        nd.off = it.off[t];
        nd.n = int((it.L == 0) ? it.N : it.node_rows(t));
        nd.oU = it.oU[t];
        nd.oV = it.oV[t];
        nd.oD = it.oD[t];
      }
      nodes.push_back(nd);
    }
  }
  e = cudaMalloc(&h->d_nodes, nodes.size() * sizeof(hbs::ApplyNode));
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_nodes, nodes.data(), nodes.size() * sizeof(hbs::ApplyNode),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_handle(h);
    return fail(HBS_ERR_NOMEM, "node table: %s", cudaGetErrorString(e));
  }
  // the fixed arrays of hbs_apply_static on this device, looked up (and so loaded) now, while
  // the plan may allocate; a failure here is reported by hbs_apply_static itself
  double* sws = nullptr;
  GemmTask* stk = nullptr;
  if (static_arrays(&sws, &stk) != HBS_OK) cudaGetLastError();
  *out = h;
  return ok();
}

namespace {

// Checks probs against the plan and points the tasks at its blocks (rebuilt and uploaded on st
// when a pointer changed).
int bind_problems(hbs_handle* h, const hbs_problem* probs, cudaStream_t st, const char* who) {
  bool changed = !h->tasks_uploaded;
  for (size_t i = 0; i < h->items.size(); ++i) {
    Item& it = h->items[i];
    const hbs_problem& p = probs[i];
    if (p.N != it.N || p.r != it.r || p.s != it.s || p.leaf_max != it.leaf_max)
      return fail(HBS_ERR_ARG, "%s: problem %zu differs from the plan", who, i);
    if (!p.Omega || !p.Psi || !p.Y || !p.Z)
      return fail(HBS_ERR_ARG, "%s: problem %zu has a NULL input", who, i);
    if (p.Omega != it.Om || p.Psi != it.Ps || p.Y != it.Y || p.Z != it.Z) changed = true;
    it.Om = p.Omega;
    it.Ps = p.Psi;
    it.Y = p.Y;
    it.Z = p.Z;
  }
  if (changed) {
    build_tasks(h);
    const int rc = upload_tasks(h, st);
    if (rc != HBS_OK) return rc;
    h->tasks_uploaded = true;
    drop_graphs(h);
  }
  return HBS_OK;
}

// The leaf height takes its factorizations from node_lq when it runs the one-CTA side form with
// FP64 sample rows. (With a reduced finish the rows stream in double-float, and the fused side
// kernel, 2.06 ms at the leaves of the N = 32768 log-kernel tree, beats node_lq + the copying
// kernel, 1.20 + 1.02 ms, which the products leave no room to overlap.)
bool leaves_prefactorable(const hbs_handle* h) {
  if (h->items.size() != 1 || h->items[0].L < 1 || h->heights.empty()) return false;
  const Height& H = h->heights[0];
  return hbs::side_shape(int(H.tasks.size()), H.max_n, H.max_s, H.R) > 0 &&
         hbs::effective_finish(H.max_n, H.max_r, finish_of(h->precision)) == hbs::kFinishF64;
}

// lq_buf, the second stream (the highest priority, so that its CTAs are placed among the
// products' as SMs free up) and the two events, made on first use.
int ensure_lq_resources(hbs_handle* h) {
  const Height& H = h->heights[0];
  const size_t need = size_t(2) * H.tasks.size() * size_t(hbs::side_lq_stride(H.max_n, H.max_s));
  if (need > h->lq_doubles) {
    cudaFree(h->lq_buf);
    h->lq_buf = nullptr;
    h->lq_doubles = 0;
    drop_graphs(h);                                    // graph_pre holds the old address
    cudaError_t e = cudaMalloc(&h->lq_buf, need * sizeof(double));
    if (e != cudaSuccess) return fail(HBS_ERR_NOMEM, "leaf LQ images: %s", cudaGetErrorString(e));
    h->lq_doubles = need;
  }
  if (!h->lq_stream) {
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess)
      e = cudaStreamCreateWithPriority(&h->lq_stream, cudaStreamNonBlocking, greatest);
    if (e != cudaSuccess) {
      h->lq_stream = nullptr;
      return cuda_fail(e, "leaf LQ stream");
    }
  }
  for (cudaEvent_t* ev : {&h->ev_drawn, &h->ev_lq}) {
    if (!*ev) {
      cudaError_t e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
      if (e != cudaSuccess) {
        *ev = nullptr;
        return cuda_fail(e, "leaf LQ event");
      }
    }
  }
  return HBS_OK;
}

}  // namespace

int hbs_execute(hbs_handle* h, const hbs_problem* probs, void* cuda_stream) {
  if (!h || !probs) return fail(HBS_ERR_ARG, "hbs_execute: NULL argument");
  if (check_device(h, "hbs_execute") != HBS_OK) return HBS_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  int rc = bind_problems(h, probs, st, "hbs_execute");
  if (rc != HBS_OK) return rc;
  rc = launch_sweep(h, st);
  if (rc != HBS_OK) return rc;
  return ok();
}

int hbs_sample_execute(hbs_handle* h, const hbs_operator* op, uint64_t seed, int32_t precision,
                       const hbs_problem* probs, void* cuda_stream) {
  if (!h || !probs || !op) return fail(HBS_ERR_ARG, "hbs_sample_execute: NULL argument");
  if (h->items.size() != 1)
    return fail(HBS_ERR_ARG, "hbs_sample_execute: the handle must hold one problem");
  if (check_device(h, "hbs_sample_execute") != HBS_OK) return HBS_ERR_ARG;
  const hbs_problem& p = probs[0];
  if (op->N != p.N) return fail(HBS_ERR_ARG, "hbs_sample_execute: operator N differs from the problem's");
  int rc = check_operator(op, p.s, precision, p.Omega, p.Psi, p.Y, p.Z, "hbs_sample_execute");
  if (rc != HBS_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  rc = bind_problems(h, probs, st, "hbs_sample_execute");
  if (rc != HBS_OK) return rc;
  // the problem's blocks are the sweep's inputs (const there); here they are written
  double* Om = const_cast<double*>(p.Omega);
  double* Ps = const_cast<double*>(p.Psi);
  double* Y = const_cast<double*>(p.Y);
  double* Z = const_cast<double*>(p.Z);
  const int64_t count = p.N * int64_t(p.s);
  cudaError_t e = hbs::launch_gaussian(count, 0u, seed, Om, st);
  if (e == cudaSuccess) e = hbs::launch_gaussian(count, 1u, seed, Ps, st);
  if (e != cudaSuccess) return cuda_fail(e, "gaussian kernel");
  const bool pre = leaves_prefactorable(h);
  if (pre) {
    rc = ensure_lq_resources(h);
    if (rc != HBS_OK) return rc;
    const Height& H = h->heights[0];
    e = cudaEventRecord(h->ev_drawn, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->lq_stream, h->ev_drawn, 0);
    if (e == cudaSuccess)
      e = hbs::launch_side_lq(H.d_tasks, int(H.tasks.size()), H.max_n, H.max_s, h->lq_buf,
                              h->d_status, h->lq_stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_lq, h->lq_stream);
    if (e != cudaSuccess) return cuda_fail(e, "leaf LQ");
  }
  rc = hbs_sample_products(op, p.s, precision, Om, Ps, Y, Z, cuda_stream);
  if (pre) {                                         // join the second stream in every case
    e = cudaStreamWaitEvent(st, h->ev_lq, 0);
    if (e != cudaSuccess && rc == HBS_OK) rc = cuda_fail(e, "leaf LQ join");
  }
  if (rc != HBS_OK) return rc;
  rc = launch_sweep(h, st, pre);
  if (rc != HBS_OK) return rc;
  return ok();
}

int hbs_compress(int32_t batch, const hbs_problem* probs, int32_t precision, hbs_handle** out,
                 void* cuda_stream) {
  int rc = hbs_plan(batch, probs, precision, out);
  if (rc != HBS_OK) return rc;
  rc = hbs_execute(*out, probs, cuda_stream);
  if (rc != HBS_OK) {
    free_handle(*out);
    *out = nullptr;
  }
  return rc;
}

int hbs_apply(hbs_handle* h, int32_t item, int trans, int32_t ncols, const double* X,
              double* Out, void* cuda_stream) {
  if (!h || !X || !Out || ncols < 1 || item < 0 || item >= int(h->items.size()))
    return fail(HBS_ERR_ARG, "hbs_apply: bad arguments");
  if (check_device(h, "hbs_apply") != HBS_OK) return HBS_ERR_ARG;
  const Item& it = h->items[item];
  const int c = ncols;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // workspace: q-hat and u-hat for every node on levels 1..L, level-major, r x c per node
  const size_t need = apply_ws_doubles(it, c);
  if (need > h->apply_ws_doubles) {
    cudaFree(h->apply_ws);
    h->apply_ws = nullptr;
    h->apply_ws_doubles = 0;
    cudaError_t e = cudaMalloc(&h->apply_ws, need * sizeof(double));
    if (e != cudaSuccess) return fail(HBS_ERR_NOMEM, "apply workspace: %s", cudaGetErrorString(e));
    h->apply_ws_doubles = need;
  }
  double* ws = h->apply_ws;
  // same arguments on the same stream as the last call: its work list is still in d_gemm (the
  // factors are addressed through the arena, whose contents may have changed, not its address)
  hbs_handle::ApplyKey key;
  key.item = item; key.trans = trans; key.ncols = c; key.X = X; key.Out = Out; key.ws = ws; key.st = st;
  if (!(key == h->apply_key)) {
    h->apply_key = hbs_handle::ApplyKey{};            // invalid until the new list is built
    const size_t total = apply_task_count(it);
    if (total > h->d_gemm_cap) {
      cudaFree(h->d_gemm);
      h->d_gemm = nullptr;
      h->d_gemm_cap = 0;
      cudaError_t e = cudaMalloc(&h->d_gemm, total * sizeof(GemmTask));
      if (e != cudaSuccess) return fail(HBS_ERR_NOMEM, "apply task list: %s", cudaGetErrorString(e));
      h->d_gemm_cap = total;
    }
    cudaError_t e = hbs::launch_build_apply_tasks(h->d_nodes + h->node_base[item], it.L, it.r, it.N,
                                                  trans, c, h->arena, X, Out, ws, h->d_gemm, st);
    if (e != cudaSuccess) return cuda_fail(e, "apply work list");
    h->apply_key = key;
  }
  const int rc = launch_apply_passes(it, h->d_gemm, c, st, "apply kernel");
  if (rc != HBS_OK) return rc;
  return ok();
}

int hbs_sync_status(hbs_handle* h, void* cuda_stream) {
  if (!h) return fail(HBS_ERR_ARG, "hbs_sync_status: NULL handle");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  int status = 0;
  e = cudaMemcpy(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, hbs::kStatusWords * sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (status & hbs::kStatusTimeout)
    return fail(HBS_ERR_TIMEOUT, "a bounded device-side wait of the sweep gave up%s",
                (status & hbs::kStatusNumeric) ? " (a zero or non-finite pivot was also met)" : "");
  if (status & hbs::kStatusNumeric)
    return fail(HBS_ERR_NUMERIC, "zero or non-finite pivot in a triangular factor");
  return ok();
}

int hbs_test_inject_status(hbs_handle* h, int32_t bits) {
  if (bits & ~(hbs::kStatusNumeric | hbs::kStatusTimeout))
    return fail(HBS_ERR_ARG, "hbs_test_inject_status: unknown bits %d", bits);
  if (!h) {
    cudaError_t e = hbs::sample_tc_inject(bits);
    if (e == cudaSuccess) e = hbs::sample_oz_inject(bits);
    if (e != cudaSuccess) return cuda_fail(e, "hbs_test_inject_status");
    return ok();
  }
  int now[hbs::kStatusWords];
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(now, h->d_status, sizeof(now), cudaMemcpyDeviceToHost);
  now[0] |= bits;
  if (bits & hbs::kStatusTimeout) now[hbs::kAbortWord] = 1;
  if (e == cudaSuccess) e = cudaMemcpy(h->d_status, now, sizeof(now), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "hbs_test_inject_status");
  return ok();
}

void hbs_free(hbs_handle* h) { free_handle(h); }

int hbs_tree_build(int64_t N, int32_t leaf_max, int32_t* L, int64_t* offsets, int64_t* sizes,
                   int64_t max_nodes) {
  if (N < 1 || leaf_max < 1 || !L) return fail(HBS_ERR_ARG, "hbs_tree_build: bad arguments");
  int depth;
  std::vector<int64_t> off, size;
  build_tree(N, leaf_max, &depth, &off, &size);
  *L = depth;
  const int64_t count = (int64_t(2) << depth) - 1;
  if (offsets || sizes) {
    if (max_nodes < count) return fail(HBS_ERR_ARG, "hbs_tree_build: arrays hold %lld < %lld nodes",
                                       (long long)max_nodes, (long long)count);
    for (int64_t t = 1; t <= count; ++t) {
      if (offsets) offsets[t - 1] = off[t];
      if (sizes) sizes[t - 1] = size[t];
    }
  }
  return ok();
}

int hbs_tree(const hbs_handle* h, int32_t item, int32_t* L, int64_t* offsets, int64_t* sizes) {
  if (!h || !L || item < 0 || item >= int(h->items.size()))
    return fail(HBS_ERR_ARG, "hbs_tree: bad arguments");
  const Item& it = h->items[item];
  *L = it.L;
  const int64_t count = (int64_t(2) << it.L) - 1;
  for (int64_t t = 1; t <= count; ++t) {
    if (offsets) offsets[t - 1] = it.off[t];
    if (sizes) sizes[t - 1] = it.size[t];
  }
  return ok();
}

int hbs_get_node(const hbs_handle* h, int32_t item, int64_t node, int32_t* n, double* U,
                 double* V, double* D) {
  if (!h || item < 0 || item >= int(h->items.size())) return fail(HBS_ERR_ARG, "hbs_get_node: bad item");
  const Item& it = h->items[item];
  if (node < 1 || node >= (int64_t(2) << it.L)) return fail(HBS_ERR_ARG, "hbs_get_node: bad node");
  const int64_t rows = (it.L == 0) ? it.N : it.node_rows(node);
  if (n) *n = int(rows);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && node > 1 && U)
    e = cudaMemcpy(U, h->arena + it.oU[node], rows * it.r * sizeof(double), cudaMemcpyDefault);
  if (e == cudaSuccess && node > 1 && V)
    e = cudaMemcpy(V, h->arena + it.oV[node], rows * it.r * sizeof(double), cudaMemcpyDefault);
  if (e == cudaSuccess && D)
    e = cudaMemcpy(D, h->arena + it.oD[node], rows * rows * sizeof(double), cudaMemcpyDefault);
  if (e != cudaSuccess) return cuda_fail(e, "hbs_get_node copy");
  return ok();
}

size_t hbs_factor_bytes(const hbs_handle* h) { return h ? h->factor_doubles * sizeof(double) : 0; }

int hbs_copy_factors(const hbs_handle* h, void* dst, void* cuda_stream) {
  if (!h || !dst) return fail(HBS_ERR_ARG, "hbs_copy_factors: bad arguments");
  cudaError_t e = cudaMemcpyAsync(dst, h->arena, h->factor_doubles * sizeof(double),
                                  cudaMemcpyDefault, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(e, "hbs_copy_factors");
  return ok();
}

int hbs_load_factors(hbs_handle* h, const void* src, void* cuda_stream) {
  if (!h || !src) return fail(HBS_ERR_ARG, "hbs_load_factors: bad arguments");
  cudaError_t e = cudaMemcpyAsync(h->arena, src, h->factor_doubles * sizeof(double),
                                  cudaMemcpyDefault, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(e, "hbs_load_factors");
  return ok();
}

int hbs_apply_batch(hbs_handle* h, int trans, const double* const* X, double* const* Out,
                    const int32_t* ncols, void* cuda_stream) {
  if (!h || !X || !Out || !ncols) return fail(HBS_ERR_ARG, "hbs_apply_batch: bad arguments");
  if (check_device(h, "hbs_apply_batch") != HBS_OK) return HBS_ERR_ARG;
  const int nitems = int(h->items.size());
  int maxL = 0;
  size_t need = 0;
  std::vector<size_t> base(nitems);
  for (int i = 0; i < nitems; ++i) {
    if (!X[i] || !Out[i] || ncols[i] < 1) return fail(HBS_ERR_ARG, "hbs_apply_batch: item %d", i);
    const Item& it = h->items[i];
    maxL = std::max(maxL, it.L);
    base[i] = need;
    need += 2 * ((size_t(2) << it.L) - 2) * size_t(it.r) * size_t(ncols[i]);
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  std::vector<uintptr_t> key;
  key.reserve(3 + 3 * size_t(nitems));
  key.push_back(uintptr_t(trans));
  key.push_back(reinterpret_cast<uintptr_t>(st));
  for (int i = 0; i < nitems; ++i) {
    key.push_back(reinterpret_cast<uintptr_t>(X[i]));
    key.push_back(reinterpret_cast<uintptr_t>(Out[i]));
    key.push_back(uintptr_t(ncols[i]));
  }
  if (need <= h->batch_ws_doubles) {
    key.push_back(reinterpret_cast<uintptr_t>(h->batch_ws));
    if (key == h->batch_key) {                         // the uploaded list still applies
      size_t at = 0;
      for (int cnt : h->batch_sizes) {
        if (cnt > 0) {
          cudaError_t e = hbs::launch_gemm_tasks_f64(h->d_batch + at, cnt, h->batch_ncols, st);
          if (e != cudaSuccess) return cuda_fail(e, "apply kernel");
        }
        at += size_t(cnt);
      }
      return ok();
    }
    key.pop_back();
  }
  h->batch_key.clear();
  if (need > h->batch_ws_doubles) {
    cudaFree(h->batch_ws);
    h->batch_ws = nullptr;
    h->batch_ws_doubles = 0;
    cudaError_t e = cudaMalloc(&h->batch_ws, std::max<size_t>(need, 1) * sizeof(double));
    if (e != cudaSuccess) return fail(HBS_ERR_NOMEM, "apply workspace: %s", cudaGetErrorString(e));
    h->batch_ws_doubles = need;
  }
  // passes: upward by height (0 = leaves), then downward by depth (0 = root)
  std::vector<std::vector<GemmTask>> up(std::max(maxL, 1)), down(maxL + 1);
  const double* A = h->arena;
  for (int i = 0; i < nitems; ++i) {
    const Item& it = h->items[i];
    const int r = it.r, c = ncols[i], L = it.L;
    double* ws = h->batch_ws + base[i];
    const size_t half = ((size_t(2) << L) - 2) * size_t(r) * size_t(c);
    // q-hat / u-hat of node t (levels 1..L) at level-major offsets
    auto off = [&](int64_t t) {
      int l = 0;
      while ((int64_t(2) << l) <= t) ++l;
      return ((size_t(1) << l) - 2 + size_t(t - (int64_t(1) << l))) * size_t(r) * size_t(c);
    };
    auto qhat = [&](int64_t t) { return ws + off(t); };
    auto uhat = [&](int64_t t) { return ws + half + off(t); };
    const std::vector<int64_t>& oIn = trans ? it.oU : it.oV;
    const std::vector<int64_t>& oOut = trans ? it.oV : it.oU;
    if (L == 0) {
      GemmTask g{};
      g.A1 = A + it.oD[1]; g.lda1 = int(it.N); g.t1 = trans; g.k1 = int(it.N);
      g.B1 = X[i]; g.ldb1 = c; g.C = Out[i]; g.ldc = c; g.m = int(it.N); g.ncols = c;
      down[0].push_back(g);
      continue;
    }
    for (int l = L; l >= 1; --l) {
      for (int64_t t = int64_t(1) << l; t < (int64_t(2) << l); ++t) {
        GemmTask g{};
        const int n = int(it.node_rows(t));
        g.A1 = A + oIn[t]; g.lda1 = r; g.t1 = 1; g.k1 = n; g.m = r; g.ncols = c;
        g.B1 = (l == L) ? X[i] + it.off[t] * c : qhat(2 * t);
        g.ldb1 = c; g.C = qhat(t); g.ldc = c;
        up[L - l].push_back(g);
      }
    }
    for (int l = 0; l <= L; ++l) {
      for (int64_t t = int64_t(1) << l; t < (int64_t(2) << l); ++t) {
        GemmTask g{};
        g.ncols = c;
        const int n = (l == 0) ? 2 * r : int(it.node_rows(t));
        if (l == 0) {
          g.A1 = A + it.oD[1]; g.lda1 = n; g.t1 = trans; g.k1 = n; g.m = n;
          g.B1 = qhat(2); g.ldb1 = c; g.C = uhat(2); g.ldc = c;
        } else {
          g.A1 = A + oOut[t]; g.lda1 = r; g.t1 = 0; g.k1 = r; g.m = n;
          g.B1 = uhat(t); g.ldb1 = c;
          g.A2 = A + it.oD[t]; g.lda2 = n; g.t2 = trans; g.k2 = n;
          if (l < L) {
            g.B2 = qhat(2 * t); g.ldb2 = c; g.C = uhat(2 * t); g.ldc = c;
          } else {
            g.B2 = X[i] + it.off[t] * c; g.ldb2 = c; g.C = Out[i] + it.off[t] * c; g.ldc = c;
          }
        }
        down[l].push_back(g);
      }
    }
  }
  std::vector<GemmTask> flat;
  std::vector<int> sizes;
  for (auto& p : up) { flat.insert(flat.end(), p.begin(), p.end()); sizes.push_back(int(p.size())); }
  for (auto& p : down) { flat.insert(flat.end(), p.begin(), p.end()); sizes.push_back(int(p.size())); }
  if (flat.size() > h->d_batch_cap) {
    cudaFree(h->d_batch);
    h->d_batch = nullptr;
    h->d_batch_cap = 0;
    cudaError_t e = cudaMalloc(&h->d_batch, flat.size() * sizeof(GemmTask));
    if (e != cudaSuccess) return fail(HBS_ERR_NOMEM, "apply task list: %s", cudaGetErrorString(e));
    h->d_batch_cap = flat.size();
  }
  cudaError_t e = cudaMemcpyAsync(h->d_batch, flat.data(), flat.size() * sizeof(GemmTask),
                                  cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "apply task upload");
  // one column count for every item: the launch can take the skinny kernel; otherwise each task
  // carries its own (0)
  int common = nitems > 0 ? ncols[0] : 0;
  for (int i = 1; i < nitems; ++i)
    if (ncols[i] != common) common = 0;
  size_t at = 0;
  for (int cnt : sizes) {
    if (cnt > 0) {
      e = hbs::launch_gemm_tasks_f64(h->d_batch + at, cnt, common, st);
      if (e != cudaSuccess) return cuda_fail(e, "apply kernel");
    }
    at += size_t(cnt);
  }
  key.push_back(reinterpret_cast<uintptr_t>(h->batch_ws));
  h->batch_key = std::move(key);
  h->batch_sizes = sizes;
  h->batch_ncols = common;
  return ok();
}

int hbs_autotune(hbs_handle* h, void* cuda_stream) {
  if (!h) return fail(HBS_ERR_ARG, "hbs_autotune: NULL handle");
  if (!h->tasks_uploaded) return fail(HBS_ERR_ARG, "hbs_autotune: execute the handle once first");
  if (check_device(h, "hbs_autotune") != HBS_OK) return HBS_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t ce = cudaMemsetAsync(h->d_status + hbs::kAbortWord, 0, sizeof(int), st);
  if (ce != cudaSuccess) return cuda_fail(ce, "hbs_autotune: status");
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cuda_fail(cudaGetLastError(), "hbs_autotune: events");
  h->tuned_R.assign(h->heights.size(), 0);
  for (size_t t = 0; t < h->heights.size(); ++t) {
    Height& H = h->heights[t];
    const int ntasks = int(H.tasks.size());
    float best_ms = 1e30f;
    int best = hbs::side_row_splits(ntasks, H.max_n, H.max_s);
    // With a reduced finish (FP32 or double-float) the one-CTA form streams the sample rows in
    // double-float and the cluster form in FP64, so the tuner keeps the automatic form there
    // (every shape within a form rounds alike; the factors of a tuned run equal the automatic
    // ones).
    const bool df = hbs::effective_finish(H.max_n, H.max_r, finish_of(h->precision)) != hbs::kFinishF64;
    const int form = best > 0 ? 1 : -1;
    // row slices (each CTA factors the test block) and clusters of C CTAs sharing one
    // factorization (R = -C)
    for (int R : {1, 2, 3, 4, 6, 8, 12, 16, -1, -2, -3, -4, -6, -8}) {
      if (std::abs(R) > std::max(1, H.max_n / 8)) continue;
      if (R < 0 && !hbs::side_cluster_fits(H.max_n, H.max_s, -R)) continue;
      if (df && R * form < 0) continue;
      // one untimed launch, then the mean of three
      cudaError_t e = hbs::launch_side_only(H.d_tasks, ntasks, H.max_n, H.max_s, R, h->d_status, st,
                                            nullptr, df);
      if (R < 0 && e != cudaSuccess && e != cudaErrorLaunchFailure) {
        cudaGetLastError();                            // a cluster shape the GPU cannot place
        continue;
      }
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        e = hbs::launch_side_only(H.d_tasks, ntasks, H.max_n, H.max_s, R, h->d_status, st,
                                  nullptr, df);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_fail(e, "hbs_autotune");
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = R;
      }
    }
    H.R = best;
    h->tuned_R[t] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // The finish kernels' grids per height: the merge chunk, then (FP64 finish) the D column
  // blocks, each timed over the D and merge launches of one run of the whole height (side,
  // bases, D, merges: the height's outputs are recomputed from the same inputs, and every
  // grid rounds alike, so the factors do not change).
  cudaEvent_t ev[5];
  int made = 0;
  cudaError_t fe = cudaSuccess;
  for (; made < 5 && fe == cudaSuccess; ++made) fe = cudaEventCreate(&ev[made]);
  const int finish = finish_of(h->precision);
  h->tuned_fs.assign(h->heights.size(), hbs::FinishShape{});
  auto time_finish = [&](Height& H, hbs::FinishShape fs, float* ms) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep)     // untimed, then timed
      e = hbs::launch_sweep_level(H.d_tasks, int(H.tasks.size()), H.max_n, H.max_r, H.max_s,
                                  finish, H.R, h->d_status, st, ev, fs);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[4]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, ev[2], ev[4]);
    return e;
  };
  for (size_t t = 0; t < h->heights.size() && fe == cudaSuccess; ++t) {
    Height& H = h->heights[t];
    if (H.tasks.size() == 1 && H.tasks[0].is_root) continue;   // the root has no finish
    hbs::FinishShape best{};
    float best_ms = 1e30f;
    for (int chunk : {0, 8, 16, 32}) {
      hbs::FinishShape fs = best;
      fs.merge_chunk = chunk;
      float ms = 0.f;
      fe = time_finish(H, fs, &ms);
      if (fe != cudaSuccess) break;
      if (ms < best_ms) { best_ms = ms; best = fs; }
    }
    if (finish == hbs::kFinishF64 || hbs::effective_finish(H.max_n, H.max_r, finish) == hbs::kFinishF64) {
      const hbs::FinishShape base = best;
      for (int blocks : {1, 2, 4, 8}) {
        if (fe != cudaSuccess) break;
        hbs::FinishShape fs = base;
        fs.d_blocks = blocks;
        float ms = 0.f;
        fe = time_finish(H, fs, &ms);
        if (fe == cudaSuccess && ms < best_ms) { best_ms = ms; best = fs; }
      }
    }
    H.fs = best;
    h->tuned_fs[t] = best;
  }
  for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
  if (fe != cudaSuccess) return cuda_fail(fe, "hbs_autotune: finish shapes");
  drop_graphs(h);
  return ok();
}

int hbs_profile_sweep(hbs_handle* h, void* cuda_stream, float* ms, int32_t count,
                      int32_t* heights) {
  if (!h || !heights) return fail(HBS_ERR_ARG, "hbs_profile_sweep: bad arguments");
  if (!h->tasks_uploaded) return fail(HBS_ERR_ARG, "hbs_profile_sweep: execute the handle once first");
  if (check_device(h, "hbs_profile_sweep") != HBS_OK) return HBS_ERR_ARG;
  *heights = int32_t(h->heights.size());
  if (!ms) return ok();
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaEvent_t ev[5];
  int made = 0;
  cudaError_t e = cudaSuccess;
  for (; made < 5 && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_status + hbs::kAbortWord, 0, sizeof(int), st);
  const int finish = finish_of(h->precision);
  for (size_t t = 0; t < h->heights.size() && e == cudaSuccess; ++t) {
    Height& H = h->heights[t];
    e = hbs::launch_sweep_level(H.d_tasks, int(H.tasks.size()), H.max_n, H.max_r, H.max_s, finish,
                                H.R, h->d_status, st, ev, H.fs);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[4]);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
      float v = 0.f;
      e = cudaEventElapsedTime(&v, ev[k], ev[k + 1]);
      if (e == cudaSuccess && int(4 * t) + k < count) ms[4 * t + k] = v;
    }
  }
  for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
  if (e != cudaSuccess) return cuda_fail(e, "hbs_profile_sweep");
  return ok();
}

int hbs_get_tuning(const hbs_handle* h, int32_t* R, int32_t count, int32_t* heights) {
  if (!h || !heights) return fail(HBS_ERR_ARG, "hbs_get_tuning: bad arguments");
  *heights = int32_t(h->heights.size());
  for (int t = 0; R && t < count && t < int(h->heights.size()); ++t) R[t] = h->heights[t].R;
  return ok();
}

int hbs_set_tuning(hbs_handle* h, const int32_t* R, int32_t count) {
  if (!h || !R || count < 0) return fail(HBS_ERR_ARG, "hbs_set_tuning: bad arguments");
  h->tuned_R.assign(R, R + count);
  for (int t = 0; t < count && t < int(h->heights.size()); ++t)
    h->heights[t].R = std::max(-hbs::kMaxSideCluster, R[t]);
  drop_graphs(h);
  return ok();
}

int hbs_set_graph(hbs_handle* h, int enable) {
  if (!h) return fail(HBS_ERR_ARG, "hbs_set_graph: NULL handle");
  h->use_graph = enable != 0;
  drop_graphs(h);
  return ok();
}

}  // extern "C"


extern "C" int hbs_apply_static(const hbs_handle* h, int32_t item, int trans, int32_t ncols,
                                const double* X, double* Out, void* cuda_stream) {
  if (!h || !X || !Out || ncols < 1 || item < 0 || item >= int(h->items.size()))
    return fail(HBS_ERR_ARG, "hbs_apply_static: bad arguments");
  if (check_device(h, "hbs_apply_static") != HBS_OK) return HBS_ERR_ARG;
  const Item& it = h->items[item];
  const int c = ncols;
  // size checks first: nothing is queued for a request beyond the fixed arrays
  const size_t need = apply_ws_doubles(it, c);
  const size_t ntasks = apply_task_count(it);
  if (need > size_t(HBS_APPLY_STATIC_MAX_DOUBLES))
    return fail(HBS_ERR_UNSUPPORTED,
                "hbs_apply_static: workspace of %zu doubles exceeds the fixed %d (L=%d, r=%d, ncols=%d)",
                need, HBS_APPLY_STATIC_MAX_DOUBLES, it.L, it.r, c);
  if (ntasks > size_t(HBS_APPLY_STATIC_MAX_TASKS))
    return fail(HBS_ERR_UNSUPPORTED, "hbs_apply_static: %zu node products exceed the fixed %d (L=%d)",
                ntasks, HBS_APPLY_STATIC_MAX_TASKS, it.L);
  double* ws = nullptr;
  GemmTask* d_tasks = nullptr;
  const int rc = static_arrays(&ws, &d_tasks);
  if (rc != HBS_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the work list is written into the fixed array by a kernel on the caller's stream: no host
  // copy, no allocation
  cudaError_t e = hbs::launch_build_apply_tasks(h->d_nodes + h->node_base[item], it.L, it.r, it.N,
                                                trans, c, h->arena, X, Out, ws, d_tasks, st);
  if (e != cudaSuccess) return cuda_fail(e, "hbs_apply_static: work list");
  const int prc = launch_apply_passes(it, d_tasks, c, st, "hbs_apply_static: apply kernel");
  if (prc != HBS_OK) return prc;
  return ok();
}
