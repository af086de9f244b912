// Per-level node sweep of Algorithm 2 in FP64 (one CTA per node of a tree level).
//
// For a node tau with blocks Omega_tau, Psi_tau, Y_tau, Z_tau (n x s) the CTA computes
//   P = null(Omega_tau, r), U = col(Y_tau P, r)              (Section 4.1, Eq. u_tau_formula)
//   Q = null(Psi_tau, r),   V = col(Z_tau Q, r)              (Eq. v_tau_formula)
//   D = (I - UU^*) Y Omega^+ + UU^* ((I - VV^*) Z Psi^+)^*   (Eq. d_tau_formula)
// and the node's rows of the parent's blocks (Eq. omega_tau_and_y_tau, Algorithm 2):
//   V^* Omega_tau, U^* Psi_tau, U^* (Y_tau - D Omega_tau), V^* (Z_tau - D^* Psi_tau).
// At the root only D = Y Omega^+ (Section 4.3).
//
// One Householder factorization of Omega_tau serves both `null` and the pseudo-inverse:
// Omega_tau = L Q^* (an LQ factorization, i.e. the QR of Omega_tau^* of Section 2.4), Q
// square. The last r columns of Q are null(Omega_tau, r) (Section 2.4), and because
// Omega_tau = L_1 Q_1^* with L_1 the leading n x n lower triangle, Omega^+ = Q_1 L_1^{-1}.
// Each row y of Y_tau is pushed once through all n reflectors (y Q = y H_0 ... H_{n-1}):
// its last r entries are the row of Y_tau P, and its first n entries, solved against L_1,
// are the row of Y_tau Omega^+. The factored block keeps L_1's strictly lower part in place,
// its diagonal as reciprocals in `rdiag`, and each reflector with an explicit leading 1. Neither P nor Q is formed. col(., r) is an unpivoted
// Householder QR whose first r orthonormal columns are formed explicitly. Reflectors use
// LAPACK's sign choice (beta = -sign(alpha) ||x||; identity when the tail is zero).
//
// Since UU^* U = U, the product U^* D needed by the merge equals U^* T2^*, with
// T2 = (I - VV^*) Z Psi^+; it is taken from there. D V is formed from D.
//
// Mapping: 256 threads = 32 groups of 8 lanes. A group owns one row (of the factored block,
// of a streamed sample row, or of a basis column); lane q of a group holds columns
// q, q + 8, q + 16, ... in registers or reads them from shared memory. Reductions inside a
// group take 3 shuffles. The FP64 pipe is the bound; shared memory holds the factored n x s
// test block and the r x n sample block of `col`; n x n intermediates live in the node's
// global workspace (L1/L2 resident).
#include <algorithm>

#include "hbs_internal.cuh"

namespace hbs {
namespace {

constexpr int THREADS = 256;
constexpr int G = 8;                    // lanes per row
constexpr int NGROUPS = THREADS / G;    // rows processed at once
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double group_sum(double v) {
  v += __shfl_xor_sync(FULL, v, 4);
  v += __shfl_xor_sync(FULL, v, 2);
  v += __shfl_xor_sync(FULL, v, 1);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

// Reflector of row j of M over columns j..cols-1 (warp 0 only). Leaves v_j in M[j][j..] with
// the leading 1 stored explicitly (so that applying it needs no special case), tau_j in tau[j];
// with rdiag, also 1/beta_j (the diagonal of L) and a NUMERIC flag if beta_j is zero or not
// finite.
__device__ void make_reflector(double* M, int ld, int j, int cols, double* tau, double* rdiag,
                               int* status) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double* row = M + static_cast<size_t>(j) * ld;
  double ss = 0.0;
  for (int k = j + 1 + lane; k < cols; k += 32) ss = fma(row[k], row[k], ss);
  ss = warp_sum(ss);
  const double alpha = row[j];
  double beta = alpha, t = 0.0, scale = 1.0;
  if (ss != 0.0) {
    beta = -copysign(sqrt(fma(alpha, alpha, ss)), alpha);
    t = (beta - alpha) / beta;
    scale = 1.0 / (alpha - beta);
  }
  for (int k = j + 1 + lane; k < cols; k += 32) row[k] *= scale;
  __syncwarp();
  if (lane == 0) {
    row[j] = 1.0;
    tau[j] = t;
    if (rdiag != nullptr) {
      rdiag[j] = 1.0 / beta;
      if (!(fabs(beta) > 0.0) || !isfinite(beta)) atomicOr(status, kStatusNumeric);
    }
  }
}

// In-place Householder LQ of M (rows x cols, rows <= cols, leading dimension ld).
__device__ void lq_factor(double* M, int ld, int rows, int cols, double* tau, double* rdiag,
                          int* status) {
  const int gid = threadIdx.x / G, q = threadIdx.x % G;
  for (int j = 0; j < rows; ++j) {
    make_reflector(M, ld, j, cols, tau, rdiag, status);
    __syncthreads();
    const double tj = tau[j];
    const double* v = M + static_cast<size_t>(j) * ld;
    const int remaining = rows - j - 1;
    for (int base = 0; base < remaining; base += NGROUPS) {
      const int i = j + 1 + base + gid;
      const bool active = i < rows;
      double* ri = M + static_cast<size_t>(active ? i : j) * ld;
      double part = 0.0;
      for (int k = j + q; k < cols; k += G) part = fma(ri[k], v[k], part);
      const double w = group_sum(part) * tj;
      if (active)
        for (int k = j + q; k < cols; k += G) ri[k] = fma(-w, v[k], ri[k]);
    }
    __syncthreads();
  }
}

// y <- y H_j for the reflector stored in row j of M (columns j..cols-1, leading 1 explicit).
// Slots wholly left of column j are skipped (warp-uniform); inside the boundary slot the
// columns k < j select a zero, so every slot costs exactly one FP64 instruction per pass.
template <int T>
__device__ __forceinline__ void apply_reflector(double (&y)[T], const double* v, double tj, int j,
                                                int cols, int q) {
  double part = 0.0;
#pragma unroll
  for (int t = 0; t < T; ++t) {
    if (G * t + G - 1 < j || G * t >= cols) continue;
    const int k = q + G * t;
    const double vk = (k >= j && k < cols) ? v[min(k, cols - 1)] : 0.0;
    part = fma(y[t], vk, part);
  }
  const double w = group_sum(part) * tj;
#pragma unroll
  for (int t = 0; t < T; ++t) {
    if (G * t + G - 1 < j || G * t >= cols) continue;
    const int k = q + G * t;
    const double vk = (k >= j && k < cols) ? v[min(k, cols - 1)] : 0.0;
    y[t] = fma(-w, vk, y[t]);
  }
}

// Streams the n rows of the sample block S (n x s, leading dimension s) through the n
// reflectors of the factored test block F. Writes the last r entries of each transformed row
// to XT (r x ldX, transposed) when XT != NULL, and W = S Omega^+ (n x n, leading dimension ldW).
template <int T>
__device__ void stream_rows(const double* __restrict__ S, int n, int s, int r, const double* F,
                            int ldF, const double* tau, const double* rdiag, double* XT, int ldX,
                            double* __restrict__ W, int ldW) {
  const int gid = threadIdx.x / G, q = threadIdx.x % G;
  const int gbase = (threadIdx.x % 32) & ~(G - 1);
  for (int base = 0; base < n; base += NGROUPS) {
    const int i = base + gid;
    const bool active = i < n;
    double y[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
      const int k = q + G * t;
      y[t] = (active && k < s) ? S[static_cast<size_t>(i) * s + k] : 0.0;
    }
    for (int j = 0; j < n; ++j)
      apply_reflector<T>(y, F + static_cast<size_t>(j) * ldF, tau[j], j, s, q);
    if (XT != nullptr && active) {
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const int k = q + G * t;
        if (k >= s - r && k < s) XT[static_cast<size_t>(k - (s - r)) * ldX + i] = y[t];
      }
    }
    // W L_1 = (y Q)(0:n): column-oriented back substitution, L_1 = lower triangle of F.
#pragma unroll
    for (int t = T - 1; t >= 0; --t) {
      if (G * t >= n) continue;
#pragma unroll 1
      for (int qq = G - 1; qq >= 0; --qq) {
        const int j = qq + G * t;
        if (j >= n) continue;
        const double wj = __shfl_sync(FULL, y[t], gbase + qq) * rdiag[j];
        if (q == qq) y[t] = wj;
        const double* Lj = F + static_cast<size_t>(j) * ldF;
#pragma unroll
        for (int tt = 0; tt <= t; ++tt) {
          const int k = q + G * tt;
          if (k < j) y[tt] = fma(-wj, Lj[k], y[tt]);
        }
      }
    }
    if (active) {
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const int k = q + G * t;
        if (k < n) W[static_cast<size_t>(i) * ldW + k] = y[t];
      }
    }
  }
}

// Basis B (n x r, leading dimension ldB) = first r columns of H_0 ... H_{r-1}, the reflectors
// of the LQ of XT (r x n) -- i.e. col(X, r) for X = XT^*.
template <int T>
__device__ void form_basis(const double* XT, int ldX, const double* tau2, int r, int n,
                           double* __restrict__ B, int ldB) {
  const int gid = threadIdx.x / G, q = threadIdx.x % G;
  for (int base = 0; base < r; base += NGROUPS) {
    const int c = base + gid;
    const bool active = c < r;
    double u[T];
#pragma unroll
    for (int t = 0; t < T; ++t) u[t] = (q + G * t == c) ? 1.0 : 0.0;
    const int jmax = min(r, base + NGROUPS) - 1;
    for (int j = jmax; j >= 0; --j)
      apply_reflector<T>(u, XT + static_cast<size_t>(j) * ldX, tau2[j], j, n, q);
    if (active) {
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const int k = q + G * t;
        if (k < n) B[static_cast<size_t>(k) * ldB + c] = u[t];
      }
    }
  }
}

__device__ void load_block(double* F, int ldF, const double* __restrict__ X, int n, int s) {
  for (int e = threadIdx.x; e < n * s; e += THREADS) {
    const int i = e / s, k = e % s;
    F[static_cast<size_t>(i) * ldF + k] = X[e];
  }
}

template <int T>
__global__ void __launch_bounds__(THREADS, 1)
    node_sweep_f64(const NodeTask* __restrict__ tasks, int* status) {
  extern __shared__ double smem[];
  const NodeTask tk = tasks[blockIdx.x];
  const int n = tk.n, r = tk.r, s = tk.s;
  const int ldF = s + 1, ldX = n + 1;
  double* F = smem;                                   // n x ldF
  double* XT = F + static_cast<size_t>(n) * ldF;      // r x ldX
  double* tau = XT + static_cast<size_t>(r) * ldX;    // n
  double* rdiag = tau + n;                            // n
  double* tau2 = rdiag + n;                           // r

  // ---- Omega / Y side: LQ of Omega_tau, rows of Y_tau -> Y Omega^+ and Y P ----
  load_block(F, ldF, tk.Om, n, s);
  __syncthreads();
  lq_factor(F, ldF, n, s, tau, rdiag, status);
  if (tk.is_root) {
    stream_rows<T>(tk.Y, n, s, 0, F, ldF, tau, rdiag, nullptr, 0, tk.D, n);
    return;
  }
  stream_rows<T>(tk.Y, n, s, r, F, ldF, tau, rdiag, XT, ldX, tk.WY, n);
  __syncthreads();
  lq_factor(XT, ldX, r, n, tau2, nullptr, status);
  form_basis<T>(XT, ldX, tau2, r, n, tk.U, r);
  __syncthreads();

  // ---- Psi / Z side ----
  load_block(F, ldF, tk.Ps, n, s);
  __syncthreads();
  lq_factor(F, ldF, n, s, tau, rdiag, status);
  stream_rows<T>(tk.Z, n, s, r, F, ldF, tau, rdiag, XT, ldX, tk.WZ, n);
  __syncthreads();
  lq_factor(XT, ldX, r, n, tau2, nullptr, status);
  form_basis<T>(XT, ldX, tau2, r, n, tk.V, r);
  __syncthreads();

  // ---- D_tau (Eq. d_tau_formula) ----
  // written earlier in this kernel: plain (coherent) loads, no __restrict__
  const double* U = tk.U;
  const double* V = tk.V;
  const double* WY = tk.WY;
  const double* WZ = tk.WZ;
  const int ldT = n + 1;
  double* G1 = XT;                                    // r x ldX: V^* WZ, later U^* T2^*
  double* T2 = F;                                     // n x ldT: (I - VV^*) WZ, later D
  double* Hs = F + static_cast<size_t>(n) * ldT;      // r x n: U^*(T2^* - WY), later (D V)^*
  for (int e = threadIdx.x; e < r * n; e += THREADS) {
    const int c = e / n, j = e % n;
    double acc = 0.0;
    for (int i = 0; i < n; ++i) acc = fma(V[i * r + c], WZ[static_cast<size_t>(i) * n + j], acc);
    G1[c * ldX + j] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += THREADS) {
    const int i = e / n, j = e % n;
    double acc = WZ[e];
    for (int c = 0; c < r; ++c) acc = fma(-V[i * r + c], G1[c * ldX + j], acc);
    T2[i * ldT + j] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * n; e += THREADS) {
    const int c = e / n, j = e % n;
    double h2 = 0.0, ky = 0.0;
    for (int i = 0; i < n; ++i) {
      const double u = U[i * r + c];
      h2 = fma(u, T2[j * ldT + i], h2);
      ky = fma(u, WY[static_cast<size_t>(i) * n + j], ky);
    }
    G1[c * ldX + j] = h2;
    Hs[c * n + j] = h2 - ky;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += THREADS) {
    const int i = e / n, j = e % n;
    double acc = WY[e];
    for (int c = 0; c < r; ++c) acc = fma(U[i * r + c], Hs[c * n + j], acc);
    tk.D[e] = acc;
    T2[i * ldT + j] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * n; e += THREADS) {
    const int c = e / n, i = e % n;
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc = fma(T2[i * ldT + j], V[j * r + c], acc);
    Hs[c * n + i] = acc;
  }
  __syncthreads();

  // ---- this node's rows of the parent's blocks (Eq. omega_tau_and_y_tau) ----
  for (int e = threadIdx.x; e < r * s; e += THREADS) {
    const int c = e / s, k = e % s;
    double om = 0.0, ps = 0.0, y = 0.0, z = 0.0;
    for (int i = 0; i < n; ++i) {
      const size_t ik = static_cast<size_t>(i) * s + k;
      const double u = U[i * r + c], v = V[i * r + c];
      const double omk = tk.Om[ik], psk = tk.Ps[ik];
      om = fma(v, omk, om);
      ps = fma(u, psk, ps);
      y = fma(u, tk.Y[ik], y);
      y = fma(-G1[c * ldX + i], omk, y);
      z = fma(v, tk.Z[ik], z);
      z = fma(-Hs[c * n + i], psk, z);
    }
    tk.Om_p[e] = om;
    tk.Ps_p[e] = ps;
    tk.Y_p[e] = y;
    tk.Z_p[e] = z;
  }
}

}  // namespace

size_t node_smem_doubles(int n, int r, int s) {
  return static_cast<size_t>(n) * (s + 1) + static_cast<size_t>(r) * (n + 1) + 2 * n + r;
}

cudaError_t launch_node_sweep_f64(const NodeTask* d_tasks, int ntasks, int max_n, int max_r,
                                  int max_s, int* d_status, cudaStream_t st) {
  if (ntasks <= 0) return cudaSuccess;
  const size_t bytes = node_smem_doubles(max_n, max_r, max_s) * sizeof(double);
  if (bytes > kMaxNodeSmemBytes || max_s > kMaxS) return cudaErrorInvalidValue;
  auto launch = [&](auto kernel) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kMaxNodeSmemBytes));
    if (e != cudaSuccess) return e;
    kernel<<<ntasks, THREADS, bytes, st>>>(d_tasks, d_status);
    return cudaGetLastError();
  };
  if (max_s <= 8 * G) return launch(node_sweep_f64<8>);
  if (max_s <= 16 * G) return launch(node_sweep_f64<16>);
  return launch(node_sweep_f64<24>);
}

}  // namespace hbs
