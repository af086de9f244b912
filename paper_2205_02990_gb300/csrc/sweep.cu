// Per-level sweep of Algorithm 2: the kernels of one tree level.
//
// For a node tau with blocks Omega_tau, Psi_tau, Y_tau, Z_tau (n x s) the sweep computes
//   P = null(Omega_tau, r), U = col(Y_tau P, r)              (Section 4.1, Eq. u_tau_formula)
//   Q = null(Psi_tau, r),   V = col(Z_tau Q, r)              (Eq. v_tau_formula)
//   D = (I - UU^*) Y Omega^+ + UU^* ((I - VV^*) Z Psi^+)^*   (Eq. d_tau_formula)
// and the node's rows of the parent's blocks (Eq. omega_tau_and_y_tau, Algorithm 2):
//   V^* Omega_tau, U^* Psi_tau, U^* (Y_tau - D Omega_tau), V^* (Z_tau - D^* Psi_tau).
// At the root only D = Y Omega^+ (Section 4.3).
//
// Side kernel (the LQ in FP64 in every precision: it holds the nullspace and the pseudo-inverse;
// with the reduced finishes the one-CTA form pushes the sample rows through it in double-float,
// the cluster form in FP64); side 0
// works on Omega_tau and Y_tau, side 1 on Psi_tau and Z_tau. One Householder LQ of the test
// block, Omega_tau = L Q^* (the QR of Omega_tau^* of Section 2.4, Q square), serves both `null`
// and the pseudo-inverse: the last r columns of Q are null(Omega_tau, r), and
// Omega_tau = L_1 Q_1^* with L_1 the leading n x n lower triangle gives Omega^+ = Q_1 L_1^{-1}.
// Each sample row y is pushed once through the n reflectors (y Q = y H_0 ... H_{n-1}): its last
// r entries are the row of Y_tau P, its first n entries, solved against L_1, the row of
// Y_tau Omega^+. Neither P nor Q is formed. Two forms, which round alike: node_side (one CTA per
// (node, side), or per row slice, each slice refactoring the block) and node_side_cluster (a
// thread-block cluster shares one factorization, below), for the levels with few nodes.
//
// Finish kernels, per level after the side kernel: node_bases (col(., r): an unpivoted
// Householder QR whose first r columns are formed by backward accumulation; FP64, or FP32 in the
// plain mixed finish), then D_tau from D = WY + U (Q - P - R V^*) (node_dblk_a / node_dblk_b in
// FP64, over column blocks; node_dchain in FP32 or in double-float, which also forms U^* D and
// (D V)^*), then the parent's blocks (node_merge in FP64 / node_merge_r in FP32 or double-float,
// over column chunks). The double-float finish (compensated FP32 pairs, dfloat.cuh) keeps ~48
// bits on the FP32 pipe.
//
// Reflectors use LAPACK's sign choice (beta = -sign(alpha) ||x||; identity when the tail is
// zero) and are stored with their leading 1 explicit. Mapping: 256 threads = 32 groups of 8
// lanes; a group owns one row (of the factored block or of a streamed sample row) and lane q of
// a group holds columns q, q + 8, ... Reductions inside a group take 3 shuffles. The FP64 pipe
// (2 DFMA per clock per SM on GB300) bounds the side kernel where a level has many nodes.
#include <algorithm>
#include <type_traits>

#include <cooperative_groups.h>

#include "dfloat.cuh"
#include "hbs_internal.cuh"
#include "tc_ptx.cuh"

namespace hbs {
namespace {

namespace cg = cooperative_groups;

constexpr int THREADS = 256;
constexpr int G = 8;                    // lanes per row
constexpr int NGROUPS = THREADS / G;    // rows processed at once
constexpr unsigned FULL = 0xffffffffu;

template <class Real>
__device__ __forceinline__ Real group_sum(Real v) {
  v += __shfl_xor_sync(FULL, v, 4);
  v += __shfl_xor_sync(FULL, v, 2);
  v += __shfl_xor_sync(FULL, v, 1);
  return v;
}

template <class Real>
__device__ __forceinline__ Real warp_sum(Real v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return ::rsqrt(x); }
__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }

// Reflector of row j of M over columns j..cols-1 (warp 0 only). Leaves v_j in M[j][j..] with
// the leading 1 stored explicitly, tau_j in tau[j]; with rdiag, also 1/beta_j (the diagonal of
// L) and a NUMERIC flag if beta_j is zero or not finite.
// With rho = 1/||x|| (one reciprocal square root) the scalars need one more reciprocal only:
// beta = -sign(alpha)/rho, 1/beta = -sign(alpha) rho, tau = (beta - alpha)/beta = 1 + |alpha| rho
// and 1/(alpha - beta) = sign(alpha)/(|alpha| + |beta|). On GB300 a dependent FP64 square root
// or division costs ~650-700 cycles and a reciprocal or reciprocal square root ~450, and this
// chain is serial in the factorization.
template <class Real>
__device__ void make_reflector(Real* M, int ld, int j, int cols, Real* tau, Real* rdiag,
                               int* status) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  Real* row = M + static_cast<size_t>(j) * ld;
  Real ss = 0;
  for (int k = j + 1 + lane; k < cols; k += 32) ss = fma(row[k], row[k], ss);
  ss = warp_sum(ss);
  const Real alpha = row[j];
  Real beta = alpha, t = 0, scale = 1, inv_beta;
  if (ss != Real(0)) {
    const Real s2 = fma(alpha, alpha, ss);
    const Real rho = rsqrt_r(s2);
    const Real nb = s2 * rho;                          // ||x||
    beta = -copysign(nb, alpha);
    inv_beta = -copysign(rho, alpha);
    t = fma(fabs(alpha), rho, Real(1));
    scale = copysign(recip(fabs(alpha) + nb), alpha);
  } else {
    inv_beta = Real(1) / alpha;                        // H = I; L keeps alpha
  }
  for (int k = j + 1 + lane; k < cols; k += 32) row[k] *= scale;
  __syncwarp();
  if (lane == 0) {
    row[j] = 1;
    tau[j] = t;
    if (rdiag != nullptr) {
      rdiag[j] = inv_beta;
      if (!(fabs(beta) > Real(0)) || !isfinite(beta)) atomicOr(status, kStatusNumeric);
    }
  }
}

// In-place Householder LQ of M (rows x cols, rows <= cols, leading dimension ld), with a
// one-step look-ahead: while warps 1.. apply reflector j to rows j+2.., warp 0 applies it to row
// j+1 and at once generates reflector j+1, so the serial reflector generation (a norm, a square
// root and two divisions on the FP64 pipe) is off the critical path of the other warps. Row j+1
// is updated by a whole warp (a 32-lane reduction), the other rows by groups of G lanes.
template <class Real>
__device__ void lq_factor(Real* M, int ld, int rows, int cols, Real* tau, Real* rdiag,
                          int* status) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int gid = (threadIdx.x - 32) / G, q = threadIdx.x % G;   // groups of warps 1..
  constexpr int kGroups = (THREADS - 32) / G;
  make_reflector(M, ld, 0, cols, tau, rdiag, status);
  __syncthreads();
  for (int j = 0; j < rows; ++j) {
    const Real tj = tau[j];
    const Real* v = M + static_cast<size_t>(j) * ld;
    if (warp == 0) {
      if (j + 1 < rows) {                                         // row j+1, then reflector j+1
        Real* ri = M + static_cast<size_t>(j + 1) * ld;
        Real part = 0;
        for (int k = j + lane; k < cols; k += 32) part = fma(ri[k], v[k], part);
        const Real w = warp_sum(part) * tj;
        for (int k = j + lane; k < cols; k += 32) ri[k] = fma(-w, v[k], ri[k]);
        __syncwarp();
        make_reflector(M, ld, j + 1, cols, tau, rdiag, status);
      }
    } else {
      const int remaining = rows - j - 2;                       // rows j+2 .. rows-1
      for (int base = 0; base < remaining; base += kGroups) {
        if (base + (warp - 1) * (32 / G) >= remaining) break;     // no row for this warp
        const int i = j + 2 + base + gid;
        const bool active = i < rows;
        Real* ri = M + static_cast<size_t>(active ? i : j) * ld;
        Real part = 0;
        for (int k = j + q; k < cols; k += G) part = fma(ri[k], v[k], part);
        const Real w = group_sum(part) * tj;
        if (active)
          for (int k = j + q; k < cols; k += G) ri[k] = fma(-w, v[k], ri[k]);
      }
    }
    __syncthreads();
  }
}

// y <- y H_j for the reflector stored in row j of M (columns j..cols-1, leading 1 explicit).
// Slots wholly left of column j are skipped (warp-uniform); inside the boundary slot the
// columns k < j select a zero, so every slot costs exactly one FMA per pass.
template <class Real, int NS>
__device__ __forceinline__ void apply_reflector(Real (&y)[NS], const Real* v, Real tj, int j,
                                                int cols, int q) {
  Real part = 0;
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    if (G * t + G - 1 < j || G * t >= cols) continue;
    const int k = q + G * t;
    const Real vk = (k >= j && k < cols) ? v[min(k, cols - 1)] : Real(0);
    part = fma(y[t], vk, part);
  }
  const Real w = group_sum(part) * tj;
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    if (G * t + G - 1 < j || G * t >= cols) continue;
    const int k = q + G * t;
    const Real vk = (k >= j && k < cols) ? v[min(k, cols - 1)] : Real(0);
    y[t] = fma(-w, vk, y[t]);
  }
}

// Finishes one transformed sample row y (= s_i Q, lane q holding columns q, q + G, ...): its last
// r entries to row i of X (n x r, row-major) when X != NULL, and the row of W = S Omega^+ (n x n)
// from the back substitution W L_1 = (S Q)(:, 0:n), L_1 = lower triangle of F.
template <int NS>
__device__ __forceinline__ void store_row(double (&y)[NS], int i, bool active, int n, int s, int r,
                                          const double* F, int ldF, const double* rdiag,
                                          double* __restrict__ X, double* __restrict__ W) {
  const int q = threadIdx.x % G;
  const int gbase = (threadIdx.x % 32) & ~(G - 1);
  if (X != nullptr && active) {
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int k = q + G * t;
      if (k >= s - r && k < s) X[static_cast<size_t>(i) * r + (k - (s - r))] = y[t];
    }
  }
  // column-oriented back substitution
#pragma unroll
  for (int t = NS - 1; t >= 0; --t) {
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
    for (int t = 0; t < NS; ++t) {
      const int k = q + G * t;
      if (k < n) W[static_cast<size_t>(i) * n + k] = y[t];
    }
  }
}

// Streams rows [row0, row1) of the sample block S (n x s, leading dimension s) through the n
// reflectors of the factored test block F, then finishes them (store_row).
template <int NS>
__device__ void stream_rows(const double* __restrict__ S, int n, int s, int r, int row0, int row1,
                            const double* F, int ldF, const double* tau, const double* rdiag,
                            double* __restrict__ X, double* __restrict__ W) {
  const int gid = threadIdx.x / G, q = threadIdx.x % G;
  for (int base = row0; base < row1; base += NGROUPS) {
    if (base + (threadIdx.x / 32) * (32 / G) >= row1) break;   // no row for this warp
    const int i = base + gid;
    const bool active = i < row1;
    double y[NS];
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int k = q + G * t;
      y[t] = (active && k < s) ? S[static_cast<size_t>(i) * s + k] : 0.0;
    }
    for (int j = 0; j < n; ++j)
      apply_reflector<double, NS>(y, F + static_cast<size_t>(j) * ldF, tau[j], j, s, q);
    store_row<NS>(y, i, active, n, s, r, F, ldF, rdiag, X, W);
  }
}

// ---- the same streaming in double-float (compensated finish, single-CTA side form) -----------
// The LQ stays FP64; its shared-memory image (reflectors with L_1 below the diagonal, tau, 1/beta)
// is then converted in place to double-float pairs, and the sample rows go through it on the
// FP32 pipe: a double-float multiply-add is ~15 FP32 instructions against one FP64 instruction
// that holds the FP64 unit as long as 64 FP32 ones on GB300. Where two CTAs share an SM the rows
// take the reflectors two at a time (compact WY of two), which halves the latency of the 8-lane
// reductions that bound this streaming.

// Sum over the 8 lanes of a row group (butterfly: every lane ends with the same bits).
__device__ __forceinline__ dfloat df_group_sum(dfloat v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const dfloat w{__shfl_xor_sync(FULL, v.hi, o), __shfl_xor_sync(FULL, v.lo, o)};
    v = df_add(v, w);
  }
  return v;
}

template <int NS>
__device__ __forceinline__ void apply_reflector_df(dfloat (&y)[NS], const dfloat* v, dfloat tj, int j,
                                                   int cols, int q) {
  dfloat part = df_zero();
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    if (G * t + G - 1 < j || G * t >= cols) continue;
    const int k = q + G * t;
    const dfloat vk = (k >= j && k < cols) ? v[min(k, cols - 1)] : df_zero();
    part = df_fma_acc(y[t], vk, part);
  }
  const dfloat w = df_neg(df_fma(df_group_sum(df_norm(part)), tj, df_zero()));
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    if (G * t + G - 1 < j || G * t >= cols) continue;
    const int k = q + G * t;
    const dfloat vk = (k >= j && k < cols) ? v[min(k, cols - 1)] : df_zero();
    y[t] = df_fma(w, vk, y[t]);
  }
}

// y <- y H_j H_{j+1} in one pass (the compact WY form of two reflectors, Schreiber and Van Loan
// 1989): with a = tau_j (y . v_j) and b = tau_{j+1} (y . v_{j+1} - a c_j), c_j = v_j . v_{j+1},
// the product is y - a v_j - b v_{j+1}. The two dot products share one pass over the row and
// their 8-lane sums interleave, so each pair pays one reduction's latency instead of two.
template <int NS>
__device__ __forceinline__ void apply_reflector_pair_df(dfloat (&y)[NS], const dfloat* v,
                                                        const dfloat* u, dfloat tj, dfloat tj1,
                                                        dfloat cj, int j, int cols, int q) {
  dfloat p1 = df_zero(), p2 = df_zero();
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    if (G * t + G - 1 < j || G * t >= cols) continue;
    const int k = q + G * t;
    const int kc = min(k, cols - 1);
    const dfloat vk = (k >= j && k < cols) ? v[kc] : df_zero();
    const dfloat uk = (k > j && k < cols) ? u[kc] : df_zero();
    p1 = df_fma_acc(y[t], vk, p1);
    p2 = df_fma_acc(y[t], uk, p2);
  }
  p1 = df_norm(p1);
  p2 = df_norm(p2);
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const dfloat w1{__shfl_xor_sync(FULL, p1.hi, o), __shfl_xor_sync(FULL, p1.lo, o)};
    const dfloat w2{__shfl_xor_sync(FULL, p2.hi, o), __shfl_xor_sync(FULL, p2.lo, o)};
    p1 = df_add(p1, w1);
    p2 = df_add(p2, w2);
  }
  const dfloat a = df_fma(p1, tj, df_zero());
  const dfloat na = df_neg(a);
  const dfloat nb = df_neg(df_fma(df_fma(na, cj, p2), tj1, df_zero()));
#pragma unroll
  for (int t = 0; t < NS; ++t) {
    if (G * t + G - 1 < j || G * t >= cols) continue;
    const int k = q + G * t;
    const int kc = min(k, cols - 1);
    const dfloat vk = (k >= j && k < cols) ? v[kc] : df_zero();
    const dfloat uk = (k > j && k < cols) ? u[kc] : df_zero();
    y[t] = df_fma(nb, uk, df_fma(na, vk, y[t]));
  }
}

// c_j = v_j . v_{j+1} for the reflector pairs (j even, j + 1 < n) of a double-float image, into
// the image's spare column `cols` of row j. One pair per group of 8 lanes; a warp stops only when
// none of its groups has a pair, so every lane takes part in the shuffles.
__device__ void pair_dots_df(dfloat* F, int ldF, int n, int cols) {
  const int warp = threadIdx.x / 32, gid = threadIdx.x / G, q = threadIdx.x % G;
  const int npairs = n / 2;
  for (int base = 0; base < npairs; base += NGROUPS) {
    if (base + warp * (32 / G) >= npairs) break;                // no pair for this warp
    const int pr = base + gid;
    const bool active = pr < npairs;
    const int j = active ? 2 * pr : 0;
    const dfloat* v = F + static_cast<size_t>(j) * ldF;
    const dfloat* u = v + ldF;
    dfloat c = df_zero();
    for (int k = j + 1 + q; k < cols; k += G) c = df_fma_acc(v[k], u[k], c);
    c = df_group_sum(df_norm(c));
    if (active && q == 0) F[static_cast<size_t>(j) * ldF + cols] = c;
  }
}

// store_row in double-float: the last r entries to X, then the back substitution against L_1
// and the first n entries to W (both stored as FP64).
template <int NS>
__device__ __forceinline__ void store_row_df(dfloat (&y)[NS], int i, bool active, int n, int s, int r,
                                             const dfloat* F, int ldF, const dfloat* rdiag,
                                             double* __restrict__ X, double* __restrict__ W) {
  const int q = threadIdx.x % G;
  const int gbase = (threadIdx.x % 32) & ~(G - 1);
  if (X != nullptr && active) {
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int k = q + G * t;
      if (k >= s - r && k < s) X[static_cast<size_t>(i) * r + (k - (s - r))] = df_to(y[t]);
    }
  }
#pragma unroll
  for (int t = NS - 1; t >= 0; --t) {
    if (G * t >= n) continue;
#pragma unroll 1
    for (int qq = G - 1; qq >= 0; --qq) {
      const int j = qq + G * t;
      if (j >= n) continue;
      const dfloat yj{__shfl_sync(FULL, y[t].hi, gbase + qq), __shfl_sync(FULL, y[t].lo, gbase + qq)};
      const dfloat wj = df_fma(yj, rdiag[j], df_zero());
      if (q == qq) y[t] = wj;
      const dfloat nwj = df_neg(wj);
      const dfloat* Lj = F + static_cast<size_t>(j) * ldF;
#pragma unroll
      for (int tt = 0; tt <= t; ++tt) {
        const int k = q + G * tt;
        if (k < j) y[tt] = df_fma(nwj, Lj[k], y[tt]);
      }
    }
  }
  if (active) {
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int k = q + G * t;
      if (k < n) W[static_cast<size_t>(i) * n + k] = df_to(y[t]);
    }
  }
}

// PAIRS: the reflectors two at a time (apply_reflector_pair_df, with c_j in column s of row j);
// otherwise one at a time.
template <int NS, bool PAIRS>
__device__ void stream_rows_df(const double* __restrict__ S, int n, int s, int r, int row0, int row1,
                               const dfloat* F, int ldF, const dfloat* tau, const dfloat* rdiag,
                               double* __restrict__ X, double* __restrict__ W) {
  const int gid = threadIdx.x / G, q = threadIdx.x % G;
  for (int base = row0; base < row1; base += NGROUPS) {
    if (base + (threadIdx.x / 32) * (32 / G) >= row1) break;   // no row for this warp
    const int i = base + gid;
    const bool active = i < row1;
    dfloat y[NS];
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int k = q + G * t;
      y[t] = (active && k < s) ? df_from(S[static_cast<size_t>(i) * s + k]) : df_zero();
    }
    int j = 0;
    if constexpr (PAIRS) {
      for (; j + 1 < n; j += 2) {
        const dfloat* v = F + static_cast<size_t>(j) * ldF;
        apply_reflector_pair_df<NS>(y, v, v + ldF, tau[j], tau[j + 1], v[s], j, s, q);
      }
    }
    for (; j < n; ++j)
      apply_reflector_df<NS>(y, F + static_cast<size_t>(j) * ldF, tau[j], j, s, q);
    store_row_df<NS>(y, i, active, n, s, r, F, ldF, rdiag, X, W);
  }
}

// The side kernel's shared-memory image (len values) from FP64 to double-float, in place.
__device__ __forceinline__ void image_to_df(double* img, int len) {
  __syncthreads();
  for (int e = threadIdx.x; e < len; e += THREADS) {
    const dfloat v = df_from(img[e]);
    reinterpret_cast<dfloat*>(img)[e] = v;
  }
  __syncthreads();
}

// Basis B (n x r, leading dimension ldB, FP64 storage) = first r columns of H_0 ... H_{r-1},
// the reflectors of the LQ of XT (r x n) -- i.e. col(X, r) for X = XT^*. Backward accumulation
// on an n x r tile W in shared memory: W = [I_r; 0], then W <- H_j W for j = r-1 .. 0. H_j acts
// on rows j.. only, where the columns c < j of W are still zero, so step j touches the block of
// rows j.. and columns j.. . Lanes run over columns and warps over rows: the dot products
// v_j^* W are summed per warp, the eight partial sums added by one thread per column (no
// shuffles, no integer divisions). scratch: 8 r + r Reals.
template <class Real>
__device__ void form_basis(const Real* XT, int ldX, const Real* tau2, int r, int n, Real* W,
                           Real* scratch, double* __restrict__ B, int ldB) {
  constexpr int kWarps = THREADS / 32;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int ldW = r + 1;
  Real* part = scratch;                                // kWarps x r
  Real* wsum = scratch + kWarps * r;                   // r
  for (int i = warp; i < n; i += kWarps)
    for (int c = lane; c < r; c += 32) W[i * ldW + c] = (i == c) ? Real(1) : Real(0);
  __syncthreads();
  for (int j = r - 1; j >= 0; --j) {
    const Real* v = XT + static_cast<size_t>(j) * ldX;  // v[j] = 1, v[i > j] the tail
    for (int c = j + lane; c < r; c += 32) {
      Real acc = 0;
      for (int i = j + warp; i < n; i += kWarps) acc = fma(v[i], W[i * ldW + c], acc);
      part[warp * r + c] = acc;
    }
    __syncthreads();
    if (threadIdx.x >= j && threadIdx.x < r) {
      Real w = 0;
#pragma unroll
      for (int ww = 0; ww < kWarps; ++ww) w += part[ww * r + threadIdx.x];
      wsum[threadIdx.x] = w * tau2[j];
    }
    __syncthreads();
    for (int c = j + lane; c < r; c += 32) {
      const Real w = wsum[c];
      for (int i = j + warp; i < n; i += kWarps) W[i * ldW + c] = fma(-v[i], w, W[i * ldW + c]);
    }
    __syncthreads();
  }
  for (int i = warp; i < n; i += kWarps)
    for (int c = lane; c < r; c += 32) B[static_cast<size_t>(i) * ldB + c] = static_cast<double>(W[i * ldW + c]);
}

// ---- side kernel: LQ of one test block, its sample rows -> W rows and X rows (FP64) ---------

// MINB: CTAs per SM the registers are budgeted for (3 or 4 where the test block is small enough
// for that many tiles of shared memory per SM, so that more warps hide the FP64 latencies).
// PRE: the factorization of the test block was made beforehand by node_lq (its shared-memory
// image in `lq`, lq_stride doubles per (node, side)) and is copied in instead of recomputed;
// the same instructions made it, so the results are bit-identical.
// DF: the sample rows stream in double-float (compensated finish).
template <int NS, int MINB, bool PRE = false, bool DF = false>
__global__ void __launch_bounds__(THREADS, MINB)
    node_side(const NodeTask* __restrict__ tasks, int row_splits, int* status,
              const double* __restrict__ lq = nullptr, int64_t lq_stride = 0) {
  extern __shared__ double smem[];
  const NodeTask tk = tasks[blockIdx.x];
  const int side = blockIdx.y;
  if (tk.is_root && side == 1) return;                 // the root needs Y Omega^+ only
  const int n = tk.n, r = tk.r, s = tk.s;
  const int chunk = (n + row_splits - 1) / row_splits;
  const int row0 = blockIdx.z * chunk, row1 = min(n, row0 + chunk);
  if (row0 >= row1) return;
  const int ldF = s + 1;
  double* F = smem;                                    // n x ldF
  double* tau = F + static_cast<size_t>(n) * ldF;      // n
  double* rdiag = tau + n;                             // n
  if constexpr (PRE) {
    const double* img = lq + (2 * static_cast<int64_t>(blockIdx.x) + side) * lq_stride;
    const int len = n * ldF + 2 * n;
    for (int e = threadIdx.x; e < len; e += THREADS) F[e] = img[e];
    __syncthreads();
  } else {
    const double* T = side ? tk.Ps : tk.Om;
    for (int e = threadIdx.x; e < n * s; e += THREADS) F[(e / s) * ldF + e % s] = T[e];
    __syncthreads();
    lq_factor<double>(F, ldF, n, s, tau, rdiag, status);
  }
  if constexpr (DF) {
    image_to_df(F, n * ldF + 2 * n);
    // Reflector pairs where two CTAs share an SM (128 registers a thread); at three CTAs per SM
    // (80 registers) the pair form measured slower than one reflector at a time.
    constexpr bool kPairs = MINB <= 2;
    if constexpr (kPairs) {
      pair_dots_df(reinterpret_cast<dfloat*>(F), ldF, n, s);    // into the spare column s
      __syncthreads();
    }
    const dfloat* Fd = reinterpret_cast<const dfloat*>(F);
    const dfloat* taud = Fd + static_cast<size_t>(n) * ldF;
    const dfloat* rdiagd = taud + n;
    if (tk.is_root) {
      stream_rows_df<NS, kPairs>(tk.Y, n, s, 0, row0, row1, Fd, ldF, taud, rdiagd, nullptr, tk.D);
      return;
    }
    stream_rows_df<NS, kPairs>(side ? tk.Z : tk.Y, n, s, r, row0, row1, Fd, ldF, taud, rdiagd,
                       side ? tk.XZ : tk.XY, side ? tk.WZ : tk.WY);
  } else {
    if (tk.is_root) {
      stream_rows<NS>(tk.Y, n, s, 0, row0, row1, F, ldF, tau, rdiag, nullptr, tk.D);
      return;
    }
    stream_rows<NS>(side ? tk.Z : tk.Y, n, s, r, row0, row1, F, ldF, tau, rdiag,
                    side ? tk.XZ : tk.XY, side ? tk.WZ : tk.WY);
  }
}

// The LQ of one test block alone (grid: node, side), its shared-memory image (F, tau, 1/beta:
// side_smem_doubles(n, s) doubles) written to lq for node_side<.., PRE = true>. The test blocks
// of the leaves need no sample, so this can run while the products are formed: registers are
// budgeted at 40 per thread (six CTAs' worth per SM) so that a CTA fits beside a product
// kernel's (e.g. 320 threads x 168 registers).
__global__ void __launch_bounds__(THREADS, 6)
    node_lq(const NodeTask* __restrict__ tasks, int* status, double* __restrict__ lq,
            int64_t lq_stride) {
  extern __shared__ double smem[];
  const NodeTask tk = tasks[blockIdx.x];
  const int side = blockIdx.y;
  if (tk.is_root && side == 1) return;
  const int n = tk.n, s = tk.s;
  const int ldF = s + 1;
  double* F = smem;
  double* tau = F + static_cast<size_t>(n) * ldF;
  double* rdiag = tau + n;
  const double* T = side ? tk.Ps : tk.Om;
  for (int e = threadIdx.x; e < n * s; e += THREADS) F[(e / s) * ldF + e % s] = T[e];
  __syncthreads();
  lq_factor<double>(F, ldF, n, s, tau, rdiag, status);
  __syncthreads();
  double* img = lq + (2 * static_cast<int64_t>(blockIdx.x) + side) * lq_stride;
  const int len = n * ldF + 2 * n;
  for (int e = threadIdx.x; e < len; e += THREADS) img[e] = F[e];
}

// ---- side kernel, cluster form: the C CTAs of a thread-block cluster share one LQ -----------
//
// A test block's LQ is a chain of n reflector steps; on one SM it is bounded by that SM's FP64
// pipe (the row updates) and by the serial reflector generation. Here the C CTAs of a cluster
// (grid z) hold one (node, side) together. LQ row i lives in CTA i mod C, which applies every
// reflector to it. When row j+1 is due, warp 0 of its owner applies reflector j to it, generates
// reflector j+1, writes tau and 1/beta into the row's two spare columns and sends the finished
// row (its part of L and the reflector) to every other CTA of the cluster with one bulk copy per
// CTA into distributed shared memory; each CTA has one mbarrier per row, armed for the row's
// bytes before the loop, and waits on it before the step that uses the row. The other warps
// meanwhile apply reflector j to the CTA's rows below j+1 and to its slice of the sample rows
// (staged in shared memory), so the sample rows ride along with the factorization. There is no
// cluster-wide barrier per step: a row depends only on earlier rows, so the CTAs run ahead or
// behind each other freely. After the n-th step every CTA holds the whole factorization and
// finishes its sample rows.
__host__ __device__ __forceinline__ int cluster_ld(int s) { return s + 2 + (s & 1); }

__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

// Row j (ldF doubles, 16-byte aligned) from this CTA to CTA d's copy of it, completing on d's
// mbarrier of that row.
__device__ __forceinline__ void send_row(const double* row, uint64_t* bar, uint32_t bytes, int d) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(cluster_addr(su32(row), d)), "r"(su32(row)), "r"(bytes), "r"(cluster_addr(su32(bar), d))
      : "memory");
}

template <int NS>
__global__ void __launch_bounds__(THREADS, 2)
    node_side_cluster(const NodeTask* __restrict__ tasks, int* status) {
  extern __shared__ __align__(16) double smem_cl[];
  cg::cluster_group cl = cg::this_cluster();
  const NodeTask tk = tasks[blockIdx.x];
  const int side = blockIdx.y;
  if (tk.is_root && side == 1) return;                 // the whole cluster leaves together
  const int C = static_cast<int>(cl.num_blocks());
  const int c = static_cast<int>(cl.block_rank());
  const int n = tk.n, r = tk.r, s = tk.s, ldF = cluster_ld(s);
  const uint32_t row_bytes = static_cast<uint32_t>(ldF) * sizeof(double);
  const int chunk = (n + C - 1) / C;
  const int row0 = min(n, c * chunk), nrows = min(n, row0 + chunk) - row0;
  double* F = smem_cl;                                 // n x ldF (every row, once received)
  double* tau = F + static_cast<size_t>(n) * ldF;      // n (owner's scratch)
  double* rdiag = tau + n;                             // n
  double* Sr = rdiag + n + (n & 1);                    // chunk x ldF: this CTA's sample rows
  uint64_t* bar = reinterpret_cast<uint64_t*>(Sr + static_cast<size_t>(chunk) * ldF);   // n
  const double* T = side ? tk.Ps : tk.Om;
  const double* S = side ? tk.Z : tk.Y;
  const int own = c < n ? (n - 1 - c) / C + 1 : 0;     // rows c, c + C, ...
  for (int e = threadIdx.x; e < own * s; e += THREADS) {
    const int i = c + (e / s) * C, k = e % s;
    F[static_cast<size_t>(i) * ldF + k] = T[static_cast<size_t>(i) * s + k];
  }
  for (int e = threadIdx.x; e < nrows * s; e += THREADS) {
    const int i = e / s, k = e % s;
    Sr[static_cast<size_t>(i) * ldF + k] = S[static_cast<size_t>(row0 + i) * s + k];
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) mbar_init(&bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int i = 0; i < n; ++i)
      if (i % C != c) mbar_expect_tx(&bar[i], row_bytes);     // armed before any copy can start
  }
  cl.sync();                     // every CTA runs and has armed its barriers before any copy
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, q = threadIdx.x % G;
  // reflector j, its tau and 1/beta into row j (columns s, s + 1), then out to the cluster
  auto finish_reflector = [&](int j) {
    make_reflector(F, ldF, j, s, tau, rdiag, status);
    __syncwarp();
    if (lane == 0) {
      F[static_cast<size_t>(j) * ldF + s] = tau[j];
      F[static_cast<size_t>(j) * ldF + s + 1] = rdiag[j];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the copies
    __syncwarp();
    if (lane < C && lane != c) send_row(F + static_cast<size_t>(j) * ldF, &bar[j], row_bytes, lane);
  };
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the loaded rows, likewise
  __syncthreads();
  if (c == 0 && warp == 0) finish_reflector(0);
  __syncthreads();
  // in a step where this CTA generates the next reflector, warps 1..7 update (warp 4, which
  // shares a scheduler and its FP64 unit with warp 0, last); in the other steps all 8 warps do
  const int wslot = warp == 4 ? 6 : (warp < 4 ? warp - 1 : warp - 2);
  for (int j = 0; j < n; ++j) {
    if (j % C != c) mbar_wait(&bar[j], 0, status);             // row j from its owner
    const double* v = F + static_cast<size_t>(j) * ldF;
    const double tj = v[s];
    const bool chain_step = j + 1 < n && (j + 1) % C == c;
    if (warp == 0 && chain_step) {                              // row j+1, then reflector j+1
      double* ri = F + static_cast<size_t>(j + 1) * ldF;
      double part = 0;
      for (int k = j + lane; k < s; k += 32) part = fma(ri[k], v[k], part);
      const double w = warp_sum(part) * tj;
      for (int k = j + lane; k < s; k += 32) ri[k] = fma(-w, v[k], ri[k]);
      __syncwarp();
      finish_reflector(j + 1);
    } else {
      // items: this CTA's LQ rows i >= j + 2, then its sample rows
      const int slot = chain_step ? wslot : warp;
      const int ngroups = (chain_step ? THREADS - 32 : THREADS) / G;
      const int gid = slot * (32 / G) + lane / G;
      const int first = j + 2 + ((c - (j + 2)) % C + C) % C;
      const int nlq = first < n ? (n - 1 - first) / C + 1 : 0;
      const int items = nlq + nrows;
      for (int base = 0; base < items; base += ngroups) {
        if (base + slot * (32 / G) >= items) break;              // no item for this warp
        const int it = base + gid;
        const bool active = it < items;
        double* ri = !active    ? F + static_cast<size_t>(j) * ldF
                     : it < nlq ? F + static_cast<size_t>(first + it * C) * ldF
                                : Sr + static_cast<size_t>(it - nlq) * ldF;
        // LQ rows split their columns as lq_factor does (lane q: j + q, j + q + G, ...), sample
        // rows as stream_rows does (lane q: columns = q mod G from the slot holding j), so both
        // round exactly as the single-CTA kernel
        const int k0 = (active && it >= nlq) ? (j & ~(G - 1)) + q : j + q;
        double part = 0;
        for (int k = k0; k < s; k += G) part = fma(ri[k], k >= j ? v[k] : 0.0, part);
        const double w = group_sum(part) * tj;
        if (active)
          for (int k = k0; k < s; k += G)
            if (k >= j) ri[k] = fma(-w, v[k], ri[k]);
      }
    }
    // rows written here are sent by a bulk copy (the async proxy) in a later step
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
  // A wait above that gave up (its own timeout, or the run's abort flag) may have left a copy
  // into this CTA's shared memory in flight. Every owner sends every row it owns whatever its
  // waits returned, so each armed row still lands: account for all of them, under one shared
  // deadline, before the cluster may leave.
  if (aborted(status)) {
    const unsigned long long deadline = now_ns() + kWaitNs;
    for (int i = threadIdx.x; i < n; i += THREADS)
      if (i % C != c) mbar_wait_until(&bar[i], 0, status, deadline);
  }
  __syncthreads();
  // every CTA has received every row: no copy is in flight from or into any CTA of the cluster
  cl.sync();
  for (int j = threadIdx.x; j < n; j += THREADS) rdiag[j] = F[static_cast<size_t>(j) * ldF + s + 1];
  __syncthreads();
  double* X = tk.is_root ? nullptr : (side ? tk.XZ : tk.XY);
  double* W = tk.is_root ? tk.D : (side ? tk.WZ : tk.WY);
  const int gidr = threadIdx.x / G;
  for (int base = 0; base < nrows; base += NGROUPS) {
    if (base + warp * (32 / G) >= nrows) break;                // no row for this warp
    const int i = base + gidr;
    const bool active = i < nrows;
    double y[NS];
#pragma unroll
    for (int t = 0; t < NS; ++t) {
      const int k = q + G * t;
      y[t] = (active && k < s) ? Sr[static_cast<size_t>(i) * ldF + k] : 0.0;
    }
    store_row<NS>(y, row0 + i, active, n, s, tk.is_root ? 0 : r, F, ldF, rdiag, X, W);
  }
}

// ---- FP64 finish: bases, D_tau and the parent's blocks in three kernels --------------------
//
// With P = U^* WY, Q = U^* WZ^* (r x n) and R = Q V (r x r), Eq. (d_tau_formula) reads
//   D = (I - UU^*) WY + UU^* ((I - VV^*) WZ)^* = WY + U (Q - P - R V^*),
// so every column block of D needs only its own columns of P and Q plus the small R. The
// merges (Eq. omega_tau_and_y_tau) are U^* (Y - D Omega) and V^* (Z - D^* Psi) and need D only.
// node_bases (node, side) -> U, V; node_dblk_a (node, column block) -> P, Q; node_dblk_b
// (node, column block) -> R, D; node_merge (node, column chunk, pass) -> the parent's blocks.
// Upper levels, which have few nodes, thus spread each node over several SMs.

// U = col(Y P, r) (side 0) or V = col(Z Q, r) (side 1): unpivoted Householder QR, first r
// columns formed explicitly.
// Real = float in the mixed precisions (the sample block converted once on load; the basis is
// stored as FP64).
template <class Real>
__global__ void __launch_bounds__(THREADS, 4)   // four CTAs per SM: more warps for the FP64 chains
    node_bases(const NodeTask* __restrict__ tasks, int* status) {
  extern __shared__ __align__(16) unsigned char bsm_bytes[];
  Real* bsm = reinterpret_cast<Real*>(bsm_bytes);
  const NodeTask tk = tasks[blockIdx.x];
  if (tk.is_root) return;
  const int n = tk.n, r = tk.r;
  const int ldX = n + 1;
  Real* XT = bsm;                                      // r x ldX: (Y P)^* or (Z Q)^*
  Real* tau2 = XT + static_cast<size_t>(r) * ldX;      // r
  Real* W = tau2 + r;                                  // n x (r + 1): the basis being formed
  Real* scratch = W + static_cast<size_t>(n) * (r + 1);  // 9 r
  const double* X = blockIdx.y ? tk.XZ : tk.XY;
  for (int e = threadIdx.x; e < n * r; e += THREADS)
    XT[(e % r) * ldX + e / r] = static_cast<Real>(X[e]);
  __syncthreads();
  lq_factor<Real>(XT, ldX, r, n, tau2, nullptr, status);
  form_basis<Real>(XT, ldX, tau2, r, n, W, scratch, blockIdx.y ? tk.V : tk.U, r);
}

// Columns [j0, j0 + nb) of P = U^* WY and Q = U^* WZ^*, into the spent XZ and XY (r x n).
__global__ void __launch_bounds__(THREADS)
    node_dblk_a(const NodeTask* __restrict__ tasks, int nb) {
  const NodeTask tk = tasks[blockIdx.x];
  if (tk.is_root) return;
  const int n = tk.n, r = tk.r;
  const int j0 = blockIdx.y * nb;
  const int w = min(nb, n - j0);
  if (w <= 0) return;
  for (int e = threadIdx.x; e < r * w; e += THREADS) {
    const int c = e / w, j = j0 + e % w;
    double p = 0.0, q = 0.0;
    for (int i = 0; i < n; ++i) {
      const double u = tk.U[i * r + c];
      p = fma(u, tk.WY[static_cast<size_t>(i) * n + j], p);
      q = fma(u, tk.WZ[static_cast<size_t>(j) * n + i], q);
    }
    tk.XZ[c * n + j] = p;
    tk.XY[c * n + j] = q;
  }
}

// R = Q V (every column block forms it: r^2 n flops), then columns [j0, j0 + nb) of
// M = Q - P - R V^* and of D = WY + U M.
__global__ void __launch_bounds__(THREADS)
    node_dblk_b(const NodeTask* __restrict__ tasks, int nb) {
  extern __shared__ double dsm[];
  const NodeTask tk = tasks[blockIdx.x];
  if (tk.is_root) return;
  const int n = tk.n, r = tk.r;
  const int j0 = blockIdx.y * nb;
  const int w = min(nb, n - j0);
  if (w <= 0) return;
  const double* Q = tk.XY;                             // r x n
  const double* P = tk.XZ;                             // r x n
  double* R = dsm;                                     // r x r
  double* M = R + static_cast<size_t>(r) * r;          // r x w
  for (int e = threadIdx.x; e < r * r; e += THREADS) {
    const int c = e / r, f = e % r;
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc = fma(Q[c * n + j], tk.V[j * r + f], acc);
    R[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * w; e += THREADS) {
    const int c = e / w, j = j0 + e % w;
    double acc = Q[c * n + j] - P[c * n + j];
    for (int f = 0; f < r; ++f) acc = fma(-R[c * r + f], tk.V[j * r + f], acc);
    M[c * w + (j - j0)] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * w; e += THREADS) {
    const int i = e / w, jj = e % w;
    double acc = tk.WY[static_cast<size_t>(i) * n + j0 + jj];
    for (int c = 0; c < r; ++c) acc = fma(tk.U[i * r + c], M[c * w + jj], acc);
    tk.D[static_cast<size_t>(i) * n + j0 + jj] = acc;
  }
}

// ---- merge kernel: this node's rows of the parent's blocks (Eq. omega_tau_and_y_tau) ------------
// Grid (node, chunk of kw columns, pass). Pass 0: V^* Omega_tau and U^* (Y_tau - D Omega_tau);
// pass 1: U^* Psi_tau and V^* (Z_tau - D^* Psi_tau). The chunk of the test and sample blocks is
// staged in shared memory; D, U and V are read through L1 (each value is the same for the lanes
// of a warp). Levels with few nodes take narrow chunks, so that they still spread over the SMs.
constexpr int kMergeCols = 32;                          // widest chunk

__global__ void __launch_bounds__(THREADS)
    node_merge(const NodeTask* __restrict__ tasks, int chunk) {
  extern __shared__ double msm[];
  const NodeTask tk = tasks[blockIdx.x];
  if (tk.is_root) return;
  const int n = tk.n, r = tk.r, s = tk.s;
  const int k0 = blockIdx.y * chunk;
  if (k0 >= s) return;
  const int kw = min(chunk, s - k0);
  const int pass = blockIdx.z;
  const double* T = pass ? tk.Ps : tk.Om;
  const double* S = pass ? tk.Z : tk.Y;
  const double* Bt = pass ? tk.U : tk.V;               // reduces the test block
  const double* Bs = pass ? tk.V : tk.U;               // reduces the sample block
  double* outT = pass ? tk.Ps_p : tk.Om_p;
  double* outS = pass ? tk.Z_p : tk.Y_p;
  double* Ts = msm;                                    // n x kw
  double* Ss = Ts + static_cast<size_t>(n) * kw;       // n x kw
  for (int e = threadIdx.x; e < n * kw; e += THREADS) {
    const int i = e / kw, k = e % kw;
    Ts[e] = T[static_cast<size_t>(i) * s + k0 + k];
    Ss[e] = S[static_cast<size_t>(i) * s + k0 + k];
  }
  __syncthreads();
  // S <- S - op(D) T, each thread on its own entries (D for pass 0, D^* for pass 1)
  for (int e = threadIdx.x; e < n * kw; e += THREADS) {
    const int i = e / kw, k = e % kw;
    double acc = Ss[e];
    if (pass == 0)
      for (int j = 0; j < n; ++j) acc = fma(-tk.D[static_cast<size_t>(i) * n + j], Ts[j * kw + k], acc);
    else
      for (int j = 0; j < n; ++j) acc = fma(-tk.D[static_cast<size_t>(j) * n + i], Ts[j * kw + k], acc);
    Ss[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * kw; e += THREADS) {
    const int c = e / kw, k = e % kw;
    double t = 0.0, y = 0.0;
    for (int i = 0; i < n; ++i) {
      t = fma(Bt[i * r + c], Ts[i * kw + k], t);
      y = fma(Bs[i * r + c], Ss[i * kw + k], y);
    }
    outT[c * s + k0 + k] = t;
    outS[c * s + k0 + k] = y;
  }
}

// Arithmetic of the reduced-precision finish kernels: Real = float (plain FP32, the "mixed"
// finish) or dfloat (double-float, the compensated finish). Loads convert once from FP64, stores
// convert back.
__device__ __forceinline__ float nfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ dfloat nfma(dfloat a, dfloat b, dfloat c) { return df_fma_acc(a, b, c); }
__device__ __forceinline__ float nfinish(float a) { return a; }
__device__ __forceinline__ dfloat nfinish(dfloat a) { return df_norm(a); }
__device__ __forceinline__ float nneg(float a) { return -a; }
__device__ __forceinline__ dfloat nneg(dfloat a) { return df_neg(a); }
template <class Real> __device__ __forceinline__ Real from_f64(double x);
template <> __device__ __forceinline__ float from_f64<float>(double x) { return static_cast<float>(x); }
template <> __device__ __forceinline__ dfloat from_f64<dfloat>(double x) { return df_from(x); }
__device__ __forceinline__ double to_f64(float v) { return static_cast<double>(v); }
__device__ __forceinline__ double to_f64(dfloat v) { return df_to(v); }

// Small product in shared memory with a register tile per thread: for i < M, j < N,
// C(i, j) = init(i, j) + sum_k a(i, k) b(k, j), stored by out(i, j, value). A warp takes a tile
// of TM rows and 32 TN columns, lane l the columns l, l + 32, ...: a(i, k) is the same for the
// whole warp (one broadcast) and b(k, j) is read by consecutive lanes (no bank conflicts), so
// each k costs TM + TN shared loads per warp for 32 TM TN multiply-adds.
template <class Real, int TM, int TN, int NT = THREADS, class FA, class FB, class FI, class FO>
__device__ __forceinline__ void tile_gemm(int M, int N, int K, FA a, FB b, FI init, FO out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tn = (N + 32 * TN - 1) / (32 * TN), tm = (M + TM - 1) / TM;
  for (int t = warp; t < tm * tn; t += NT / 32) {
    const int i0 = (t / tn) * TM, j0 = (t % tn) * 32 * TN + lane;
    Real acc[TM][TN];
#pragma unroll
    for (int ii = 0; ii < TM; ++ii)
#pragma unroll
      for (int jj = 0; jj < TN; ++jj)
        acc[ii][jj] = (i0 + ii < M && j0 + 32 * jj < N) ? init(i0 + ii, j0 + 32 * jj) : Real{};
    for (int k = 0; k < K; ++k) {
      Real av[TM], bv[TN];
#pragma unroll
      for (int ii = 0; ii < TM; ++ii) av[ii] = a(min(i0 + ii, M - 1), k);
#pragma unroll
      for (int jj = 0; jj < TN; ++jj) bv[jj] = b(k, min(j0 + 32 * jj, N - 1));
#pragma unroll
      for (int ii = 0; ii < TM; ++ii)
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) acc[ii][jj] = nfma(av[ii], bv[jj], acc[ii][jj]);
    }
#pragma unroll
    for (int ii = 0; ii < TM; ++ii)
#pragma unroll
      for (int jj = 0; jj < TN; ++jj)
        if (i0 + ii < M && j0 + 32 * jj < N) out(i0 + ii, j0 + 32 * jj, nfinish(acc[ii][jj]));
  }
}

// D products with every operand staged in shared memory once. On GB300 a conversion from FP64
// runs at the FP64 rate, so converting each operand inside the product loops (one conversion
// per multiply-add) would make this kernel as slow as FP64 arithmetic; staged, a node converts
// each input entry once. One CTA per node, after node_bases has written U and V: D_tau (stored as
// FP64), then U^* D and (D V)^* (r x n) into the spent XY and XZ for node_merge_r. Real = float
// stores those as FP64; Real = dfloat stores them, and U and V, as double-float pairs (two
// floats in each 8-byte slot: U^* D and (D V)^* in XY, XZ; U, V in the spent WY, WZ), so that
// node_merge_r<dfloat> reads them without converting again.
constexpr int kDchainThreads = 512;   // 16 warps: one CTA per SM (its tile fills the shared memory)

template <class Real>
__global__ void __launch_bounds__(kDchainThreads, 1)
    node_dchain(const NodeTask* __restrict__ tasks) {
  extern __shared__ __align__(16) unsigned char dch_bytes[];
  Real* fsm = reinterpret_cast<Real*>(dch_bytes);
  const NodeTask tk = tasks[blockIdx.x];
  if (tk.is_root) return;
  const int n = tk.n, r = tk.r;
  const int ldX = n + 1, ldT = n + 1;
  Real* G1 = fsm;                                      // r x ldX: V^* WZ, later U^* D
  Real* Hs = G1 + static_cast<size_t>(r) * ldX;        // r x n: U^*(T2^* - WY), later (D V)^*
  Real* Us = Hs + static_cast<size_t>(r) * n;          // n x r
  Real* Vs = Us + static_cast<size_t>(n) * r;          // n x r
  Real* T2 = Vs + static_cast<size_t>(n) * r;          // n x ldT: WZ, then (I - VV^*) WZ, then D
  Real* WYs = T2 + static_cast<size_t>(n) * ldT;       // n x n
  for (int e = threadIdx.x; e < n * r; e += kDchainThreads) {
    Us[e] = from_f64<Real>(tk.U[e]);
    Vs[e] = from_f64<Real>(tk.V[e]);
  }
  for (int e = threadIdx.x; e < n * n; e += kDchainThreads) {
    WYs[e] = from_f64<Real>(tk.WY[e]);
    T2[(e / n) * ldT + e % n] = from_f64<Real>(tk.WZ[e]);
  }
  __syncthreads();
  // G1 = V^* WZ (r x n)
  tile_gemm<Real, 4, 1, kDchainThreads>(r, n, n, [&](int c, int i) { return Vs[i * r + c]; },
                        [&](int i, int j) { return T2[i * ldT + j]; }, [](int, int) { return Real{}; },
                        [&](int c, int j, Real v) { G1[c * ldX + j] = v; });
  __syncthreads();
  // T2 = WZ - V G1 (n x n), in place: each entry reads only its own WZ value
  tile_gemm<Real, 8, 1, kDchainThreads>(n, n, r, [&](int i, int c) { return nneg(Vs[i * r + c]); },
                        [&](int c, int j) { return G1[c * ldX + j]; },
                        [&](int i, int j) { return T2[i * ldT + j]; },
                        [&](int i, int j, Real v) { T2[i * ldT + j] = v; });
  __syncthreads();
  // G1 = U^* T2^* (= U^* D), then Hs = G1 - U^* WY
  tile_gemm<Real, 4, 1, kDchainThreads>(r, n, n, [&](int c, int i) { return Us[i * r + c]; },
                        [&](int i, int j) { return T2[j * ldT + i]; }, [](int, int) { return Real{}; },
                        [&](int c, int j, Real v) { G1[c * ldX + j] = v; });
  __syncthreads();
  tile_gemm<Real, 4, 1, kDchainThreads>(r, n, n, [&](int c, int i) { return nneg(Us[i * r + c]); },
                        [&](int i, int j) { return WYs[i * n + j]; },
                        [&](int c, int j) { return G1[c * ldX + j]; },
                        [&](int c, int j, Real v) { Hs[c * n + j] = v; });
  __syncthreads();
  // D = WY + U Hs (n x n), stored as FP64 and kept in T2
  tile_gemm<Real, 8, 1, kDchainThreads>(n, n, r, [&](int i, int c) { return Us[i * r + c]; },
                        [&](int c, int j) { return Hs[c * n + j]; },
                        [&](int i, int j) { return WYs[i * n + j]; },
                        [&](int i, int j, Real v) {
                          tk.D[static_cast<size_t>(i) * n + j] = to_f64(v);
                          T2[i * ldT + j] = v;
                        });
  __syncthreads();
  // Hs = (D V)^* (r x n)
  tile_gemm<Real, 4, 1, kDchainThreads>(r, n, n, [&](int c, int j) { return Vs[j * r + c]; },
                        [&](int j, int i) { return T2[i * ldT + j]; }, [](int, int) { return Real{}; },
                        [&](int c, int i, Real v) { Hs[c * n + i] = v; });
  __syncthreads();
  if constexpr (sizeof(Real) == sizeof(double)) {
    Real* XYd = reinterpret_cast<Real*>(tk.XY);
    Real* XZd = reinterpret_cast<Real*>(tk.XZ);
    Real* Ud = reinterpret_cast<Real*>(tk.WY);
    Real* Vd = reinterpret_cast<Real*>(tk.WZ);
    for (int e = threadIdx.x; e < r * n; e += kDchainThreads) {
      const int c = e / n, i = e % n;
      XYd[e] = G1[c * ldX + i];
      XZd[e] = Hs[e];
      Ud[e] = Us[e];
      Vd[e] = Vs[e];
    }
  } else {
    for (int e = threadIdx.x; e < r * n; e += kDchainThreads) {
      const int c = e / n, i = e % n;
      tk.XY[e] = to_f64(G1[c * ldX + i]);
      tk.XZ[e] = to_f64(Hs[e]);
    }
  }
}

// Merges (Eq. omega_tau_and_y_tau): grid (node, chunk of kw columns, pass) as node_merge, from U,
// V and the products U^* D, (D V)^* that node_dchain left behind; the chunk, the bases and the
// product are staged in shared memory.
// Threads of the merges: 256 in FP32 (three CTAs per SM fit), 512 in double-float, whose 8-byte
// tiles at n = 80 leave one CTA per SM.
template <class Real>
__host__ __device__ constexpr int merge_threads() { return sizeof(Real) == sizeof(double) ? 512 : THREADS; }

template <class Real>
__global__ void __launch_bounds__(merge_threads<Real>())
    node_merge_r(const NodeTask* __restrict__ tasks, int chunk) {
  extern __shared__ __align__(16) unsigned char mr_bytes[];
  Real* msf = reinterpret_cast<Real*>(mr_bytes);
  const NodeTask tk = tasks[blockIdx.x];
  if (tk.is_root) return;
  const int n = tk.n, r = tk.r, s = tk.s;
  const int k0 = blockIdx.y * chunk;
  if (k0 >= s) return;
  const int kw = min(chunk, s - k0);
  const int pass = blockIdx.z;
  const double* T = pass ? tk.Ps : tk.Om;
  const double* S = pass ? tk.Z : tk.Y;
  double* outT = pass ? tk.Ps_p : tk.Om_p;
  double* outS = pass ? tk.Z_p : tk.Y_p;
  Real* Ts = msf;                                      // n x kw
  Real* Ss = Ts + static_cast<size_t>(n) * kw;         // n x kw
  Real* Bts = Ss + static_cast<size_t>(n) * kw;        // n x r: reduces the test block
  Real* Bss = Bts + static_cast<size_t>(n) * r;        // n x r: reduces the sample block
  Real* Hsm = Bss + static_cast<size_t>(n) * r;        // r x n: (D V)^* or U^* D
  for (int e = threadIdx.x; e < n * kw; e += merge_threads<Real>()) {
    const int i = e / kw, k = e % kw;
    Ts[e] = from_f64<Real>(T[static_cast<size_t>(i) * s + k0 + k]);
    Ss[e] = from_f64<Real>(S[static_cast<size_t>(i) * s + k0 + k]);
  }
  if constexpr (sizeof(Real) == sizeof(double)) {      // left as pairs by node_dchain
    const Real* Ud = reinterpret_cast<const Real*>(tk.WY);
    const Real* Vd = reinterpret_cast<const Real*>(tk.WZ);
    const Real* H = reinterpret_cast<const Real*>(pass ? tk.XZ : tk.XY);
    const Real* Bt = pass ? Ud : Vd;
    const Real* Bs = pass ? Vd : Ud;
    for (int e = threadIdx.x; e < n * r; e += merge_threads<Real>()) {
      Bts[e] = Bt[e];
      Bss[e] = Bs[e];
      Hsm[e] = H[e];
    }
  } else {
    const double* Bt = pass ? tk.U : tk.V;
    const double* Bs = pass ? tk.V : tk.U;
    const double* H = pass ? tk.XZ : tk.XY;
    for (int e = threadIdx.x; e < n * r; e += merge_threads<Real>()) {
      Bts[e] = from_f64<Real>(Bt[e]);
      Bss[e] = from_f64<Real>(Bs[e]);
      Hsm[e] = from_f64<Real>(H[e]);
    }
  }
  __syncthreads();
  tile_gemm<Real, 2, 1, merge_threads<Real>()>(r, kw, n, [&](int c, int i) { return Bts[i * r + c]; },
                        [&](int i, int k) { return Ts[i * kw + k]; }, [](int, int) { return Real{}; },
                        [&](int c, int k, Real v) { outT[c * s + k0 + k] = to_f64(v); });
  // U^* S - H T as two products: Pm = U^* S, then Pm - H T
  Real* Pm = Hsm + static_cast<size_t>(r) * n;         // r x kw
  tile_gemm<Real, 2, 1, merge_threads<Real>()>(r, kw, n, [&](int c, int i) { return Bss[i * r + c]; },
                        [&](int i, int k) { return Ss[i * kw + k]; }, [](int, int) { return Real{}; },
                        [&](int c, int k, Real v) { Pm[c * kw + k] = v; });
  __syncthreads();
  tile_gemm<Real, 2, 1, merge_threads<Real>()>(r, kw, n, [&](int c, int i) { return nneg(Hsm[c * n + i]); },
                        [&](int i, int k) { return Ts[i * kw + k]; },
                        [&](int c, int k) { return Pm[c * kw + k]; },
                        [&](int c, int k, Real v) { outS[c * s + k0 + k] = to_f64(v); });
}

int merge_threads_of(int finish) {
  return finish == kFinishF32 ? merge_threads<float>() : merge_threads<dfloat>();
}

template <class Kernel>
cudaError_t allow_smem(Kernel kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(kMaxNodeSmemBytes));
}

}  // namespace

size_t side_smem_doubles(int n, int s) {
  return static_cast<size_t>(n) * (s + 1) + 2 * static_cast<size_t>(n);
}


size_t merge_smem_doubles(int n) { return 2 * static_cast<size_t>(n) * kMergeCols; }
size_t bases_smem_doubles(int n, int r) {   // in units of the kernel's Real
  return static_cast<size_t>(r) * (n + 1) + r + static_cast<size_t>(n) * (r + 1) + 9 * static_cast<size_t>(r);
}
size_t dblk_smem_doubles(int r, int nb) {
  return static_cast<size_t>(r) * r + static_cast<size_t>(r) * nb;
}

// Column blocks per node for the D kernels: several where a level has few nodes (each block
// re-forms the r x r product R, r^2 n flops, against ~4 r n^2 / blocks of its own work).
int dblk_blocks(int ntasks) { return std::max(1, std::min(8, (2 * 152) / std::max(1, ntasks))); }

// Reduced-precision D products (node_dchain): G1, Hs, the staged U, V, T2 (which holds WZ) and
// WY, in units of the kernel's Real.
size_t dchain_smem_reals(int n, int r) {
  return static_cast<size_t>(r) * (n + 1) + static_cast<size_t>(r) * n +
         2 * static_cast<size_t>(n) * r + static_cast<size_t>(n) * (n + 1) +
         static_cast<size_t>(n) * n;
}
size_t merge_r_smem_reals(int n, int r, int chunk) {
  return 2 * static_cast<size_t>(n) * chunk + 3 * static_cast<size_t>(n) * r +
         static_cast<size_t>(r) * chunk;
}

size_t finish_smem_bytes(int n, int r, int finish) {
  if (finish == kFinishF32 || finish == kFinishDF32) {
    const size_t w = finish == kFinishF32 ? sizeof(float) : sizeof(dfloat);
    return std::max(dchain_smem_reals(n, r) * w, merge_r_smem_reals(n, r, kMergeCols) * w);
  }
  return std::max(dblk_smem_doubles(r, n) * sizeof(double), merge_smem_doubles(n) * sizeof(double));
}

// The finish a height of nodes of up to n rows runs: the double-float tiles of the one-CTA-per-
// node D kernel grow as 8 (2 n^2 + 4 n r) bytes and pass 227 KB near n = 96; such heights run the
// FP64 finish (spread over several CTAs per node), which is at least as accurate.
int effective_finish(int n, int r, int finish) {
  if (finish == kFinishDF32 && finish_smem_bytes(n, r, finish) > kMaxNodeSmemBytes) return kFinishF64;
  return finish;
}

// The largest shared-memory tile the sweep kernels need for a node of n rows.
size_t node_smem_bytes(int n, int r, int s, int finish) {
  const size_t d = sizeof(double);
  const size_t common = std::max(side_smem_doubles(n, s) * d, bases_smem_doubles(n, r) * d);
  return std::max(common, finish_smem_bytes(n, r, effective_finish(n, r, finish)));
}

int side_row_splits(int ntasks, int n, int s) {
  // Where a height has fewer (node, side) pairs than SMs, give each a cluster of about
  // 152 / (2 ntasks) CTAs (at most 6, at least 8 rows each) sharing its factorization; otherwise
  // one CTA each. (Measured on the N = 32768, r = 40 log-kernel tree and the 256-tree batch, the
  // tuner picks these shapes or ones within a few percent of them.)
  const int want = (152 + ntasks) / (2 * ntasks);
  int C = std::max(1, std::min({want, 6, n / 8}));
  while (C >= 2 && !side_cluster_fits(n, s, C)) --C;
  return C >= 2 ? -C : 1;
}

int side_shape(int ntasks, int n, int s, int row_splits) {
  return row_splits != 0 ? row_splits : side_row_splits(ntasks, n, s);
}

size_t side_cluster_smem_doubles(int n, int s, int C) {
  const size_t chunk = (static_cast<size_t>(n) + C - 1) / C;
  const size_t ld = static_cast<size_t>(cluster_ld(s));
  // F, tau, 1/beta, the sample rows, one mbarrier per row
  return static_cast<size_t>(n) * ld + 2 * static_cast<size_t>(n) + (n & 1) + chunk * ld + n;
}

bool side_cluster_fits(int n, int s, int C) {
  return C >= 1 && C <= kMaxSideCluster && s <= kMaxS &&
         side_cluster_smem_doubles(n, s, C) * sizeof(double) <= kMaxNodeSmemBytes;
}

int64_t side_lq_stride(int max_n, int max_s) {
  return static_cast<int64_t>(side_smem_doubles(max_n, max_s));
}

cudaError_t launch_side_lq(const NodeTask* d_tasks, int ntasks, int max_n, int max_s, double* lq,
                           int* d_status, cudaStream_t st) {
  if (ntasks <= 0) return cudaSuccess;
  const size_t bytes = side_smem_doubles(max_n, max_s) * sizeof(double);
  if (max_s > kMaxS || bytes > kMaxNodeSmemBytes || lq == nullptr) return cudaErrorInvalidValue;
  const dim3 grid(static_cast<unsigned>(ntasks), 2u);
  cudaError_t e = allow_smem(node_lq);
  if (e != cudaSuccess) return e;
  node_lq<<<grid, THREADS, bytes, st>>>(d_tasks, d_status, lq, side_lq_stride(max_n, max_s));
  return cudaGetLastError();
}

// The side kernel of one height. R > 0: R row slices per (node, side), each CTA factoring the
// test block itself (or, with lq, copying the factorization node_lq left there); R < 0: a
// cluster of -R CTAs per (node, side) sharing one factorization (lq must be NULL).
cudaError_t launch_side_only(const NodeTask* d_tasks, int ntasks, int max_n, int max_s,
                             int R, int* d_status, cudaStream_t st, const double* lq, bool df) {
  if (ntasks <= 0) return cudaSuccess;
  if (max_s > kMaxS) return cudaErrorInvalidValue;
  if (lq != nullptr && R < 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  if (R < 0) {
    const int C = std::min(-R, kMaxSideCluster);
    const size_t bytes = side_cluster_smem_doubles(max_n, max_s, C) * sizeof(double);
    if (bytes > kMaxNodeSmemBytes) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(ntasks), 2u, static_cast<unsigned>(C));
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = static_cast<unsigned>(C);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    auto side = [&](auto kernel) {
      e = allow_smem(kernel);
      if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, kernel, d_tasks, d_status);
    };
    if (max_s <= 8 * G) side(node_side_cluster<8>);
    else if (max_s <= 16 * G) side(node_side_cluster<16>);
    else side(node_side_cluster<24>);
    return e;
  }
  const size_t side_bytes = side_smem_doubles(max_n, max_s) * sizeof(double);
  if (side_bytes > kMaxNodeSmemBytes) return cudaErrorInvalidValue;
  const int splits = std::max(1, std::min(R, std::max(1, max_n)));
  // four or three CTAs per SM where that many tiles (plus the 1 KB the runtime reserves per
  // CTA) fit; the register budget follows (64, 80 or 128 per thread, no spills)
  const int fit = static_cast<int>((228 * 1024) / (side_bytes + 1024));
  const dim3 grid(static_cast<unsigned>(ntasks), 2u, static_cast<unsigned>(splits));
  const int64_t stride = side_lq_stride(max_n, max_s);
  auto side = [&](auto kernel) {
    e = allow_smem(kernel);
    if (e == cudaSuccess) {
      kernel<<<grid, THREADS, side_bytes, st>>>(d_tasks, splits, d_status, lq, stride);
      e = cudaGetLastError();
    }
  };
  auto pick = [&](auto pre, auto dfl) {
    constexpr bool P = decltype(pre)::value, D = decltype(dfl)::value;
    if (max_s <= 8 * G) {
      if (fit >= 4) side(node_side<8, 4, P, D>);
      else if (fit == 3) side(node_side<8, 3, P, D>);
      else side(node_side<8, 2, P, D>);
    } else if (max_s <= 16 * G) {
      if (fit >= 4) side(node_side<16, 4, P, D>);
      else if (fit == 3) side(node_side<16, 3, P, D>);
      else side(node_side<16, 2, P, D>);
    } else {
      if (fit >= 3) side(node_side<24, 3, P, D>);
      else side(node_side<24, 2, P, D>);
    }
  };
  if (lq != nullptr) {
    if (df) pick(std::true_type{}, std::true_type{});
    else pick(std::true_type{}, std::false_type{});
  } else {
    if (df) pick(std::false_type{}, std::true_type{});
    else pick(std::false_type{}, std::false_type{});
  }
  return e;
}

cudaError_t launch_sweep_level(const NodeTask* d_tasks, int ntasks, int max_n, int max_r,
                               int max_s, int finish, int row_splits, int* d_status,
                               cudaStream_t st, cudaEvent_t* marks, FinishShape shape,
                               const double* lq) {
  if (ntasks <= 0) return cudaSuccess;
  auto mark = [&](int i) { return marks ? cudaEventRecord(marks[i], st) : cudaSuccess; };
  if (max_s > kMaxS) return cudaErrorInvalidValue;
  finish = effective_finish(max_n, max_r, finish);
  const bool reduced = finish == kFinishF32 || finish == kFinishDF32;
  const size_t rsize = finish == kFinishF32 ? sizeof(float) : sizeof(dfloat);
  // automatic: about four merge CTAs per SM in all; chunks of 8 .. 32 columns
  const int want = std::max(1, (4 * 152) / (2 * ntasks));
  const int chunk = shape.merge_chunk > 0 ? std::max(8, std::min(kMergeCols, shape.merge_chunk))
                                          : std::max(8, std::min(kMergeCols, (max_s + want - 1) / want));
  const size_t side_bytes = side_smem_doubles(max_n, max_s) * sizeof(double);
  const size_t bases_bytes = bases_smem_doubles(max_n, max_r) *
                             (finish == kFinishF32 ? sizeof(float) : sizeof(double));
  const int blocks = shape.d_blocks > 0 ? std::min(8, shape.d_blocks) : dblk_blocks(ntasks);
  const int nb = (max_n + blocks - 1) / blocks;
  const size_t dblk_bytes = reduced ? dchain_smem_reals(max_n, max_r) * rsize
                                    : dblk_smem_doubles(max_r, nb) * sizeof(double);
  const size_t merge_bytes = reduced ? merge_r_smem_reals(max_n, max_r, chunk) * rsize
                                     : merge_smem_doubles(max_n) * sizeof(double);
  if (side_bytes > kMaxNodeSmemBytes || bases_bytes > kMaxNodeSmemBytes ||
      dblk_bytes > kMaxNodeSmemBytes || merge_bytes > kMaxNodeSmemBytes)
    return cudaErrorInvalidValue;
  cudaError_t e = mark(0);
  if (e == cudaSuccess)
    e = launch_side_only(d_tasks, ntasks, max_n, max_s, side_shape(ntasks, max_n, max_s, row_splits),
                         d_status, st, lq, reduced);
  if (e == cudaSuccess) e = mark(1);
  if (e != cudaSuccess) return e;
  // bases: one CTA per (node, side); the register slots span the n <= s columns of a basis
  // (FP32 in the plain mixed finish; FP64 otherwise, the double-float finish included)
  const dim3 bgrid(static_cast<unsigned>(ntasks), 2u);
  auto bases = [&](auto kernel) {
    e = allow_smem(kernel);
    if (e == cudaSuccess) {
      kernel<<<bgrid, THREADS, bases_bytes, st>>>(d_tasks, d_status);
      e = cudaGetLastError();
    }
  };
  if (finish == kFinishF32) {
    bases(node_bases<float>);
  } else {
    bases(node_bases<double>);
  }
  if (e == cudaSuccess) e = mark(2);
  if (e != cudaSuccess) return e;
  const dim3 merge_grid(static_cast<unsigned>(ntasks),
                        static_cast<unsigned>((max_s + chunk - 1) / chunk), 2u);
  if (reduced) {
    auto finish_pair = [&](auto dchain, auto merge) {
      e = allow_smem(dchain);
      if (e != cudaSuccess) return;
      dchain<<<ntasks, kDchainThreads, dblk_bytes, st>>>(d_tasks);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = mark(3);
      if (e != cudaSuccess) return;
      e = allow_smem(merge);
      if (e != cudaSuccess) return;
      merge<<<merge_grid, merge_threads_of(finish), merge_bytes, st>>>(d_tasks, chunk);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = mark(4);
    };
    if (finish == kFinishF32) finish_pair(node_dchain<float>, node_merge_r<float>);
    else finish_pair(node_dchain<dfloat>, node_merge_r<dfloat>);
    return e;
  }
  const dim3 dgrid(static_cast<unsigned>(ntasks), static_cast<unsigned>(blocks));
  node_dblk_a<<<dgrid, THREADS, 0, st>>>(d_tasks, nb);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = allow_smem(node_dblk_b);
  if (e != cudaSuccess) return e;
  node_dblk_b<<<dgrid, THREADS, dblk_bytes, st>>>(d_tasks, nb);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = mark(3);
  if (e != cudaSuccess) return e;
  e = allow_smem(node_merge);
  if (e != cudaSuccess) return e;
  node_merge<<<merge_grid, THREADS, merge_bytes, st>>>(d_tasks, chunk);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = mark(4);
  return e;
}

}  // namespace hbs
