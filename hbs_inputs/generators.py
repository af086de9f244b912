"""Input generators (see the package docstring). No compression arithmetic lives here."""

from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 220502990


def seed_for(workload, role):
    """Deterministic seed per (workload number, role): 0 Omega, 1 Psi, 2 generator, 3 probe."""
    return BASE_SEED + 100 * int(workload) + int(role)


def gaussian(shape, seed):
    """i.i.d. standard normal float64 array."""
    return np.random.default_rng(seed).standard_normal(shape)


@dataclass
class CurvePoints:
    x: np.ndarray
    y: np.ndarray


def curve_points(N):
    """N points at theta_i = 2 pi i / N on r(theta) = 1 + 0.3 cos(5 theta)."""
    theta = 2.0 * np.pi * np.arange(N, dtype=np.float64) / N
    rad = 1.0 + 0.3 * np.cos(5.0 * theta)
    return CurvePoints(rad * np.cos(theta), rad * np.sin(theta))


def log_kernel_rows(N, rows, cols=None):
    """Rows ``rows`` (and columns ``cols``, default all) of the dense log kernel, float64."""
    p = curve_points(N)
    rows = np.asarray(rows)
    cols = np.arange(N) if cols is None else np.asarray(cols)
    dx = p.x[rows][:, None] - p.x[cols][None, :]
    dy = p.y[rows][:, None] - p.y[cols][None, :]
    d = np.hypot(dx, dy)
    same = rows[:, None] == cols[None, :]
    with np.errstate(divide="ignore"):
        out = np.log(np.where(same, 1.0, d))
    out[same] = 0.0
    return out


def log_kernel(N):
    """Dense N x N log kernel, float64 (small N only: N^2 doubles on the host)."""
    return log_kernel_rows(N, np.arange(N))


def log_kernel_torch(N, device, dtype=None, row_block=4096):
    """Dense N x N log kernel built by torch on ``device`` (float64 arithmetic, then cast).

    Built in row blocks so that the float64 temporaries stay small next to the result.
    """
    import torch
    dtype = dtype or torch.float64
    p = curve_points(N)
    x = torch.as_tensor(p.x, device=device)
    y = torch.as_tensor(p.y, device=device)
    A = torch.empty((N, N), dtype=dtype, device=device)
    for r0 in range(0, N, row_block):
        r1 = min(N, r0 + row_block)
        d = torch.hypot(x[r0:r1, None] - x[None, :], y[r0:r1, None] - y[None, :])
        idx = torch.arange(r0, r1, device=device)
        d[idx - r0, idx] = 1.0
        blk = torch.log(d)
        blk[idx - r0, idx] = 0.0
        A[r0:r1] = blk.to(dtype)
        del d, blk
    return A


def _tree(N, leaf_max):
    """Section 3.1 tree: (L, offsets, sizes) by node id (1-based heap numbering)."""
    sizes = [N]
    L = 0
    while max(sizes) > leaf_max:
        sizes = [h for n in sizes for h in ((n + 1) // 2, n // 2)]
        L += 1
    offsets = [0] * 2 ** (L + 1)
    sz = [0] * 2 ** (L + 1)
    sz[1] = N
    for t in range(1, 2 ** L):
        left = (sz[t] + 1) // 2
        offsets[2 * t], sz[2 * t] = offsets[t], left
        offsets[2 * t + 1], sz[2 * t + 1] = offsets[t] + left, sz[t] - left
    return L, offsets, sz


def _orthonormal(rng, n, k):
    q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return q


@dataclass
class ExactHBS:
    """Exact-rank HBS matrix: classical generators plus telescoping factors (node ids 1-based)."""
    N: int
    k: int
    L: int
    offsets: list
    sizes: list
    U: dict = field(default_factory=dict)        # levels 1..L
    V: dict = field(default_factory=dict)
    D: dict = field(default_factory=dict)        # leaves: diagonal block; parents/root: [[0,B],[B',0]]
    B: dict = field(default_factory=dict)        # (alpha, beta) -> k x k coupling

    def dense(self):
        """Assemble A block by block: A(I_a, I_b) = Ubar_a B_ab Vbar_b^T for siblings a != b,
        leaf diagonal blocks D; Ubar is the expanded basis (leaf U, or blockdiag of the
        children's expanded bases times the node's U)."""
        N, L = self.N, self.L
        if L == 0:
            return self.D[1].copy()
        Ubar, Vbar = {}, {}
        for level in range(L, 0, -1):
            for t in range(2 ** level, 2 ** (level + 1)):
                if level == L:
                    Ubar[t], Vbar[t] = self.U[t], self.V[t]
                else:
                    a, b = 2 * t, 2 * t + 1
                    Ubar[t] = np.vstack([Ubar[a] @ self.U[t][:self.k], Ubar[b] @ self.U[t][self.k:]])
                    Vbar[t] = np.vstack([Vbar[a] @ self.V[t][:self.k], Vbar[b] @ self.V[t][self.k:]])
        A = np.zeros((N, N))
        for t in range(2 ** L, 2 ** (L + 1)):
            o, n = self.offsets[t], self.sizes[t]
            A[o:o + n, o:o + n] = self.D[t]
        for t in range(1, 2 ** L):
            a, b = 2 * t, 2 * t + 1
            ia = slice(self.offsets[a], self.offsets[a] + self.sizes[a])
            ib = slice(self.offsets[b], self.offsets[b] + self.sizes[b])
            A[ia, ib] = Ubar[a] @ self.B[(a, b)] @ Vbar[b].T
            A[ib, ia] = Ubar[b] @ self.B[(b, a)] @ Vbar[a].T
        return A


def exact_hbs(N, leaf_max, k, seed):
    """Random HBS matrix of exact block rank k on the Section 3.1 tree with threshold leaf_max."""
    rng = np.random.default_rng(seed)
    L, offsets, sizes = _tree(N, leaf_max)
    g = ExactHBS(N=N, k=k, L=L, offsets=offsets, sizes=sizes)
    if L == 0:
        g.D[1] = rng.standard_normal((N, N))
        return g
    for t in range(2 ** L, 2 ** (L + 1)):
        n = sizes[t]
        if n < k:
            raise ValueError("leaf smaller than k")
        g.U[t] = _orthonormal(rng, n, k)
        g.V[t] = _orthonormal(rng, n, k)
        g.D[t] = rng.standard_normal((n, n))
    for level in range(L - 1, 0, -1):
        for t in range(2 ** level, 2 ** (level + 1)):
            g.U[t] = _orthonormal(rng, 2 * k, k)
            g.V[t] = _orthonormal(rng, 2 * k, k)
    for t in range(1, 2 ** L):
        a, b = 2 * t, 2 * t + 1
        g.B[(a, b)] = rng.standard_normal((k, k))
        g.B[(b, a)] = rng.standard_normal((k, k))
        Dt = np.zeros((2 * k, 2 * k))
        Dt[:k, k:] = g.B[(a, b)]
        Dt[k:, :k] = g.B[(b, a)]
        g.D[t] = Dt
    return g


def packed_layout(N, leaf_max, r):
    """Node sizes and offsets (in doubles) of the packed telescoping-factor order used by the
    library's factor load/copy calls: per node id 1 .., U (n x r) and V (n x r) for nodes below the
    root, then D (n x n). Returns (L, {node: (offU, offV, offD, n)}, total)."""
    L, offsets, sizes = _tree(N, leaf_max)
    out, cur = {}, 0
    for t in range(1, 2 ** (L + 1)):
        level = t.bit_length() - 1
        n = N if L == 0 else (sizes[t] if level == L else 2 * r)
        oU = oV = None
        if t > 1:
            oU, oV = cur, cur + n * r
            cur += 2 * n * r
        out[t] = (oU, oV, cur, n)
        cur += n * n
    return L, out, cur


def pack_telescoping(g):
    """The generator's telescoping factors (U, V, D per node, Section 3.3) in the packed order."""
    L, lay, total = packed_layout(g.N, max(g.sizes[2 ** g.L: 2 ** (g.L + 1)]) if g.L else g.N, g.k)
    flat = np.zeros(total)
    for t, (oU, oV, oD, n) in lay.items():
        if oU is not None:
            flat[oU:oU + n * g.k] = g.U[t].ravel()
            flat[oV:oV + n * g.k] = g.V[t].ravel()
        flat[oD:oD + n * n] = g.D[t].ravel()
    return flat


def exact_hbs_packed_torch(N, leaf_max, k, seed, device):
    """Packed telescoping factors of a random exact-rank HBS matrix (same construction as
    ``exact_hbs``: orthonormal leaf and parent bases, Gaussian couplings and leaf blocks), drawn
    with torch on ``device`` for sizes where the dense matrix cannot be formed. Needs equal leaf
    sizes (N a multiple of 2^L)."""
    import torch
    L, lay, total = packed_layout(N, leaf_max, k)
    out = torch.zeros(total, dtype=torch.float64, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))

    def gauss(*shape):
        return torch.randn(*shape, dtype=torch.float64, device=device, generator=gen)

    def orth(cnt, n):
        q, _ = torch.linalg.qr(gauss(cnt, n, k))
        return q

    if L == 0:
        out[:] = gauss(N * N)
        return out
    m = N >> L
    if m << L != N:
        raise ValueError("exact_hbs_packed_torch needs N divisible by 2^L")
    for level in range(0, L + 1):
        cnt = 1 << level
        first = lay[cnt]
        start = first[0] if first[0] is not None else first[2]
        n = first[3]
        blk = (2 * n * k if level > 0 else 0) + n * n
        view = out[start:start + cnt * blk].view(cnt, blk)
        if level > 0:
            view[:, :n * k] = orth(cnt, n).reshape(cnt, n * k)
            view[:, n * k:2 * n * k] = orth(cnt, n).reshape(cnt, n * k)
        if level == L:
            view[:, blk - n * n:] = gauss(cnt, n * n)
        else:
            D = torch.zeros(cnt, 2 * k, 2 * k, dtype=torch.float64, device=device)
            D[:, :k, k:] = gauss(cnt, k, k)
            D[:, k:, :k] = gauss(cnt, k, k)
            view[:, blk - n * n:] = D.reshape(cnt, n * n)
    return out


def _curve_geometry(N):
    """Points, outward unit normals, arc-length weights (trapezoid rule) and curvature of
    r(theta) = 1 + 0.3 cos 5 theta at theta_i = 2 pi i / N (counter-clockwise)."""
    th = 2.0 * np.pi * np.arange(N) / N
    r = 1.0 + 0.3 * np.cos(5 * th)
    dr = -1.5 * np.sin(5 * th)
    d2r = -7.5 * np.cos(5 * th)
    x, y = r * np.cos(th), r * np.sin(th)
    dx, dy = dr * np.cos(th) - r * np.sin(th), dr * np.sin(th) + r * np.cos(th)
    d2x = d2r * np.cos(th) - 2 * dr * np.sin(th) - r * np.cos(th)
    d2y = d2r * np.sin(th) + 2 * dr * np.cos(th) - r * np.sin(th)
    speed = np.hypot(dx, dy)
    nx, ny = dy / speed, -dx / speed
    kappa = (dx * d2y - dy * d2x) / speed ** 3
    w = speed * 2.0 * np.pi / N
    return x, y, nx, ny, w, kappa


def double_layer_rows(N, rows, cols=None):
    """Rows of the Nystrom matrix of the boundary integral equation of Section 5.1 on the same
    curve: (1/2) delta_ij + w_j (x_i - y_j) . n(y_j) / (4 pi |x_i - y_j|^2) (constant as printed
    in the paper), with the kernel's smooth diagonal limit -kappa_i / (8 pi) times w_i."""
    x, y, nx, ny, w, kappa = _curve_geometry(N)
    rows = np.asarray(rows)
    cols = np.arange(N) if cols is None else np.asarray(cols)
    ddx = x[rows][:, None] - x[cols][None, :]
    ddy = y[rows][:, None] - y[cols][None, :]
    num = ddx * nx[cols][None, :] + ddy * ny[cols][None, :]
    den = ddx ** 2 + ddy ** 2
    same = rows[:, None] == cols[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        K = num / (4.0 * np.pi * np.where(same, 1.0, den))
    diag = -kappa / (8.0 * np.pi)
    K = np.where(same, diag[rows][:, None], K) * w[cols][None, :]
    return K + 0.5 * same


def double_layer(N):
    return double_layer_rows(N, np.arange(N))


def double_layer_torch(N, device, dtype=None, row_block=4096):
    """Dense double-layer Nystrom matrix built by torch on ``device`` in row blocks."""
    import torch
    dtype = dtype or torch.float64
    x, y, nx, ny, w, kappa = (torch.as_tensor(v, device=device) for v in _curve_geometry(N))
    A = torch.empty((N, N), dtype=dtype, device=device)
    for r0 in range(0, N, row_block):
        r1 = min(N, r0 + row_block)
        ddx = x[r0:r1, None] - x[None, :]
        ddy = y[r0:r1, None] - y[None, :]
        den = ddx * ddx + ddy * ddy
        idx = torch.arange(r0, r1, device=device)
        den[idx - r0, idx] = 1.0
        K = (ddx * nx[None, :] + ddy * ny[None, :]) / (4.0 * np.pi * den)
        K[idx - r0, idx] = -kappa[idx] / (8.0 * np.pi)
        K = K * w[None, :]
        K[idx - r0, idx] += 0.5
        A[r0:r1] = K.to(dtype)
        del ddx, ddy, den, K
    return A
