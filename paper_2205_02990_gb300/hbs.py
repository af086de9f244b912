"""Thin Python binding of include/hbs.h (ctypes; argument marshalling only).

Every computation runs in libhbs.so; this module only checks tensors, passes
``tensor.data_ptr()`` and the current torch CUDA stream, and turns status codes into
exceptions. Loading fails loudly when the library has not been built: there is no fallback.
Function names follow the C ABI (``hbs_sample``, ``hbs_compress``, ``hbs_apply``, ``hbs_free``
and the rest).
"""

import ctypes
import os
from dataclasses import dataclass

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libhbs.so")

HBS_OK = 0
HBS_ERR_ARG = -1
HBS_ERR_SHAPE = -2
HBS_ERR_NOMEM = -3
HBS_ERR_CUDA = -4
HBS_ERR_NUMERIC = -5
HBS_ERR_TIMEOUT = -6
HBS_ERR_CALLBACK = -7
HBS_ERR_UNSUPPORTED = -8
HBS_PREC_FP64 = 0
HBS_PREC_MIXED_BF16X3 = 1
HBS_PREC_MIXED_BF16X6 = 2
HBS_PREC_FP64_TC = 3
HBS_PREC_MIXED_COMPENSATED = 4
HBS_F64 = 0
HBS_F32 = 1

EXPORTED = ["hbs_draw_gaussian", "hbs_sample", "hbs_sample_products", "hbs_plan", "hbs_execute", "hbs_compress",
            "hbs_apply", "hbs_sync_status", "hbs_free", "hbs_last_error", "hbs_tree",
            "hbs_tree_build", "hbs_get_node", "hbs_factor_bytes", "hbs_copy_factors",
            "hbs_apply_static", "hbs_sample_sync", "hbs_apply_batch", "hbs_load_factors",
            "hbs_autotune", "hbs_get_tuning", "hbs_set_tuning", "hbs_set_graph",
            "hbs_test_inject_status", "hbs_probe_peaks", "hbs_profile_sweep", "hbs_probe_dmma",
            "hbs_sample_execute", "hbs_probe_mma_issue"]


class HBSError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"hbs status {code}: {message}")
        self.code = code


MATMAT_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64,
                             ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class _Operator(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("dtype", ctypes.c_int32), ("A", ctypes.c_void_p),
                ("lda", ctypes.c_int64), ("fn", MATMAT_FN), ("user", ctypes.c_void_p)]


class _Problem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("r", ctypes.c_int32), ("s", ctypes.c_int32),
                ("leaf_max", ctypes.c_int32), ("Omega", ctypes.c_void_p),
                ("Psi", ctypes.c_void_p), ("Y", ctypes.c_void_p), ("Z", ctypes.c_void_p)]


_lib = None


def load():
    """The loaded libhbs.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with "
                           "`python -m paper_2205_02990_gb300.build`")
    lib = ctypes.CDLL(_LIB_PATH)
    c = ctypes
    sig = {
        "hbs_draw_gaussian": (c.c_int, [c.c_int64, c.c_int32, c.c_uint32, c.c_uint64, c.c_void_p, c.c_void_p]),
        "hbs_sample": (c.c_int, [c.POINTER(_Operator), c.c_int32, c.c_uint64, c.c_int32, c.c_void_p,
                                 c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p]),
        "hbs_sample_products": (c.c_int, [c.POINTER(_Operator), c.c_int32, c.c_int32, c.c_void_p,
                                          c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p]),
        "hbs_sample_sync": (c.c_int, [c.c_void_p]),
        "hbs_apply_batch": (c.c_int, [c.c_void_p, c.c_int, c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p]),
        "hbs_load_factors": (c.c_int, [c.c_void_p, c.c_void_p, c.c_void_p]),
        "hbs_autotune": (c.c_int, [c.c_void_p, c.c_void_p]),
        "hbs_get_tuning": (c.c_int, [c.c_void_p, c.c_void_p, c.c_int32, c.POINTER(c.c_int32)]),
        "hbs_set_tuning": (c.c_int, [c.c_void_p, c.c_void_p, c.c_int32]),
        "hbs_set_graph": (c.c_int, [c.c_void_p, c.c_int]),
        "hbs_plan": (c.c_int, [c.c_int32, c.POINTER(_Problem), c.c_int32, c.POINTER(c.c_void_p)]),
        "hbs_execute": (c.c_int, [c.c_void_p, c.POINTER(_Problem), c.c_void_p]),
        "hbs_sample_execute": (c.c_int, [c.c_void_p, c.POINTER(_Operator), c.c_uint64, c.c_int32,
                                         c.POINTER(_Problem), c.c_void_p]),
        "hbs_compress": (c.c_int, [c.c_int32, c.POINTER(_Problem), c.c_int32, c.POINTER(c.c_void_p),
                                   c.c_void_p]),
        "hbs_apply": (c.c_int, [c.c_void_p, c.c_int32, c.c_int, c.c_int32, c.c_void_p, c.c_void_p,
                                c.c_void_p]),
        "hbs_sync_status": (c.c_int, [c.c_void_p, c.c_void_p]),
        "hbs_test_inject_status": (c.c_int, [c.c_void_p, c.c_int32]),
        "hbs_probe_peaks": (c.c_int, [c.POINTER(c.c_double), c.POINTER(c.c_double), c.c_void_p]),
        "hbs_probe_dmma": (c.c_int, [c.POINTER(c.c_double), c.c_void_p]),
        "hbs_probe_mma_issue": (c.c_int, [c.POINTER(c.c_double), c.c_void_p]),
        "hbs_profile_sweep": (c.c_int, [c.c_void_p, c.c_void_p, c.c_void_p, c.c_int32,
                                        c.POINTER(c.c_int32)]),
        "hbs_free": (None, [c.c_void_p]),
        "hbs_last_error": (c.c_char_p, []),
        "hbs_tree": (c.c_int, [c.c_void_p, c.c_int32, c.POINTER(c.c_int32), c.c_void_p, c.c_void_p]),
        "hbs_tree_build": (c.c_int, [c.c_int64, c.c_int32, c.POINTER(c.c_int32), c.c_void_p, c.c_void_p,
                                     c.c_int64]),
        "hbs_get_node": (c.c_int, [c.c_void_p, c.c_int32, c.c_int64, c.POINTER(c.c_int32), c.c_void_p,
                                   c.c_void_p, c.c_void_p]),
        "hbs_factor_bytes": (c.c_size_t, [c.c_void_p]),
        "hbs_copy_factors": (c.c_int, [c.c_void_p, c.c_void_p, c.c_void_p]),
        "hbs_apply_static": (c.c_int, [c.c_void_p, c.c_int32, c.c_int, c.c_int32, c.c_void_p,
                                       c.c_void_p, c.c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(code):
    if code != HBS_OK:
        raise HBSError(code, load().hbs_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, shape=None, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous (row-major)")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def hbs_draw_gaussian(N, s, stream_id, seed, out):
    """Fill ``out`` (N x s, float64, CUDA) from the counter-based generator."""
    _check(load().hbs_draw_gaussian(N, s, stream_id, seed, _dev(out, (N, s), "out"), _stream()))


def _operator(A, N):
    """(ctypes operator, keep-alive) for a dense matrix or a callable black box. A dense A is a
    CUDA tensor, or a page-locked (pinned) CPU float64 tensor, which the FP64 products stream
    through the device."""
    if isinstance(A, torch.Tensor):
        where_ok = A.is_cuda or (A.dtype == torch.float64 and A.is_pinned())
        if (not where_ok or A.dtype not in (torch.float64, torch.float32) or A.dim() != 2
                or A.shape[0] != A.shape[1] or A.stride(1) != 1 or A.stride(0) < A.shape[0]):
            raise TypeError("A must be a square row-major CUDA float64 or float32 matrix, "
                            "or a pinned CPU float64 matrix")
        N = A.shape[0]
        dt = HBS_F64 if A.dtype == torch.float64 else HBS_F32
        op = _Operator(N=N, dtype=dt, A=A.data_ptr(), lda=A.stride(0), fn=MATMAT_FN(), user=None)
        return op, None, N
    if N is None:
        raise ValueError("N is required with a callable operator")

    def trampoline(user, trans, n, ncols, X, Out, stream):
        try:
            A(int(trans), _wrap(X, n, ncols), _wrap(Out, n, ncols))
            return 0
        except Exception:            # reported to the caller as HBS_ERR_CALLBACK
            return 1

    keep = MATMAT_FN(trampoline)
    return _Operator(N=N, dtype=HBS_F64, A=None, lda=0, fn=keep, user=None), keep, N


def hbs_sample(A, s, seed, Omega, Psi, Y, Z, precision=HBS_PREC_FP64, N=None):
    """Draw Omega, Psi and form Y = A Omega, Z = A^* Psi.

    ``A`` is a dense CUDA float64 tensor (N x N, row-major; a pinned CPU float64 tensor is
    streamed through the device in row blocks) or a callable
    ``fn(trans, X, Out)`` that writes A X (trans = 0) or A^* X (trans = 1) into ``Out``
    (both N x s CUDA float64 tensors) on the current stream.
    """
    op, keep, N = _operator(A, N)
    ptrs = [_dev(x, (N, s), nm) for x, nm in ((Omega, "Omega"), (Psi, "Psi"), (Y, "Y"), (Z, "Z"))]
    _check(load().hbs_sample(ctypes.byref(op), s, seed, precision, *ptrs, _stream()))
    del keep


def hbs_sample_sync():
    """Wait for the current stream; raise if the tensor-core sampling reported a timeout."""
    _check(load().hbs_sample_sync(_stream()))


def hbs_sample_products(A, s, Omega, Psi, Y, Z, precision=HBS_PREC_FP64, N=None):
    """Y = A Omega, Z = A^* Psi for test matrices already drawn (same operator rules)."""
    op, keep, N = _operator(A, N)
    ptrs = [_dev(x, (N, s), nm) for x, nm in ((Omega, "Omega"), (Psi, "Psi"), (Y, "Y"), (Z, "Z"))]
    _check(load().hbs_sample_products(ctypes.byref(op), s, precision, *ptrs, _stream()))
    del keep


class _CudaView:
    """A device buffer described by __cuda_array_interface__ (viewed by torch without a copy)."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8",
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def _wrap(ptr, n, ncols):
    return torch.as_tensor(_CudaView(ptr, (n, ncols)), device="cuda")


@dataclass
class Problem:
    """One compression problem: test matrices and samples (N x s CUDA float64 tensors)."""
    N: int
    r: int
    s: int
    leaf_max: int
    Omega: torch.Tensor
    Psi: torch.Tensor
    Y: torch.Tensor
    Z: torch.Tensor

    def _c(self):
        sh = (self.N, self.s)
        return _Problem(N=self.N, r=self.r, s=self.s, leaf_max=self.leaf_max,
                        Omega=_dev(self.Omega, sh, "Omega").value, Psi=_dev(self.Psi, sh, "Psi").value,
                        Y=_dev(self.Y, sh, "Y").value, Z=_dev(self.Z, sh, "Z").value)


def _problems(problems):
    arr = (_Problem * len(problems))(*[p._c() for p in problems])
    return arr


class Handle:
    """Owns an hbs_handle (factors + workspace); freed by ``hbs_free`` or on deletion."""

    def __init__(self, ptr, problems):
        self._ptr = ptr
        self.problems = list(problems)

    @property
    def ptr(self):
        if not self._ptr:
            raise RuntimeError("handle already freed")
        return self._ptr

    def free(self):
        if self._ptr:
            load().hbs_free(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def hbs_plan(problems, precision=HBS_PREC_FP64):
    h = ctypes.c_void_p()
    arr = _problems(problems)
    _check(load().hbs_plan(len(problems), arr, precision, ctypes.byref(h)))
    return Handle(h, problems)


def hbs_execute(handle, problems=None):
    problems = handle.problems if problems is None else list(problems)
    _check(load().hbs_execute(handle.ptr, _problems(problems), _stream()))
    handle.problems = problems


def hbs_sample_execute(handle, A, seed, precision=HBS_PREC_FP64, problems=None, N=None):
    """hbs_sample into the problem's Omega, Psi, Y, Z, then hbs_execute (a one-problem
    handle); with an FP64 sweep the leaves' test-block LQ runs on a second stream while the
    products run."""
    problems = handle.problems if problems is None else list(problems)
    op, keep, _ = _operator(A, problems[0].N if N is None else N)
    _check(load().hbs_sample_execute(handle.ptr, ctypes.byref(op), seed, precision,
                                     _problems(problems), _stream()))
    handle.problems = problems
    del keep


def hbs_compress(problems, precision=HBS_PREC_FP64):
    """Plan and run Algorithm 2 for a batch of problems; returns a Handle."""
    h = ctypes.c_void_p()
    arr = _problems(problems)
    _check(load().hbs_compress(len(problems), arr, precision, ctypes.byref(h), _stream()))
    return Handle(h, problems)


def hbs_apply(handle, X, Out, item=0, trans=False):
    """Out = A~ X (or A~^* X) by Algorithm 1; X, Out N x c CUDA float64."""
    N = handle.problems[item].N
    if X.dim() != 2:
        raise ValueError("X must be 2-D (N x c)")
    c = X.shape[1]
    _check(load().hbs_apply(handle.ptr, item, int(bool(trans)), c, _dev(X, (N, c), "X"),
                            _dev(Out, (N, c), "Out"), _stream()))


def hbs_apply_static(handle, X, Out, item=0, trans=False):
    """As ``hbs_apply``, but allocating nothing: the workspace and work list live in fixed
    device arrays inside the library (see the limits and sharing rules in include/hbs.h)."""
    N = handle.problems[item].N
    if X.dim() != 2:
        raise ValueError("X must be 2-D (N x c)")
    c = X.shape[1]
    _check(load().hbs_apply_static(handle.ptr, item, int(bool(trans)), c, _dev(X, (N, c), "X"),
                                   _dev(Out, (N, c), "Out"), _stream()))


def hbs_apply_batch(handle, Xs, Outs, trans=False):
    """Algorithm 1 for every problem of the handle: Outs[i] = A~_i Xs[i] (or A~_i^* Xs[i])."""
    n = len(handle.problems)
    if len(Xs) != n or len(Outs) != n:
        raise ValueError("one X and one Out per problem")
    xp = (ctypes.c_void_p * n)(*[_dev(x, (p.N, x.shape[1]), "X").value for x, p in zip(Xs, handle.problems)])
    op = (ctypes.c_void_p * n)(*[_dev(o, (p.N, x.shape[1]), "Out").value
                                 for o, x, p in zip(Outs, Xs, handle.problems)])
    nc = (ctypes.c_int32 * n)(*[x.shape[1] for x in Xs])
    _check(load().hbs_apply_batch(handle.ptr, int(bool(trans)), xp, op, nc, _stream()))


def hbs_load_factors(handle, src):
    """Overwrite every factor of the handle from ``src`` (order of hbs_copy_factors)."""
    if src.numel() * src.element_size() < hbs_factor_bytes(handle):
        raise ValueError("source too small")
    _check(load().hbs_load_factors(handle.ptr, ctypes.c_void_p(src.data_ptr()), _stream()))


def hbs_autotune(handle):
    """Time the side kernel's shapes (row slices R > 0, clusters R = -C) per tree height on the
    current inputs; keep the best."""
    _check(load().hbs_autotune(handle.ptr, _stream()))


def hbs_profile_sweep(handle):
    """Per tree height (finest first): device ms of the side, bases, D and merge phases of one
    more sweep with plain launches."""
    lib = load()
    n = ctypes.c_int32()
    _check(lib.hbs_profile_sweep(handle.ptr, _stream(), None, 0, ctypes.byref(n)))
    ms = (ctypes.c_float * max(4 * n.value, 1))()
    _check(lib.hbs_profile_sweep(handle.ptr, _stream(), ms, 4 * n.value, ctypes.byref(n)))
    return [list(ms[4 * t:4 * t + 4]) for t in range(n.value)]


def hbs_get_tuning(handle):
    lib = load()
    n = ctypes.c_int32()
    _check(lib.hbs_get_tuning(handle.ptr, None, 0, ctypes.byref(n)))
    R = (ctypes.c_int32 * max(n.value, 1))()
    _check(lib.hbs_get_tuning(handle.ptr, R, n.value, ctypes.byref(n)))
    return list(R)[:n.value]


def hbs_set_tuning(handle, R):
    arr = (ctypes.c_int32 * max(len(R), 1))(*R)
    _check(load().hbs_set_tuning(handle.ptr, arr, len(R)))


def hbs_set_graph(handle, enable):
    _check(load().hbs_set_graph(handle.ptr, int(bool(enable))))


def factor_layout(N, r, leaf_max):
    """Offsets (in doubles) of U, V, D per node id in the packed factor order of one problem,
    and the total length: {node: (offU, offV, offD, n)}, total."""
    L, off, size = hbs_tree_build(N, leaf_max)
    out, cur = {}, 0
    for t in range(1, 2 ** (L + 1)):
        level = t.bit_length() - 1
        n = N if L == 0 else (size[t - 1] if level == L else 2 * r)
        oU = oV = None
        if t > 1:
            oU, oV = cur, cur + n * r
            cur += 2 * n * r
        out[t] = (oU, oV, cur, n)
        cur += n * n
    return out, cur


def hbs_sync_status(handle):
    _check(load().hbs_sync_status(handle.ptr, _stream()))


def hbs_test_inject_status(handle, bits):
    """Tests only: OR ``bits`` (1 numeric, 2 timeout) into the status word of ``handle`` (or,
    with ``handle=None``, of the current device's tensor-core sampling) as a device-side failure
    would, without running a kernel."""
    _check(load().hbs_test_inject_status(None if handle is None else handle.ptr, bits))


def hbs_probe_peaks():
    """(FP64, FP32) multiply-add throughput of the current GPU in TFLOP/s (measured now)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().hbs_probe_peaks(ctypes.byref(a), ctypes.byref(b), _stream()))
    return a.value, b.value


def hbs_probe_dmma():
    """FP64 tensor-instruction (DMMA) throughput of the current GPU in TFLOP/s (measured now)."""
    a = ctypes.c_double()
    _check(load().hbs_probe_dmma(ctypes.byref(a), _stream()))
    return a.value


def hbs_probe_mma_issue():
    """Cycles per tcgen05 MMA (M = N = 128, K = 16) issued by one thread: with the CTA's other
    warps idle, with FP32 work on every warp scheduler, and with FP32 work only on the schedulers
    the issuing warp does not use (measured now, one CTA per SM)."""
    a = (ctypes.c_double * 3)()
    _check(load().hbs_probe_mma_issue(a, _stream()))
    return {"alone": a[0], "fp32_all_schedulers": a[1], "fp32_other_schedulers": a[2]}


def hbs_free(handle):
    handle.free()


def hbs_tree_build(N, leaf_max):
    """(L, offsets, sizes) of the Section 3.1 tree, node ids 1.. at index 0.."""
    lib = load()
    L = ctypes.c_int32()
    _check(lib.hbs_tree_build(N, leaf_max, ctypes.byref(L), None, None, 0))
    count = (2 << L.value) - 1
    off = (ctypes.c_int64 * count)()
    size = (ctypes.c_int64 * count)()
    _check(lib.hbs_tree_build(N, leaf_max, ctypes.byref(L), off, size, count))
    return L.value, list(off), list(size)


def hbs_tree(handle, item=0):
    lib = load()
    L = ctypes.c_int32()
    _check(lib.hbs_tree(handle.ptr, item, ctypes.byref(L), None, None))
    count = (2 << L.value) - 1
    off = (ctypes.c_int64 * count)()
    size = (ctypes.c_int64 * count)()
    _check(lib.hbs_tree(handle.ptr, item, ctypes.byref(L), off, size))
    return L.value, list(off), list(size)


def hbs_get_node(handle, node, item=0):
    """(U, V, D) of a node as float64 CPU tensors (U, V are None for the root)."""
    lib = load()
    n = ctypes.c_int32()
    _check(lib.hbs_get_node(handle.ptr, item, node, ctypes.byref(n), None, None, None))
    r = handle.problems[item].r
    D = torch.empty((n.value, n.value), dtype=torch.float64)
    if node == 1:
        _check(lib.hbs_get_node(handle.ptr, item, node, ctypes.byref(n), None, None,
                                ctypes.c_void_p(D.data_ptr())))
        return None, None, D
    U = torch.empty((n.value, r), dtype=torch.float64)
    V = torch.empty((n.value, r), dtype=torch.float64)
    _check(lib.hbs_get_node(handle.ptr, item, node, ctypes.byref(n), ctypes.c_void_p(U.data_ptr()),
                            ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(D.data_ptr())))
    return U, V, D


def hbs_factor_bytes(handle):
    return int(load().hbs_factor_bytes(handle.ptr))


def hbs_copy_factors(handle, dst):
    """Asynchronous copy of every factor into ``dst`` (uint8/float64 tensor, host or device)."""
    if dst.numel() * dst.element_size() < hbs_factor_bytes(handle):
        raise ValueError("destination too small")
    _check(load().hbs_copy_factors(handle.ptr, ctypes.c_void_p(dst.data_ptr()), _stream()))
