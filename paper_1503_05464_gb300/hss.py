"""Thin ctypes binding of libhss.so (include/hss.h).

Argument marshalling only: every step of the compression, product,
factorization and solve runs in the library's CUDA kernels.  Tensors are
PyTorch CUDA tensors (device memory and streams come from PyTorch); the
functions keep the C names.  If the library has not been built, or no CUDA
device is present, the calls raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhss.so")

HSS_OK, HSS_ERR_INVALID, HSS_ERR_OOM, HSS_ERR_CUDA, HSS_ERR_RANK_CAP, HSS_ERR_SINGULAR, \
    HSS_ERR_TIMEOUT, HSS_ERR_STATE = range(8)
HSS_F32, HSS_F64 = 0, 1
HSS_FAULT_NONE, HSS_FAULT_OOM, HSS_FAULT_WAIT_LIMIT = 0, 1, 2
SAMPLE_MODES = {"native": 0, "tf32": 1, "bf16x2": 2, "bf16x3": 3}

STATUS_NAMES = {0: "HSS_OK", 1: "HSS_ERR_INVALID", 2: "HSS_ERR_OOM", 3: "HSS_ERR_CUDA",
                4: "HSS_ERR_RANK_CAP", 5: "HSS_ERR_SINGULAR", 6: "HSS_ERR_TIMEOUT",
                7: "HSS_ERR_STATE"}


class HssError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class HssOpts(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int32), ("rtol", ctypes.c_double),
                ("atol", ctypes.c_double), ("d0", ctypes.c_int32), ("d_step", ctypes.c_int32),
                ("d_max", ctypes.c_int32), ("oversample_p", ctypes.c_int32),
                ("sample_mode", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("tree", ctypes.POINTER(ctypes.c_int64)), ("tree_nodes", ctypes.c_int32),
                ("symmetric", ctypes.c_int32)]


class HssInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nodes", ctypes.c_int32), ("leaves", ctypes.c_int32),
                ("levels", ctypes.c_int32), ("max_rank_r", ctypes.c_int32),
                ("max_rank_c", ctypes.c_int32), ("d_final", ctypes.c_int32),
                ("passes", ctypes.c_int32), ("bytes_hss", ctypes.c_int64),
                ("bytes_ulv", ctypes.c_int64), ("ms_compress", ctypes.c_double),
                ("ms_sample", ctypes.c_double), ("ms_id", ctypes.c_double),
                ("ms_levels", ctypes.c_double), ("flops_sample", ctypes.c_double),
                ("flops_id", ctypes.c_double), ("factored", ctypes.c_int32),
                ("launches", ctypes.c_int64), ("bytes_d2h", ctypes.c_int64),
                ("ms_host_id_launch", ctypes.c_double), ("ms_host_wait", ctypes.c_double),
                ("ms_host_sample", ctypes.c_double), ("id_launches", ctypes.c_int64),
                ("flops_id_solve", ctypes.c_double)]


# hss_matfree (include/hss.h): the caller's products and entries of A
SAMPLE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                             ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                             ctypes.c_void_p)
EXTRACT_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                              ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                              ctypes.c_void_p)


class HssMatfree(ctypes.Structure):
    _fields_ = [("sample", SAMPLE_FN), ("extract", EXTRACT_FN), ("ctx", ctypes.c_void_p)]


_lib = None
EXPORTS = ["hss_default_opts", "hss_compress", "hss_matvec", "hss_factor", "hss_solve",
           "hss_info", "hss_node_ranks", "hss_destroy", "hss_last_error",
           "hss_random_gaussian", "hss_sample", "hss_id_batched", "hss_kernel_launches", "hss_sample_noalloc",
           "hss_pool_bytes", "hss_set_fault", "hss_tuner_stats",
           "hss_batch_create", "hss_batch_submit", "hss_batch_step", "hss_batch_take",
           "hss_batch_last_error", "hss_batch_destroy", "hss_compress_batched",
           "hss_factor_batched", "hss_solve_batched", "hss_compress_matfree"]


def load(path: str = LIB_PATH):
    """Load libhss.so and declare the C signatures (no CUDA call is made)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1503_05464_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64, f64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
    L.hss_default_opts.argtypes = [ctypes.POINTER(HssOpts)]
    L.hss_compress.argtypes = [vp, i64, i64, i32, ctypes.POINTER(HssOpts), vp, ctypes.POINTER(vp)]
    L.hss_matvec.argtypes = [vp, vp, i64, i64, vp, i64, vp]
    L.hss_factor.argtypes = [vp, vp]
    L.hss_solve.argtypes = [vp, vp, i64, i64, vp, i64, vp]
    L.hss_info.argtypes = [vp, ctypes.POINTER(HssInfo)]
    L.hss_node_ranks.argtypes = [vp, vp, vp, vp, vp, i32, ctypes.POINTER(i32)]
    L.hss_destroy.argtypes = [vp]
    L.hss_destroy.restype = None
    L.hss_last_error.argtypes = [vp]
    L.hss_last_error.restype = ctypes.c_char_p
    L.hss_random_gaussian.argtypes = [u64, i64, i64, i64, vp, i64, i32, vp]
    L.hss_sample.argtypes = [vp, i64, i64, i32, vp, i64, i64, i64, vp, vp, i64, vp, i32, i32, vp]
    L.hss_id_batched.argtypes = [i32, vp, vp, vp, vp, i32, f64, f64, vp, vp, vp, vp]
    L.hss_sample_noalloc.argtypes = L.hss_sample.argtypes
    L.hss_pool_bytes.argtypes = [ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.hss_set_fault.argtypes = [i32, i64]
    L.hss_tuner_stats.argtypes = [ctypes.POINTER(i32)] * 3
    L.hss_kernel_launches.argtypes = []
    L.hss_kernel_launches.restype = ctypes.c_int64
    L.hss_batch_create.argtypes = [i32, vp, ctypes.POINTER(vp)]
    L.hss_batch_submit.argtypes = [vp, vp, i64, i64, ctypes.POINTER(HssOpts), ctypes.POINTER(i64)]
    L.hss_batch_step.argtypes = [vp, ctypes.POINTER(i32)]
    L.hss_batch_take.argtypes = [vp, i64, ctypes.POINTER(vp)]
    L.hss_batch_last_error.argtypes = [vp]
    L.hss_batch_last_error.restype = ctypes.c_char_p
    L.hss_batch_destroy.argtypes = [vp]
    L.hss_batch_destroy.restype = None
    L.hss_compress_batched.argtypes = [i32, vp, vp, vp, i32, ctypes.POINTER(HssOpts), i32, vp,
                                       vp, vp]
    L.hss_factor_batched.argtypes = [i32, vp, vp, vp]
    L.hss_compress_matfree.argtypes = [i64, i32, ctypes.POINTER(HssMatfree),
                                       ctypes.POINTER(HssOpts), vp, ctypes.POINTER(vp)]
    L.hss_solve_batched.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp]
    for name in EXPORTS:
        if name not in ("hss_destroy", "hss_last_error", "hss_kernel_launches",
                        "hss_batch_last_error", "hss_batch_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(st, handle=None):
    if st != HSS_OK:
        msg = load().hss_last_error(handle).decode(errors="replace")
        raise HssError(st, msg)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return HSS_F32
    if t.dtype == torch.float64:
        return HSS_F64
    raise TypeError(f"unsupported dtype {t.dtype} (float32 or float64)")


def _require_cuda(*ts):
    for t in ts:
        if not t.is_cuda:
            raise ValueError("tensors must live on a CUDA device")
        if t.dim() == 2 and t.stride(1) != 1:
            raise ValueError("matrices must be row-major with unit column stride")


def hss_default_opts(**kw) -> HssOpts:
    """hss_opts with the library defaults, then the keyword fields.  tree: a
    list of split points, one per node in breadth-first order (-1 = leaf),
    the format of hss_opts.tree.  symmetric: True when A = A^T."""
    o = HssOpts()
    _check(load().hss_default_opts(ctypes.byref(o)))
    for k, v in kw.items():
        if k == "sample_mode" and isinstance(v, str):
            v = SAMPLE_MODES[v]
        if k == "tree":
            if v is None:
                o.tree, o.tree_nodes = None, 0
                continue
            arr = (ctypes.c_int64 * len(v))(*[int(x) for x in v])
            o._tree_keep = arr          # the array must outlive the options
            o.tree = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int64))
            o.tree_nodes = len(v)
            continue
        if k == "symmetric":
            v = int(bool(v))
        setattr(o, k, v)
    return o


class HSS:
    """Owner of an hss_t handle (hss_destroy on deletion)."""

    def __init__(self, handle: int, n: int, dtype: torch.dtype):
        self.handle = ctypes.c_void_p(handle)
        self.n = n
        self.dtype = dtype

    def __del__(self):
        if getattr(self, "handle", None) and self.handle.value and _lib is not None:
            _lib.hss_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def close(self):
        self.__del__()


def hss_compress(A: torch.Tensor, opts: HssOpts | None = None, stream=None, **kw) -> HSS:
    """Randomized HSS compression of the square row-major CUDA matrix A."""
    _require_cuda(A)
    n = A.shape[0]
    if A.dim() != 2 or A.shape[1] != n:
        raise ValueError("A must be square")
    if opts is None:
        opts = hss_default_opts(**kw)
    out = ctypes.c_void_p()
    st = load().hss_compress(ctypes.c_void_p(A.data_ptr()), n, A.stride(0), _dtype(A),
                             ctypes.byref(opts), _stream(stream), ctypes.byref(out))
    if st == HSS_ERR_RANK_CAP and out.value:
        msg = load().hss_last_error(out).decode()
        load().hss_destroy(out)
        raise HssError(st, msg)
    _check(st)
    return HSS(out.value, n, A.dtype)


def hss_compress_batched(As, opts=None, stream=None, **kw):
    """Compresses a list of square CUDA matrices together (one dtype); the
    level work of all of them shares launches.  Returns a list of HSS
    handles (None for a matrix that failed) and the per-matrix statuses."""
    if not As:
        return [], []
    _require_cuda(*As)
    cnt = len(As)
    dt = _dtype(As[0])
    if opts is None:
        opts = hss_default_opts(**kw)
    ptrs = (ctypes.c_void_p * cnt)(*[a.data_ptr() for a in As])
    ns = (ctypes.c_int64 * cnt)(*[a.shape[0] for a in As])
    lds = (ctypes.c_int64 * cnt)(*[a.stride(0) for a in As])
    outs = (ctypes.c_void_p * cnt)()
    sts = (ctypes.c_int * cnt)()
    if isinstance(opts, (list, tuple)):
        arr = (HssOpts * cnt)(*opts)
        optp, stride = ctypes.cast(arr, ctypes.POINTER(HssOpts)), 1
    else:
        optp, stride = ctypes.pointer(opts), 0
    load().hss_compress_batched(cnt, ptrs, ns, lds, dt, optp, stride, _stream(stream), outs, sts)
    handles = [HSS(outs[i], As[i].shape[0], As[i].dtype) if outs[i] else None for i in range(cnt)]
    return handles, [sts[i] for i in range(cnt)]


class HssBatch:
    """Incremental batch (continuous batching): submit matrices at any time,
    step() runs one round for every job, take() hands over finished ones."""

    def __init__(self, dtype=torch.float32, stream=None):
        self.b = ctypes.c_void_p()
        dt = HSS_F32 if dtype == torch.float32 else HSS_F64
        self.dtype = dtype
        self.stream = stream
        _check(load().hss_batch_create(dt, _stream(stream), ctypes.byref(self.b)))
        self.keep = {}

    def submit(self, A: torch.Tensor, opts: HssOpts | None = None, **kw) -> int:
        _require_cuda(A)
        if opts is None:
            opts = hss_default_opts(**kw)
        t = ctypes.c_int64()
        st = load().hss_batch_submit(self.b, ctypes.c_void_p(A.data_ptr()), A.shape[0],
                                     A.stride(0), ctypes.byref(opts), ctypes.byref(t))
        if st != HSS_OK:
            raise HssError(st, load().hss_batch_last_error(self.b).decode())
        self.keep[t.value] = A          # A must outlive its job
        return t.value

    def step(self) -> int:
        act = ctypes.c_int32()
        st = load().hss_batch_step(self.b, ctypes.byref(act))
        if st != HSS_OK:
            raise HssError(st, load().hss_batch_last_error(self.b).decode())
        return act.value

    def take(self, ticket: int):
        """(HSS or None, status); status HSS_ERR_STATE while still running."""
        out = ctypes.c_void_p()
        st = load().hss_batch_take(self.b, ticket, ctypes.byref(out))
        if st == HSS_ERR_STATE:
            return None, st
        A = self.keep.pop(ticket, None)
        h = HSS(out.value, A.shape[0], A.dtype) if out.value else None
        return h, st

    def close(self):
        if self.b and self.b.value and _lib is not None:
            _lib.hss_batch_destroy(self.b)
            self.b = ctypes.c_void_p(0)

    def __del__(self):
        self.close()


def hss_matvec(h: HSS, X: torch.Tensor, B: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """B = H X (Algorithm 2); X is n x nrhs (or length n)."""
    vec = X.dim() == 1
    X2 = X.view(-1, 1) if vec else X
    _require_cuda(X2)
    if B is None:
        B = torch.empty((h.n, X2.shape[1]), dtype=X2.dtype, device=X2.device)
    B2 = B.view(-1, 1) if B.dim() == 1 else B
    _check(load().hss_matvec(h.handle, ctypes.c_void_p(X2.data_ptr()), X2.stride(0), X2.shape[1],
                             ctypes.c_void_p(B2.data_ptr()), B2.stride(0), _stream(stream)),
           h.handle)
    return B2.view(-1) if vec else B2


def hss_factor(h: HSS, stream=None) -> None:
    """ULV-like factorization (Algorithm 3)."""
    _check(load().hss_factor(h.handle, _stream(stream)), h.handle)


def hss_factor_batched(hs, stream=None):
    """ULV factorization of several handles together (one launch per level
    round across all of them).  Returns the per-handle statuses."""
    cnt = len(hs)
    if cnt == 0:
        return []
    arr = (ctypes.c_void_p * cnt)(*[h.handle.value for h in hs])
    sts = (ctypes.c_int * cnt)()
    load().hss_factor_batched(cnt, arr, _stream(stream), sts)
    return [sts[i] for i in range(cnt)]


def hss_solve_batched(hs, Bs, stream=None):
    """X_q = H_q^{-1} B_q for every pair (one launch per sweep round across
    all of them).  Returns (list of X, list of statuses)."""
    cnt = len(hs)
    if cnt == 0:
        return [], []
    B2 = [b.view(-1, 1) if b.dim() == 1 else b for b in Bs]
    _require_cuda(*B2)
    Xs = [torch.empty((h.n, b.shape[1]), dtype=b.dtype, device=b.device) for h, b in zip(hs, B2)]
    vp = ctypes.c_void_p
    harr = (vp * cnt)(*[h.handle.value for h in hs])
    barr = (vp * cnt)(*[b.data_ptr() for b in B2])
    xarr = (vp * cnt)(*[x.data_ptr() for x in Xs])
    ldb = (ctypes.c_int64 * cnt)(*[b.stride(0) for b in B2])
    nr = (ctypes.c_int64 * cnt)(*[b.shape[1] for b in B2])
    ldx = (ctypes.c_int64 * cnt)(*[x.stride(0) for x in Xs])
    sts = (ctypes.c_int * cnt)()
    load().hss_solve_batched(cnt, harr, barr, ldb, nr, xarr, ldx, _stream(stream), sts)
    Xs = [x.view(-1) if b.dim() == 1 else x for x, b in zip(Xs, Bs)]
    return Xs, [sts[i] for i in range(cnt)]


def hss_solve(h: HSS, B: torch.Tensor, X: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """X = H^{-1} B with the ULV factors (Algorithm 4)."""
    vec = B.dim() == 1
    B2 = B.view(-1, 1) if vec else B
    _require_cuda(B2)
    if X is None:
        X = torch.empty((h.n, B2.shape[1]), dtype=B2.dtype, device=B2.device)
    X2 = X.view(-1, 1) if X.dim() == 1 else X
    _check(load().hss_solve(h.handle, ctypes.c_void_p(B2.data_ptr()), B2.stride(0), B2.shape[1],
                            ctypes.c_void_p(X2.data_ptr()), X2.stride(0), _stream(stream)),
           h.handle)
    return X2.view(-1) if vec else X2


def hss_kernel_launches() -> int:
    """Kernels libhss has launched in this process so far."""
    return int(load().hss_kernel_launches())


def hss_set_fault(kind: int, value: int = 0) -> None:
    """Arm an injected fault (HSS_FAULT_OOM: the value-th allocation from now
    fails; HSS_FAULT_WAIT_LIMIT: the ID's group barrier gives up after value
    cycles) or clear them (HSS_FAULT_NONE)."""
    _check(load().hss_set_fault(kind, value))


def hss_tuner_stats() -> dict:
    """Shape classes seen / settled and timed trials of the ID launch tuner."""
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().hss_tuner_stats(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"classes": a.value, "settled": b.value, "trials": c.value}


def hss_pool_bytes() -> tuple[int, int]:
    """(used, reserved) bytes of the library's device memory pool on the
    current device."""
    u, r = ctypes.c_int64(), ctypes.c_int64()
    _check(load().hss_pool_bytes(ctypes.byref(u), ctypes.byref(r)))
    return u.value, r.value


def hss_info(h: HSS) -> dict:
    info = HssInfo()
    _check(load().hss_info(h.handle, ctypes.byref(info)), h.handle)
    return {name: getattr(info, name) for name, _ in HssInfo._fields_}


def hss_node_ranks(h: HSS):
    """[(lo, hi, kr, kc)] for every node, breadth-first (root first, kr = kc = -1)."""
    L = load()
    cnt = ctypes.c_int32()
    _check(L.hss_node_ranks(h.handle, None, None, None, None, 0, ctypes.byref(cnt)), h.handle)
    n = cnt.value
    arrs = [(ctypes.c_int32 * n)() for _ in range(4)]
    _check(L.hss_node_ranks(h.handle, *arrs, n, ctypes.byref(cnt)), h.handle)
    return [(arrs[0][i], arrs[1][i], arrs[2][i], arrs[3][i]) for i in range(n)]


def hss_random_gaussian(seed: int, n: int, c0: int, c1: int, R: torch.Tensor, stream=None):
    """Columns [c0, c1) of the random matrix R into the row-major CUDA tensor R."""
    _require_cuda(R)
    _check(load().hss_random_gaussian(seed, n, c0, c1, ctypes.c_void_p(R.data_ptr()), R.stride(0),
                                      _dtype(R), _stream(stream)))
    return R


def hss_sample(A, R, c0, c1, Sr, Sc, leaf_starts=None, mode="native", stream=None):
    """Fused sampling of columns [c0, c1): Sr = (A-D) R, Sc = (A-D)^T R
    (Sc None: the row samples only)."""
    _require_cuda(A, R, Sr, *([Sc] if Sc is not None else []))
    if Sc is not None and Sr.stride(0) != Sc.stride(0):
        raise ValueError("Sr and Sc must share a leading dimension")
    if isinstance(mode, str):
        mode = SAMPLE_MODES[mode]
    if leaf_starts is None:
        ls, nleaf = None, 0
    else:
        arr = (ctypes.c_int64 * len(leaf_starts))(*[int(x) for x in leaf_starts])
        ls, nleaf = ctypes.cast(arr, ctypes.c_void_p), len(leaf_starts) - 1
    _check(load().hss_sample(ctypes.c_void_p(A.data_ptr()), A.shape[0], A.stride(0), _dtype(A),
                             ctypes.c_void_p(R.data_ptr()), R.stride(0), c0, c1,
                             ctypes.c_void_p(Sr.data_ptr()),
                             ctypes.c_void_p(Sc.data_ptr() if Sc is not None else None),
                             Sr.stride(0), ls, nleaf, mode, _stream(stream)))


def hss_sample_noalloc(A, R, c0, c1, Sr, Sc, leaf_starts=None, mode="native", stream=None):
    """hss_sample without any device allocation, for callers that may not
    allocate (fixed library scratch; small problems only: n <= 2048,
    c1 - c0 <= 64, at most 2048 leaves)."""
    _require_cuda(A, R, Sr, Sc)
    if Sr.stride(0) != Sc.stride(0):
        raise ValueError("Sr and Sc must share a leading dimension")
    if isinstance(mode, str):
        mode = SAMPLE_MODES[mode]
    if leaf_starts is None:
        ls, nleaf = None, 0
    else:
        arr = (ctypes.c_int64 * len(leaf_starts))(*[int(x) for x in leaf_starts])
        ls, nleaf = ctypes.cast(arr, ctypes.c_void_p), len(leaf_starts) - 1
    _check(load().hss_sample_noalloc(ctypes.c_void_p(A.data_ptr()), A.shape[0], A.stride(0),
                                     _dtype(A), ctypes.c_void_p(R.data_ptr()), R.stride(0), c0, c1,
                                     ctypes.c_void_p(Sr.data_ptr()), ctypes.c_void_p(Sc.data_ptr()),
                                     Sr.stride(0), ls, nleaf, mode, _stream(stream)))


def hss_id_batched(Ys, rtol, atol=0.0, stream=None):
    """Batched FP64 CPQR interpolative decompositions.

    Ys: list of CUDA tensors Y_b^T (m_b x d_b, row j = column j of Y_b), one
    dtype.  Returns [(k, perm (m,), E ((m-k) x k))] as CUDA tensors.
    """
    if not Ys:
        return []
    dev = Ys[0].device
    dt = _dtype(Ys[0])
    _require_cuda(*Ys)
    cnt = len(Ys)
    m = torch.tensor([y.shape[0] for y in Ys], dtype=torch.int32, device=dev)
    d = torch.tensor([y.shape[1] for y in Ys], dtype=torch.int32, device=dev)
    ld = torch.tensor([y.stride(0) for y in Ys], dtype=torch.int32, device=dev)
    ptrs = torch.tensor([y.data_ptr() for y in Ys], dtype=torch.int64, device=dev)
    perms = [torch.empty(max(y.shape[0], 1), dtype=torch.int32, device=dev) for y in Ys]
    Es = [torch.empty(max(y.shape[0] * min(y.shape), 1), dtype=torch.float64, device=dev) for y in Ys]
    pp = torch.tensor([p.data_ptr() for p in perms], dtype=torch.int64, device=dev)
    ep = torch.tensor([e.data_ptr() for e in Es], dtype=torch.int64, device=dev)
    k = torch.empty(cnt, dtype=torch.int32, device=dev)
    vp = ctypes.c_void_p
    _check(load().hss_id_batched(cnt, vp(ptrs.data_ptr()), vp(m.data_ptr()), vp(d.data_ptr()),
                                 vp(ld.data_ptr()), dt, rtol, atol, vp(pp.data_ptr()),
                                 vp(ep.data_ptr()), vp(k.data_ptr()), _stream(stream)))
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    ks = k.tolist()
    out = []
    for y, kk, p, e in zip(Ys, ks, perms, Es):
        mm = y.shape[0]
        out.append((kk, p[:mm], e[: (mm - kk) * kk].view(mm - kk, kk)))
    return out


class _DeviceArray:
    """A device buffer of the library seen through the CUDA array interface
    (torch.as_tensor wraps it without a copy)."""

    def __init__(self, ptr, shape, strides, typestr, itemsize):
        self.__cuda_array_interface__ = {
            "shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
            "strides": tuple(x * itemsize for x in strides), "version": 3}


def _device_view(ptr, rows, cols, ld, dtype):
    typestr, size = {torch.float32: ("<f4", 4), torch.float64: ("<f8", 8),
                     torch.int32: ("<i4", 4)}[dtype]
    shape = (rows,) if cols is None else (rows, cols)
    strides = (1,) if cols is None else (ld, 1)
    return torch.as_tensor(_DeviceArray(ptr, shape, strides, typestr, size), device="cuda")


def hss_compress_matfree(n: int, sample, extract, dtype=torch.float32,
                         opts: HssOpts | None = None, stream=None, **kw) -> HSS:
    """Matrix-free compression (hss_compress_matfree).  sample(R, Sr, Sc)
    must write Sr = A R and, when Sc is not None, Sc = A^T R (torch views of
    the library's n x c device buffers); extract(rows, cols, out) must write
    out[i, j] = A[rows[i], cols[j]] (int32 index tensors, an nr x nc view).
    Both run with the compression's stream as torch's current stream."""
    if opts is None:
        opts = hss_default_opts(**kw)
    failure = []
    tstream = stream if stream is not None else torch.cuda.current_stream()
    sp = _stream(tstream)

    def _sample(ctx, c, r, ldr, sr, sc, lds, st):
        try:
            with torch.cuda.stream(tstream):
                R = _device_view(r, n, c, ldr, dtype)
                Sr = _device_view(sr, n, c, lds, dtype)
                Sc = _device_view(sc, n, c, lds, dtype) if sc else None
                sample(R, Sr, Sc)
            return 0
        except Exception as e:   # reported after the call returns
            failure.append(e)
            return 1

    def _extract(ctx, rows, nr, cols, nc, out, ldo, st):
        try:
            with torch.cuda.stream(tstream):
                rw = _device_view(rows, nr, None, 1, torch.int32)
                cl = _device_view(cols, nc, None, 1, torch.int32)
                extract(rw, cl, _device_view(out, nr, nc, ldo, dtype))
            return 0
        except Exception as e:
            failure.append(e)
            return 1

    ops = HssMatfree(SAMPLE_FN(_sample), EXTRACT_FN(_extract), None)
    out = ctypes.c_void_p()
    st = load().hss_compress_matfree(n, HSS_F64 if dtype == torch.float64 else HSS_F32,
                                     ctypes.byref(ops), ctypes.byref(opts), sp,
                                     ctypes.byref(out))
    if failure:
        if out.value:
            load().hss_destroy(out)
        raise failure[0]
    if st == HSS_ERR_RANK_CAP and out.value:
        msg = load().hss_last_error(out).decode()
        load().hss_destroy(out)
        raise HssError(st, msg)
    _check(st)
    return HSS(out.value, n, dtype)
