"""tcdtw: exact multivariate DTW nearest-neighbour search on GB300 (sm_103a).

Thin Python binding of ``libtcdtw.so`` (C ABI in ``include/tcdtw.h``): argument
marshalling only.  Every step of the search and of the differentiable distance
runs in the library's CUDA kernels; PyTorch supplies device memory and the
current CUDA stream.  There is no CPU fallback: if the library is not built, or no
CUDA device is present, calls raise.

Main entry points
  ``Index(cand, W, K).nn(q) -> (idx, dist)``   exact 1-NN under windowed DTW
  ``dtw(A, B, W)``                              differentiable DTW of pairs (autograd)
  ``batch_nn(sets)``                            many uneven searches in one launch
and the pipeline stages ``envelope``, ``query_dq``, ``pc_boxes``,
``lower_bounds`` and ``compact``.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

__all__ = ["Index", "dtw", "dtw_pairs", "dtw_pairs_backward", "batch_nn", "batch_tiles", "batch_release", "batch_selftest_timeout", "lb_mv_selftest_timeout", "envelope", "query_dq",
           "pc_boxes", "lower_bounds", "compact", "Opts", "Stats", "TcdtwError", "lib_path",
           "LB_MV", "LB_PC", "LB_TI", "LB_MV_REV", "default_opts"]

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libtcdtw.so")
_lib = None

LB_MV, LB_PC, LB_TI, LB_MV_REV = 0, 1, 2, 3
# status codes of the C ABI (tcdtw.h)
OK, ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_NONFINITE, ERR_UNSUPPORTED = range(7)


def lib_path() -> str:
    return _LIB_PATH


class TcdtwError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _load().tcdtw_strerror(code).decode() if _lib is not None else str(code)
        if code in (2, 3) and _lib is not None:
            detail = _lib.tcdtw_last_error_detail().decode()
            if detail:
                msg += f" [{detail}]"
        super().__init__(f"{where}: {msg} (code {code})")
        self.code = code


class Opts(C.Structure):
    _fields_ = [("P", C.c_int32), ("Lq", C.c_int32), ("w", C.c_int32), ("e_pc", C.c_float),
                ("e_ti", C.c_float), ("use_pc", C.c_int32), ("use_ti", C.c_int32),
                ("seed_s", C.c_int32), ("qblock", C.c_int32), ("tile", C.c_int32),
                ("check_finite", C.c_int32), ("no_prune", C.c_int32), ("use_graph", C.c_int32),
                ("select", C.c_int32), ("use_rev", C.c_int32), ("ti_top", C.c_int32),
                ("mv_abandon", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("pairs", "pruned_mv", "pruned_pc", "pruned_ti", "dtw_started",
                                          "dtw_abandoned", "cells", "refined",
                                          "refined64", "pruned_rev", "mv_terms")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class Dataset(C.Structure):
    _fields_ = [("cand", C.c_void_p), ("N", C.c_int64), ("L", C.c_int32), ("D", C.c_int32),
                ("W", C.c_int32), ("K", C.c_int32), ("q", C.c_void_p), ("M", C.c_int64),
                ("idx", C.c_void_p), ("dist", C.c_void_p)]


_P, _I32, _I64, _F = C.c_void_p, C.c_int32, C.c_int64, C.c_float
_SIGS = {
    "tcdtw_default_opts": (None, [C.POINTER(Opts)]),
    "tcdtw_strerror": (C.c_char_p, [C.c_int]),
    "tcdtw_last_error_detail": (C.c_char_p, []),
    "tcdtw_build": (C.c_int, [_P, _I64, _I32, _I32, _I32, _I32, C.POINTER(Opts), _P, C.POINTER(_P)]),
    "tcdtw_nn": (C.c_int, [_P, _P, _I64, _P, _P, C.POINTER(Stats), _P]),
    "tcdtw_free": (None, [_P]),
    "tcdtw_dtw_pairs": (C.c_int, [_P, _P, _I64, _I32, _I32, _I32, _P, _P, _I64, _P]),
    "tcdtw_dtw_pairs_ckpt_bytes": (C.c_int, [_I64, _I32, _I32, _I32, C.POINTER(_I64)]),
    "tcdtw_dtw_pairs_backward": (C.c_int, [_P, _P, _P, _I64, _P, _I64, _I32, _I32, _I32, _P, _P, _P]),
    "tcdtw_envelope": (C.c_int, [_P, _I64, _I32, _I32, _I32, _P, _P, _P]),
    "tcdtw_query_dq": (C.c_int, [_P, _I64, _I32, _I32, _P, _P, _P]),
    "tcdtw_pc_boxes": (C.c_int, [_P, _I64, _I32, _I32, _I32, _I32, _I32, _I32, _P, _P, _P]),
    "tcdtw_lower_bounds": (C.c_int, [_P, _I64, _P, _I64, _I32, _I32, _I32, _I32, C.POINTER(Opts), _I32, _P,
                                     _P]),
    "tcdtw_compact": (C.c_int, [_P, _I64, _I64, _P, _P, _P, _P]),
    "tcdtw_lb_mv_abandon": (C.c_int, [_P, _I64, _P, _I64, _I32, _I32, _I32, _P, _P, _P]),
    "tcdtw_lb_mv_noalloc": (C.c_int, [_P, _I64, _P, _I64, _I32, _I32, _I32, _P, _P]),
    "tcdtw_batch_nn": (C.c_int, [C.POINTER(Dataset), _I32, C.POINTER(Opts), C.POINTER(Stats), _P]),
    "tcdtw_batch_selftest_timeout": (C.c_int, [_I64, _P]),
    "tcdtw_lb_mv_selftest_timeout": (C.c_int, [_I64, _P]),
    "tcdtw_lb_mv_rest_selftest_timeout": (C.c_int, [_I64, _P]),
    "tcdtw_batch_release": (C.c_int, []),
    "tcdtw_batch_tiles": (C.c_int, [C.POINTER(Dataset), _I32, C.POINTER(Opts), C.POINTER(_I32), C.POINTER(_I32), _P]),
    "tcdtw_inject_alloc_failure": (C.c_int, [_I64]),
    "tcdtw_tile_count": (C.c_int, []),
    "tcdtw_set_profiling": (C.c_int, [_P, _I32]),
    "tcdtw_stage_times": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(_I64)]),
    "tcdtw_kernel_launches": (C.c_uint64, []),
    "tcdtw_index_info": (C.c_int, [_P, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32)]),
    "tcdtw_index_opts": (C.c_int, [_P, C.POINTER(Opts)]),
    "tcdtw_tile_info": (C.c_int, [_I32, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I32)]),
}


def _load():
    """Load the in-tree library; raise (no fallback) if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; "
                               f"g.build()'` (needs nvcc)")
        L = C.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _call(name, *args):
    fn = getattr(_load(), name)
    code = fn(*args)
    if code != 0:
        raise TcdtwError(code, name)


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _series(x: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not x.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if x.dtype != torch.float32:
        raise ValueError(f"{name} must be float32")
    if x.dim() != 3:
        raise ValueError(f"{name} must have shape [count][L][D]")
    return x.contiguous()


def _ptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


def default_opts(**kw) -> Opts:
    o = Opts()
    _load().tcdtw_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, v)
    return o


# ----------------------------------------------------------------- DTW of pairs

def ckpt_bytes(P: int, L: int, D: int, W: int) -> int:
    b = _I64(0)
    _call("tcdtw_dtw_pairs_ckpt_bytes", P, L, D, W, C.byref(b))
    return int(b.value)


def dtw_pairs(A: torch.Tensor, B: torch.Tensor, W: int, ckpt: torch.Tensor | None = None) -> torch.Tensor:
    """DTW distance of each pair (A[p], B[p]) [P][L][D] -> float32 [P]."""
    A, B = _series(A, "A"), _series(B, "B")
    if A.shape != B.shape:
        raise ValueError("A and B must have the same shape")
    P, L, D = A.shape
    dist = torch.empty(P, dtype=torch.float32, device=A.device)
    ck_ptr, ck_n = C.c_void_p(0), 0
    if ckpt is not None:
        ck_ptr, ck_n = _ptr(ckpt), ckpt.numel() * ckpt.element_size()
    _call("tcdtw_dtw_pairs", _ptr(A), _ptr(B), P, L, D, int(W), _ptr(dist), ck_ptr, ck_n, _stream())
    return dist


def dtw_pairs_backward(A, B, W, ckpt, grad_dist):
    A, B = _series(A, "A"), _series(B, "B")
    P, L, D = A.shape
    grad_dist = grad_dist.contiguous().to(torch.float32)
    gA = torch.empty_like(A)
    gB = torch.empty_like(B)
    n = ckpt.numel() * ckpt.element_size() if ckpt is not None else 0
    _call("tcdtw_dtw_pairs_backward", _ptr(A), _ptr(B), _ptr(ckpt) if ckpt is not None else C.c_void_p(0), n,
          _ptr(grad_dist), P, L, D, int(W), _ptr(gA), _ptr(gB), _stream())
    return gA, gB


class _DTWFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, W):
        A = _series(A, "A")
        B = _series(B, "B")
        P, L, D = A.shape
        ck = torch.empty(max(1, ckpt_bytes(P, L, D, W) // 4), dtype=torch.float32, device=A.device)
        dist = dtw_pairs(A, B, W, ck)
        ctx.save_for_backward(A, B, ck)
        ctx.W = W
        return dist

    @staticmethod
    def backward(ctx, grad):
        A, B, ck = ctx.saved_tensors
        gA, gB = dtw_pairs_backward(A, B, ctx.W, ck, grad)
        return gA, gB, None


def dtw(A: torch.Tensor, B: torch.Tensor, W: int) -> torch.Tensor:
    """Differentiable windowed DTW of pairs: float32 [P], gradients w.r.t. A and B
    through the optimal warping path (recomputed from checkpointed band rows)."""
    return _DTWFunction.apply(A, B, int(W))


# ----------------------------------------------------------------- NN search

class Index:
    """A candidate set prepared for exact DTW-NN search.

    ``cand`` (CUDA float32 [N][L][D]) is borrowed: keep it alive and unchanged
    while the index exists (the index holds a reference)."""

    def __init__(self, cand: torch.Tensor, W: int, K: int = 16, **opts):
        cand = _series(cand, "cand")
        self.cand = cand
        self.N, self.L, self.D = cand.shape
        self.W, self.K = int(W), int(K)
        self.opts = default_opts(**opts)
        h = C.c_void_p(0)
        _call("tcdtw_build", _ptr(cand), self.N, self.L, self.D, self.W, self.K, C.byref(self.opts), _stream(),
              C.byref(h))
        self._h = h

    def nn(self, q: torch.Tensor, stats: bool = False, out=None):
        """(idx int64 [M], dist float64 [M]) of each query's nearest candidate;
        with ``stats=True`` also the search counters (synchronises).  ``out`` =
        (idx, dist) reuses caller buffers.  Calls of up to one query block with a
        query count seen before replay a captured CUDA graph, whatever the buffers."""
        q = _series(q, "q")
        if q.shape[1:] != (self.L, self.D):
            raise ValueError("query shape must be [M][L][D] with the index's L and D")
        M = q.shape[0]
        if out is not None:
            idx, dist = out
            if idx.dtype != torch.int64 or dist.dtype != torch.float64 or idx.numel() < M or dist.numel() < M:
                raise ValueError("out must be (int64 [M], float64 [M]) tensors")
        else:
            idx = torch.empty(M, dtype=torch.int64, device=q.device)
            dist = torch.empty(M, dtype=torch.float64, device=q.device)
        st = Stats()
        _call("tcdtw_nn", self._h, _ptr(q), M, _ptr(idx), _ptr(dist), C.byref(st) if stats else None, _stream())
        return (idx, dist, st.as_dict()) if stats else (idx, dist)

    def info(self):
        """{tile, R, DM, G, qblock}: the band tile the search uses (autotuned at build)."""
        t, g, qb = _I32(), _I32(), _I32()
        _call("tcdtw_index_info", self._h, C.byref(t), C.byref(g), C.byref(qb))
        r, dm = _I32(), _I32()
        _call("tcdtw_tile_info", t.value, None, C.byref(r), C.byref(dm))
        return {"tile": t.value, "R": r.value, "DM": dm.value, "G": g.value, "qblock": qb.value}

    def options(self):
        """The options the index searches with (after TC-DTW's bound selection, made by
        the first nn() call when select=1)."""
        o = Opts()
        _call("tcdtw_index_opts", self._h, C.byref(o))
        return {n: getattr(o, n) for n, _ in o._fields_}

    STAGES = ("check", "prep", "lb_mv", "seed", "lb_rest", "seed2", "compact", "cascade", "dtw", "refine")

    def set_profiling(self, enable: bool = True):
        """Record per-stage CUDA-event times in every nn() call (synchronises)."""
        _call("tcdtw_set_profiling", self._h, int(bool(enable)))

    def stage_times(self):
        """{stage: milliseconds} summed over the profiled nn() calls, and block count."""
        ms = (C.c_double * len(self.STAGES))()
        nb = _I64(0)
        _call("tcdtw_stage_times", self._h, ms, C.byref(nb))
        return dict(zip(self.STAGES, list(ms))), int(nb.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _load().tcdtw_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches() -> int:
    """Kernels launched by libtcdtw.so in this process so far."""
    return int(_load().tcdtw_kernel_launches())


def batch_nn(sets, stats: bool = False, out=None, **opts):
    """Search many independent (cand, q, W, K) problems in one persistent launch.
    ``sets``: iterable of dicts with keys cand, q, W and optionally K (16).
    ``out``: optional list of (idx int64 [M], dist float64 [M]) device tensors, one
    pair per set, written in place (the launch is cached per batch description, so
    reusing the same tensors lets later calls replay a captured graph).
    Returns a list of (idx, dist) per set (and the summed counters if stats)."""
    sets = list(sets)
    if out is not None and len(out) != len(sets):
        raise ValueError("out must hold one (idx, dist) pair per set")
    descs, outs, keep = [], [], []
    for k, s in enumerate(sets):
        cand, q = _series(s["cand"], "cand"), _series(s["q"], "q")
        N, L, D = cand.shape
        M = q.shape[0]
        if q.shape[1:] != cand.shape[1:]:
            raise ValueError(f"set {k}: query and candidate series differ in shape")
        if out is not None:
            idx, dist = out[k]
            if (idx.dtype != torch.int64 or dist.dtype != torch.float64 or idx.numel() != M
                    or dist.numel() != M or not idx.is_contiguous() or not dist.is_contiguous()
                    or idx.device != q.device or dist.device != q.device):
                raise ValueError(f"set {k}: out must be contiguous int64 / float64 [M] on the queries' device")
        else:
            idx = torch.empty(M, dtype=torch.int64, device=q.device)
            dist = torch.empty(M, dtype=torch.float64, device=q.device)
        descs.append(Dataset(cand.data_ptr(), N, L, D, int(s["W"]), int(s.get("K", 16)), q.data_ptr(), M,
                             idx.data_ptr(), dist.data_ptr()))
        outs.append((idx, dist))
        keep += [cand, q]
    arr = (Dataset * len(descs))(*descs)
    o = default_opts(**opts)
    st = Stats()
    _call("tcdtw_batch_nn", arr, len(descs), C.byref(o), C.byref(st) if stats else None, _stream())
    return (outs, st.as_dict()) if stats else outs


def batch_tiles(sets, **opts):
    """[(R, G)] per set: the band tile (rows per lane, lanes per pair) the batched
    search gives each set -- the single-set tuner's choice for its shape; (0, 0) for a
    set searched one at a time."""
    sets = list(sets)
    descs = []
    for s in sets:
        cand, q = _series(s["cand"], "cand"), _series(s["q"], "q")
        N, L, D = cand.shape
        descs.append(Dataset(cand.data_ptr(), N, L, D, int(s["W"]), int(s.get("K", 16)), q.data_ptr(), q.shape[0],
                             None, None))
    arr = (Dataset * len(descs))(*descs)
    R = (_I32 * max(1, len(descs)))()
    G = (_I32 * max(1, len(descs)))()
    o = default_opts(**opts)
    _call("tcdtw_batch_tiles", arr, len(descs), C.byref(o), R, G, _stream())
    return [(int(R[k]), int(G[k])) for k in range(len(descs))]


def batch_release():
    """Free the cached batch sequences (graphs and workspaces)."""
    _call("tcdtw_batch_release")


def batch_selftest_timeout(spin_limit: int = 200000) -> int:
    """Run the batched launch's wait-limit self-test; returns the status code
    (TIMEOUT when the device-side wait ran out and the launch ended by itself)."""
    return int(_load().tcdtw_batch_selftest_timeout(int(spin_limit), _stream()))


def lb_mv_selftest_timeout(wait_us: int = 20000) -> int:
    """Run the TMA LB_MV stream's wait-limit self-test; returns the status code
    (TIMEOUT when the device-side wait ran out and the launch ended by itself)."""
    return int(_load().tcdtw_lb_mv_selftest_timeout(int(wait_us), _stream()))


def lb_mv_rest_selftest_timeout(wait_us: int = 20000) -> int:
    """Run the wait-limit self-test of the abandoning LB_MV's completion kernel;
    returns the status code (TIMEOUT when its consumers' wait ran out and the launch
    ended by itself)."""
    return int(_load().tcdtw_lb_mv_rest_selftest_timeout(int(wait_us), _stream()))


# ----------------------------------------------------------------- pipeline stages

def envelope(q: torch.Tensor, W: int):
    q = _series(q, "q")
    M, L, D = q.shape
    U, Lo = torch.empty_like(q), torch.empty_like(q)
    _call("tcdtw_envelope", _ptr(q), M, L, D, int(W), _ptr(U), _ptr(Lo), _stream())
    return U, Lo


def query_dq(q: torch.Tensor):
    q = _series(q, "q")
    M, L, D = q.shape
    lo = torch.empty(M, L, dtype=torch.float32, device=q.device)
    hi = torch.empty_like(lo)
    _call("tcdtw_query_dq", _ptr(q), M, L, D, _ptr(lo), _ptr(hi), _stream())
    return lo, hi


def pc_boxes(q: torch.Tensor, W: int, K: int, Lq: int = 2, w: int = 6):
    q = _series(q, "q")
    M, L, D = q.shape
    G = (L + w - 1) // w
    boxes = torch.full((M, G, K, 2, D), float("nan"), dtype=torch.float32, device=q.device)
    counts = torch.empty(M, G, dtype=torch.int32, device=q.device)
    _call("tcdtw_pc_boxes", _ptr(q), M, L, D, int(W), int(K), int(Lq), int(w), _ptr(boxes), _ptr(counts),
          _stream())
    return boxes, counts


def lower_bounds(q: torch.Tensor, c: torch.Tensor, W: int, which: int = LB_MV, K: int = 16, **opts):
    q, c = _series(q, "q"), _series(c, "c")
    M, L, D = q.shape
    N = c.shape[0]
    out = torch.empty(M, N, dtype=torch.float32, device=q.device)
    o = default_opts(**opts)
    _call("tcdtw_lower_bounds", _ptr(q), M, _ptr(c), N, L, D, int(W), int(K), C.byref(o), int(which), _ptr(out),
          _stream())
    return out


def lb_mv_abandon(q: torch.Tensor, c: torch.Tensor, W: int, thresh: torch.Tensor):
    """LB_MV of every pair with early abandoning against ``thresh`` ([M] float32):
    out[m][n] is the (rounded-down) LB_MV where that is at most thresh[m], else a
    partial sum that already exceeds thresh[m]; always a lower bound of DTW."""
    q, c = _series(q, "q"), _series(c, "c")
    M, L, D = q.shape
    N = c.shape[0]
    thresh = thresh.contiguous().to(device=q.device, dtype=torch.float32)
    if thresh.numel() != M:
        raise ValueError("thresh must hold one threshold per query")
    out = torch.empty(M, N, dtype=torch.float32, device=q.device)
    _call("tcdtw_lb_mv_abandon", _ptr(q), M, _ptr(c), N, L, D, int(W), _ptr(thresh), _ptr(out), _stream())
    return out


def compact(lb: torch.Tensor, thresh: torch.Tensor):
    lb = lb.contiguous()
    M, N = lb.shape
    thresh = thresh.contiguous().to(torch.float32)
    idx = torch.empty(M, N, dtype=torch.int32, device=lb.device)
    cnt = torch.empty(M, dtype=torch.int32, device=lb.device)
    _call("tcdtw_compact", _ptr(lb), M, N, _ptr(thresh), _ptr(idx), _ptr(cnt), _stream())
    return idx, cnt


def lb_mv_noalloc(q: torch.Tensor, c: torch.Tensor, W: int, out: torch.Tensor | None = None):
    """LB_MV of every (query, candidate) pair with no device allocation inside the
    library (scratch in a fixed in-library array; see tcdtw_lb_mv_noalloc for who
    needs that and for the size limit).  Pass ``out`` ([M][N] float32, on the GPU)
    to avoid the one allocation this wrapper would otherwise make."""
    q, c = _series(q, "q"), _series(c, "c")
    M, L, D = q.shape
    N = c.shape[0]
    if out is None:
        out = torch.empty(M, N, dtype=torch.float32, device=q.device)
    _call("tcdtw_lb_mv_noalloc", _ptr(q), M, _ptr(c), N, L, D, int(W), _ptr(out), _stream())
    return out
