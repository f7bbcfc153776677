"""ctypes front end of the FP64 CPU oracle (``tcdtw_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may use this module; the product package never does.
It shares no code with the CUDA path.

All array arguments are numpy float32 ``[count][L][D]`` series (C-contiguous);
results are float64.  The library is compiled with gcc on first use (or by
``build()``), with ``-ffp-contract=off`` so that no multiply-add is fused and the
FP64 results depend only on the operation order in the C source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tcdtw_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in
                ("pairs", "pruned_mv", "pruned_pc", "pruned_ti", "dtw_started", "dtw_abandoned")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile the oracle into ``liboracle.so`` (OpenMP if the compiler has it)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-lm"]
    tmp = _LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base[:-1] + ["-fopenmp", "-o", tmp, "-lm"], check=True,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        I, D_, I64 = C.c_int, C.c_double, C.c_int64
        L.orc_num_threads.restype = I
        L.orc_cost.restype = D_
        L.orc_cost.argtypes = [_f32p, _f32p, I]
        L.orc_dtw.restype = D_
        L.orc_dtw.argtypes = [_f32p, _f32p, I, I, I]
        L.orc_dtw_abandon.restype = D_
        L.orc_dtw_abandon.argtypes = [_f32p, _f32p, I, I, I, D_]
        L.orc_dtw_pairs.restype = None
        L.orc_dtw_pairs.argtypes = [_f32p, _f32p, I64, I, I, I, _f64p, I]
        L.orc_envelope.restype = None
        L.orc_envelope.argtypes = [_f32p, I, I, I, _f64p, _f64p]
        L.orc_lb_mv.restype = D_
        L.orc_lb_mv.argtypes = [_f32p, _f32p, I, I, I]
        L.orc_lb_ad.restype = D_
        L.orc_lb_ad.argtypes = [_f32p, _f32p, I, I, I]
        L.orc_query_dq.restype = None
        L.orc_query_dq.argtypes = [_f32p, I, I, _f64p]
        L.orc_lb_ti.restype = D_
        L.orc_lb_ti.argtypes = [_f32p, _f32p, I, I, I, I]
        L.orc_lb_ti_var.restype = D_
        L.orc_lb_ti_var.argtypes = [_f32p, _f32p, I, I, I, I, I]
        L.orc_pc_boxes.restype = None
        L.orc_pc_boxes.argtypes = [_f32p, I, I, I, I, I, I, _f64p, _i32p]
        L.orc_lb_pc.restype = D_
        L.orc_lb_pc.argtypes = [_f32p, _f32p, I, I, I, I, I, I]
        L.orc_nn_brute.restype = None
        L.orc_nn_brute.argtypes = [_f32p, I64, _f32p, I64, I, I, I, _i64p, _f64p, I]
        L.orc_nn_pruned.restype = None
        L.orc_nn_pruned.argtypes = [_f32p, I64, _f32p, I64, I, I, I, I, I, I, I, I, I, D_, D_,
                                    _i64p, _f64p, C.POINTER(Stats), I]
        L.orc_dtw_grad.restype = D_
        L.orc_dtw_grad.argtypes = [_f32p, _f32p, I, I, I, _f64p, _f64p, _i32p, _i32p,
                                   C.POINTER(C.c_int), C.POINTER(C.c_double)]
        _lib = L
    return _lib


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def cost(a, b) -> float:
    a, b = _f32(a), _f32(b)
    return float(lib().orc_cost(a, b, a.shape[-1]))


def dtw(a, b, W: int, abandon_at: float = np.inf) -> float:
    """Windowed DTW of two [L][D] series (Eq. 1), squared-Euclidean point cost."""
    a, b = _f32(a), _f32(b)
    L, D = a.shape
    return float(lib().orc_dtw_abandon(a, b, L, D, W, float(abandon_at)))


def dtw_pairs(A, B, W: int, nthreads: int = 0) -> np.ndarray:
    A, B = _f32(A), _f32(B)
    P, L, D = A.shape
    out = np.empty(P, dtype=np.float64)
    lib().orc_dtw_pairs(A, B, P, L, D, W, out, nthreads)
    return out


def envelope(q, W: int):
    q = _f32(q)
    L, D = q.shape
    U = np.empty((L, D)); Lo = np.empty((L, D))
    lib().orc_envelope(q, L, D, W, U, Lo)
    return U, Lo


def lb_mv(q, c, W: int) -> float:
    q, c = _f32(q), _f32(c)
    L, D = q.shape
    return float(lib().orc_lb_mv(q, c, L, D, W))


def lb_ad(q, c, W: int) -> float:
    q, c = _f32(q), _f32(c)
    L, D = q.shape
    return float(lib().orc_lb_ad(q, c, L, D, W))


def query_dq(q) -> np.ndarray:
    q = _f32(q)
    L, D = q.shape
    out = np.empty(L)
    lib().orc_query_dq(q, L, D, out)
    return out


def lb_ti(q, c, W: int, P: int = 5) -> float:
    q, c = _f32(q), _f32(c)
    L, D = q.shape
    return float(lib().orc_lb_ti(q, c, L, D, W, P))


def lb_ti_var(q, c, W: int, P: int, top: int) -> float:
    """LB_TI variants (Section 4.2): top=1 exact window tops (TIP_TOP, or LB_TI_TOP
    when P >= L), top=0 window tops from the candidate-side triangle (LB_TIP, or the
    basic LB_TI when P >= L)."""
    q, c = _f32(q), _f32(c)
    L, D = q.shape
    return float(lib().orc_lb_ti_var(q, c, L, D, W, P, int(top)))


def pc_boxes(q, W: int, K: int, Lq: int = 2, w: int = 6):
    """Boxes [G][K][2][D] (lower, upper corner) and counts [G] of one query."""
    q = _f32(q)
    L, D = q.shape
    G = (L + w - 1) // w
    boxes = np.full((G, K, 2, D), np.nan)
    counts = np.zeros(G, dtype=np.int32)
    lib().orc_pc_boxes(q, L, D, W, K, Lq, w, boxes, counts)
    return boxes, counts


def lb_pc(q, c, W: int, K: int, Lq: int = 2, w: int = 6) -> float:
    q, c = _f32(q), _f32(c)
    L, D = q.shape
    return float(lib().orc_lb_pc(q, c, L, D, W, K, Lq, w))


def nn_brute(Q, Cands, W: int, nthreads: int = 0):
    """Exact FP64 DTW-NN: (idx int64[M], dist float64[M]), ties to the smallest index."""
    Q, Cands = _f32(Q), _f32(Cands)
    M, L, D = Q.shape
    N = Cands.shape[0]
    idx = np.empty(M, dtype=np.int64); dist = np.empty(M)
    lib().orc_nn_brute(Q, M, Cands, N, L, D, W, idx, dist, nthreads)
    return idx, dist


def nn_pruned(Q, Cands, W: int, K: int = 16, Lq: int = 2, w: int = 6, P: int = 5,
              use_pc: bool = True, use_ti: bool = True, e_pc: float = 0.1, e_ti: float = 0.1,
              nthreads: int = 0):
    """The paper's pruned search (LB_MV, gated LB_PC / LB_TI, abandoning DTW)."""
    Q, Cands = _f32(Q), _f32(Cands)
    M, L, D = Q.shape
    N = Cands.shape[0]
    idx = np.empty(M, dtype=np.int64); dist = np.empty(M)
    st = Stats()
    lib().orc_nn_pruned(Q, M, Cands, N, L, D, W, K, Lq, w, P, int(use_pc), int(use_ti),
                        float(e_pc), float(e_ti), idx, dist, C.byref(st), nthreads)
    return idx, dist, st.as_dict()


def dtw_grad(a, b, W: int):
    """(dist, dA [L][D], dB [L][D], path [(i, j)], margin) -- see orc_dtw_grad."""
    a, b = _f32(a), _f32(b)
    L, D = a.shape
    ga = np.empty((L, D)); gb = np.empty((L, D))
    pi = np.empty(2 * L, dtype=np.int32); pj = np.empty(2 * L, dtype=np.int32)
    n = C.c_int(0); mg = C.c_double(0.0)
    d = lib().orc_dtw_grad(a, b, L, D, W, ga, gb, pi, pj, C.byref(n), C.byref(mg))
    path = list(zip(pi[:n.value].tolist(), pj[:n.value].tolist()))
    return float(d), ga, gb, path, float(mg.value)
