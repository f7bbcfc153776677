"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/tcdtw.h; host-side argument validation and the host-only
helpers behave as documented (no kernel is launched here)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tcdtw.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2101_07731_gb300 import build as B
    path = B.build()
    return C.CDLL(path)


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tcdtw_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tcdtw_build", "tcdtw_nn", "tcdtw_free", "tcdtw_dtw_pairs", "tcdtw_dtw_pairs_backward",
                     "tcdtw_dtw_pairs_ckpt_bytes", "tcdtw_batch_nn", "tcdtw_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], stdout=subprocess.PIPE, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (tcdtw_[a-z_0-9]+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert getattr(lib, n) is not None


def test_strerror_and_default_opts(lib):
    lib.tcdtw_strerror.restype = C.c_char_p
    assert lib.tcdtw_strerror(0) == b"ok"
    assert b"invalid" in lib.tcdtw_strerror(1)
    assert b"non-finite" in lib.tcdtw_strerror(5)
    import paper_2101_07731_gb300 as tc
    o = tc.default_opts()
    assert (o.P, o.Lq, o.w, o.use_pc, o.use_ti, o.seed_s, o.check_finite) == (5, 2, 6, 1, 1, 4, 1)
    assert abs(o.e_pc - 0.1) < 1e-7 and abs(o.e_ti - 0.1) < 1e-7


def test_tile_table(lib):
    n = lib.tcdtw_tile_count()
    assert n >= 8
    R, D = C.c_int32(), C.c_int32()
    seen = set()
    for t in range(n):
        assert lib.tcdtw_tile_info(t, None, C.byref(R), C.byref(D)) == 0
        assert R.value >= 1 and D.value >= 1
        seen.add(D.value)
    assert max(seen) >= 64
    assert lib.tcdtw_tile_info(n, None, C.byref(R), C.byref(D)) == 1


def test_ckpt_bytes_formula(lib):
    b = C.c_int64()
    # one band row (2W+1 floats) per 48 rows, except after the last segment
    assert lib.tcdtw_dtw_pairs_ckpt_bytes(C.c_int64(1024), 512, 8, 51, C.byref(b)) == 0
    n_seg = -(-512 // 48)
    assert b.value == 1024 * (n_seg - 1) * 103 * 4
    assert lib.tcdtw_dtw_pairs_ckpt_bytes(C.c_int64(3), 10, 2, 50, C.byref(b)) == 0   # W clamped to L-1
    assert b.value == 0
    assert lib.tcdtw_dtw_pairs_ckpt_bytes(C.c_int64(3), 0, 2, 5, C.byref(b)) == 1


def test_host_validation_rejects_bad_shapes_without_touching_the_gpu(lib):
    P = C.c_void_p
    lib.tcdtw_dtw_pairs.argtypes = [P, P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, P, P, C.c_int64, P]
    dummy = P(16)
    assert lib.tcdtw_dtw_pairs(dummy, dummy, 4, 0, 3, 2, dummy, None, 0, None) == 1      # L < 1
    assert lib.tcdtw_dtw_pairs(dummy, dummy, 4, 8, 0, 2, dummy, None, 0, None) == 1      # D < 1
    assert lib.tcdtw_dtw_pairs(dummy, dummy, 4, 8, 3, -1, dummy, None, 0, None) == 1     # W < 0
    assert lib.tcdtw_dtw_pairs(None, dummy, 4, 8, 3, 2, dummy, None, 0, None) == 1       # null
    assert lib.tcdtw_dtw_pairs(dummy, dummy, 0, 8, 3, 2, dummy, None, 0, None) == 0      # nothing to do
    assert lib.tcdtw_dtw_pairs(dummy, dummy, 4, 8, 65, 2, dummy, None, 0, None) == 6     # D > max
    lib.tcdtw_build.argtypes = [P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, P, C.POINTER(P)]
    h = P()
    assert lib.tcdtw_build(dummy, 0, 8, 3, 2, 4, None, None, C.byref(h)) == 1             # N < 1
    assert lib.tcdtw_build(dummy, 10, 8, 3, 2, 0, None, None, C.byref(h)) == 1            # K < 1
    assert lib.tcdtw_build(None, 10, 8, 3, 2, 4, None, None, C.byref(h)) == 1             # null
    assert h.value is None
    lib.tcdtw_nn.argtypes = [P, P, C.c_int64, P, P, P, P]
    assert lib.tcdtw_nn(None, dummy, 3, dummy, dummy, None, None) == 1
    lib.tcdtw_pc_boxes.argtypes = [P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                   C.c_int32, P, P, P]
    assert lib.tcdtw_pc_boxes(dummy, 2, 64, 64, 4, 8, 3, 6, dummy, dummy, None) == 1     # 3^64 overflows
    lib.tcdtw_batch_nn.argtypes = [P, C.c_int32, P, P, P]
    assert lib.tcdtw_batch_nn(None, 2, None, None, None) == 1
    assert lib.tcdtw_batch_nn(None, 0, None, None, None) == 0


def test_product_path_has_no_cpu_fallback():
    """The package refuses CPU tensors instead of computing on the host."""
    import torch
    import paper_2101_07731_gb300 as tc
    x = torch.zeros(2, 8, 3)
    with pytest.raises(ValueError, match="CUDA"):
        tc.dtw_pairs(x, x, 2)
    with pytest.raises(ValueError, match="CUDA"):
        tc.Index(x, 2)
    src = open(os.path.join(ROOT, "paper_2101_07731_gb300", "__init__.py")).read()
    assert "import oracle" not in src and "from oracle" not in src


def test_binding_structs_mirror_the_header():
    # the ctypes mirrors of tcdtw_opts / tcdtw_stats / tcdtw_dataset must list the
    # header's fields in the header's order (the C side writes whole structs)
    import paper_2101_07731_gb300 as tc
    hdr = open(os.path.join(ROOT, "include", "tcdtw.h")).read()
    for cname, py in (("tcdtw_opts", tc.Opts), ("tcdtw_stats", tc.Stats), ("tcdtw_dataset", tc.Dataset)):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + ";", hdr).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = [re.findall(r"(\w+)\s*$", part)[0] for stmt in body.split(";") if stmt.strip()
                 for part in stmt.split(",")]
        assert names == [n for n, _ in py._fields_], (cname, names)


def test_argument_errors_of_the_newer_calls(lib):
    # every check below returns before any CUDA call (no GPU needed; the dummy
    # addresses are never dereferenced)
    import paper_2101_07731_gb300 as tc
    o = tc.default_opts()
    assert (o.use_rev, o.ti_top, o.select, o.mv_abandon) == (0, 1, 1, 1)
    dummy = C.c_void_p(256)
    f = lib.tcdtw_lower_bounds
    f.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                  C.POINTER(tc.Opts), C.c_int32, C.c_void_p, C.c_void_p]
    for which in (-1, 4):
        assert f(dummy, 1, dummy, 1, 30, 2, 3, 4, C.byref(o), which, dummy, None) == tc.ERR_INVALID
    # the row-sweep LB_TI variants hold the window in up to 8 x 32 lanes: W <= 127
    o2 = tc.default_opts(ti_top=0)
    assert f(dummy, 1, dummy, 1, 300, 2, 200, 4, C.byref(o2), tc.LB_TI, dummy, None) == tc.ERR_UNSUPPORTED
    build = lib.tcdtw_build
    build.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(tc.Opts),
                      C.c_void_p, C.POINTER(C.c_void_p)]
    h = C.c_void_p()
    assert build(dummy, 1, 300, 2, 200, 4, C.byref(o2), None, C.byref(h)) == tc.ERR_UNSUPPORTED
    lib.tcdtw_lb_mv_selftest_timeout.argtypes = [C.c_int64, C.c_void_p]
    lib.tcdtw_batch_selftest_timeout.argtypes = [C.c_int64, C.c_void_p]
    assert lib.tcdtw_lb_mv_selftest_timeout(0, None) == tc.ERR_INVALID
    assert lib.tcdtw_lb_mv_selftest_timeout(10_000_001, None) == tc.ERR_INVALID
    assert lib.tcdtw_batch_selftest_timeout(0, None) == tc.ERR_INVALID
    lib.tcdtw_lb_mv_rest_selftest_timeout.argtypes = [C.c_int64, C.c_void_p]
    assert lib.tcdtw_lb_mv_rest_selftest_timeout(0, None) == tc.ERR_INVALID
    assert lib.tcdtw_lb_mv_rest_selftest_timeout(10_000_001, None) == tc.ERR_INVALID


def test_noalloc_refuses_what_the_allocating_call_refuses(lib):
    # tcdtw_lb_mv_noalloc promises the values of tcdtw_lower_bounds(TCDTW_LB_MV), so it
    # must refuse the same arguments with the same codes, before any CUDA call
    import paper_2101_07731_gb300 as tc
    dummy = C.c_void_p(256)
    f = lib.tcdtw_lower_bounds
    f.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                  C.POINTER(tc.Opts), C.c_int32, C.c_void_p, C.c_void_p]
    g = lib.tcdtw_lb_mv_noalloc
    g.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                  C.c_void_p]
    o = tc.default_opts()
    cases = [(2, 3, 8, 65, 2),            # D > TCDTW_MAX_D: UNSUPPORTED
             (70000, 70000, 8, 2, 2),     # M*N >= 4.29e9: UNSUPPORTED
             (-1, 3, 8, 2, 2), (2, 3, 0, 2, 2), (2, 3, 8, 0, 2), (2, 3, 8, 2, -1),   # INVALID
             (0, 3, 8, 2, 2), (2, 0, 8, 2, 2)]                                         # nothing to do
    for M, N, L, D, W in cases:
        a = f(dummy, M, dummy, N, L, D, W, 16, C.byref(o), tc.LB_MV, dummy, None)
        b = g(dummy, M, dummy, N, L, D, W, dummy, None)
        assert a == b, (M, N, L, D, W, a, b)
    assert g(dummy, 2, dummy, 3, 8, 65, 2, dummy, None) == tc.ERR_UNSUPPORTED
    assert g(None, 2, dummy, 3, 8, 2, 2, dummy, None) == tc.ERR_INVALID


def test_abandoning_lb_mv_argument_errors(lib):
    # tcdtw_lb_mv_abandon checks its arguments like tcdtw_lower_bounds(TCDTW_LB_MV), plus
    # the threshold array, before any CUDA call
    import paper_2101_07731_gb300 as tc
    dummy = C.c_void_p(256)
    g = lib.tcdtw_lb_mv_abandon
    g.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                  C.c_void_p, C.c_void_p]
    assert g(dummy, 2, dummy, 3, 8, 65, 2, dummy, dummy, None) == tc.ERR_UNSUPPORTED
    assert g(dummy, 70000, dummy, 70000, 8, 2, 2, dummy, dummy, None) == tc.ERR_UNSUPPORTED
    for M, N, L, D, W in [(-1, 3, 8, 2, 2), (2, 3, 0, 2, 2), (2, 3, 8, 0, 2), (2, 3, 8, 2, -1)]:
        assert g(dummy, M, dummy, N, L, D, W, dummy, dummy, None) == tc.ERR_INVALID
    assert g(dummy, 2, dummy, 3, 8, 2, 2, None, dummy, None) == tc.ERR_INVALID      # no thresholds
    assert g(None, 2, dummy, 3, 8, 2, 2, dummy, dummy, None) == tc.ERR_INVALID
    assert g(dummy, 0, dummy, 3, 8, 2, 2, None, None, None) == 0                   # nothing to do


def test_alloc_failure_injection_switch(lib):
    lib.tcdtw_inject_alloc_failure.argtypes = [C.c_int64]
    assert lib.tcdtw_inject_alloc_failure(-2) == 1          # INVALID
    assert lib.tcdtw_inject_alloc_failure(5) == 0
    assert lib.tcdtw_inject_alloc_failure(-1) == 0          # off again
