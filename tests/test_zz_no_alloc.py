"""The allocation-free LB_MV entry point (tcdtw_lb_mv_noalloc) against the
allocating one (tcdtw_lower_bounds with TCDTW_LB_MV), both called through the C ABI.

Callers that cannot allocate device memory -- latency-critical serving loops
(cudaMalloc/cudaFree can synchronise the device) and processes whose memory belongs
to a caching allocator or a fixed budget -- use the variant whose scratch is a fixed
array inside the library.  This file is collected last so that a failure here does
not hide the other tests; it passes alone in a fresh process and after the rest.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

tc = pytest.importorskip("paper_2101_07731_gb300")


def _lb_rtol(L, D):
    # the bar of tests/test_gpu_nn.py for rounded-down bounds
    return max(1e-5, (D + 32 + (L * D + 31) // 32 + 8) * 2.0 ** -23)


def _abi_lower_bounds_mv(lib, q, c, W, stream):
    M, L, D = q.shape
    N = c.shape[0]
    out = torch.empty(M, N, dtype=torch.float32, device=q.device)
    opts = tc.default_opts()
    rc = lib.tcdtw_lower_bounds(C.c_void_p(q.data_ptr()), M, C.c_void_p(c.data_ptr()), N, L, D, W, 16,
                                C.byref(opts), tc.LB_MV, C.c_void_p(out.data_ptr()), stream)
    assert rc == 0, rc
    return out


def _abi_noalloc(lib, q, c, W, out, stream):
    M, L, D = q.shape
    N = c.shape[0]
    return lib.tcdtw_lb_mv_noalloc(C.c_void_p(q.data_ptr()), M, C.c_void_p(c.data_ptr()), N, L, D, W,
                                   C.c_void_p(out.data_ptr()), stream)


def test_noalloc_lb_mv_matches_allocating_entry_point_twice():
    lib = tc._load()
    dev = torch.device("cuda:0")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [  # calls in a row, different shapes: odd M, ragged L*D, one query, a query
        # tile of at most 8 queries, and the largest block the scratch holds
        # (2*ceil(M/2) * ceil32(L*D) == 2^20)
        (synth.SeriesSpec("proto_warp", 96, 5, 31, n_proto=4, sigma=0.1), 37, 700, 9),
        (synth.SeriesSpec("random_walk", 67, 3, 32), 20, 333, 6),
        (synth.SeriesSpec("random_walk", 40, 2, 33), 1, 150, 4),
        (synth.SeriesSpec("proto_warp", 50, 7, 34, n_proto=3, sigma=0.1), 5, 260, 5),
        (synth.SeriesSpec("random_walk", 512, 32, 35), 64, 40, 25),
    ]
    for spec, M, N, W in cases:
        Q = torch.from_numpy(synth.generate(spec, synth.ROLE_QUERY, M)).to(dev)
        Cn = torch.from_numpy(synth.generate(spec, synth.ROLE_CAND, N)).to(dev)
        out = torch.full((M, N), float("nan"), dtype=torch.float32, device=dev)
        assert _abi_noalloc(lib, Q, Cn, W, out, stream) == 0
        ref = _abi_lower_bounds_mv(lib, Q, Cn, W, stream)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        np.testing.assert_allclose(got, want, rtol=_lb_rtol(spec.L, spec.D), atol=1e-6)


def test_noalloc_rejects_sizes_beyond_its_scratch_and_wide_points():
    lib = tc._load()
    dev = torch.device("cuda:0")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # 2*ceil(M/2) * ceil32(L*D) = 1024 * 2048 > 2^20: refused before any work
    Q = torch.zeros(1024, 512, 4, dtype=torch.float32, device=dev)
    Cn = torch.zeros(2, 512, 4, dtype=torch.float32, device=dev)
    out = torch.zeros(1024, 2, dtype=torch.float32, device=dev)
    assert _abi_noalloc(lib, Q, Cn, 5, out, stream) == 6      # TCDTW_ERR_UNSUPPORTED
    # one query more than the largest block that fits (65 * 16384 > 2^20)
    Q2 = torch.zeros(65, 512, 32, dtype=torch.float32, device=dev)
    C2 = torch.zeros(2, 512, 32, dtype=torch.float32, device=dev)
    out2 = torch.zeros(65, 2, dtype=torch.float32, device=dev)
    assert _abi_noalloc(lib, Q2, C2, 5, out2, stream) == 6
    # more dimensions than the kernels are compiled for: refused like the allocating call
    Q3 = torch.zeros(2, 8, 65, dtype=torch.float32, device=dev)
    C3 = torch.zeros(2, 8, 65, dtype=torch.float32, device=dev)
    out3 = torch.zeros(2, 2, dtype=torch.float32, device=dev)
    assert _abi_noalloc(lib, Q3, C3, 2, out3, stream) == 6
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
    assert torch.count_nonzero(out2).item() == 0 and torch.count_nonzero(out3).item() == 0
