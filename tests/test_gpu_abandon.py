"""GPU parity of LB_MV with early abandoning (Section 7.1: abandoning applies to the
lower bounds as well as to DTW) against the FP64 oracle.

tcdtw_lb_mv_abandon's contract, checked pair by pair: the value never exceeds the
oracle's LB_MV; where that LB_MV is at most the query's threshold the value is the
complete bound (within the round-down bar of the plain LB_MV tests); where it is
above the threshold, the value is either the complete bound or a partial sum that
already exceeds the threshold.  End to end, the search with and without abandoning
returns the oracle's nearest neighbours.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

tc = pytest.importorskip("paper_2101_07731_gb300")
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
DF_RTOL = 1e-9


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def _set(kind, M, N, L, D, seed, n_proto=5, sigma=0.1):
    spec = synth.SeriesSpec(kind, L, D, seed, n_proto=n_proto, sigma=sigma)
    return synth.generate(spec, synth.ROLE_QUERY, M), synth.generate(spec, synth.ROLE_CAND, N)


def _lb_rtol(L, D):
    """The round-down bar of the LB_MV tests: chains of at most D + 32 + L*D/32 + 8
    round-down operations, 2^-23 relative each; 1e-5 at least."""
    return max(1e-5, (D + 32 + (L * D + 31) // 32 + 8) * 2.0 ** -23)


def _oracle_lb(Q, Cn, W):
    return np.array([[O.lb_mv(q, c, W) for c in Cn] for q in Q])


def _check_contract(out, ref, thr, L, D):
    """Returns how many pairs hold a partial (abandoned) sum."""
    rt = _lb_rtol(L, D)
    lo = ref * (1 - rt) - 1e-6
    thr = thr[:, None].astype(np.float64)
    assert np.all(out <= ref * (1 + 1e-12) + 1e-30), np.argwhere(out > ref * (1 + 1e-12) + 1e-30)[:5]
    under = ref <= thr
    assert np.all(out[under] >= lo[under]), "a bound at or under its threshold was not completed"
    over = lo > thr
    assert np.all(out[over] > np.broadcast_to(thr, out.shape)[over]), "an abandoned value is not above the threshold"
    # between the two: complete, or partial above the threshold
    mid = ~under & ~over
    ok = (out >= lo) | (out > thr)
    assert np.all(ok[mid])
    return int(np.sum(out < lo))


@pytest.mark.parametrize("kind,M,N,L,D,W,q", [
    ("random_walk", 70, 600, 67, 3, 6, 0.1),     # E = 201: 4-byte copies, ragged last chunk
    ("random_walk", 70, 600, 67, 3, 6, None),    # threshold +inf: every pair complete, two rounds per tile
    ("proto_warp", 300, 40, 40, 4, 4, 0.5),      # 300 queries: two query passes per tile
    ("proto_warp", 20, 300, 512, 8, 51, 0.05),   # long rows: pairs abandoned inside the completion too
    ("proto_warp", 9, 257, 64, 4, 6, 0.2),       # E = 256: 16-byte copies; ragged candidate tiles
    ("random_walk", 5, 100, 30, 3, 3, 0.3),      # E = 90: too short to abandon, summed whole
])
def test_lb_mv_abandon_contract(kind, M, N, L, D, W, q):
    Q, Cn = _set(kind, M, N, L, D, 40 + M)
    ref = _oracle_lb(Q, Cn, W)
    thr = np.full(M, np.inf, np.float32) if q is None else np.quantile(ref, q, axis=1).astype(np.float32)
    out = tc.lb_mv_abandon(_gpu(Q), _gpu(Cn), W, _gpu(thr)).cpu().numpy().astype(np.float64)
    partial = _check_contract(out, ref, thr, L, D)
    if q is None or L * D < 128:
        assert partial == 0
    else:
        assert partial > 0, "no pair was abandoned"


def test_lb_mv_abandon_complete_values_match_the_plain_stream():
    # with no threshold every value is the complete bound: the same bound as
    # tcdtw_lower_bounds up to the summation order
    Q, Cn = _set("proto_warp", 37, 450, 96, 5, 8, 77)
    inf = torch.full((37,), float("inf"), device=DEV)
    a = tc.lb_mv_abandon(_gpu(Q), _gpu(Cn), 8, inf).cpu().numpy().astype(np.float64)
    b = tc.lower_bounds(_gpu(Q), _gpu(Cn), 8, which=tc.LB_MV).cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(a, b, rtol=2 * _lb_rtol(96, 5), atol=1e-6)


def test_lb_mv_completion_wait_limit_selftest():
    # a completion launch whose producer issues nothing: its consumers' first wait runs
    # out, the launch reports TIMEOUT and ends, and the context stays usable
    assert tc.lb_mv_rest_selftest_timeout(2000) == tc.ERR_TIMEOUT
    Q, Cn = _set("proto_warp", 33, 200, 128, 4, 91)
    ref = _oracle_lb(Q, Cn, 6)
    thr = np.quantile(ref, 0.2, axis=1).astype(np.float32)
    out = tc.lb_mv_abandon(_gpu(Q), _gpu(Cn), 6, _gpu(thr)).cpu().numpy().astype(np.float64)
    _check_contract(out, ref, thr, 128, 4)


def _check_nn(Q, Cn, W, K=16, **opts):
    index = tc.Index(_gpu(Cn), W, K, **opts)
    idx, dist, st = index.nn(_gpu(Q), stats=True)
    index.close()
    ridx, rdist = O.nn_brute(Q, Cn, W)
    gi, gd = idx.cpu().numpy(), dist.cpu().numpy()
    assert np.array_equal(gi, ridx), np.nonzero(gi != ridx)
    np.testing.assert_allclose(gd, rdist, rtol=DF_RTOL, atol=0)
    assert (st["pruned_mv"] + st["pruned_pc"] + st["pruned_ti"] + st["pruned_rev"] + st["dtw_started"] ==
            st["pairs"]), st
    return st


@pytest.mark.parametrize("mv_abandon", [0, 1])
@pytest.mark.parametrize("kind,M,N,L,D,W,n_proto", [
    ("proto_warp", 40, 2000, 128, 5, 13, 20),    # prototype classes: most pairs abandon after the sample
    ("random_walk", 36, 500, 100, 3, 10, 0),     # loose LB_MV: most pairs complete
    ("proto_warp", 32, 500, 200, 32, 20, 8),     # wide points (ring DTW tile)
    ("proto_warp", 7, 300, 64, 4, 6, 5),         # a block of fewer than 32 queries: never abandons
])
def test_nn_with_and_without_abandoning(mv_abandon, kind, M, N, L, D, W, n_proto):
    Q, Cn = _set(kind, M, N, L, D, 60 + M, n_proto=n_proto)
    _check_nn(Q, Cn, W, 8, mv_abandon=mv_abandon)


def test_nn_abandoning_counts_both_seed_rounds():
    # a block of 40 queries: two seed rounds of seed_s each; every pair is still
    # accounted for exactly once, the second round's DTWs are among those started, and
    # fewer LB_MV terms are summed than pairs x L x D (all of them without abandoning)
    M, N, L, D = 40, 1500, 96, 4
    Q, Cn = _set("proto_warp", M, N, L, D, 70, n_proto=10)
    st1 = _check_nn(Q, Cn, 9, 8, mv_abandon=1, seed_s=3, select=0)
    st0 = _check_nn(Q, Cn, 9, 8, mv_abandon=0, seed_s=3, select=0)
    assert st1["dtw_started"] >= M * 6 and st0["dtw_started"] >= M * 3
    assert st0["mv_terms"] == M * N * L * D
    assert M * N * 32 <= st1["mv_terms"] < 0.5 * M * N * L * D
