"""GPU parity of the search pipeline against the FP64 oracle, stage by stage and
end to end.

Bars: envelopes, LB_PC boxes, box counts and compaction are bit-exact; lower
bounds are rounded down (never above the FP64 bound, never above the FP64 DTW) and
within 1e-5 relative of it, or of the directed-rounding error bound where that is
larger (see _lb_rtol); NN indices are bit-exact (ties to the smallest index)
and distances within 1e-5 relative of FP64.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

tc = pytest.importorskip("paper_2101_07731_gb300")
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
RTOL = 1e-5
# Returned distances come from the double-float recompute, whose proven relative
# error is below ~2e-10 at these sizes (or from FP64 itself): far inside RTOL.
DF_RTOL = 1e-9


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def _set(kind, M, N, L, D, seed, n_proto=5, sigma=0.1):
    spec = synth.SeriesSpec(kind, L, D, seed, n_proto=n_proto, sigma=sigma)
    return synth.generate(spec, synth.ROLE_QUERY, M), synth.generate(spec, synth.ROLE_CAND, N)


# ------------------------------------------------------------------ stages

@pytest.mark.parametrize("M,L,D,W", [(5, 70, 3, 7), (3, 257, 5, 26), (2, 40, 12, 0), (2, 33, 2, 100),
                                     (4, 1, 3, 0), (2, 300, 32, 30), (2, 2048, 32, 102), (3, 205, 7, 102),
                                     (2, 9000, 1, 50), (2, 600, 64, 299)])
def test_envelope_bit_exact(M, L, D, W):
    Q, _ = _set("random_walk", M, 1, L, D, 11)
    U, Lo = tc.envelope(_gpu(Q), W)
    U, Lo = U.cpu().numpy(), Lo.cpu().numpy()
    for m in range(M):
        rU, rL = O.envelope(Q[m], W)
        assert np.array_equal(U[m].astype(np.float64), rU)
        assert np.array_equal(Lo[m].astype(np.float64), rL)


def test_query_dq_interval_contains_exact():
    Q, _ = _set("random_walk", 4, 1, 97, 6, 12)
    lo, hi = tc.query_dq(_gpu(Q))
    lo, hi = lo.cpu().numpy().astype(np.float64), hi.cpu().numpy().astype(np.float64)
    for m in range(4):
        ref = O.query_dq(Q[m])
        assert np.all(lo[m] <= ref) and np.all(ref <= hi[m])
        np.testing.assert_allclose(lo[m], ref, rtol=1e-6)
        np.testing.assert_allclose(hi[m], ref, rtol=1e-6)


@pytest.mark.parametrize("L,D,W,K,Lq,w", [(64, 3, 5, 4, 2, 6), (256, 5, 26, 16, 2, 6), (100, 4, 9, 3, 3, 4),
                                          (50, 2, 60, 8, 2, 1), (90, 32, 10, 64, 2, 6), (30, 6, 3, 1, 2, 6)])
def test_pc_boxes_bit_exact(L, D, W, K, Lq, w):
    Q, _ = _set("proto_warp", 3, 1, L, D, 13)
    boxes, counts = tc.pc_boxes(_gpu(Q), W, K, Lq, w)
    boxes, counts = boxes.cpu().numpy(), counts.cpu().numpy()
    for m in range(3):
        rb, rc = O.pc_boxes(Q[m], W, K, Lq, w)
        assert np.array_equal(counts[m], rc)
        for g in range(len(rc)):
            assert np.array_equal(boxes[m, g, :rc[g]].astype(np.float64), rb[g, :rc[g]])


def _lb_rtol(L, D):
    """Closeness bar for a rounded-down bound: every operation rounds the same
    way, so errors add up instead of cancelling.  The longest chain of round-down
    operations feeding one bound is at most D (one point's terms) + 32 (one chunk or
    one lane's points) + L*D/32 (chunk sums) + 8 (warp reduction, sqrt), each
    costing at most 2^-23 relative; 1e-5 is the floor."""
    return max(1e-5, (D + 32 + (L * D + 31) // 32 + 8) * 2.0 ** -23)


@pytest.mark.parametrize("which", [tc.LB_MV, tc.LB_PC, tc.LB_TI])
@pytest.mark.parametrize("L,D,W", [(64, 3, 6), (129, 5, 13), (50, 8, 0), (40, 2, 60), (70, 33, 7)])
def test_lower_bounds_rounded_down_and_close(which, L, D, W):
    Q, Cn = _set("proto_warp", 4, 37, L, D, 14)
    K = 8
    out = tc.lower_bounds(_gpu(Q), _gpu(Cn), W, which=which, K=K).cpu().numpy().astype(np.float64)
    for m in range(4):
        for n in range(37):
            if which == tc.LB_MV:
                ref = O.lb_mv(Q[m], Cn[n], W)
            elif which == tc.LB_PC:
                ref = O.lb_pc(Q[m], Cn[n], W, K, 2, 6)
            else:
                ref = O.lb_ti(Q[m], Cn[n], W, 5)
            g = out[m, n]
            assert g <= ref * (1 + 1e-12) + 1e-30, (m, n, g, ref)
            tol = ref * _lb_rtol(L, D) + 1e-6
            if which == tc.LB_TI:   # exact cells widened, carried through the recursion
                tol = max(tol, _ti_chain_tol(Q[m], Cn[n]))
            assert g >= ref - tol, (m, n, g, ref)
    # never above the DTW distance
    for m in range(2):
        for n in range(10):
            assert out[m, n] <= O.dtw(Q[m], Cn[n], W) * (1 + 1e-12)


def test_lower_bounds_large_ragged_lb_mv():
    # several CTA tiles of candidates and queries, E = L*D not a multiple of 32 or of 4
    Q, Cn = _set("random_walk", 45, 300, 67, 3, 15)
    out = tc.lower_bounds(_gpu(Q), _gpu(Cn), 6, which=tc.LB_MV).cpu().numpy().astype(np.float64)
    for m in (0, 17, 44):
        for n in (0, 127, 128, 299):
            ref = O.lb_mv(Q[m], Cn[n], 6)
            assert out[m, n] <= ref * (1 + 1e-12) and out[m, n] >= ref * (1 - _lb_rtol(67, 3)) - 1e-6


@pytest.mark.parametrize("M", [1, 2, 3, 5, 8, 13, 16, 17, 33, 70])
def test_lower_bounds_lb_mv_tma_stream(M):
    # E = L*D a multiple of 4 (the bulk-tensor stream) but not of 32 (a ragged last
    # chunk), several candidate tiles with a ragged last tile, every query-tile width
    L, D, W, N = 67, 4, 7, 300
    Q, Cn = _set("proto_warp", M, N, L, D, 16 + M)
    out = tc.lower_bounds(_gpu(Q), _gpu(Cn), W, which=tc.LB_MV).cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(M)
    ms = sorted({0, M - 1, *rng.integers(0, M, 3).tolist()})
    ns = sorted({0, 127, 128, 255, 256, N - 1, *rng.integers(0, N, 4).tolist()})
    for m in ms:
        for n in ns:
            ref = O.lb_mv(Q[m], Cn[n], W)
            assert out[m, n] <= ref * (1 + 1e-12) + 1e-30, (m, n, out[m, n], ref)
            assert out[m, n] >= ref * (1 - _lb_rtol(L, D)) - 1e-6, (m, n, out[m, n], ref)


@pytest.mark.parametrize("M,N,L,D", [(1, 40, 67, 4), (5, 130, 67, 4), (2, 7, 8, 4), (16, 129, 300, 8)])
def test_lower_bounds_lb_mv_tma_shared_tiles(M, N, L, D):
    # few candidate tiles: the stream-K split gives each tile several CTAs (N = 40,
    # E = 268: one tile of 9 chunks over 9 CTAs), whose parts the last one adds up
    W = 5
    Q, Cn = _set("proto_warp", M, N, L, D, 26 + M)
    out = tc.lower_bounds(_gpu(Q), _gpu(Cn), W, which=tc.LB_MV).cpu().numpy().astype(np.float64)
    for m in range(M):
        for n in range(N):
            ref = O.lb_mv(Q[m], Cn[n], W)
            assert out[m, n] <= ref * (1 + 1e-12) + 1e-30, (m, n, out[m, n], ref)
            assert out[m, n] >= ref * (1 - _lb_rtol(L, D)) - 1e-6, (m, n, out[m, n], ref)


def test_lb_mv_tma_wait_limit_selftest():
    # the consumers' first wait runs out; the launch reports TIMEOUT and the context
    # stays usable for the next call
    assert tc.lb_mv_selftest_timeout(20000) == tc.ERR_TIMEOUT
    Q, Cn = _set("proto_warp", 2, 40, 32, 4, 17)
    out = tc.lower_bounds(_gpu(Q), _gpu(Cn), 3, which=tc.LB_MV).cpu().numpy().astype(np.float64)
    ref = O.lb_mv(Q[1], Cn[39], 3)
    assert out[1, 39] <= ref * (1 + 1e-12) + 1e-30 and out[1, 39] >= ref * (1 - _lb_rtol(32, 4)) - 1e-6


@pytest.mark.parametrize("M,N,L,D,W", [(4, 37, 64, 3, 6), (3, 130, 129, 5, 13), (2, 20, 50, 8, 0), (3, 25, 40, 2, 60),
                                       (2, 9, 70, 33, 7), (2, 600, 96, 1, 9)])
def test_lower_bounds_candidate_side_lb_mv(M, N, L, D, W):
    # the reverse bound is LB_MV with the roles exchanged: the candidate's envelope,
    # summed over the query's points
    Q, Cn = _set("proto_warp", M, N, L, D, 18)
    out = tc.lower_bounds(_gpu(Q), _gpu(Cn), W, which=tc.LB_MV_REV).cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(N)
    for m in range(M):
        for n in sorted({0, N - 1, *rng.integers(0, N, 6).tolist()}):
            ref = O.lb_mv(Cn[n], Q[m], W)
            assert out[m, n] <= ref * (1 + 1e-12) + 1e-30, (m, n, out[m, n], ref)
            assert out[m, n] >= ref * (1 - _lb_rtol(L, D)) - 1e-6, (m, n, out[m, n], ref)
            assert out[m, n] <= O.dtw(Q[m], Cn[n], W) * (1 + 1e-12) + 1e-30


def _ti_chain_tol(q, c):
    """Closeness bar of the FP32 triangle recursions without periodic exact rows: every
    step rounds Ub up and Lb down (4 roundings of at most 2^-24 relative), a chain is at
    most L steps long, and Lb = dc - Ub can cancel, so a column minimum may sit up to
    4 L 2^-24 Umax below its FP64 value, Umax bounding every Ub (the sum of all neighbour
    distances of both series plus the largest point distance); an exact cell from one
    rounded square root is widened by (D + 4) 2^-24 of its value (<= Umax) on top.
    Summed over the L squared minima (m <= Umax): 2 L Umax err + L err^2."""
    q, c = q.astype(np.float64), c.astype(np.float64)
    L, D = q.shape
    umax = (np.linalg.norm(np.diff(q, axis=0), axis=1).sum() + np.linalg.norm(np.diff(c, axis=0), axis=1).sum()
            + np.linalg.norm(q[:, None, :] - c[None, :, :], axis=2).max())
    err = (4.0 * L + D + 4) * 2.0 ** -24 * umax
    return 2.0 * L * umax * err + L * err * err


@pytest.mark.parametrize("L,D,W", [(40, 3, 0), (48, 1, 1), (64, 3, 6), (129, 5, 26), (70, 8, 60), (90, 2, 100),
                                   (35, 33, 7)])
@pytest.mark.parametrize("P,top", [(1000, 0), (5, 0), (1000, 1)])
def test_lower_bounds_lb_ti_variants(L, D, W, P, top):
    # basic LB_TI (P >= L, window tops from the candidate-side triangle), LB_TIP (P = 5)
    # and LB_TI_TOP (exact tops, P >= L) against the oracle's variants
    Q, Cn = _set("proto_warp", 3, 9, L, D, 19)
    out = tc.lower_bounds(_gpu(Q), _gpu(Cn), W, which=tc.LB_TI, P=P, ti_top=top).cpu().numpy().astype(np.float64)
    for m in range(3):
        for n in range(9):
            ref = O.lb_ti_var(Q[m], Cn[n], W, P, top)
            g = out[m, n]
            assert g <= ref * (1 + 1e-12) + 1e-30, (m, n, g, ref)
            assert g >= ref - _ti_chain_tol(Q[m], Cn[n]), (m, n, g, ref)


@pytest.mark.parametrize("L,W", [(3, 1), (40, 0), (40, 3), (129, 26), (96, 60), (150, 100)])
def test_lower_bounds_lb_ti_variants_exact_on_small_integers(L, W):
    # D = 1 and small integer values: every distance, neighbour distance and recursion
    # step is an exact integer in FP32 (a square root of a perfect square is exact),
    # so the variants with triangle window tops (top = 0) must equal the oracle exactly,
    # however long their triangle chains.  With exact window tops (top = 1) the exact
    # cells come from one correctly rounded square root widened by k = (D + 4) 2^-24
    # (exact_interval): those bounds may sit below the oracle by at most what that
    # widening, carried through the recursion and squared, allows -- and never above.
    rng = np.random.default_rng(L + W)
    if L == 3:  # the hand-worked example (tests/golden/ti_variants_hand.txt)
        Q = np.array([[[0.], [1.], [2.]]], np.float32)
        Cn = np.array([[[0.], [0.], [-5.]]], np.float32)
    else:
        Q = np.clip(np.cumsum(rng.integers(-2, 3, (3, L, 1)), axis=1), -60, 60).astype(np.float32)
        Cn = (np.clip(np.cumsum(rng.integers(-3, 4, (5, L, 1)), axis=1), -40, 40) + 25).astype(np.float32)
    k = 5 * 2.0 ** -24
    dmax = float(np.abs(Q.max() - Cn.min())) + float(np.abs(Cn.max() - Q.min()))
    for P, top in ((1000, 0), (2, 0), (5, 0), (1000, 1), (5, 1)):
        out = tc.lower_bounds(_gpu(Q), _gpu(Cn), W, which=tc.LB_TI, P=P, ti_top=top).cpu().numpy()
        for m in range(len(Q)):
            for n in range(len(Cn)):
                ref = O.lb_ti_var(Q[m], Cn[n], W, P, top)
                if top == 0:
                    assert float(out[m, n]) == ref, (P, top, m, n)
                else:
                    assert ref - L * (2 * dmax * dmax * k + 1e-6) <= float(out[m, n]) <= ref, (P, top, m, n)
    if L == 3:
        got = [float(tc.lower_bounds(_gpu(Q), _gpu(Cn), 1, which=tc.LB_TI, P=P, ti_top=t).item())
               for P, t in ((3, 0), (3, 1), (2, 0), (2, 1))]
        assert got[0] == 9.0 and got[2] == 16.0
        assert 25.0 * (1 - 4 * k) <= got[1] <= 25.0 and 36.0 * (1 - 4 * k) <= got[3] <= 36.0


def test_compact_bit_exact():
    rng = np.random.default_rng(0)
    lb = rng.random((7, 1000)).astype(np.float32)
    lb[3, :] = np.inf
    thr = np.array([0.1, 0.5, 0.0, 1.0, 2.0, 0.25, 0.999], np.float32)
    idx, cnt = tc.compact(_gpu(lb), _gpu(thr))
    idx, cnt = idx.cpu().numpy(), cnt.cpu().numpy()
    for m in range(7):
        ref = np.nonzero(lb[m] <= thr[m])[0]
        assert cnt[m] == len(ref)
        assert np.array_equal(idx[m, :cnt[m]], ref)


# ------------------------------------------------------------------ end to end

def _check_nn(Q, Cn, W, K=16, **opts):
    index = tc.Index(_gpu(Cn), W, K, **opts)
    idx, dist, st = index.nn(_gpu(Q), stats=True)
    index.close()
    ridx, rdist = O.nn_brute(Q, Cn, W)
    gi, gd = idx.cpu().numpy(), dist.cpu().numpy()
    assert np.array_equal(gi, ridx), np.nonzero(gi != ridx)
    np.testing.assert_allclose(gd, rdist, rtol=DF_RTOL, atol=0)
    M, N = len(Q), len(Cn)
    assert st["pairs"] == M * N
    assert (st["pruned_mv"] + st["pruned_pc"] + st["pruned_ti"] + st["pruned_rev"] + st["dtw_started"] ==
            st["pairs"]), st
    assert st["refined"] >= M
    assert st["refined64"] <= st["refined"]
    return gd, rdist, st


def test_nn_rw_16x256_L128_D3_W13_exact():
    wl = synth.RW_16x256_L128
    gd, rd, st = _check_nn(wl.queries(), wl.candidates(), wl.W, wl.K)
    # no near-ties on random walks: double-float separates every query's best
    # candidate, so FP64 never runs, and the distances are within its error bound
    assert st["refined64"] == 0
    np.testing.assert_allclose(gd, rd, rtol=1e-11, atol=0)


@pytest.mark.parametrize("use_pc,use_ti", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_nn_proto_warp_cascade_settings(use_pc, use_ti):
    Q, Cn = _set("proto_warp", 24, 1500, 96, 4, 21, n_proto=6)
    _check_nn(Q, Cn, 10, 8, use_pc=use_pc, use_ti=use_ti, e_pc=0.0, e_ti=0.0)


@pytest.mark.parametrize("seed_s,qblock", [(1, 7), (8, 0), (3, 32)])
def test_nn_query_blocks_and_seeds(seed_s, qblock):
    Q, Cn = _set("proto_warp", 50, 700, 64, 3, 22)
    _check_nn(Q, Cn, 6, 8, seed_s=seed_s, qblock=qblock)


@pytest.mark.parametrize("M,N,L,D,W", [(1, 1, 16, 2, 3), (3, 5, 1, 3, 0), (4, 9, 20, 1, 0), (5, 40, 30, 2, 100),
                                       (2, 300, 50, 12, 5), (2, 80, 40, 32, 4), (2, 60, 24, 64, 3),
                                       (3, 150, 60, 9, 6), (4, 130, 70, 10, 30), (2, 90, 33, 11, 3),
                                       (3, 200, 120, 32, 30), (2, 150, 300, 16, 40), (3, 120, 97, 21, 25),
                                       (2, 100, 64, 44, 20),
                                       # long bands: the refine's cost table in global memory
                                       (2, 60, 400, 3, 150), (3, 80, 300, 6, 70)])
def test_nn_edge_shapes(M, N, L, D, W):
    Q, Cn = _set("random_walk", M, N, L, D, 23)
    _check_nn(Q, Cn, W, 4)


def test_nn_candidate_side_bound_keeps_answers():
    # use_rev adds the candidate-side LB_MV to the cascade: different pruning, same NN
    Q, Cn = _set("proto_warp", 30, 1200, 80, 4, 33, n_proto=6)
    gd, rd, st = _check_nn(Q, Cn, 8, 8, use_rev=1, select=0)
    plain = tc.Index(_gpu(Cn), 8, 8, use_rev=0, select=0)
    i0, d0, st0 = plain.nn(_gpu(Q), stats=True)
    plain.close()
    assert st["pruned_rev"] >= 0 and st0["pruned_rev"] == 0
    np.testing.assert_array_equal(gd, d0.cpu().numpy())
    # random walks: the two envelopes differ, so the reverse bound prunes some pairs
    Q2, C2 = _set("random_walk", 12, 800, 64, 2, 34)
    _, _, st2 = _check_nn(Q2, C2, 6, 4, use_rev=1, select=0, use_pc=0, use_ti=0)
    assert st2["pruned_rev"] > 0


@pytest.mark.parametrize("P", [5, 1000])
def test_nn_lb_ti_without_exact_tops_keeps_answers(P):
    # LB_TIP (P = 5) and the basic LB_TI (P >= L) in the cascade, on every survivor
    Q, Cn = _set("proto_warp", 20, 900, 72, 3, 35, n_proto=6)
    _check_nn(Q, Cn, 7, 8, use_pc=0, use_ti=1, ti_top=0, P=P, e_ti=0.0, select=0)


@pytest.mark.parametrize("use_pc,use_ti,ti_top", [(1, 0, 1), (0, 1, 1), (0, 1, 0)])
def test_nn_tight_bounds_prune_on_smooth_series(use_pc, use_ti, ti_top):
    """On smooth 2-D circles of different radii the query envelope is a loose box
    around an arc, so LB_MV lets through pairs that the point-based bounds reject:
    LB_PC (Section 5), LB_TI in its TIP_TOP form and LB_TIP (Section 4.2, P = 5) each
    prune pairs inside the GPU pipeline (the oracle's pairwise bounds, evaluated in
    the pipeline's order on the same data, prune 713, 261 and 260 of 1,534 LB_MV
    survivors), and the answers stay the oracle's."""
    spec = synth.SeriesSpec("circle", 96, 2, 51, sigma=0.01)
    Q, Cn = synth.generate(spec, synth.ROLE_QUERY, 12), synth.generate(spec, synth.ROLE_CAND, 500)
    _, _, st = _check_nn(Q, Cn, 12, 8, use_pc=use_pc, use_ti=use_ti, ti_top=ti_top, P=5, e_pc=0.0, e_ti=0.0,
                         select=0)
    if use_pc:
        assert st["pruned_pc"] > 0, st
    if use_ti:
        assert st["pruned_ti"] > 0, st


def test_sharded_index_single_rank_nccl():
    # the candidate-sharded search through a real process group (NCCL, one rank: the
    # shard is the whole set, offset 0) equals the plain index
    import os
    import socket
    import torch.distributed as dist
    from paper_2101_07731_gb300.sharded import ShardedIndex
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda:0"))
    try:
        Q, Cn = _set("proto_warp", 10, 400, 48, 3, 37)
        sh = ShardedIndex(_gpu(Cn), 0, 5, 8)
        gi, gd = sh.nn(_gpu(Q))
        sh.close()
        ridx, rdist = O.nn_brute(Q, Cn, 5)
        assert np.array_equal(gi.cpu().numpy(), ridx)
        np.testing.assert_allclose(gd.cpu().numpy(), rdist, rtol=DF_RTOL, atol=0)
    finally:
        dist.destroy_process_group()


def test_nn_tc_dtw_selection_keeps_answers():
    # TC-DTW's data-adaptive bound choice changes which DTWs run, never the answer
    Q, Cn = _set("proto_warp", 40, 2000, 80, 4, 31, n_proto=6)
    fixed = tc.Index(_gpu(Cn), 8, 8, select=0)
    i0, d0 = fixed.nn(_gpu(Q))
    assert fixed.options()["use_pc"] == 1 and fixed.options()["use_ti"] == 1
    fixed.close()
    chosen = tc.Index(_gpu(Cn), 8, 8)
    i1, d1 = chosen.nn(_gpu(Q))
    opts = chosen.options()
    assert not (opts["use_pc"] and opts["use_ti"])      # one of the two bounds, or LB_MV alone
    if opts["use_ti"]:
        assert opts["e_ti"] in (pytest.approx(0.05), pytest.approx(0.1), pytest.approx(0.2))
    if opts["use_pc"]:
        assert opts["Lq"] in (2, 3) and opts["e_pc"] in (pytest.approx(0.1), pytest.approx(0.5))
    i2, d2 = chosen.nn(_gpu(Q))                            # the choice is kept
    assert chosen.options() == opts
    chosen.close()
    assert torch.equal(i0, i1) and torch.equal(i1, i2)
    assert torch.equal(d0, d1) and torch.equal(d1, d2)
    ridx, rdist = O.nn_brute(Q, Cn, 8)
    assert np.array_equal(i1.cpu().numpy(), ridx)


def test_nn_duplicates_tie_to_smallest_index():
    _, Cn = _set("random_walk", 1, 64, 40, 3, 24)
    Cn = np.concatenate([Cn, Cn[[10, 5, 10]]])          # copies at 64, 65, 66
    Q = (Cn[[10, 5, 33]] + np.float32(0.01)).astype(np.float32)
    index = tc.Index(_gpu(Cn), 4, 4)
    idx, dist = index.nn(_gpu(Q))
    assert idx.cpu().tolist() == [10, 5, 33]
    # the query equal to a candidate: distance 0, smallest duplicate index
    idx2, dist2 = index.nn(_gpu(Cn[[65, 66]]))
    assert idx2.cpu().tolist() == [5, 10] and dist2.cpu().tolist() == [0.0, 0.0]
    # exact duplicates have equal double-float values: FP64 settles them
    _, _, st = index.nn(_gpu(Cn[[65, 66]] + np.float32(0.25)), stats=True)
    assert st["refined64"] >= 4, st


def test_nn_constant_series():
    Cn = np.zeros((20, 32, 3), np.float32)
    Cn[7] += 1.0
    Q = np.zeros((2, 32, 3), np.float32)
    Q[1] += 0.9
    index = tc.Index(_gpu(Cn), 3, 4)
    idx, dist = index.nn(_gpu(Q))
    assert idx.cpu().tolist() == [0, 7]


def test_nn_rejects_non_finite():
    Q, Cn = _set("random_walk", 2, 30, 20, 2, 25)
    Cbad = Cn.copy()
    Cbad[3, 4, 1] = np.nan
    with pytest.raises(tc.TcdtwError) as ei:
        tc.Index(_gpu(Cbad), 3, 4)
    assert ei.value.code == 5
    index = tc.Index(_gpu(Cn), 3, 4)
    Qbad = Q.copy()
    Qbad[1, 0, 0] = np.inf
    with pytest.raises(tc.TcdtwError) as ei:
        index.nn(_gpu(Qbad))
    assert ei.value.code == 5
    # the index stays usable
    idx, _ = index.nn(_gpu(Q))
    ridx, _ = O.nn_brute(Q, Cn, 3)
    assert np.array_equal(idx.cpu().numpy(), ridx)


def test_nn_proto_256x20000_L256_D5_W26_all_queries():
    """The full 256 x 20,000 search (L=256, D=5, W=26, K=16) against the oracle for
    every query: the oracle's pruned search (LB_MV and early abandoning, pinned equal
    to brute force) over all 20,000 candidates."""
    wl = synth.PROTO_256x20000_L256
    Q, Cn = wl.queries(), wl.candidates()
    index = tc.Index(_gpu(Cn), wl.W, wl.K)
    idx, dist, st = index.nn(_gpu(Q), stats=True)
    index.close()
    gi, gd = idx.cpu().numpy(), dist.cpu().numpy()
    ridx, rdist, _ = O.nn_pruned(Q, Cn, wl.W, K=wl.K, use_pc=False, use_ti=False)
    assert np.array_equal(gi, ridx), np.nonzero(gi != ridx)
    np.testing.assert_allclose(gd, rdist, rtol=DF_RTOL, atol=0)
    assert st["pruned_mv"] + st["pruned_pc"] + st["pruned_ti"] + st["dtw_started"] == st["pairs"]
    # pruning must avoid most DTWs on this prototype data
    assert st["dtw_started"] < 0.5 * st["pairs"]


def test_nn_graph_replay_with_new_query_contents():
    """Repeated calls with the same buffers run eagerly once, then capture and
    replay a CUDA graph; the graph reads whatever the buffers hold at replay time."""
    spec = synth.SeriesSpec("proto_warp", 80, 4, 27, n_proto=5, sigma=0.1)
    Cn = synth.generate(spec, synth.ROLE_CAND, 900)
    index = tc.Index(_gpu(Cn), 8, 8)
    q = torch.empty(19, 80, 4, dtype=torch.float32, device=DEV)
    idx = torch.empty(19, dtype=torch.int64, device=DEV)
    dist = torch.empty(19, dtype=torch.float64, device=DEV)
    for rep in range(4):
        Qn = synth.generate(spec, synth.ROLE_QUERY, 19, start=19 * rep)
        q.copy_(torch.from_numpy(Qn))
        index.nn(q, out=(idx, dist))
        ridx, rdist = O.nn_brute(Qn, Cn, 8)
        assert np.array_equal(idx.cpu().numpy(), ridx), rep
        np.testing.assert_allclose(dist.cpu().numpy(), rdist, rtol=DF_RTOL, atol=0)
    index.close()


def test_nn_graph_replay_with_fresh_buffers_every_call():
    """A caller that allocates new query and answer tensors for every call (the
    caching allocator hands out alternating addresses) still gets the replayed graph's
    answers right: the graph runs on the index's own buffers, keyed by the query count."""
    spec = synth.SeriesSpec("proto_warp", 64, 3, 28, n_proto=5, sigma=0.1)
    Cn = synth.generate(spec, synth.ROLE_CAND, 700)
    index = tc.Index(_gpu(Cn), 6, 8)
    keep = []
    for rep in range(5):
        Qn = synth.generate(spec, synth.ROLE_QUERY, 13, start=13 * rep)
        q = _gpu(Qn)
        idx, dist = index.nn(q)
        keep.append((q, idx, dist))                    # keep the buffers alive: new addresses
        ridx, rdist = O.nn_brute(Qn, Cn, 6)
        assert np.array_equal(idx.cpu().numpy(), ridx), rep
        np.testing.assert_allclose(dist.cpu().numpy(), rdist, rtol=DF_RTOL, atol=0)
    # a different query count gets its own graph; the first one stays valid
    Qn = synth.generate(spec, synth.ROLE_QUERY, 5, start=200)
    for _ in range(3):
        idx, _ = index.nn(_gpu(Qn))
        assert np.array_equal(idx.cpu().numpy(), O.nn_brute(Qn, Cn, 6)[0])
    index.close()


def test_allocation_failures_are_reported_and_leak_nothing():
    """Allocation failure injected on the host (tcdtw_inject_alloc_failure): building an
    index with every possible allocation failing in turn returns TCDTW_ERR_NOMEM and
    frees what was allocated; a search and a stage call whose allocation fails do the
    same; afterwards the context and the index are fully usable."""
    lib = tc._load()
    spec = synth.SeriesSpec("proto_warp", 48, 3, 29, n_proto=4, sigma=0.1)
    Qn, Cn = synth.generate(spec, synth.ROLE_QUERY, 9), synth.generate(spec, synth.ROLE_CAND, 300)
    cand, q = _gpu(Cn), _gpu(Qn)
    out = (torch.empty(9, dtype=torch.int64, device=DEV), torch.empty(9, dtype=torch.float64, device=DEV))
    ridx, _ = O.nn_brute(Qn, Cn, 5)
    # warm up everything a first use loads or caches (modules, the tile cache, torch's pool)
    x = tc.Index(cand, 5, 8)
    for _ in range(3):
        x.nn(q, out=out)
    x.close()
    tc.lower_bounds(q, cand, 5)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    try:
        for n in range(400):
            lib.tcdtw_inject_alloc_failure(n)
            try:
                x = tc.Index(cand, 5, 8)
            except tc.TcdtwError as e:
                assert e.code == tc.ERR_NOMEM, e
                failed += 1
                continue
            break
        torch.cuda.synchronize()
        lib.tcdtw_inject_alloc_failure(0)
        with pytest.raises(tc.TcdtwError) as ei:        # the first search allocates (TC-DTW's choice)
            x.nn(q, out=out)
        assert ei.value.code == tc.ERR_NOMEM
        with pytest.raises(tc.TcdtwError) as ei:        # a stage call with its own scratch
            tc.lower_bounds(q, cand, 5)
        assert ei.value.code == tc.ERR_NOMEM
    finally:
        assert lib.tcdtw_inject_alloc_failure(-1) == 0
    assert failed >= 20, failed                           # every workspace of the index was tried
    for _ in range(3):                                    # usable: selection, eager run, graph replay
        x.nn(q, out=out)
        assert np.array_equal(out[0].cpu().numpy(), ridx)
    x.close()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
