"""Pins of the FP64 oracle to things other than itself (no GPU needed).

Each test checks the oracle against what the paper and the mathematics fix:
exhaustive enumeration of warping paths, closed forms, library routines (scipy
sliding-window filters), invariants and special cases that reduce to another
bound, so that a dropped term, a wrong sign or index or a transposed operand in
the oracle fails at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy.ndimage import maximum_filter1d, minimum_filter1d

import oracle as O
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def rw(n, L, D, seed, role=0):
    return synth.generate(synth.SeriesSpec("random_walk", L, D, seed), role, n)


# ---------------------------------------------------------------- DTW (Eq. 1)

def _enumerate_band_paths(L, W):
    """All warping paths from (0,0) to (L-1,L-1) with steps (1,0),(0,1),(1,1)
    that stay inside |i-j| <= W (brute force, independent of any recurrence)."""
    out = []

    def rec(i, j, path):
        if abs(i - j) > W:
            return
        path.append((i, j))
        if i == L - 1 and j == L - 1:
            out.append(list(path))
        else:
            if i + 1 < L:
                rec(i + 1, j, path)
            if j + 1 < L:
                rec(i, j + 1, path)
            if i + 1 < L and j + 1 < L:
                rec(i + 1, j + 1, path)
        path.pop()

    rec(0, 0, [])
    return out


@pytest.mark.parametrize("L", [1, 2, 3, 5, 6])
@pytest.mark.parametrize("D", [1, 2, 3])
def test_dtw_equals_min_over_enumerated_paths(L, D):
    rng = np.random.default_rng(L * 10 + D)
    for W in sorted({0, 1, 2, L - 1, L + 3}):
        a = rng.standard_normal((L, D)).astype(np.float32)
        b = rng.standard_normal((L, D)).astype(np.float32)
        best = math.inf
        for path in _enumerate_band_paths(L, W):
            s = sum(float(np.sum((a[i].astype(np.float64) - b[j].astype(np.float64)) ** 2))
                    for i, j in path)
            best = min(best, s)
        assert O.dtw(a, b, W) == pytest.approx(best, rel=1e-12, abs=1e-12)


def test_dtw_w0_is_pointwise_sum():
    a, b = rw(2, 64, 4, 3)
    ref = float(np.sum((a.astype(np.float64) - b.astype(np.float64)) ** 2))
    assert O.dtw(a, b, 0) == pytest.approx(ref, rel=1e-13)


def test_dtw_symmetry_and_identity():
    X = rw(6, 40, 3, 5)
    for W in (0, 3, 39):
        for x in X:
            assert O.dtw(x, x, W) == 0.0
        for x, y in itertools.combinations(X, 2):
            assert O.dtw(x, y, W) == pytest.approx(O.dtw(y, x, W), rel=1e-13)


def test_dtw_window_monotone_and_saturates():
    a, b = rw(2, 30, 2, 11)
    vals = [O.dtw(a, b, W) for W in range(0, 32)]
    # a wider band admits more paths: never larger
    assert all(vals[k + 1] <= vals[k] * (1 + 1e-13) for k in range(len(vals) - 1))
    # W >= L-1 is unconstrained
    assert vals[29] == vals[30] == vals[31]


def test_dtw_hand_example_1d():
    """Eq. (1) worked by hand.  a = [0,1,2], b = [0,0,2], W = 1.  In-band costs:
    (0,0)=0 (0,1)=0 (1,0)=1 (1,1)=1 (1,2)=1 (2,1)=4 (2,2)=0, so
    R(0,0)=0, R(0,1)=0, R(1,0)=1, R(1,1)=1+min(0,1,0)=1, R(1,2)=1+min(inf,1,0)=1,
    R(2,1)=4+min(1,inf,1)=5, R(2,2)=0+min(R(1,2)=1, R(2,1)=5, R(1,1)=1)=1."""
    a = np.array([[0], [1], [2]], np.float32)
    b = np.array([[0], [0], [2]], np.float32)
    assert O.dtw(a, b, 1) == 1.0
    assert O.dtw(a, b, 0) == 1.0          # diagonal: 0 + 1 + 0
    # 2-D: a' = [(0,0),(3,4)], b' = [(0,0),(0,0)], W = 1: the path must end at
    # (1,1) with cost 25; the best path is (0,0),(1,1): 0 + 25 = 25.
    a2 = np.array([[0, 0], [3, 4]], np.float32)
    b2 = np.zeros((2, 2), np.float32)
    assert O.dtw(a2, b2, 1) == 25.0


def test_dtw_early_abandon_is_exact_or_inf():
    a, b = rw(2, 50, 3, 21)
    d = O.dtw(a, b, 5)
    assert O.dtw(a, b, 5, abandon_at=d * 1.0001) == d
    assert O.dtw(a, b, 5, abandon_at=d * 0.5) == math.inf


# ---------------------------------------------------------------- envelope / LB_MV

@pytest.mark.parametrize("W", [0, 1, 4, 100])
def test_envelope_matches_scipy_sliding_filters(W):
    q = rw(1, 57, 3, 7)[0]
    U, Lo = O.envelope(q, W)
    size = 2 * min(W, 57) + 1
    for p in range(3):
        # 'nearest' padding repeats edge values, which equals clipping the window
        assert np.array_equal(U[:, p], maximum_filter1d(q[:, p], size, mode="nearest").astype(np.float64))
        assert np.array_equal(Lo[:, p], minimum_filter1d(q[:, p], size, mode="nearest").astype(np.float64))


def test_lb_mv_d1_equals_lb_keogh_with_library_envelope():
    q, c = rw(2, 80, 1, 9)
    W = 6
    u = maximum_filter1d(q[:, 0], 2 * W + 1, mode="nearest").astype(np.float64)
    l = minimum_filter1d(q[:, 0], 2 * W + 1, mode="nearest").astype(np.float64)
    x = c[:, 0].astype(np.float64)
    keogh = float(np.sum(np.where(x > u, (x - u) ** 2, 0) + np.where(x < l, (x - l) ** 2, 0)))
    assert O.lb_mv(q, c, W) == pytest.approx(keogh, rel=1e-13)


# ---------------------------------------------------------------- bound chain

def _bounds(q, c, W, K=16, Lq=2, w=6, P=5):
    return dict(mv=O.lb_mv(q, c, W), ad=O.lb_ad(q, c, W), ti=O.lb_ti(q, c, W, P),
                pc=O.lb_pc(q, c, W, K, Lq, w), pc1=O.lb_pc(q, c, W, K, Lq, 1),
                dtw=O.dtw(q, c, W))


@pytest.mark.parametrize("kind", ["random_walk", "proto_warp"])
def test_lower_bound_chain(kind):
    spec = synth.SeriesSpec(kind, 48, 3, 4, n_proto=3, sigma=0.1)
    Q = synth.generate(spec, synth.ROLE_QUERY, 4)
    Cs = synth.generate(spec, synth.ROLE_CAND, 12)
    eps = 1e-12
    for W in (0, 2, 5, 47):
        for q in Q:
            for c in Cs:
                b = _bounds(q, c, W)
                assert 0.0 <= b["mv"]
                assert b["mv"] <= b["ad"] * (1 + eps) + eps
                assert b["ad"] <= b["dtw"] * (1 + eps) + eps
                assert b["ti"] <= b["ad"] * (1 + eps) + eps
                assert b["pc"] <= b["dtw"] * (1 + eps) + eps
                assert b["mv"] <= b["pc1"] * (1 + eps) + eps
                assert b["pc1"] <= b["ad"] * (1 + eps) + eps


def test_lb_ad_equals_dtw_at_w0():
    q, c = rw(2, 33, 4, 13)
    assert O.lb_ad(q, c, 0) == pytest.approx(O.dtw(q, c, 0), rel=1e-13)


# ---------------------------------------------------------------- LB_TI (Section 4)

def test_lb_ti_period_one_equals_lb_ad():
    Q = rw(3, 40, 3, 15, role=1)
    Cs = rw(5, 40, 3, 15)
    for W in (1, 4, 39):
        for q in Q:
            for c in Cs:
                assert O.lb_ti(q, c, W, 1) == pytest.approx(O.lb_ad(q, c, W), rel=1e-13)


@pytest.mark.parametrize("P", [2, 3, 5, 1000])
def test_lb_ti_exact_on_collinear_monotone_series(P):
    """On a line, with the query increasing and every candidate point beyond the
    query's maximum, the triangle d(q_i,c) = d(q_{i-1},c) - d(q_{i-1},q_i) is
    degenerate and exact, so Lb = Ub = true distance for every P and LB_TI equals
    LB_AD.  A wrong sign, a dropped dq term or a mis-indexed Lb/Ub breaks this."""
    rng = np.random.default_rng(P)
    L, W = 30, 4
    t = np.cumsum(rng.uniform(0.1, 1.0, L))
    dirv = np.array([0.6, -0.8], np.float64)          # unit direction in 2-D
    # exactly representable coordinates: multiples of 1/64
    tq = np.round(t * 64) / 64
    tc = np.round((t.max() + 1 + rng.uniform(0, 5, L)) * 64) / 64
    q = (tq[:, None] * dirv[None, :]).astype(np.float32)
    c = (tc[:, None] * dirv[None, :]).astype(np.float32)
    assert O.lb_ti(q, c, W, P) == pytest.approx(O.lb_ad(q, c, W), rel=1e-9)


def test_lb_ti_dq_is_neighbour_distance():
    q = rw(1, 20, 3, 17)[0].astype(np.float64)
    dq = O.query_dq(q)
    assert dq[0] == 0.0
    assert np.allclose(dq[1:], np.linalg.norm(q[1:] - q[:-1], axis=1), rtol=1e-13)


def _read_golden_ti():
    q = c = None
    vals = []
    with open(os.path.join(HERE, "golden", "ti_variants_hand.txt")) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "query":
                q = np.array([float(x) for x in t[1:]], np.float32)[:, None]
            elif t[0] == "cand":
                c = np.array([float(x) for x in t[1:]], np.float32)[:, None]
            elif t[0] == "lbti":
                vals.append((int(t[1]), int(t[2]), float(t[3])))
    return q, c, vals


def test_lb_ti_variants_hand_worked_example():
    q, c, vals = _read_golden_ti()
    assert len(vals) == 6
    for P, top, want in vals:
        assert O.lb_ti_var(q, c, 1, P, top) == want, (P, top)
    assert O.lb_ad(q, c, 1) == 36.0


def test_lb_ti_variants_order_and_soundness():
    """Exact window tops and more exact rows only tighten the triangle bounds (the
    recursions are monotone in (Lb, -Ub)), and every variant stays below LB_AD:
    basic <= TOP <= TIP_TOP, basic <= TIP <= TIP_TOP <= LB_AD, the top = 1 variant
    is orc_lb_ti, and P = 1 gives LB_AD for both tops.  A wrong sign or a mis-indexed
    neighbour in the candidate-side triangle breaks soundness or the order."""
    Q = rw(3, 36, 3, 41, role=1)
    Cs = rw(4, 36, 3, 41)
    for W in (0, 1, 3, 8, 35):
        for q in Q:
            for c in Cs:
                ad = O.lb_ad(q, c, W)
                basic = O.lb_ti_var(q, c, W, 1000, 0)
                top = O.lb_ti_var(q, c, W, 1000, 1)
                tip = O.lb_ti_var(q, c, W, 4, 0)
                tiptop = O.lb_ti_var(q, c, W, 4, 1)
                tol = 1e-12 * max(1.0, ad)
                assert basic <= top + tol and basic <= tip + tol
                assert top <= tiptop + tol and tip <= tiptop + tol and tiptop <= ad + tol
                assert tiptop == O.lb_ti(q, c, W, 4)
                assert O.lb_ti_var(q, c, W, 1, 0) == pytest.approx(ad, rel=1e-13)
                assert O.lb_ti_var(q, c, W, 1, 1) == pytest.approx(ad, rel=1e-13)
                if W == 0:  # single-point windows: every top is exact, the variants agree
                    assert basic == top and tip == tiptop


# ---------------------------------------------------------------- LB_PC (Section 5)

def _read_golden_boxes():
    pts, boxes, box1, vals = [], [], None, {}
    with open(os.path.join(HERE, "golden", "pc_boxes_hand.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "box":
                boxes.append([float(v) for v in tok[1:]])
            elif tok[0] == "box1":
                box1 = [float(v) for v in tok[1:]]
            elif tok[0].startswith("lbpc"):
                vals[tok[0]] = float(tok[1])
            else:
                pts.append([float(v) for v in tok])
    return np.array(pts, np.float32), boxes, box1, vals


def test_pc_boxes_hand_example():
    q, boxes, box1, vals = _read_golden_boxes()
    b, cnt = O.pc_boxes(q, W=3, K=2, Lq=2, w=4)
    assert cnt.tolist() == [1] * 0 + [2]
    for k, (lx, ly, hx, hy) in enumerate(boxes):
        assert b[0, k, 0].tolist() == [lx, ly] and b[0, k, 1].tolist() == [hx, hy]
    b1, cnt1 = O.pc_boxes(q, W=3, K=1, Lq=2, w=4)
    assert cnt1.tolist() == [1]
    assert b1[0, 0, 0].tolist() == box1[:2] and b1[0, 0, 1].tolist() == box1[2:]
    c = np.full((4, 2), 5.0, np.float32)
    assert O.lb_pc(q, c, 3, 2, 2, 4) == vals["lbpc_k2"]
    assert O.lb_pc(q, c, 3, 1, 2, 4) == vals["lbpc_k1"]


def test_lb_pc_single_box_equals_lb_mv():
    Q = rw(3, 45, 3, 19, role=1)
    Cs = rw(4, 45, 3, 19)
    for W in (0, 3, 44):
        for q in Q:
            for c in Cs:
                mv = O.lb_mv(q, c, W)
                assert O.lb_pc(q, c, W, K=1, Lq=2, w=1) == pytest.approx(mv, rel=1e-13, abs=1e-13)
                assert O.lb_pc(q, c, W, K=8, Lq=1, w=1) == pytest.approx(mv, rel=1e-13, abs=1e-13)


def test_lb_pc_point_boxes_equal_lb_ad():
    """With w=1, a very fine quantisation (every point its own cell) and K at least
    the window size, every box is a single query point, so LB_PC is LB_AD."""
    Q = rw(2, 36, 2, 23, role=1)
    Cs = rw(3, 36, 2, 23)
    W = 3
    for q in Q:
        b, cnt = O.pc_boxes(q, W, K=2 * W + 1, Lq=4096, w=1)
        # every point alone in its cell: box count = number of window points
        assert all(cnt[g] == min(35, g + W) - max(0, g - W) + 1 for g in range(36))
        for c in Cs:
            assert O.lb_pc(q, c, W, K=2 * W + 1, Lq=4096, w=1) == pytest.approx(O.lb_ad(q, c, W), rel=1e-13)


def test_pc_boxes_cover_their_expanded_window_and_cap():
    q = rw(1, 64, 3, 29)[0]
    W, K, Lq, w = 5, 4, 3, 6
    b, cnt = O.pc_boxes(q, W, K, Lq, w)
    for g in range(len(cnt)):
        assert 1 <= cnt[g] <= K
        pts = q[max(0, g * w - W): min(63, g * w + w - 1 + W) + 1].astype(np.float64)
        inside = np.zeros(len(pts), bool)
        for k in range(cnt[g]):
            inside |= np.all((pts >= b[g, k, 0]) & (pts <= b[g, k, 1]), axis=1)
        assert inside.all()
        # the union of boxes is exactly the envelope of the expanded window
        assert np.array_equal(np.min(b[g, :cnt[g], 0], axis=0), pts.min(axis=0))
        assert np.array_equal(np.max(b[g, :cnt[g], 1], axis=0), pts.max(axis=0))


# ---------------------------------------------------------------- NN search

@pytest.mark.parametrize("kind", ["random_walk", "proto_warp"])
@pytest.mark.parametrize("use_pc,use_ti", [(False, False), (True, False), (False, True), (True, True)])
def test_pruned_nn_equals_brute_force(kind, use_pc, use_ti):
    spec = synth.SeriesSpec(kind, 64, 3, 31, n_proto=4, sigma=0.1)
    Q = synth.generate(spec, synth.ROLE_QUERY, 12)
    Cs = synth.generate(spec, synth.ROLE_CAND, 300)
    W = 6
    bi, bd = O.nn_brute(Q, Cs, W)
    pi, pd, st = O.nn_pruned(Q, Cs, W, K=8, use_pc=use_pc, use_ti=use_ti, e_pc=0.1, e_ti=0.1)
    assert np.array_equal(bi, pi)
    assert np.array_equal(bd, pd)
    assert st["pairs"] == 12 * 300
    assert st["pruned_mv"] + st["pruned_pc"] + st["pruned_ti"] + st["dtw_started"] == st["pairs"]
    # the brute-force NN really is the argmin (spot check with the single-pair call)
    for m in range(3):
        d = [O.dtw(Q[m], c, W) for c in Cs]
        assert int(np.argmin(d)) == bi[m] and min(d) == bd[m]


def test_nn_ties_go_to_smallest_index():
    Cs = rw(20, 32, 2, 37)
    Cs = np.concatenate([Cs, Cs[[7, 3]]])            # duplicates at 20 and 21
    Q = Cs[[7, 3]] + np.float32(0.01)
    bi, bd = O.nn_brute(Q, Cs, 3)
    assert bi.tolist() == [7, 3]
    pi, pd, _ = O.nn_pruned(Q, Cs, 3, K=4)
    assert pi.tolist() == [7, 3]


# ---------------------------------------------------------------- gradient

def test_grad_path_is_valid_and_costs_the_distance():
    a, b = rw(2, 40, 3, 41)
    W = 5
    d, ga, gb, path, mg = O.dtw_grad(a, b, W)
    assert path[0] == (0, 0) and path[-1] == (39, 39)
    for (i0, j0), (i1, j1) in zip(path, path[1:]):
        assert (i1 - i0, j1 - j0) in {(1, 0), (0, 1), (1, 1)}
        assert abs(i1 - j1) <= W
    cost = sum(float(np.sum((a[i].astype(np.float64) - b[j].astype(np.float64)) ** 2)) for i, j in path)
    assert cost == pytest.approx(d, rel=1e-12)
    assert d == O.dtw(a, b, W)


def test_grad_matches_central_finite_differences():
    """The DTW cost is quadratic in the inputs along a fixed path, so central
    differences are exact up to rounding on pairs whose optimal path is unique by a
    margin that the perturbation cannot close: with h = 1e-4 a cell's cost moves by at
    most ~2 * |a - b| * h ~ 1e-3 here, so pairs with a margin >= 1e-3 keep their path.
    Eight pairs, every dimension, 16 coordinates per input; at least seven pairs must
    pass the margin filter (all 12 of the first pairs have margins 1.9e-3 .. 1.7e-2)."""
    rng = np.random.default_rng(0)
    A, B = synth.PAIRS_1024_L512.pairs(count=8)
    D = A.shape[2]
    h = 1e-4
    checked = 0
    for a, b in zip(A[:, :48], B[:, :48]):          # a shorter prefix keeps this fast
        W = 5
        d, ga, gb, path, mg = O.dtw_grad(a, b, W)
        if mg < 1e-3:
            continue
        for which, g in (("a", ga), ("b", gb)):
            for _ in range(16):
                i, p = int(rng.integers(0, 48)), int(rng.integers(0, D))
                x = (a if which == "a" else b).copy()
                x0 = x[i, p]
                xp, xm = x.copy(), x.copy()
                xp[i, p] = np.float32(x0 + h)
                xm[i, p] = np.float32(x0 - h)
                hp = float(xp[i, p]) - float(x0)
                hm = float(x0) - float(xm[i, p])
                fp = O.dtw(xp, b, W) if which == "a" else O.dtw(a, xp, W)
                fm = O.dtw(xm, b, W) if which == "a" else O.dtw(a, xm, W)
                fd = (fp - fm) / (hp + hm)
                scale = max(abs(g[i, p]), float(np.mean(np.abs(g))))
                assert abs(fd - g[i, p]) <= 1e-5 * scale + 1e-6, (which, i, p, fd, g[i, p])
        checked += 1
    assert checked >= 7
