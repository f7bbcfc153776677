"""GPU parity of the banded DTW kernel and its adjoint against the FP64 oracle.

Distances: within 1e-5 relative of FP64.  Gradients (on pairs whose optimal path
is unique by a margin): |g - g_ref| <= 1e-5 * max(|g_ref|, mean|g_ref|) per entry,
and against central finite differences (h = 1e-3) of the FP64 oracle distance.
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


def _rw(n, L, D, seed, role=0):
    return synth.generate(synth.SeriesSpec("random_walk", L, D, seed), role, n)


def _gpu(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


# (P, L, D, W): several tiles, ragged tails (L not a multiple of R, P not a
# multiple of the groups per block), W = 0, W >= L, D = 1, L = 1, wide D.
CASES = [
    (37, 70, 3, 7), (64, 128, 3, 13), (33, 256, 5, 26), (19, 100, 8, 10), (8, 64, 12, 6),
    (5, 90, 16, 9), (4, 60, 32, 6), (3, 50, 64, 4), (17, 40, 1, 0), (9, 31, 2, 200),
    (6, 1, 3, 0), (7, 2, 4, 5), (11, 129, 6, 47), (5, 300, 4, 120),
    (9, 77, 9, 8), (10, 64, 10, 30), (7, 45, 11, 4),   # exact-width tiles of D = 9..11
    # wide points through the shared-memory rings: D not a multiple of 4 (4-byte
    # copies), ragged L, one pair per warp (large W), the 2,048 x 32 shape with W = 102
    (6, 75, 17, 20), (5, 200, 27, 102), (4, 130, 40, 35), (3, 64, 13, 3), (5, 301, 32, 60),
    (3, 2048, 32, 102),
]


@pytest.mark.parametrize("P,L,D,W", CASES)
def test_dtw_pairs_matches_oracle(P, L, D, W):
    A, B = _rw(P, L, D, 100 + L), _rw(P, L, D, 100 + L, role=1)
    got = tc.dtw_pairs(_gpu(A), _gpu(B), W).cpu().numpy().astype(np.float64)
    ref = O.dtw_pairs(A, B, W)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0)


def test_dtw_pairs_identity_is_zero_and_symmetric():
    A = _rw(16, 77, 3, 5)
    B = _rw(16, 77, 3, 6)
    z = tc.dtw_pairs(_gpu(A), _gpu(A), 9).cpu().numpy()
    assert np.all(z == 0)
    ab = tc.dtw_pairs(_gpu(A), _gpu(B), 9).cpu().numpy()
    ba = tc.dtw_pairs(_gpu(B), _gpu(A), 9).cpu().numpy()
    np.testing.assert_allclose(ab, ba, rtol=RTOL)


def test_dtw_pairs_full_size_1024_L512_D8_W51():
    wl = synth.PAIRS_1024_L512
    A, B = wl.pairs()
    got = tc.dtw_pairs(_gpu(A), _gpu(B), wl.W).cpu().numpy().astype(np.float64)
    ref = O.dtw_pairs(A, B, wl.W)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0)


def _check_grad(ga, gref):
    scale = np.maximum(np.abs(gref), np.mean(np.abs(gref)))
    err = np.abs(ga - gref)
    assert np.all(err <= RTOL * scale + 1e-6), float(np.max(err / (scale + 1e-30)))


@pytest.mark.parametrize("P,L,D,W", [(12, 64, 3, 6), (8, 150, 5, 15), (6, 97, 8, 20), (4, 60, 32, 6),
                                     (5, 33, 1, 40), (3, 1, 2, 0)])
def test_dtw_backward_matches_oracle_gradient(P, L, D, W):
    A, B = _rw(P, L, D, 300 + L), _rw(P, L, D, 300 + L, role=1)
    At, Bt = _gpu(A).requires_grad_(True), _gpu(B).requires_grad_(True)
    d = tc.dtw(At, Bt, W)
    g = torch.linspace(0.5, 1.5, P, device=DEV)
    (d * g).sum().backward()
    gA, gB = At.grad.cpu().numpy(), Bt.grad.cpu().numpy()
    checked = 0
    for p in range(P):
        rd, ra, rb, path, margin = O.dtw_grad(A[p], B[p], W)
        assert abs(float(d[p].detach()) - rd) <= RTOL * max(rd, 1e-30)
        if margin < 1e-4:
            continue   # path not unique by a safe margin: FP32 may pick another optimum
        gp = float(g[p])
        _check_grad(gA[p], gp * ra)
        _check_grad(gB[p], gp * rb)
        checked += 1
    assert checked >= 1


def _gamma32(L, D):
    """Relative FP32 error bound of the DTW value (gamma_n, n = 2L+D+2 roundings)."""
    n = 2 * L + D + 2
    u = 2.0 ** -24
    return n * u / (1 - n * u)


def _grad_ok(ga, gref):
    scale = np.maximum(np.abs(gref), np.mean(np.abs(gref)))
    return bool(np.all(np.abs(ga - gref) <= RTOL * scale + 1e-6))


def test_dtw_backward_full_size_1024_L512_D8_W51():
    """All 1024 pairs.  Where the oracle's backtracking margin is at least twice
    the FP32 error bound, the FP32 argmin decisions provably equal the FP64 ones, so
    the gradient must match; there the FP64 distance is also checked by central
    differences.  Below that margin another (equally optimal within rounding) path
    is legitimate; among pairs above typical rounding noise (1e-5) at least 95%
    must still match."""
    wl = synth.PAIRS_1024_L512
    A, B = wl.pairs()
    At, Bt = _gpu(A).requires_grad_(True), _gpu(B).requires_grad_(True)
    d = tc.dtw(At, Bt, wl.W)
    d.sum().backward()
    gA, gB = At.grad.cpu().numpy(), Bt.grad.cpu().numpy()
    dist = d.detach().cpu().numpy().astype(np.float64)
    g2 = 2 * _gamma32(wl.L, wl.D)
    rng = np.random.default_rng(1)
    rigorous = noisy_ok = noisy = 0
    for p in range(wl.P):
        rd, ra, rb, path, margin = O.dtw_grad(A[p], B[p], wl.W)
        assert abs(dist[p] - rd) <= RTOL * rd
        ok = _grad_ok(gA[p], ra) and _grad_ok(gB[p], rb)
        if margin >= g2:
            assert ok, (p, margin)
            rigorous += 1
            for _ in range(4):
                i, k = int(rng.integers(0, wl.L)), int(rng.integers(0, wl.D))
                x = A[p].copy()
                xp, xm = x.copy(), x.copy()
                xp[i, k] = np.float32(x[i, k] + 1e-3)
                xm[i, k] = np.float32(x[i, k] - 1e-3)
                h = (float(xp[i, k]) - float(x[i, k])) + (float(x[i, k]) - float(xm[i, k]))
                fd = (O.dtw(xp, B[p], wl.W) - O.dtw(xm, B[p], wl.W)) / h
                scale = max(abs(ra[i, k]), float(np.mean(np.abs(ra))))
                assert abs(gA[p][i, k] - fd) <= 1e-4 * scale + 1e-4
        elif margin >= 1e-5:
            noisy += 1
            noisy_ok += ok
    assert rigorous >= 1
    assert noisy_ok >= 0.95 * noisy, (noisy_ok, noisy)
