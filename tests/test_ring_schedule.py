"""Host-side check of the shared-memory ring schedule of the wide-point DTW tiles.

The ring variant of the band sweep (csrc/dtw_core.cuh) copies candidate columns and the
query rows of upcoming virtual lanes into per-group rings every kRingFill steps, for the
steps of the next kRingAhead + 1 periods, and waits for the fills of kRingAhead periods
ago.  The ring sizes (ring_cols(G) column slots, kRingRows row slots) follow from the
schedule.  This test replays that schedule exactly -- which virtual lane reads which
column and when it loads its rows -- with the constants read from the source, and checks
that every read comes after the copy it needs completed and that no slot is refilled
before its last read.  A ring one size class too small must fail the same check.
"""
import os
import random
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2101_07731_gb300", "csrc", "dtw_core.cuh")


def _constants():
    text = open(SRC).read()
    get = lambda name: int(re.search(rf"constexpr int {name} = (\d+);", text).group(1))
    return get("kRingFill"), get("kRingAhead"), get("kRingRows")


F, A, ROWS = _constants()


def ring_cols(G):
    n = F * (A + 1) + G
    return 16 if n <= 16 else 32 if n <= 32 else 64


def v_jlo(v, R, W):
    return max(0, v * R - W)


def v_jhi(v, R, W, L):
    return min(L - 1, v * R + R - 1 + W)


def ring_vmin(T, R, W, L):
    x = T - R + 1 - W
    a = 0 if x <= 0 else (x + R) // (R + 1)
    return max(a, T - L + 1)


def ring_vmax(T, R, W, v1):
    return min(v1 - 1, min(T, (T + W) // (R + 1)))


def check(L, W, R, G, RC=None, RR=None):
    """None if the schedule is safe, else a description of the first violation."""
    RC = ring_cols(G) if RC is None else RC
    RR = ROWS if RR is None else RR
    v1 = (L + R - 1) // R
    tau0, tau_end = 0, v_jhi(v1 - 1, R, W, L) + v1 - 1
    col_fill, row_fill, fill_step = {}, {}, {}
    hi = {"col": 0, "v": 0}

    def fill(T, period):
        c_end = min(L, T - ring_vmin(T, R, W, L) + 1)
        for c in range(hi["col"], c_end):
            col_fill[c] = period
        hi["col"] = max(hi["col"], c_end)
        v_end = min(v1, ring_vmax(T, R, W, v1) + 1)
        for v in range(hi["v"], v_end):
            row_fill[v] = period
        hi["v"] = max(hi["v"], v_end)

    fill(tau0 + F * A - 1, -1)  # prologue, complete before the loop
    col_reads, row_reads = {}, {}
    for t in range(tau0, tau_end + 1):
        p = (t - tau0) // F
        if (t - tau0) % F == 0:
            fill(t + F * (A + 1) - 1, p)
            fill_step[p] = t
        for v in range(v1):
            lo, hi_t = v_jlo(v, R, W) + v, v_jhi(v, R, W, L) + v
            if lo <= t <= hi_t:
                j = t - v
                if j not in col_fill or col_fill[j] > p - A:
                    return f"column {j} read at step {t} (period {p}) before its copy completed"
                col_reads.setdefault(j, []).append(t)
                if t == lo:
                    if v not in row_fill or row_fill[v] > p - A:
                        return f"rows of virtual lane {v} read at step {t} before their copy completed"
                    row_reads.setdefault(v, []).append(t)
    for j, ts in col_reads.items():
        k = j + RC  # the next column to use j's slot
        if k in col_fill:
            q = col_fill[k]
            if q < 0 or max(ts) >= fill_step[q]:
                return f"column slot of {j} refilled with {k} before its last read at step {max(ts)}"
    for v, ts in row_reads.items():
        k = v + RR
        if k in row_fill:
            q = row_fill[k]
            if q < 0 or max(ts) >= fill_step[q]:
                return f"row slot of virtual lane {v} refilled before its read at step {max(ts)}"
    return None


def _valid(L, W, R, G):
    return G * (R + 1) >= 2 * W + R


def test_constants_are_consistent():
    assert ROWS >= F * (A + 1)
    assert F & (F - 1) == 0 and ROWS & (ROWS - 1) == 0


@pytest.mark.parametrize("L,W,R,G", [(2048, 102, 6, 32), (2048, 109, 6, 32), (512, 51, 8, 16), (256, 26, 16, 4),
                                     (1, 0, 4, 4), (7, 6, 2, 32), (300, 120, 16, 16)])
def test_ring_schedule_named_shapes(L, W, R, G):
    if not _valid(L, W, R, G):
        pytest.skip("not a valid (tile, G) for this W")
    assert check(L, W, R, G) is None


def test_ring_schedule_random_shapes():
    rng = random.Random(7)
    n = 0
    while n < 250:
        L = rng.randint(1, 300)
        R = rng.choice([2, 4, 6, 8, 16])
        G = rng.choice([4, 8, 16, 32])
        W = rng.randint(0, min(L - 1, 140))
        if not _valid(L, W, R, G):
            continue
        n += 1
        assert check(L, W, R, G) is None, (L, W, R, G)


def test_a_smaller_ring_fails():
    # the headline shape needs more than 32 column slots at G = 32 (and the check sees it)
    assert check(2048, 102, 6, 32, RC=32) is not None
    assert check(2048, 102, 6, 32, RC=40) is not None
    # the row ring: at the start of the sweep virtual lanes begin one per step, so the
    # headline shape needs every one of the kRingRows slots
    assert check(2048, 102, 6, 32, RR=ROWS - 4) is not None
