"""Full-size parity of the largest search: 1,024 queries x 100,000 candidates,
L = 2,048, D = 32, W = 102 (5% of L), 100 prototypes, sigma = 0.2, LB_PC K = 64
(26 GB of candidates resident in HBM), in the configuration of the library's
defaults.

The GPU searches all 1,024 queries once (module fixture).  The oracle's brute force
over 1e8 pairs of 4e5 cells each is out of reach, so:
  * for 16 sampled queries, the oracle's pruned search (LB_MV and early abandoning in
    FP64, pinned equal to brute force by the oracle's own tests) runs over all
    100,000 candidates: indices must be identical, distances within 1e-9 relative
    (the double-float refine's bound);
  * for 6 more sampled queries, the returned distance is the FP64 DTW of the
    returned candidate and no candidate of a random sample beats it;
  * for a few queries, the pruned search and a search with every bound and every
    abandoning switched off (no_prune: the DTW of all 100,000 pairs) agree exactly;
  * counters: every pair is accounted for, and pruning removed most DTWs.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

tc = pytest.importorskip("paper_2101_07731_gb300")
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
WL = synth.PROTO_1024x100000_L2048


def _fill(args):
    """Worker: generate candidate chunk c into the shared buffer."""
    name, c, N, L, D = args
    from multiprocessing import shared_memory
    shm = shared_memory.SharedMemory(name=name)
    try:
        buf = np.ndarray((N, L, D), dtype=np.float32, buffer=shm.buf)
        lo = c * synth.CHUNK
        n = min(synth.CHUNK, N - lo)
        buf[lo:lo + n] = WL.candidates(n, lo)
    finally:
        shm.close()
    return c


@pytest.fixture(scope="module")
def large():
    if DEV is None:
        pytest.skip("needs a GPU")
    from multiprocessing import shared_memory
    N, L, D = WL.N, WL.spec.L, WL.spec.D
    nbytes = N * L * D * 4
    shm = shared_memory.SharedMemory(create=True, size=nbytes)
    try:
        chunks = -(-N // synth.CHUNK)
        with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
            pool.map(_fill, [(shm.name, c, N, L, D) for c in range(chunks)])
        host = np.ndarray((N, L, D), dtype=np.float32, buffer=shm.buf)
        cand = torch.from_numpy(host).to(DEV)
        sample = host[:: N // 4096].copy()  # a fixed sample of candidates for the oracle checks
        sample_idx = np.arange(0, N, N // 4096)
        Qn = WL.queries()
        yield cand, Qn, host, sample, sample_idx
    finally:
        del cand
        torch.cuda.empty_cache()
        shm.close()
        shm.unlink()


@pytest.fixture(scope="module")
def search(large):
    cand, Qn, host, sample, sample_idx = large
    index = tc.Index(cand, WL.W, WL.K)
    idx, dist, st = index.nn(torch.from_numpy(Qn).to(DEV), stats=True)
    index.close()
    return idx.cpu().numpy(), dist.cpu().numpy(), st


def test_nn_large_16_queries_match_oracle_over_all_candidates(large, search):
    cand, Qn, host, sample, sample_idx = large
    gi, gd, _ = search
    qs = np.sort(np.random.default_rng(5).choice(WL.M, size=16, replace=False))
    ridx, rdist, _ = O.nn_pruned(Qn[qs], host, WL.W, K=WL.K, use_pc=False, use_ti=False)
    assert np.array_equal(gi[qs], ridx), (qs, gi[qs], ridx)
    np.testing.assert_allclose(gd[qs], rdist, rtol=1e-9, atol=0)


def test_nn_proto_1024x100000_L2048_D32_W102_sampled(large, search):
    cand, Qn, host, sample, sample_idx = large
    gi, gd, st = search
    M, N = WL.M, WL.N
    assert st["pairs"] == M * N
    assert st["pruned_mv"] + st["pruned_pc"] + st["pruned_ti"] + st["dtw_started"] == st["pairs"], st
    assert st["dtw_started"] < 0.5 * st["pairs"]
    assert np.all((gi >= 0) & (gi < N))
    rng = np.random.default_rng(11)
    qs = rng.choice(M, size=6, replace=False)
    for m in qs:
        # the distance is the FP64 DTW of the returned candidate
        ref = O.dtw(Qn[m], host[gi[m]], WL.W)
        assert abs(gd[m] - ref) <= 1e-9 * ref, (m, gd[m], ref)
        # no sampled candidate is closer (ties: only a larger index may tie)
        sub = rng.choice(len(sample_idx), size=48, replace=False)
        d = O.dtw_pairs(np.repeat(Qn[m][None], len(sub), 0), sample[sub], WL.W)
        for n, dv in zip(sample_idx[sub], d):
            assert dv > ref or (dv == ref and n >= gi[m]), (m, n, dv, ref)


def test_nn_large_pruned_equals_unpruned(large):
    cand, Qn, host, sample, sample_idx = large
    q = torch.from_numpy(Qn[:3]).to(DEV)
    a = tc.Index(cand, WL.W, WL.K)
    ia, da = a.nn(q)
    a.close()
    b = tc.Index(cand, WL.W, WL.K, no_prune=1)
    ib, db = b.nn(q)
    b.close()
    assert torch.equal(ia, ib)
    assert torch.equal(da, db)
