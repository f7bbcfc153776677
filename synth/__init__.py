"""Seeded synthetic time-series generators (inputs only; no DTW arithmetic here).

This module is the one piece shared by the FP64 oracle runs and the CUDA runs: it
produces float32 arrays ``[count][L][D]`` (D innermost) and computes nothing that
is being tested.  The paper measures on UEA/UCR multivariate datasets (Section 7.1,
Table 2); those are not available, so seeded stand-ins with the same structure are
used instead:

* ``random_walk``: per-dimension Gaussian random walk, x_0 ~ N(0,1),
  x_t = x_{t-1} + N(0,1).
* ``proto_warp``: ``n_proto`` prototype random walks; each series picks a prototype
  uniformly, applies a random monotone time warp (local stretch factors
  U(0.9, 1.1), cumulative sum rescaled onto [0, L-1], linear interpolation per
  dimension) and adds N(0, sigma^2) noise.
* ``circle`` (D = 2): one turn of a circle, radius U(0.5, 1.5), phase U(-0.3, 0.3),
  plus N(0, sigma^2) noise.  Smooth series whose query envelopes are loose boxes
  around an arc, so that the point-based bounds (LB_TI, LB_PC) are much tighter
  than LB_MV -- the situation of the paper's trajectory datasets.

Every ``random_walk`` and ``proto_warp`` series is then z-normalised per dimension
(a constant dimension becomes all zeros), as the paper normalises its data and
replaces NA values by zero (Section 7.1); ``circle`` series are not (that would
give every circle the same radius).

Series are generated in chunks of ``CHUNK`` with an independent PCG64 stream per
chunk (``SeedSequence([seed, role, chunk])``), so any subset of a large set can be
regenerated without producing the rest.  ``role`` separates candidates (0),
queries (1) and prototypes (2); candidates use seed s, queries seed s + 1000.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

CHUNK = 1024
ROLE_CAND, ROLE_QUERY, ROLE_PROTO = 0, 1, 2


def window_for(L: int, frac_tenths: int = 1) -> int:
    """Sakoe-Chiba half-width W = round(frac * L), halves rounded up.

    ``frac_tenths`` is not used for the 5%-of-L workload; use ``window_pct``."""
    return (L * frac_tenths + 5) // 10


def window_pct(L: int, pct: int) -> int:
    """W = round(pct% of L) with halves rounded up (integer arithmetic)."""
    return (L * pct + 50) // 100


def _rng(seed: int, role: int, chunk: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), role, chunk])))


def _znorm(x: np.ndarray) -> np.ndarray:
    """Per-series, per-dimension z-normalisation in float64; std 0 -> all zeros."""
    mu = x.mean(axis=1, keepdims=True)
    sd = x.std(axis=1, keepdims=True)
    out = np.where(sd > 0, (x - mu) / np.where(sd > 0, sd, 1.0), 0.0)
    return out


def _random_walk_chunk(rng: np.random.Generator, n: int, L: int, D: int) -> np.ndarray:
    steps = rng.standard_normal((n, L, D))
    return np.cumsum(steps, axis=1)


def prototypes(seed: int, n_proto: int, L: int, D: int) -> np.ndarray:
    """The ``n_proto`` prototype walks shared by candidates and queries of one set."""
    rng = _rng(seed, ROLE_PROTO, 0)
    return _random_walk_chunk(rng, n_proto, L, D)


def _proto_warp_chunk(rng: np.random.Generator, protos: np.ndarray, n: int, sigma: float) -> np.ndarray:
    n_proto, L, D = protos.shape
    k = rng.integers(0, n_proto, size=n)
    stretch = rng.uniform(0.9, 1.1, size=(n, L))
    tau = np.cumsum(stretch, axis=1)
    if L > 1:
        tau = (tau - tau[:, :1]) / (tau[:, -1:] - tau[:, :1]) * (L - 1)
    else:
        tau = np.zeros((n, 1))
    i0 = np.clip(np.floor(tau).astype(np.int64), 0, max(L - 2, 0))
    i1 = np.minimum(i0 + 1, L - 1)
    frac = (tau - i0)[:, :, None]
    p = protos[k]                                     # n x L x D
    rows = np.arange(n)[:, None]
    x = p[rows, i0] * (1.0 - frac) + p[rows, i1] * frac
    x = x + sigma * rng.standard_normal((n, L, D))
    return x


def _circle_chunk(rng: np.random.Generator, n: int, L: int, D: int, sigma: float) -> np.ndarray:
    if D != 2:
        raise ValueError("circle series have D = 2")
    t = np.linspace(0.0, 2.0 * np.pi, L)
    r = rng.uniform(0.5, 1.5, size=(n, 1))
    ph = rng.uniform(-0.3, 0.3, size=(n, 1))
    x = np.stack([r * np.cos(t + ph), r * np.sin(t + ph)], axis=-1)
    return x + sigma * rng.standard_normal((n, L, D))


@dataclasses.dataclass(frozen=True)
class SeriesSpec:
    """Recipe for one set of series (candidates or queries)."""
    kind: str            # "random_walk" | "proto_warp" | "circle"
    L: int
    D: int
    seed: int
    n_proto: int = 0
    sigma: float = 0.0


def generate(spec: SeriesSpec, role: int, count: int, start: int = 0) -> np.ndarray:
    """Series ``start .. start+count-1`` of the set, float32 [count][L][D].

    The chunk structure means ``generate(spec, r, n, s)`` equals rows s..s+n-1 of
    ``generate(spec, r, s+n, 0)``."""
    L, D = spec.L, spec.D
    out = np.empty((count, L, D), dtype=np.float32)
    if count == 0:
        return out
    protos = prototypes(spec.seed, spec.n_proto, L, D) if spec.kind == "proto_warp" else None
    seed = spec.seed + (1000 if role == ROLE_QUERY else 0)
    c0, c1 = start // CHUNK, (start + count - 1) // CHUNK
    for c in range(c0, c1 + 1):
        rng = _rng(seed, role, c)
        if spec.kind == "random_walk":
            x = _random_walk_chunk(rng, CHUNK, L, D)
        elif spec.kind == "proto_warp":
            x = _proto_warp_chunk(rng, protos, CHUNK, spec.sigma)
        elif spec.kind == "circle":
            x = _circle_chunk(rng, CHUNK, L, D, spec.sigma)
        else:
            raise ValueError(f"unknown kind {spec.kind!r}")
        x = (x if spec.kind == "circle" else _znorm(x)).astype(np.float32)
        lo = max(start, c * CHUNK) - c * CHUNK
        hi = min(start + count, (c + 1) * CHUNK) - c * CHUNK
        dst = max(start, c * CHUNK) - start
        out[dst:dst + (hi - lo)] = x[lo:hi]
    return out


@dataclasses.dataclass(frozen=True)
class Workload:
    """One named NN-search workload: M queries against N candidates."""
    name: str
    M: int
    N: int
    spec: SeriesSpec
    W: int
    K: int = 16

    def candidates(self, count=None, start=0):
        return generate(self.spec, ROLE_CAND, self.N if count is None else count, start)

    def queries(self, count=None, start=0):
        return generate(self.spec, ROLE_QUERY, self.M if count is None else count, start)

    @property
    def band_cells(self) -> int:
        return band_cells(self.spec.L, self.W)


def band_cells(L: int, W: int) -> int:
    """Number of cells (i, j) of an L x L grid with |i - j| <= W."""
    W = min(W, L - 1)
    return L * (2 * W + 1) - W * (W + 1)


# The five workloads (names state what they are, with their sizes).
RW_16x256_L128 = Workload("rw_16q_256c_L128_D3_W13", 16, 256,
                          SeriesSpec("random_walk", 128, 3, 0), W=13, K=16)
PROTO_256x20000_L256 = Workload("proto_256q_20000c_L256_D5_W26_K16", 256, 20000,
                                SeriesSpec("proto_warp", 256, 5, 0, n_proto=20, sigma=0.1), W=26, K=16)
PROTO_1024x100000_L2048 = Workload("proto_1024q_100000c_L2048_D32_W102_K64", 1024, 100000,
                                   SeriesSpec("proto_warp", 2048, 32, 0, n_proto=100, sigma=0.2),
                                   W=102, K=64)


@dataclasses.dataclass(frozen=True)
class PairsWorkload:
    """P independent (A, B) series pairs for the differentiable DTW distance."""
    name: str
    P: int
    L: int
    D: int
    W: int
    seed: int = 0

    def pairs(self, count=None, start=0):
        n = self.P if count is None else count
        spec = SeriesSpec("random_walk", self.L, self.D, self.seed)
        a = generate(spec, ROLE_CAND, n, start)
        b = generate(spec, ROLE_QUERY, n, start)
        return a, b


PAIRS_1024_L512 = PairsWorkload("pairs_1024_L512_D8_W51", 1024, 512, 8, 51)


def batched_sets(n_sets: int = 32, M: int = 64, seed: int = 0, scale: float = 1.0):
    """The uneven batch: per set, L ~ U[64, 1024], D ~ U{2..12}, N ~ U[1k, 20k]
    (``scale`` shrinks N for small test runs), W = round(10% of L), prototype-warp
    data with 20 prototypes and sigma 0.1; set i uses seed ``seed + i``."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), 7, 7])))
    out = []
    for i in range(n_sets):
        L = int(rng.integers(64, 1025))
        D = int(rng.integers(2, 13))
        N = int(rng.integers(1000, 20001))
        N = max(1, int(math.ceil(N * scale)))
        W = window_for(L)
        out.append(Workload(f"set{i}_L{L}_D{D}_N{N}_W{W}", M, N,
                            SeriesSpec("proto_warp", L, D, seed + i, n_proto=20, sigma=0.1),
                            W=W, K=16))
    return out
