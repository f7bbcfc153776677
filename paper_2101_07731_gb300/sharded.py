"""Candidate sharding across GPUs (one process per GPU, torch.distributed).

Each rank holds a contiguous shard [offset, offset + n) of the candidate set and runs
the whole search on it (its own index: envelopes, bounds, DTW and refine); the exact
nearest neighbour over all shards is then one exchange: the minimum FP64 distance per
query (all_reduce MIN), and among the ranks holding that distance the smallest global
candidate index (a second all_reduce MIN), which is the search's tie rule (Def. 1:
the nearest member of the whole candidate set; equal distances go to the smaller
index).  The merge is the only collective on the data path."""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import Index

_IDX_NONE = torch.iinfo(torch.int64).max


def merge_nn_shards(idx: torch.Tensor, d: torch.Tensor, offset: int, group=None):
    """Exact merge of per-shard results: idx (int64, shard-local indices) and d
    (float64) of every query on this rank's shard -> (global idx, distance), the same
    on every rank.  Tensors must live where the process group's backend reduces them
    (CUDA for NCCL, CPU for gloo)."""
    gidx = idx.to(torch.int64) + int(offset)
    best = d.to(torch.float64).clone()
    dist.all_reduce(best, op=dist.ReduceOp.MIN, group=group)
    cand = torch.where(d.to(torch.float64) == best, gidx, torch.full_like(gidx, _IDX_NONE))
    dist.all_reduce(cand, op=dist.ReduceOp.MIN, group=group)
    return cand, best


class ShardedIndex:
    """An index over this rank's candidate shard; nn() returns the global answer."""

    def __init__(self, cand_shard: torch.Tensor, offset: int, W: int, K: int = 16, group=None, **opts):
        self.index = Index(cand_shard, W, K, **opts)
        self.offset = int(offset)
        self.group = group

    def nn(self, q: torch.Tensor):
        idx, d = self.index.nn(q)
        return merge_nn_shards(idx, d, self.offset, self.group)

    def close(self):
        self.index.close()
