"""Host-side block parallelism: one process (GPU) per group of KD-tree blocks, no
communication on the data path (the paper trains blocks independently, one GPU each, and
merges the block models at the end; Sec. 3, Fig. 1 caption, Sec. 5.1 "System Configuration").

- ``assign_blocks``: longest-processing-time assignment of blocks to ranks by a predicted
  cost (the paper's workload proxy is the block's camera count, Eq. L(B) = |C(B)|), so the
  slowest rank -- the one that sets T_E2E = T_coarse + T_partition + max_b T_fine -- is as
  fast as a greedy assignment can make it.
- ``prune_to_block`` / ``merge_blocks``: keep each block's Gaussians whose means lie inside its
  box, then concatenate (the final prune-and-merge of Fig. 1).
- ``max_over_ranks``: the timing reduction bench.py uses (a collective on a scalar only).
"""
from __future__ import annotations

import math

import torch


def assign_blocks(costs, world: int):
    """Greedy LPT: blocks sorted by decreasing cost (ties by index), each to the least loaded
    rank (ties by rank). Returns (list of block lists per rank, per-rank load)."""
    order = sorted(range(len(costs)), key=lambda b: (-costs[b], b))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(b)
        load[r] += costs[b]
    for lst in out:
        lst.sort()
    return out, load


def inside_mask(means: torch.Tensor, lo, hi) -> torch.Tensor:
    """lo <= mu < hi on every axis (infinite bounds allowed)."""
    lo = torch.as_tensor([float(x) for x in lo], dtype=means.dtype, device=means.device)
    hi = torch.as_tensor([float(x) for x in hi], dtype=means.dtype, device=means.device)
    return ((means >= lo) & (means < hi)).all(dim=1)


def prune_to_block(params: dict, box) -> dict:
    keep = inside_mask(params["means"], box.lo, box.hi)
    return {k: v[keep] for k, v in params.items()}


def merge_blocks(block_params: list, boxes: list) -> dict:
    """Prune each block model to its box and concatenate them in block order."""
    pruned = [prune_to_block(p, b) for p, b in zip(block_params, boxes)]
    return {k: torch.cat([p[k] for p in pruned], dim=0) for k in pruned[0]}


def max_over_ranks(x: float) -> float:
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def e2e_time(t_coarse: float, t_partition: float, t_fine: list) -> float:
    """End-to-end runtime of the paper's protocol: coarse + partition + slowest block."""
    return t_coarse + t_partition + (max(t_fine) if t_fine else 0.0)


def makespan(costs, assignment) -> float:
    return max((sum(costs[b] for b in blocks) for blocks in assignment), default=0.0) if assignment else math.nan
