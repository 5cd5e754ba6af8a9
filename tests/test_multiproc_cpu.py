"""Block parallelism across processes, on CPU with the gloo backend (world size 2).

Each rank takes the blocks ``assign_blocks`` gives it, renders them with the FP64 oracle
(standing in for one GPU per rank; there is no data-path collective), and rank 0 checks that
the gathered per-block images and the pruned-and-merged model equal a single-process run,
and that the max-over-ranks timing reduction is the maximum.
"""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import scenes
from paper_2510_01767_b300.shard import (assign_blocks, e2e_time, makespan, max_over_ranks, merge_blocks,
                                         prune_to_block)


def blocks_workload():
    rng = np.random.default_rng(9)
    g = scenes.uniform_gaussians(rng, 600, 1.0, 2.0, 6.0)
    leaves = scenes.kd_median_leaves(g.means, 2)
    cams = [scenes.pinhole(64, 48, 60.0, viewmat=scenes.look_at((x, y, -1.0), (x, y, 4.0), up=(0, -1, 0)))
            for x, y in ((-0.5, -0.5), (0.5, -0.5), (-0.5, 0.5), (0.5, 0.5))]
    return g, leaves, cams


def render_block(g, box, cam):
    idx = np.nonzero(((g.means >= np.array(box.lo, np.float32)) & (g.means < np.array(box.hi, np.float32))).all(1))[0]
    sub = oracle.set_dict(g.subset(idx))
    return oracle.forward(sub, cam.as_dict(), (16, 16)).image.rgb


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g, leaves, cams = blocks_workload()
        costs = [float(len(ix)) for ix, _ in leaves]
        mine, _ = assign_blocks(costs, world)
        out = {b: render_block(g, leaves[b][1], cams[b]) for b in mine[rank]}
        gathered = [None] * world
        dist.all_gather_object(gathered, out)
        t = max_over_ranks(float(rank + 1))
        # per-rank block models (the raw Gaussians of each block here) -> prune & merge
        params = {b: {"means": torch.as_tensor(g.means), "sh": torch.as_tensor(g.sh)} for b in mine[rank]}
        models = [None] * world
        dist.all_gather_object(models, params)
        if rank == 0:
            # numpy copies travel by value (torch tensors would be shared through file
            # descriptors that vanish when this process exits)
            models = [{b: {k: v.numpy() for k, v in d.items()} for b, d in m.items()} for m in models]
            q.put(("ok", gathered, t, models))
    except Exception as e:  # report to the parent instead of hanging it
        q.put(("err", repr(e), None, None))
        raise
    finally:
        dist.destroy_process_group()


def test_two_ranks_equal_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    status, gathered, t, models = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
    assert status == "ok", gathered
    assert t == 2.0
    g, leaves, cams = blocks_workload()
    merged_imgs = {}
    for d in gathered:
        merged_imgs.update(d)
    assert sorted(merged_imgs) == list(range(len(leaves)))
    for b, (_, box) in enumerate(leaves):
        np.testing.assert_array_equal(merged_imgs[b], render_block(g, box, cams[b]))
    per_block = {}
    for d in models:
        per_block.update({b: {k: torch.as_tensor(v) for k, v in p.items()} for b, p in d.items()})
    boxes = [box for _, box in leaves]
    merged = merge_blocks([per_block[b] for b in range(len(leaves))], boxes)
    # every Gaussian lies in exactly one KD leaf: the merge is a permutation of the scene
    assert merged["means"].shape[0] == g.n
    key = lambda m: np.lexsort(m.T)
    np.testing.assert_array_equal(np.asarray(merged["means"])[key(np.asarray(merged["means"]))],
                                  g.means[key(g.means)])


def test_assign_blocks_lpt():
    costs = [7, 5, 4, 4, 3, 3, 2]
    a, load = assign_blocks(costs, 3)
    assert sorted(sum(a, [])) == list(range(7))
    assert makespan(costs, a) == max(load) == 10
    a1, _ = assign_blocks(costs, 1)
    assert a1 == [list(range(7))]


def test_prune_to_block_half_open():
    m = torch.tensor([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.5, 0.2, 9.0]])
    box = scenes.AABB((0.0, -1.0, -math.inf), (1.0, 1.0, math.inf))
    out = prune_to_block({"means": m}, box)
    assert out["means"].shape[0] == 2  # x = 1.0 is outside [0, 1)


def test_e2e_protocol():
    assert e2e_time(38.0, 8.0, [20.0, 27.0, 25.0]) == 73.0
