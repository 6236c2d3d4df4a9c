"""Data-parallel replicas on CPU (gloo, world size 2): each rank back-propagates
its own view of a two-view anchor scene (the FP64 oracle stands in for the
GPU step here, CPU only); after allreduce_param_grads every rank holds the
gradients of the whole two-view batch computed in one process."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_2503_23044_b300 import replicas, synth


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene():
    sc = synth.tiny_anchor_scene(n_anchors=4, seed=11, n_views=2, width=32, height=24)
    grads = synth.random_image_grads(sc["cameras"], seed=4, scale=1e-2)
    return sc, grads


def _grads_of_views(views):
    sc, grads = _scene()
    leaves = O.leaves_anchor(sc)
    O.render(sc, O.RenderParams(), leaves=leaves, image_grads=grads, views=views)
    return {k: (v.grad.clone() if v.grad is not None else torch.zeros_like(v)) for k, v in leaves.items()}


def _worker(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        g = _grads_of_views([rank])
        replicas.allreduce_param_grads(g)
        out[rank] = {k: v.numpy() for k, v in g.items()}
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_allreduce_of_two_ranks_equals_the_two_view_batch():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    ref = _grads_of_views([0, 1])
    for k, v in ref.items():
        assert float(np.abs(v.numpy()).max()) > 0 or k in ("b1",), k
        for r in range(world):
            assert np.allclose(res[r][k], v.numpy(), rtol=1e-12, atol=1e-15), (k, r)
