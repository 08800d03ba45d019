"""The multi-GPU path on CPU: two gloo ranks, each owning a contiguous
global env-index range (what bench.py gives each GPU through
env_index_base), reproduce one unsharded batch exactly; the only collectives
are the ones bench.py uses outside the data path (barrier, max of the
timings, and here a gather for the check)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, n, T, out):
    import torch
    import torch.distributed as dist

    import oracle as O

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    fam = [O.DOORKEY] * n
    b = O.Batch(fam, [8] * n, seed=1, env_index_base=rank * n)  # the rank's global env range
    b.reset()
    o = b.rollout(T)
    dist.barrier()
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)  # bench.py's max over ranks
    parts = [None] * world
    dist.all_gather_object(parts, {k: o[k] for k in ("obs_sym", "reward", "terminated", "truncated")})
    if rank == 0:
        out.put((float(t.item()), {k: np.concatenate([p[k] for p in parts], axis=1) for k in parts[0]}))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_one_batch():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    n, T, world = 24, 120, 2
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, T, q)) for r in range(world)]
    for p in procs:
        p.start()
    tmax, got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert tmax == 2.0
    import oracle as O

    whole = O.Batch([O.DOORKEY] * (n * world), [8] * (n * world), seed=1)
    whole.reset()
    want = whole.rollout(T)
    for k in got:
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)
