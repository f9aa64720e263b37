"""The multi-rank (replica) path of bench.py on CPU: two gloo ranks on 127.0.0.1.  Each rank
gets its own tensor (weak scaling, no data-path collective), the ranks meet only in barriers and
in the max of their timings, and only rank 0 runs the CPU reference arm."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), BENCH_DIST_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    bench.DIMS, bench.NNZ = (40, 30, 20), 2000
    w, r, _ = bench.dist_setup(world)
    assert (w, r) == (world, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    assert bench.max_over_ranks(float(10 * (rank + 1)), w) == 10.0 * world
    X = bench.make_inputs(r)
    # every rank's tensor is its own: gather a fingerprint of each
    fp = torch.tensor([float(X.val.sum()), float(X.idx[0].astype(np.int64).sum())],
                      dtype=torch.float64)
    allfp = [torch.zeros(2, dtype=torch.float64) for _ in range(w)]
    dist.all_gather(allfp, fp)
    out[rank] = [t.tolist() for t in allfp]
    # the reference arm: rank 0 alone does work; the others return at once
    if r != 0:
        class A:
            gpus, steps, warmup = world, 1, 0
        assert bench.run_reference(A, w, r) is None
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    assert res[0] == res[1]                      # all ranks saw the same fingerprints
    assert res[0][0] != res[0][1]                # and the two ranks' tensors differ
