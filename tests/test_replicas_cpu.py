"""Replica harness on CPU: two gloo ranks, each with its own seeded system,
reduce only their timing (max over ranks); no collective touches the data."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2307_04528_gb300 import replicas
    from synthetic import make_problem
    r, w = replicas.init("gloo")
    P = make_problem(16, 8, 4, 0.1, replicas.replica_seed(1000, r))
    local = float(P["b"].sum())           # a per-rank result that differs by seed
    t = replicas.max_over_ranks(1.0 + r)  # timing reduction
    replicas.barrier()
    out[r] = (local, t)
    replicas.finalize()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    world = 2
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    (l0, t0), (l1, t1) = out[0], out[1]
    assert t0 == t1 == 2.0          # max over ranks seen by every rank
    assert l0 != l1                 # independent systems


def test_single_rank_identity():
    from paper_2307_04528_gb300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.replica_seed(3000, 0) == 3000
