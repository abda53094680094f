"""Initial states sharded over two gloo ranks on CPU: the per-rank objective
and gradient (here from the oracle) summed over ranks equal the full ones."""

import os
import socket

import numpy as np
import pytest

import workloads as W
from paper_2110_10310_gb300 import dist as D

torch = pytest.importorskip("torch")


def test_shard_indices_cover_and_balance():
    for M in (1, 3, 16, 17):
        for world in (1, 2, 3, 8):
            parts = [D.shard_indices(M, r, world) for r in range(world)]
            allv = np.concatenate(parts)
            assert np.array_equal(allv, np.arange(M))
            sizes = [p.size for p in parts]
            assert max(sizes) - min(sizes) <= 1


def test_shard_weights_and_tikhonov_split():
    p = W.random_problem(501, levels=(2,), n_states=5, gamma2=0.3)
    subs = [D.shard_problem(p, r, 3) for r in range(3)]
    # sum over ranks of (beta_i M_r / M) / M_r = beta_i / M
    total = np.concatenate([s.weights / s.M for s in subs])
    assert np.allclose(total, p.weights / p.M)
    assert subs[0].gamma2 == 0.3 and subs[1].gamma2 == 0.0 and subs[2].gamma2 == 0.0
    assert D.shard_problem(p, 4, 8) is None or D.shard_problem(p, 4, 8).M == 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from oracle import imr

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = W.random_problem(502, levels=(2, 2), n_states=3, n_steps=12, T_ns=0.3, amp=0.1, gamma2=0.2,
                             objective="trace", hermitian=False)
        sub = D.shard_problem(p, rank, world)
        G, g, _ = imr.gradient(sub)
        Gt, gt = D.allreduce_objective(G, g)
        q.put((rank, Gt, gt))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_sum_equals_full_objective():
    import torch.multiprocessing as mp

    from oracle import imr

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=240) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = W.random_problem(502, levels=(2, 2), n_states=3, n_steps=12, T_ns=0.3, amp=0.1, gamma2=0.2,
                         objective="trace", hermitian=False)
    G, g, _ = imr.gradient(p)
    for rank, Gt, gt in res:
        assert abs(Gt - G) <= 1e-13 * abs(G)
        assert np.max(np.abs(gt - g)) <= 1e-13 * np.max(np.abs(g))
