"""The CUDA path sharded over ranks (the paper's first level of parallelism,
Sec. V): two processes share the one GPU, each runs the library on its share
of the initial states (dist.shard_problem), and one gloo all-reduce sums
(G, dG/dalpha).  The sum equals the single-process result to 1e-12 and the
oracle to the method's tolerances.  The ranks' kernels never wait on each
other: each runs one CTA per state, and the only exchange is the host-side
all-reduce."""

import os
import socket

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem(objective):
    return W.random_problem(521, levels=(3, 2), n_states=5, n_steps=30, T_ns=0.6, amp=0.1, gamma2=0.15,
                            objective=objective, ckpt_every=7)


def _worker(rank, world, port, objective, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import torch as T

        from paper_2110_10310_gb300 import _lib as L
        from paper_2110_10310_gb300 import dist as D
        from paper_2110_10310_gb300.system import LindbladSystem

        T.cuda.set_device(0)
        L.load()
        sub = D.shard_problem(_problem(objective), rank, world)
        s = LindbladSystem(sub, sweep=L.LB_SWEEP_RESIDENT)
        G, g = s.gradient()
        Gt, gt = D.allreduce_objective(G, g)
        q.put((rank, sub.M, Gt, gt))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("objective", ["frob", "trace"])
def test_two_ranks_on_shards_sum_to_the_full_gradient(objective):
    import torch.multiprocessing as mp

    from oracle import imr
    from paper_2110_10310_gb300 import _lib as L
    from paper_2110_10310_gb300.system import LindbladSystem

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L.load(build_if_missing=True)
    p = _problem(objective)
    G1, g1 = LindbladSystem(p, sweep=L.LB_SWEEP_RESIDENT).gradient()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, objective, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=300) for _ in procs]
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    assert sorted(r[1] for r in res) == [2, 3]
    Go, go, _ = imr.gradient(p)
    for rank, Mr, Gt, gt in res:
        assert abs(Gt - G1) <= 1e-12 * abs(G1)
        assert np.max(np.abs(gt - g1)) <= 1e-12 * np.max(np.abs(g1))
        assert abs(Gt - Go) <= 1e-10 * abs(Go)
        assert np.max(np.abs(gt - go)) <= 1e-9 * np.max(np.abs(go))
