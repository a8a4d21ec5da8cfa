"""The multi-process path of the benchmark (CPU, two gloo ranks): every rank gets its
own, equally sized part of the scenarios, and the job's numbers are the slowest rank's
time and the sum of the ranks' work.  The solver itself has no collective (scenarios
are independent), so this host logic is all there is to check without GPUs."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from synthgrid import configs
    g = configs.grid("c0")
    t, c = bench.over_ranks(world, torch.device("cpu"), [5.0, 7.5][rank], [64, 61][rank])
    sc = bench.rank_scenarios("c0", g, rank, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, c, sc.Pd))


def test_two_ranks_split_the_scenarios_and_reduce_time_and_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        rank, t, c, Pd = q.get(timeout=120)
        out[rank] = (t, c, Pd)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from synthgrid import configs
    n = configs.CONFIGS["c0"]["n_scen"]
    for r in (0, 1):
        t, c, Pd = out[r]
        assert t == 7.5 and c == 125          # slowest rank's time, total work
        assert Pd.shape == (n, 14)
    assert not np.array_equal(out[0][2], out[1][2])   # distinct scenarios per rank
    both = configs.scenarios("c0", 2 * n)
    assert np.array_equal(np.vstack([out[0][2], out[1][2]]), both.Pd)
