"""The N>1 path of bench.py on CPU: two gloo ranks, each with its own node range, combine
their step times with one all_reduce(MAX); the whole-job rate is world * batch / max time."""

import os
import socket

import torch.distributed as dist
import torch.multiprocessing as tmp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, rate = bench.aggregate_ranks([120.0, 150.0][rank], 4096, world, dist)
    nodes = bench.rank_nodes(rank, 4096)
    out.put((rank, ms, rate, nodes.start, nodes.stop))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_disjoint_nodes():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, lo, hi in res:
        assert ms == 150.0
        assert abs(rate - 2 * 4096 / 0.150) < 1e-6
    assert (res[0][3], res[0][4]) == (0, 4096) and (res[1][3], res[1][4]) == (4096, 8192)


def test_single_rank_has_no_collective():
    ms, rate = bench.aggregate_ranks(200.0, 4096, 1, None)
    assert ms == 200.0 and abs(rate - 4096 / 0.2) < 1e-9
