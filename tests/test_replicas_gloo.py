"""The N>1 path of bench.py on CPU: one replica per rank (no data-path
collective), a barrier around the timed region, the maximum time over ranks,
and the whole-job rate from it -- two gloo ranks on 127.0.0.1."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    assert bench.dist_env() == (ws, rank, rank)
    bench.barrier(ws)
    t_rank = 100.0 + 50.0 * rank                     # ms of this rank's timed steps
    t_max = bench.max_over_ranks(t_rank, ws)
    bench.barrier(ws)
    out.put((rank, t_max, bench.job_throughput(1000, ws, 5, t_max)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_count_all_units():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]
    # 2 ranks x 1000 particles x 5 steps over the slowest rank's 150 ms
    assert all(abs(r[2] - 2 * 1000 * 5 / 0.150) < 1e-6 for r in res)
