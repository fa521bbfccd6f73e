"""bench.py's multi-process logic on CPU: two gloo ranks, barrier, max of
the per-rank times and sum of the per-rank work (the N > 1 aggregation of
the weak-scaling replicas)."""
import os
import socket
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w = bench.dist_setup("gloo")
    assert (r, w) == (rank, world)
    bench.barrier()
    mx = bench.max_over_ranks(10.0 * (rank + 1))
    sm = bench.sum_over_ranks(64 * (rank + 1))
    out.put((rank, mx, sm, bench.rank_info()))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, mx, sm, info in res:
        assert mx == 20.0 and sm == 192.0
        assert info == (rank, 2, rank)


def test_single_rank_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.rank_info() == (0, 1, 0)
    assert bench.max_over_ranks(3.5) == 3.5 and bench.sum_over_ranks(7) == 7.0
