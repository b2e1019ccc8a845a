"""The N > 1 path of bench.py (independent replicas, one per rank, no collective in the data path):
the whole-job throughput divides the units all ranks processed by the slowest rank's time.  Runs
as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, ws: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    assert bench.dist_env() == (ws, rank, rank)
    # rank r took 1000 (r + 1) ms for its 3 steps and 1500 (r + 1) ms end to end
    v, e, t, te = bench.replica_throughput(ws, 3, 1000.0 * (rank + 1), 1500.0 * (rank + 1), "cpu")
    out[rank] = (v, e, t, te)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(ws, port, out), nprocs=ws, start_method="spawn", join=True)
        res = dict(out)
    for r in range(ws):
        v, e, t, te = res[r]
        assert t == 2000.0 and te == 3000.0          # the slower rank's totals on every rank
        assert v == pytest.approx(ws * 3 / 2.0)       # 6 evaluations in 2 s
        assert e == pytest.approx(ws * 3 / 3.0)


def test_single_rank_needs_no_collective():
    import bench
    v, e, t, te = bench.replica_throughput(1, 4, 2000.0, 4000.0, "cpu")
    assert (v, e, t, te) == (2.0, 1.0, 2000.0, 4000.0)
