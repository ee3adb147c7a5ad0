"""The multi-GPU path of bench.py on the CPU: two gloo ranks (one process each, rendezvous on
127.0.0.1).  Frames are independent, so the only cross-rank steps are the barriers around the
timed region and the max over ranks of the frame time; the job value counts every rank's frame."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, _ = bench.dist_setup(world)
    assert (r, w) == (rank, world) and dist.get_backend() == "gloo"
    bench.barrier(w)
    frame_ms = 5.0 + 2.0 * rank                  # rank 1 is the slower one
    mx = bench.allmax(frame_ms, w)
    bench.barrier(w)
    out.put((rank, mx, bench.job_value(1024 * 1024, mx, w)))
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_max_frame_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(k, 2, port, q)) for k in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[1] for x in res] == [7.0, 7.0]                 # both ranks see the slowest frame
    assert res[0][2] == pytest.approx(2 * 1024 * 1024 / 7e-3)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})()) is None
