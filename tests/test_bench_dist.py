"""Multi-rank logic of bench.py on CPU (gloo, world size 2): each rank times
its own replica, the job time is the maximum over ranks, the value is the
whole-job aggregate, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as td  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    td.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, local = bench.setup_dist()
        assert (w, r, local) == (ws, rank, rank)
        local_s = 1.0 + 2.0 * rank  # rank 1 is the slow one
        t = bench.max_over_ranks(local_s, True, device="cpu")
        value = bench.whole_job_mlups(w, 128**3, 100, t)

        class Args:
            workload = "chol128_R8"
            steps = 1
            warmup = 1
        ref_rc = bench.run_reference(Args(), w, r) if r != 0 else None
        out.put((rank, t, value, ref_rc))
    finally:
        td.destroy_process_group()


def test_two_rank_timing_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, value, ref_rc in res:
        assert t == 3.0  # max over ranks
        assert value == pytest.approx(2 * 128**3 * 100 / 3.0 / 1e6)
    assert res[1][3] == 0  # the reference arm does no work on rank 1


def test_single_rank_is_local():
    import bench
    assert bench.max_over_ranks(2.5, False) == 2.5
    assert bench.whole_job_mlups(1, 10**6, 10, 2.0) == 5.0
