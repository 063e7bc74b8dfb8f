"""The bench's replica path with two ranks over gloo on the CPU: the maximum
over ranks, the whole-job aggregate, and a reference arm that only rank 0
runs (the others exit without work)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    # host-only ranks (gloo) even on a machine with a GPU: two ranks never share one
    os.environ["CUDA_VISIBLE_DEVICES"] = ""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    w, r, _ = bench.dist_setup()
    t_ms = [30.0, 50.0][r]  # the ranks' timed regions
    m = bench.max_over_ranks(t_ms, w)
    bench.barrier(w)
    ref = bench.run_reference(None, w, r, r) if r != 0 else "rank 0 runs it"
    q.put((r, w, m, bench.aggregate_qps(w, 10, 4096, m), ref))
    dist.destroy_process_group()


def test_two_ranks_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, m, qps, ref in out:
        assert w == 2 and m == 50.0  # every rank sees the slowest rank's time
        assert qps == pytest.approx(2 * 10 * 4096 / 0.050)  # all ranks' queries over that time
        if r != 0:
            assert ref is None  # the reference arm does no work off rank 0
