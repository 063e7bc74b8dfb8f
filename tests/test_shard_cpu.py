"""Grain shards on the host: the library's shard assignment and host merge
against the oracle, and the exchange of two ranks over gloo on the CPU (one
all-gather of k (id, distance) per query, then the merge) against the
oracle's sharded search."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import hntl_oracle as O
from paper_2606_08813_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_2606_08813_b300 import build_lib

    build_lib.build()
    from paper_2606_08813_b300 import hntl

    return hntl


def _case():
    m = synth.make_cluster_model(2000, 16, 8, seed=71)
    X, _ = synth.sample_points(m, 72)
    Q, _ = synth.sample_queries(m, 40, 73)
    X, Q = X.numpy(), Q.numpy()
    idx = O.build_index(X, 16, 4, synth.uniforms(16, 74).numpy())
    return X, Q, idx


def test_shard_assign_matches_oracle():
    h = _lib()
    rng = np.random.default_rng(5)
    for G, S in ((1, 1), (6, 2), (97, 3), (4096, 8)):
        rows = rng.integers(0, 3000, G)
        rows[: G // 5] = rows[0]  # equal sizes: the grain order decides
        assert h.shard_assign(rows, S).tolist() == O.shard_assign(rows, S).tolist()
    with pytest.raises(h.HntlError):
        h.shard_assign([1, 2], 3)


def test_merge_host_matches_oracle_merge():
    h = _lib()
    X, Q, idx = _case()
    sog = O.shard_assign(np.diff(idx["grain_off"]), 3)
    oi, od, per = O.sharded_search(idx, X, Q, 10, 30, 5, sog)
    ids = np.stack([p["out_id"] for p in per])
    dist = np.stack([p["out_d"][:, :10] for p in per]).astype(np.float32)
    mi, md = h.merge_topk_host(ids, dist)
    np.testing.assert_array_equal(mi, oi)
    np.testing.assert_allclose(md, od, rtol=1e-6)
    # padding ranks last; fewer than k real entries leave -1 / +inf
    ids2 = np.full((2, 1, 4), -1, dtype=np.int64)
    d2 = np.full((2, 1, 4), np.inf, dtype=np.float32)
    ids2[0, 0, :2] = [7, 3]
    d2[0, 0, :2] = [1.0, 2.0]
    ids2[1, 0, 0] = 5
    d2[1, 0, 0] = 1.0
    d2[1, 0, 1] = 0.0  # a padding entry with a small distance is still padding
    mi, md = h.merge_topk_host(ids2, d2)
    assert mi.tolist() == [[5, 7, 3, -1]] and md[0, :3].tolist() == [1.0, 1.0, 2.0] and np.isinf(md[0, 3])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["CUDA_VISIBLE_DEVICES"] = ""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    from test_shard_cpu import _case, _lib

    h = _lib()
    X, Q, idx = _case()
    sog = O.shard_assign(np.diff(idx["grain_off"]), world)
    _, _, per = O.sharded_search(idx, X, Q, 10, 30, 5, sog)  # this rank's shard: per[rank]
    ids = torch.from_numpy(per[rank]["out_id"].copy())
    dd = torch.from_numpy(per[rank]["out_d"][:, :10].astype(np.float32))
    mi, md = h.exchange_merge(ids, dd)
    q.put((rank, mi.numpy(), md.numpy()))
    dist.destroy_process_group()


def test_two_rank_exchange_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    X, Q, idx = _case()
    oi, od, _ = O.sharded_search(idx, X, Q, 10, 30, 5, O.shard_assign(np.diff(idx["grain_off"]), 2))
    for _, mi, md in out:  # every rank holds the merged result
        np.testing.assert_array_equal(mi, oi)
        np.testing.assert_allclose(md, od, rtol=1e-6)
