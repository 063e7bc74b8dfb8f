"""Grain shards on the GPU against the oracle's sharded search: each shard's
own search (probes, pool, top k) against the oracle on the same grains, the
merged top k against the oracle's merge, a single shard against the whole
index bit for bit, and the merge kernel against the host merge. Tolerances
and the gap rule are those of tests/parity.py."""
import numpy as np
import pytest
import torch

from oracle import hntl_oracle as O

from cases import clustered_case, write
from parity import GAP, check_ranked, compare_search

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hntl():
    from paper_2606_08813_b300 import build_lib

    build_lib.build()
    from paper_2606_08813_b300 import hntl as h

    return h


@pytest.fixture(scope="module")
def case(tmp_path_factory):
    """12 clusters of Zipf sizes in 48 grains (d = 64, r = 16), 512 queries."""
    X, Q, idx = clustered_case(30000, 64, 12, 48, 16, 512, seed=881, sizes="zipf")
    d = tmp_path_factory.mktemp("shard")
    return X, Q, idx, write(d, "s32", idx, X), write(d, "s8", idx, X, precision="bf16-fp8")


def _merged_ext(per, k):
    """Per query the (k+1)-th distance of the union of the shards' top-k lists
    (the next value the merge could have taken)."""
    nq = per[0]["out_id"].shape[0]
    out = np.full(nq, np.inf)
    for qi in range(nq):
        ds = sorted(float(p["out_d"][qi, j]) for p in per for j in range(k) if p["out_id"][qi, j] >= 0)
        if len(ds) > k:
            out[qi] = ds[k]
    return out


@pytest.mark.parametrize("S", [2, 3])
def test_shards_and_merge_match_oracle(hntl, case, S):
    X, Q, idx, p32, _ = case
    gi = hntl.Index.load(p32, 0, hntl.PREC_FP32)
    sh = hntl.ShardedIndex(gi, S)
    rows = np.diff(idx["grain_off"])
    assert sh.shard_of_grain.tolist() == O.shard_assign(rows, S).tolist()
    assert sum(int(s.desc.n) for s in sh.shards) == len(X)
    k, C, nprobe = 10, 100, 8
    oi, od, per = O.sharded_search(idx, X, Q, k, C, nprobe, sh.shard_of_grain)
    Qd = torch.from_numpy(Q).cuda()
    for s, shard in enumerate(sh.shards):
        ids, dist, pid, pd, probe = shard.search(Qd, k, C, nprobe, return_pool=True, return_probe=True)
        hntl.shard_global_ids(shard, ids)
        pid64 = pid.to(torch.int64).contiguous()
        hntl.shard_global_ids(shard, pid64)
        torch.cuda.synchronize()
        gpu = dict(ids=ids.cpu().numpy(), dist=dist.cpu().numpy(), pool_ids=pid64.cpu().numpy().astype(np.uint32),
                   pool_d=pd.cpu().numpy(), probe=probe.cpu().numpy())
        st = compare_search(gpu, per[s], k, C, nprobe)
        assert st["checked"] >= 0.8 * len(Q), (s, st)
        assert hntl.device_status(shard) == 0
    mi, md = sh.search(Qd, k, C, nprobe)
    mi, md = mi.cpu().numpy(), md.cpu().numpy()
    ext = _merged_ext(per, k)
    for qi in range(len(Q)):
        check_ranked(mi[qi], md[qi], oi[qi], np.append(od[qi], ext[qi]), "merged", qi, invalid=-1)


@pytest.mark.parametrize("precision", ["fp32", "bf16-fp8"])
def test_single_shard_equals_whole_index(hntl, case, precision):
    """One shard holds every grain with the same codes and rows in the same
    id order: its search equals the whole index's bit for bit."""
    X, Q, idx, p32, p8 = case
    prec = hntl.PREC_FP32 if precision == "fp32" else hntl.PREC_BF16_FP8
    gi = hntl.Index.load(p32 if precision == "fp32" else p8, 0, prec)
    one = hntl.ShardedIndex(gi, 1)
    Qd = torch.from_numpy(Q).cuda()
    a = gi.search(Qd, 10, 100, 8, return_pool=True)
    b = one.shards[0].search(Qd, 10, 100, 8, return_pool=True)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    mi, md = one.search(Qd, 10, 100, 8)
    assert torch.equal(mi, a[0]) and torch.equal(md, a[1])


def test_merge_kernel_equals_host_merge(hntl):
    rng = np.random.default_rng(9)
    S, nq, k = 5, 300, 20
    ids = rng.permutation(S * nq * k * 4)[: S * nq * k].reshape(S, nq, k).astype(np.int64)
    dist = rng.integers(0, 50, (S, nq, k)).astype(np.float32)  # many equal distances: ids decide
    pad = rng.random((S, nq, k)) < 0.3
    ids[pad] = -1
    dist[pad] = rng.choice([np.inf, 0.0], pad.sum())
    hi, hd = hntl.merge_topk_host(ids, dist)
    gi_, gd_ = hntl.merge_topk(torch.from_numpy(ids).cuda(), torch.from_numpy(dist).cuda())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(gi_.cpu().numpy(), hi)
    np.testing.assert_array_equal(gd_.cpu().numpy(), hd)
    # against a sort by (distance, id) of the real entries
    for q in range(0, nq, 37):
        c = sorted((float(dist[s, q, j]), int(ids[s, q, j])) for s in range(S) for j in range(k) if ids[s, q, j] >= 0)
        want = [i for _, i in c[:k]] + [-1] * max(0, k - len(c))
        assert hi[q].tolist() == want
