"""CUDA path against the oracle, element by element, on the same index file.

Gap rule and tolerances are in tests/parity.py: ids must match wherever the
oracle's ranking has a relative gap > 1e-4; FP32 distances within 1e-5
relative of the FP64 oracle.
"""
import numpy as np
import pytest
import torch

from oracle import hntl_oracle as O
from paper_2606_08813_b300 import synth

from cases import clustered_case, partition_index, write
from parity import compare_search

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hntl():
    from paper_2606_08813_b300 import build_lib

    build_lib.build()
    from paper_2606_08813_b300 import hntl as h

    return h


def run_gpu(h, path, Q, k, C, nprobe, filters=None, precision=0):
    gi = h.Index.load(path, 0, precision)
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    F = None if filters is None else torch.from_numpy(np.ascontiguousarray(filters)).cuda()
    ids, dist, pid, pd, probe = gi.search(Qd, k, C, nprobe, filters=F, return_pool=True, return_probe=True)
    torch.cuda.synchronize()
    out = dict(ids=ids.cpu().numpy(), dist=dist.cpu().numpy(), pool_ids=pid.cpu().numpy().view(np.uint32),
               pool_d=pd.cpu().numpy(), probe=probe.cpu().numpy())
    return gi, out


def test_plain_10k_workload(hntl, tmp_path):
    """N=10k, d=768, 32 equal clusters, G=32, r=16, 1000 queries, nprobe=4, C=20, k=10."""
    w = synth.WORKLOADS["plain-10k"]
    X, Q, idx = clustered_case(w["n"], w["d"], w["n_clusters"], w["G"], w["r"], w["nq"], w["seed"],
                               train=256 * w["G"])
    p = write(tmp_path, "plain10k", idx, X)
    ora = O.search(idx, X, Q, w["k"], w["C"], w["nprobe"])
    gi, gpu = run_gpu(hntl, p, Q, w["k"], w["C"], w["nprobe"])
    st = compare_search(gpu, ora, w["k"], w["C"], w["nprobe"])
    assert st["checked"] >= 0.95 * w["nq"], st
    # routing distances
    probe, pd = gi.route(torch.from_numpy(Q).cuda(), w["nprobe"])
    pd = pd.cpu().numpy().astype(np.float64)
    ref = ora["probe_d"][:, :w["nprobe"]]
    same = (probe.cpu().numpy() == ora["probe"]).all(1)
    assert same.mean() > 0.99
    np.testing.assert_allclose(pd[same], ref[same], rtol=1e-5)


EDGE_SIZES = [0, 1, 127, 128, 129, 300]


def _edge_case(d, r, seed, nq=40):
    G = len(EDGE_SIZES)
    n = sum(EDGE_SIZES)
    rng = np.random.default_rng(seed)
    centres = rng.standard_normal((G, d)) * 3
    assign = np.repeat(np.arange(G), EDGE_SIZES)
    X = (centres[assign] + rng.standard_normal((n, d)) * 0.7).astype(np.float32)
    perm = rng.permutation(n)
    X = X[perm]
    assign = assign[perm]
    idx = partition_index(X, assign, G, r)
    qc = rng.integers(0, G, nq)
    Q = (centres[qc] + rng.standard_normal((nq, d)) * 0.7).astype(np.float32)
    return X, Q, idx


@pytest.mark.parametrize("d,r", [(24, 5), (13, 3), (16, 16), (40, 1), (64, 64)])
@pytest.mark.parametrize("k,C,nprobe", [(10, 20, 2), (5, 200, 3), (1, 1, 1), (50, 50, 6), (10, 1024, 6),
                                        (10, 685, 6)])
def test_edge_grain_sizes(hntl, tmp_path, d, r, k, C, nprobe):
    X, Q, idx = _edge_case(d, r, seed=d * 100 + r)
    p = write(tmp_path, f"edge{d}_{r}", idx, X)
    ora = O.search(idx, X, Q, k, C, nprobe)
    _, gpu = run_gpu(hntl, p, Q, k, C, nprobe)
    st = compare_search(gpu, ora, k, C, nprobe)
    assert st["checked"] + st["route_excluded"] + st["topk_excluded"] == len(Q)
    assert st["checked"] >= len(Q) // 2, st


def test_full_basis_all_probes_equals_brute_force(hntl, tmp_path):
    X, Q, idx = _edge_case(16, 16, seed=7)
    p = write(tmp_path, "full", idx, X)
    _, gpu = run_gpu(hntl, p, Q, 10, len(X), len(EDGE_SIZES))
    bf, bd, nxt = O.brute_force(X, Q, 10)
    for qi in range(len(Q)):
        ext = np.append(bd[qi], nxt[qi])
        for m in range(1, 11):
            if (ext[m] - ext[m - 1]) / ext[m - 1] > 1e-4:
                assert set(gpu["ids"][qi][:m].tolist()) == set(bf[qi][:m].tolist())
    np.testing.assert_allclose(np.sort(gpu["dist"], 1), bd, rtol=1e-5)


def test_filters_in_scan(hntl, tmp_path):
    X, Q, idx = clustered_case(3000, 32, 8, 8, 6, 60, seed=77)
    attr = synth.attributes(len(X), 5, span=1 << 40).numpy()
    ranges = synth.range_filters(len(Q), 6, span=1 << 40, selectivity=0.2, frac_filtered=0.5).numpy()
    p = write(tmp_path, "filt", idx, X, attr=attr)
    ora = O.search(idx, X, Q, 10, 50, 3, attr=attr, ranges=ranges)
    _, gpu = run_gpu(hntl, p, Q, 10, 50, 3, filters=ranges)
    st = compare_search(gpu, ora, 10, 50, 3)
    assert st["checked"] >= 0.9 * len(Q), st


def test_many_grains_route_select(hntl, tmp_path):
    X, Q, idx = clustered_case(20000, 64, 700, 700, 8, 200, seed=88)
    p = write(tmp_path, "many", idx, X)
    ora = O.search(idx, X, Q, 10, 100, 40)
    _, gpu = run_gpu(hntl, p, Q, 10, 100, 40)
    st = compare_search(gpu, ora, 10, 100, 40)
    # 700 grains of ~28 rows probed 40 at a time: near ties at the pool boundary are common
    assert st["checked"] >= 0.75 * len(Q), st


def test_duplicate_rows_tie_break_by_id(hntl, tmp_path):
    """Groups of identical rows give exactly equal distances on both sides;
    the (distance, id) order then fixes which ids are returned."""
    rng = np.random.default_rng(5)
    base = rng.standard_normal((40, 16)).astype(np.float32)
    X = np.repeat(base, 30, axis=0)  # 1200 rows, 30 copies each
    X = X[rng.permutation(len(X))]
    idx = O.build_index(X, 4, 4, synth.uniforms(4, 1).numpy())
    Q = (base[:10] + 0.01 * rng.standard_normal((10, 16))).astype(np.float32)
    p = write(tmp_path, "dup", idx, X)
    ora = O.search(idx, X, Q, 10, 45, 2)
    _, gpu = run_gpu(hntl, p, Q, 10, 45, 2)
    np.testing.assert_array_equal(gpu["pool_ids"], ora["cand_id"])
    np.testing.assert_array_equal(gpu["ids"], ora["out_id"])


def test_more_ties_than_tie_buffer(hntl, tmp_path):
    """2000 identical rows in one grain: every D is equal, so the pool is the
    1000 smallest ids (the path that handles more ties than its buffer)."""
    rng = np.random.default_rng(6)
    X = np.repeat(rng.standard_normal((1, 8)).astype(np.float32), 2000, axis=0)
    idx = partition_index(X, np.zeros(2000, dtype=np.int64), 1, 2)
    Q = rng.standard_normal((3, 8)).astype(np.float32)
    p = write(tmp_path, "ties", idx, X)
    _, gpu = run_gpu(hntl, p, Q, 10, 1000, 1)
    for qi in range(3):
        assert gpu["pool_ids"][qi].tolist() == list(range(1000))
        assert gpu["ids"][qi].tolist() == list(range(10))


@pytest.mark.parametrize("precision", ["fp32", "bf16-fp8"])
def test_duplicated_rows_keep_ties_in_id_order(hntl, tmp_path, precision):
    """Every row three times (ids i, i + n, i + 2 n have one D): the pool holds
    all copies of every D below its last value, and of the last value's copies
    the smallest ids; equal D are listed by ascending id. Against the oracle,
    the pool sets agree at every gap between copy groups."""
    n0 = 3000
    X0, Q, idx0 = clustered_case(n0, 32, 6, 6, 8, 64, seed=131)
    assign0 = np.zeros(n0, dtype=np.int64)
    for g in range(len(idx0["grain_off"]) - 1):
        assign0[idx0["ids"][idx0["grain_off"][g]:idx0["grain_off"][g + 1]]] = g
    X = np.concatenate([X0, X0, X0])
    idx = partition_index(X, np.tile(assign0, 3), 6, 8)
    p = write(tmp_path, "dup" + precision, idx, X, precision=precision)
    C = 100  # not a multiple of 3: the last copy group is cut
    prec = hntl.PREC_BF16_FP8 if precision == "bf16-fp8" else hntl.PREC_FP32
    _, gpu = run_gpu(hntl, p, Q, 10, C, 2, precision=prec)
    cut_groups = 0
    for qi in range(len(Q)):
        ids = gpu["pool_ids"][qi].astype(np.int64)
        d = gpu["pool_d"][qi]
        assert (ids != 0xFFFFFFFF).all()
        key = list(zip(d.tolist(), ids.tolist()))
        assert key == sorted(key) and len(set(ids.tolist())) == C, f"query {qi}: not in (D, id) order"
        present = set(ids.tolist())
        last = d[-1]
        for i, dv in zip(ids.tolist(), d.tolist()):
            copies = [i % n0 + c * n0 for c in range(3)]
            if dv < last:
                assert all(c in present for c in copies), f"query {qi}: copies of {i} missing"
        tail = sorted(i for i, dv in zip(ids.tolist(), d.tolist()) if dv == last)
        base = {i % n0 for i in tail}
        group = sorted(b + c * n0 for b in base for c in range(3))
        if len(base) == 1:  # one copy group at the edge: its smallest ids are kept
            assert tail == group[:len(tail)], f"query {qi}: edge copies {tail} of {group}"
            cut_groups += len(tail) < 3
    assert cut_groups > 0  # the cut group really occurred
    if precision == "fp32":
        ora = O.search(idx, X, Q, 10, C, 2)
        st = compare_search(gpu, ora, 10, C, 2)
        # the pool edge falls inside a copy group (a tie), so the gap rule leaves
        # the top-k comparison out; the pools themselves are compared
        assert st["route_excluded"] == 0 and st["checked"] + st["topk_excluded"] == len(Q), st


def test_host_form_matches_device_form(hntl, tmp_path):
    X, Q, idx = clustered_case(2000, 32, 4, 4, 8, 50, seed=99)
    p = write(tmp_path, "host", idx, X)
    gi, gpu = run_gpu(hntl, p, Q, 10, 40, 2)
    hid, hd = gi.search_host(torch.from_numpy(Q).pin_memory(), 10, 40, 2)
    np.testing.assert_array_equal(hid.numpy(), gpu["ids"])
    np.testing.assert_array_equal(hd.numpy(), gpu["dist"])


def test_repeat_calls_are_deterministic(hntl, tmp_path):
    X, Q, idx = clustered_case(3000, 32, 6, 6, 8, 64, seed=111)
    p = write(tmp_path, "det", idx, X)
    gi = hntl.Index.load(p, 0)
    Qd = torch.from_numpy(Q).cuda()
    a = [t.cpu() for t in gi.search(Qd, 10, 60, 3, return_pool=True)]
    b = [t.cpu() for t in gi.search(Qd, 10, 60, 3, return_pool=True)]
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_invalid_arguments(hntl, tmp_path):
    X, Q, idx = clustered_case(500, 16, 4, 4, 4, 4, seed=5)
    gi = hntl.Index.load(write(tmp_path, "inv", idx, X), 0)
    Qd = torch.from_numpy(Q).cuda()
    for k, C, npb in [(0, 10, 1), (10, 2000, 1), (5, 10, 0), (5, 10, 5)]:
        with pytest.raises(hntl.HntlError) as e:
            gi.search(Qd, k, C, npb)
        assert e.value.code == hntl.EINVAL
    with pytest.raises(hntl.HntlError) as e:
        gi.search(Qd, 5, 10, 2, filters=torch.zeros(4, 2, dtype=torch.int64, device="cuda"))
    assert e.value.code == hntl.EINVAL  # no attribute column in this index
    # empty batch is a no-op
    ids, dist = gi.search(Qd[:0], 5, 10, 2)
    assert ids.shape == (0, 5)


def test_survivor_overflow_falls_back_exactly(hntl, tmp_path):
    """One 100k-row grain with C=1000: the pilot sees at most a 2048-row sample, so its
    bound admits far more than the survivor buffer holds; the pool must then
    come from every probed row, recomputed, with the same result."""
    rng = np.random.default_rng(11)
    X = (rng.standard_normal((100_000, 16)) * np.linspace(3, 0.5, 16)).astype(np.float32)
    idx = partition_index(X, np.zeros(len(X), dtype=np.int64), 1, 4)
    Q = (rng.standard_normal((6, 16)) * np.linspace(3, 0.5, 16)).astype(np.float32)
    p = write(tmp_path, "overflow", idx, X)
    ora = O.search(idx, X, Q, 10, 1000, 1)
    _, gpu = run_gpu(hntl, p, Q, 10, 1000, 1)
    st = compare_search(gpu, ora, 10, 1000, 1)
    # every query's pool was compared (dense grain: rank-1000 neighbours are near ties, so the
    # top-k comparison is often excluded by the gap rule, but the pool itself is checked)
    assert st["route_excluded"] == 0 and st["checked"] + st["topk_excluded"] == len(Q), st


def test_filtered_pilot_needs_several_probes(hntl, tmp_path):
    """A 2% selective filter leaves fewer than C rows in the nearest grain, so
    the pilot must continue through later probes (or admit everything)."""
    X, Q, idx = clustered_case(6000, 32, 6, 6, 6, 40, seed=123)
    attr = synth.attributes(len(X), 9, span=1000).numpy()
    ranges = np.tile(np.array([[100, 119]], dtype=np.int64), (len(Q), 1))
    p = write(tmp_path, "pilotfilt", idx, X, attr=attr)
    ora = O.search(idx, X, Q, 10, 30, 4, attr=attr, ranges=ranges)
    _, gpu = run_gpu(hntl, p, Q, 10, 30, 4, filters=ranges)
    st = compare_search(gpu, ora, 10, 30, 4)
    assert st["checked"] >= 0.9 * len(Q), st
