"""Precision form (BF16 rows, FP8-E4M3 coordinates with a per-grain scale,
BF16 routing and projection, FP32 accumulation and FP32 exact rerank) on the
GPU against the oracle's precision form on the same index file, plus the
per-stage error of the precision form against the plain FP32 method."""
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


def run(h, path, Q, k, C, nprobe, filters=None):
    gi = h.Index.load(path, 0, h.PREC_BF16_FP8)
    F = None if filters is None else torch.from_numpy(filters).cuda()
    ids, dist, pid, pd, probe = gi.search(torch.from_numpy(Q).cuda(), k, C, nprobe, filters=F, return_pool=True,
                                          return_probe=True)
    torch.cuda.synchronize()
    return gi, dict(ids=ids.cpu().numpy(), dist=dist.cpu().numpy(), pool_ids=pid.cpu().numpy().view(np.uint32),
                    pool_d=pd.cpu().numpy(), probe=probe.cpu().numpy())


def test_precision_10k_workload_parity(hntl, tmp_path):
    w = synth.WORKLOADS["plain-10k"]
    X, Q, idx = clustered_case(w["n"], w["d"], w["n_clusters"], w["G"], w["r"], 400, w["seed"], train=256 * w["G"])
    p = write(tmp_path, "prec10k", idx, X, precision="bf16-fp8")
    ora = O.search(idx, X, Q, 10, 20, 4, precision="bf16-fp8")
    _, gpu = run(hntl, p, Q, 10, 20, 4)
    st = compare_search(gpu, ora, 10, 20, 4)
    assert st["checked"] >= 0.95 * len(Q), st


@pytest.mark.parametrize("d,r", [(24, 5), (16, 16), (64, 8)])
@pytest.mark.parametrize("k,C,nprobe", [(10, 20, 2), (5, 200, 3), (10, 685, 6)])
def test_precision_edge_shapes(hntl, tmp_path, d, r, k, C, nprobe):
    sizes = [0, 1, 127, 128, 129, 300]
    rng = np.random.default_rng(d + r)
    centres = rng.standard_normal((len(sizes), d)) * 3
    assign = np.repeat(np.arange(len(sizes)), sizes)
    X = (centres[assign] + rng.standard_normal((len(assign), d)) * 0.7).astype(np.float32)
    idx = partition_index(X, assign, len(sizes), r)
    Q = (centres[rng.integers(0, len(sizes), 30)] + rng.standard_normal((30, d)) * 0.7).astype(np.float32)
    p = write(tmp_path, f"pe{d}_{r}", idx, X, precision="bf16-fp8")
    ora = O.search(idx, X, Q, k, C, nprobe, precision="bf16-fp8")
    _, gpu = run(hntl, p, Q, k, C, nprobe)
    st = compare_search(gpu, ora, k, C, nprobe)
    assert st["checked"] >= len(Q) // 2, st


def test_precision_filters(hntl, tmp_path):
    X, Q, idx = clustered_case(3000, 32, 8, 8, 6, 60, seed=177)
    attr = synth.attributes(len(X), 5, span=1 << 40).numpy()
    ranges = synth.range_filters(len(Q), 6, span=1 << 40, selectivity=0.2, frac_filtered=0.5).numpy()
    p = write(tmp_path, "pfilt", idx, X, attr=attr, precision="bf16-fp8")
    ora = O.search(idx, X, Q, 10, 50, 3, attr=attr, ranges=ranges, precision="bf16-fp8")
    _, gpu = run(hntl, p, Q, 10, 50, 3, filters=ranges)
    st = compare_search(gpu, ora, 10, 50, 3)
    assert st["checked"] >= 0.9 * len(Q), st


def test_precision_form_needs_d_multiple_of_8(hntl, tmp_path):
    # d = 12: BF16 rows are not a whole number of 16-byte pieces
    X, Q, idx = clustered_case(500, 12, 4, 4, 4, 4, seed=5)
    with pytest.raises(hntl.HntlError) as e:
        hntl.Index.load(write(tmp_path, "p12", idx, X, precision="bf16-fp8"), 0, hntl.PREC_BF16_FP8)
    assert e.value.code == hntl.EINVAL
    with pytest.raises(hntl.HntlError) as e:
        hntl.Index.build(torch.from_numpy(X).cuda(), 4, 4, precision=hntl.PREC_BF16_FP8)
    assert e.value.code == hntl.EINVAL


def test_per_stage_error_of_precision_form(hntl, tmp_path):
    """Per-stage distance error of the precision form against the plain FP32
    method (both FP64 oracle arithmetic), on the 10k-row workload: routing
    agreement, approximate-distance error of the pool, exact-distance error of
    the BF16 rerank, and recall against brute force."""
    w = synth.WORKLOADS["plain-10k"]
    X, Q, idx = clustered_case(w["n"], w["d"], w["n_clusters"], w["G"], w["r"], 300, w["seed"], train=256 * w["G"])
    plain = O.search(idx, X, Q, 10, 20, 4)
    prec = O.search(idx, X, Q, 10, 20, 4, precision="bf16-fp8")
    route_same = np.mean([set(a) == set(b) for a, b in zip(plain["probe"].tolist(), prec["probe"].tolist())])
    d_err = []
    for qi in range(len(Q)):
        pd = dict(zip(plain["cand_id"][qi].tolist(), plain["cand_d"][qi][:20]))
        for cid, dv in zip(prec["cand_id"][qi].tolist(), prec["cand_d"][qi][:20]):
            if cid in pd:
                d_err.append(abs(dv - pd[cid]) / pd[cid])
    x_err = []
    for qi in range(len(Q)):
        od = dict(zip(plain["out_id"][qi].tolist(), plain["out_d"][qi][:10]))
        for cid, dv in zip(prec["out_id"][qi].tolist(), prec["out_d"][qi][:10]):
            if cid in od:
                x_err.append(abs(dv - od[cid]) / od[cid])
    bf, _, _ = O.brute_force(X, Q, 10)
    rec = lambda res: np.mean([len(set(a.tolist()) & set(b.tolist())) / 10 for a, b in zip(res["out_id"], bf)])
    report = dict(route_agreement=route_same, pool_D_rel_err_median=float(np.median(d_err)),
                  pool_D_rel_err_max=float(np.max(d_err)), rerank_rel_err_max=float(np.max(x_err)),
                  recall_plain=rec(plain), recall_precision=rec(prec))
    print("precision report", report)
    assert route_same >= 0.98
    assert report["pool_D_rel_err_median"] < 1e-2
    assert report["rerank_rel_err_max"] < 2e-2      # BF16 rows: ~2^-9 relative per coordinate
    assert report["recall_precision"] >= report["recall_plain"] - 0.02
    # and the GPU precision form reproduces the oracle's precision form on this workload
    p = write(tmp_path, "prec_rep", idx, X, precision="bf16-fp8")
    _, gpu = run(hntl, p, Q, 10, 20, 4)
    st = compare_search(gpu, prec, 10, 20, 4)
    assert st["checked"] >= 0.95 * len(Q), st


def test_builder_precision_form(hntl):
    w = synth.WORKLOADS["plain-10k"]
    m = synth.make_cluster_model(w["n"], w["d"], w["n_clusters"], sizes=w["sizes"], seed=w["seed"])
    X, _ = synth.sample_points(m, w["seed"] + 1)
    Q, _ = synth.sample_queries(m, 300, w["seed"] + 2)
    gi = hntl.Index.build(X.cuda(), w["G"], w["r"], precision=hntl.PREC_BF16_FP8, u=synth.uniforms(w["G"], 3).numpy())
    exp = gi.export()
    # decoded FP8 coordinates sit within half an E4M3 step of Eq. 1-4 under the built basis
    off = exp["grain_off"]
    Xn = X.numpy()
    for g in range(0, exp["G"], 4):
        rows = exp["ids"][off[g]:off[g + 1]]
        V = Xn[rows].astype(np.float64) - exp["M"][g].astype(np.float64)
        Z = V @ exp["U"][g].astype(np.float64).T
        s = np.abs(Z).max() / 448.0
        err = np.abs(exp["Z"][off[g]:off[g + 1]] - Z)
        assert np.all(err <= np.maximum(np.abs(Z) * 2.0 ** -4, s * 2.0 ** -9) * 1.01 + 1e-6)
    ids, dist = gi.search(Q.cuda(), 10, w["C"], w["nprobe"])
    bf, _, _ = O.brute_force(Xn, Q.numpy(), 10)
    rec = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ids.cpu().numpy().tolist(), bf.tolist())])
    assert rec >= 0.95


def test_refined_rerank_matches_oracle_and_recovers_recall(hntl):
    """Precision form built on the GPU with HNTL_RERANK_REFINE: the pool is the
    precision form's, the top k comes from the two-stage rerank (the min(C, 2k)
    best by distance to the BF16 rows, ranked again on both BF16 parts). Pool
    and top k against the oracle's refined search of the exported index (the
    FP32 rows give both parts), under the gap rule; recall against brute force
    at least the unrefined form's; one shard of the index returns the same."""
    n, d, G, r, nq = 60_000, 128, 48, 16, 256
    k, C, nprobe = 10, 100, 6
    m = synth.make_cluster_model(n, d, 12, seed=731)
    X, _ = synth.sample_points(m, 732)
    Q, _ = synth.sample_queries(m, nq, 733)
    u = synth.uniforms(G, 734).numpy()
    gi = hntl.Index.build(X.cuda(), G, r, precision=hntl.PREC_BF16_FP8 | hntl.RERANK_REFINE, u=u, seed=734)
    g0 = hntl.Index.build(X.cuda(), G, r, precision=hntl.PREC_BF16_FP8, u=u, seed=734)
    Qd = Q.cuda()
    ids, dist, pid, pd, probe = gi.search(Qd, k, C, nprobe, return_pool=True, return_probe=True)
    ids0, _ = g0.search(Qd, k, C, nprobe)
    torch.cuda.synchronize()
    assert hntl.device_status(gi) == 0
    gpu = dict(ids=ids.cpu().numpy(), dist=dist.cpu().numpy(), pool_ids=pid.cpu().numpy().view(np.uint32),
               pool_d=pd.cpu().numpy(), probe=probe.cpu().numpy())
    host = gi.export()
    Xn, Qn = X.numpy(), Q.numpy()
    ora = O.search(host, Xn, Qn, k, C, nprobe, precision="bf16-fp8", Z=host["Z"], refine=True)
    st = compare_search(gpu, ora, k, C, nprobe)
    assert st["checked"] >= 0.8 * nq, st
    bf, _, _ = O.brute_force(Xn, Qn, k)
    rec = lambda a: np.mean([len(set(x.tolist()) & set(y.tolist())) / k for x, y in zip(a, bf)])
    r_ref, r_plain = rec(gpu["ids"]), rec(ids0.cpu().numpy())
    print("recall@10 refined", r_ref, "BF16 rows", r_plain)
    assert r_ref >= r_plain
    one = hntl.ShardedIndex(gi, 1)
    a = one.shards[0].search(Qd, k, C, nprobe)
    assert torch.equal(a[0], ids) and torch.equal(a[1], dist)
