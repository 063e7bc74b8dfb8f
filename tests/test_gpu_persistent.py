"""Parity of the persistent kernels on the paths full-size batches take.

The routing GEMM, the projections of both forms and both scans of the
precision form run persistent grids (about one CTA per SM) that loop over work items. Small cases
give every CTA one item at most, so these tests either cap the grids
(hntl_debug_set_persistent_cap) until each CTA loops over many items, carrying
its mbarrier phases, TMEM accumulators and prefetches from item to item, or
run a batch of the full shape (d = 768, 4096 queries, nprobe = 32, C = 200) on
a GPU-built index and compare a sample of its queries with the oracle
searching the exported index. Tolerances and the gap rule are those of
tests/parity.py."""
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

    yield h
    h.set_persistent_cap(0)


def _search(h, gi, Q, k, C, nprobe):
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    ws = gi.workspace(gi.workspace_bytes(len(Q), k, C, nprobe))
    ids, dist, pid, pd, probe = gi.search(Qd, k, C, nprobe, return_pool=True, return_probe=True, ws=ws)
    torch.cuda.synchronize()
    stats = h.search_scan_stats(gi, ws, len(Q), C, nprobe)
    return dict(ids=ids.cpu().numpy(), dist=dist.cpu().numpy(), pool_ids=pid.cpu().numpy().view(np.uint32),
                pool_d=pd.cpu().numpy(), probe=probe.cpu().numpy()), stats


@pytest.fixture(scope="module")
def clustered256(tmp_path_factory):
    """8 clusters split into 64 grains (d = 256, r = 32): each query probes
    most grains of its own cluster, so many pairs stay live in the scan."""
    X, Q, idx = clustered_case(40000, 256, 8, 64, 32, 1024, seed=4242, train=256 * 64)
    d = tmp_path_factory.mktemp("persist")
    return X, Q, idx, write(d, "c256_fp32", idx, X), write(d, "c256_p", idx, X, precision="bf16-fp8")


def _capped(h, path, prec, Q, k, C, nprobe, cap):
    h.set_persistent_cap(cap)
    try:
        gi = h.Index.load(path, 0, prec)
        gpu, stats = _search(h, gi, Q, k, C, nprobe)
        assert h.device_status(gi) == 0
    finally:
        h.set_persistent_cap(0)
    return gpu, stats


def _same(a, b):
    for key in a:
        np.testing.assert_array_equal(a[key], b[key], err_msg=key)


def test_precision_form_with_capped_grids(hntl, clustered256):
    """Routing: 8 tiles of 128 queries x 256 centres; projection: 16384 pairs
    in 32-pair slots, >= 128 items; the scans: every item of the batch. With
    cap 1 a single CTA of each kernel walks all of them; cap 3 splits them
    unevenly. Every cap gives the uncapped result bit for bit (each output is
    a function of its own item), and that result matches the oracle."""
    X, Q, idx, _, pp = clustered256
    k, C, nprobe = 10, 100, 16
    ora = O.search(idx, X, Q, k, C, nprobe, precision="bf16-fp8")
    base, stats = _capped(hntl, pp, hntl.PREC_BF16_FP8, Q, k, C, nprobe, 0)
    print("scan items", stats)
    st = compare_search(base, ora, k, C, nprobe)
    assert st["checked"] >= 0.8 * len(Q), st
    assert stats["dense"] + stats["sparse_light"] + stats["sparse_heavy"] > 0
    for cap in (1, 3):
        got, _ = _capped(hntl, pp, hntl.PREC_BF16_FP8, Q, k, C, nprobe, cap)
        _same(got, base)


def test_fp32_form_with_capped_grids(hntl, clustered256):
    """TF32 routing tiles and the FP32 tensor-core projection (z pass and
    explicit residual, persistent over 4-slot items) with many items per CTA:
    the capped run equals the uncapped one bit for bit, which matches the
    oracle."""
    X, Q, idx, pf, _ = clustered256
    k, C, nprobe = 10, 100, 16
    ora = O.search(idx, X, Q, k, C, nprobe)
    base, _ = _capped(hntl, pf, hntl.PREC_FP32, Q, k, C, nprobe, 0)
    st = compare_search(base, ora, k, C, nprobe)
    assert st["checked"] >= 0.8 * len(Q), st
    got, _ = _capped(hntl, pf, hntl.PREC_FP32, Q, k, C, nprobe, 2)
    _same(got, base)


def test_dense_tensor_core_scan_items(hntl, tmp_path):
    """Isotropic rows: a query's pilot bound lies above almost every row's
    residual floor, so most of each grain's 128 pairs stay live and the scan
    contracts them on the tensor cores (dense items); the counters show they
    ran, and the pool and top k match the oracle."""
    n, d, G, r, nq = 12000, 64, 12, 16, 384
    X = synth.isotropic(n, d, seed=501).numpy()
    Q = synth.isotropic(nq, d, seed=502).numpy()
    assign = np.random.default_rng(503).integers(0, G, n)
    idx = partition_index(X, assign, G, r)
    p = write(tmp_path, "iso", idx, X, precision="bf16-fp8")
    k, C, nprobe = 10, 200, 4
    ora = O.search(idx, X, Q, k, C, nprobe, precision="bf16-fp8")
    gpu, stats = _capped(hntl, p, hntl.PREC_BF16_FP8, Q, k, C, nprobe, 0)
    print("scan items", stats)
    assert stats["dense"] > 0, stats
    assert stats["dense_claimed"] >= stats["dense"]
    # isotropic rows crowd the pool's edge with near ties; compared under the gap rule
    st = compare_search(gpu, ora, k, C, nprobe)
    assert st["checked"] >= 0.6 * nq, st
    got, _ = _capped(hntl, p, hntl.PREC_BF16_FP8, Q, k, C, nprobe, 2)
    _same(got, gpu)


def _count_agreeing(gpu, ora, k, C, nprobe):
    """Queries of compare_search that pass, and those that fail (instead of stopping at the first)."""
    ok = bad = 0
    for qi in range(ora["out_id"].shape[0]):
        one = {key: v[qi:qi + 1] for key, v in gpu.items()}
        orq = {key: v[qi:qi + 1] for key, v in ora.items()}
        try:
            st = compare_search(one, orq, k, C, nprobe)
            ok += st["checked"]
        except AssertionError:
            bad += 1
    return ok, bad


@pytest.mark.parametrize("precision", ["bf16-fp8", "fp32"])
def test_full_shape_batch_sampled_against_oracle(hntl, precision):
    """d = 768, G = 2048 grains, 200k rows, one batch of 4096 queries with
    nprobe = 32, C = 200, k = 10 (512 routing tiles, ~4000 projection slots,
    thousands of scan items over ~1.1 CTA-waves of each persistent grid),
    uncapped. The index is built on the GPU and exported; the oracle searches
    the exported arrays (decoded FP8 coordinates, BF16 rows in the precision
    form) for 256 of the queries. Stage by stage:
      projection (Eq. 1-4): z_q and rho_q of every sampled pair against FP64
        on the same rounded inputs, z to 1e-5 of |z|, rho_q to 1e-5 of
        (rho_q + 1) (the scale of the row residual it is added to);
      scan, pool, rerank: against the oracle fed those same probes and
        projections, under the gap rule and 1e-5 of each distance;
      end to end (FP32 form): against the oracle's own projection likewise.
    In the precision form the tensor cores accumulate z in FP32 (z error
    about 1e-6 of |z|), which moves D by 2 (z_q - z_i) . dz: above 1e-5 of D
    for queries whose z is large next to sqrt(D). There the end-to-end
    agreement is reported and held to 95 % of the compared queries."""
    n, d, n_clusters, G, r, nq = 200_000, 768, 2048, 2048, 32, 4096
    k, C, nprobe = 10, 200, 32
    m = synth.make_cluster_model(n, d, n_clusters, seed=611)
    X, _ = synth.sample_points(m, 612)
    Q, _ = synth.sample_queries(m, nq, 613)
    Xd = X.cuda()
    prec = hntl.PREC_BF16_FP8 if precision == "bf16-fp8" else hntl.PREC_FP32
    gi = hntl.Index.build(Xd, G, r, precision=prec, u=synth.uniforms(G, 614).numpy(), seed=614)
    Qn = Q.numpy()
    ws = gi.workspace(gi.workspace_bytes(nq, k, C, nprobe))
    gpu, stats = _search(hntl, gi, Qn, k, C, nprobe)
    zq, rq = hntl.search_pair_proj(gi, ws, nq, C, nprobe)
    zq, rq = zq.cpu().numpy(), rq.cpu().numpy()
    print("scan items", precision, stats)
    assert hntl.device_status(gi) == 0
    host = gi.export()
    Xn = X.numpy()
    if precision == "bf16-fp8":
        Xn = O.bf16_to_f32(O.bf16_round(Xn)).reshape(Xn.shape)
    oprec = "bf16-fp8-decoded" if precision == "bf16-fp8" else "fp32"
    sample = np.random.default_rng(615).choice(nq, 256, replace=False)
    sub = {key: v[sample] for key, v in gpu.items()}
    # projection stage
    bf = (lambda a: O.bf16_to_f32(O.bf16_round(a)).reshape(a.shape)) if precision == "bf16-fp8" else (lambda a: a)
    Mb, Ub, Qb = (bf(host["M"]).astype(np.float64), bf(host["U"]).astype(np.float64),
                  bf(Qn[sample]).astype(np.float64))
    worst = 0.0
    for si, qi in enumerate(sample):
        for p, g in enumerate(gpu["probe"][qi]):
            v = Qb[si] - Mb[g]
            z = Ub[g] @ v
            rho = float(((v - Ub[g].T @ z) ** 2).sum())
            assert np.abs(zq[qi, p] - z).max() <= 1e-5 * max(np.abs(z).max(), 1e-3), (qi, p)
            worst = max(worst, abs(float(rq[qi, p]) - rho) / (rho + 1.0))
    print("projection rho_q worst error / (rho + 1):", worst)
    assert worst <= 1e-5
    # scan, pool and rerank on the GPU's own probes and projections
    ora_g = O.search(host, Xn, Qn[sample], k, C, nprobe, precision=oprec, probes=gpu["probe"][sample],
                     pair_proj=(zq[sample], rq[sample]))
    st = compare_search(sub, ora_g, k, C, nprobe)
    assert st["checked"] >= 0.9 * len(sample), st
    # end to end
    ora = O.search(host, Xn, Qn[sample], k, C, nprobe, precision=oprec)
    if precision == "fp32":
        st = compare_search(sub, ora, k, C, nprobe)
        assert st["checked"] >= 0.75 * len(sample), st
    else:
        ok, bad = _count_agreeing(sub, ora, k, C, nprobe)
        print("end to end against the oracle's own projection: agreeing", ok, "differing", bad)
        assert ok >= 0.95 * (ok + bad) and ok >= 0.7 * len(sample), (ok, bad)
