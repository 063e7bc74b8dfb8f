"""The library's GPU index builder against the oracle's build on the same rows
and the same k-means++ draws."""
import numpy as np
import pytest
import torch

from oracle import hntl_oracle as O
from paper_2606_08813_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hntl():
    from paper_2606_08813_b300 import build_lib

    build_lib.build()
    from paper_2606_08813_b300 import hntl as h

    return h


def _partition_sets(assign):
    groups = {}
    for i, g in enumerate(assign.tolist()):
        groups.setdefault(g, []).append(i)
    return sorted(tuple(v) for v in groups.values())


@pytest.fixture(scope="module")
def plain10k(hntl):
    w = synth.WORKLOADS["plain-10k"]
    m = synth.make_cluster_model(w["n"], w["d"], w["n_clusters"], sizes=w["sizes"], seed=w["seed"])
    X, _ = synth.sample_points(m, w["seed"] + 1)
    X = X.numpy()
    G, r = w["G"], w["r"]
    u = synth.uniforms(G, 12345).numpy()
    ora = O.build_index(X, G, r, u, keep_fp64=False)
    Xd = torch.from_numpy(X).cuda()
    gi = hntl.Index.build(Xd, G, r, u=u, n_train=len(X), n_seed=len(X), max_iter=25, seed=3)
    exp = gi.export()
    return X, ora, gi, exp


def test_partition_matches_oracle(plain10k):
    X, ora, gi, exp = plain10k
    g_assign = np.zeros(len(X), dtype=np.int64)
    off = exp["grain_off"]
    for g in range(exp["G"]):
        g_assign[exp["ids"][off[g]:off[g + 1]]] = g
    assert _partition_sets(g_assign) == _partition_sets(ora["assign"])


def test_centres_are_member_means(plain10k):
    X, ora, gi, exp = plain10k
    off = exp["grain_off"]
    for g in range(exp["G"]):
        mem = X[exp["ids"][off[g]:off[g + 1]]].astype(np.float64)
        np.testing.assert_allclose(exp["M"][g], mem.mean(0), rtol=0, atol=2e-6 * (1 + np.abs(mem).max()))


def test_bases_orthonormal_and_capture_top_variance(plain10k):
    X, ora, gi, exp = plain10k
    off = exp["grain_off"]
    r = exp["r"]
    for g in range(exp["G"]):
        U = exp["U"][g].astype(np.float64)
        np.testing.assert_allclose(U @ U.T, np.eye(r), atol=2e-5)
        rows = exp["ids"][off[g]:off[g + 1]]
        V = X[rows].astype(np.float64) - exp["M"][g].astype(np.float64)
        cov = V.T @ V / len(rows)
        captured = np.trace(U @ cov @ U.T)
        lam = np.linalg.eigvalsh(cov)[::-1]
        assert captured >= 0.99 * lam[:r].sum(), (g, captured, lam[:r].sum())


def test_coordinates_follow_eq1_to_eq4_under_the_built_basis(plain10k):
    X, ora, gi, exp = plain10k
    off = exp["grain_off"]
    for g in range(0, exp["G"], 5):
        rows = exp["ids"][off[g]:off[g + 1]]
        V = X[rows].astype(np.float64) - exp["M"][g].astype(np.float64)
        U = exp["U"][g].astype(np.float64)
        Z = V @ U.T
        E = V - Z @ U
        rho = (E * E).sum(1)
        np.testing.assert_allclose(exp["Z"][off[g]:off[g + 1]], Z, rtol=0, atol=2e-5 * np.abs(V).max())
        np.testing.assert_allclose(exp["rho"][off[g]:off[g + 1]], rho, rtol=1e-4, atol=1e-6)


def test_search_on_built_index_reaches_recall(plain10k, hntl):
    X, ora, gi, exp = plain10k
    w = synth.WORKLOADS["plain-10k"]
    m = synth.make_cluster_model(w["n"], w["d"], w["n_clusters"], sizes=w["sizes"], seed=w["seed"])
    Q, _ = synth.sample_queries(m, 300, w["seed"] + 2)
    ids, dist = gi.search(Q.cuda(), 10, w["C"], w["nprobe"])
    bf, _, _ = O.brute_force(X, Q.numpy(), 10)
    rec = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ids.cpu().numpy().tolist(), bf.tolist())])
    assert rec >= 0.95


def test_small_and_degenerate_grains(hntl):
    """More grains than distinct clusters, a grain with fewer rows than r and
    duplicated rows: bases must still be orthonormal (completed)."""
    rng = np.random.default_rng(3)
    base = rng.standard_normal((5, 32)).astype(np.float32) * 5
    dup = np.repeat(base[:1], 200, 0)                                   # 200 identical rows
    few = base[1:2] + 0.01 * rng.standard_normal((3, 32))               # 3 rows (< r)
    rest = base[2 + np.arange(600) % 3] + rng.standard_normal((600, 32))
    X = np.concatenate([dup, few, rest]).astype(np.float32)
    gi = hntl.Index.build(torch.from_numpy(X).cuda(), 12, 8, seed=1)
    exp = gi.export()
    for g in range(12):
        U = exp["U"][g].astype(np.float64)
        np.testing.assert_allclose(U @ U.T, np.eye(8), atol=2e-5)
    assert exp["grain_off"][-1] == len(X)
    assert sorted(exp["ids"].tolist()) == list(range(len(X)))


def test_built_int16_form_matches_oracle_quantisation_and_search(hntl, plain10k):
    """The builder's 16-bit form is the oracle's quantisation (int16_form) of the
    same build's FP32 coordinates, value for value, and searching it agrees
    with the oracle's 16-bit search on that index."""
    X, ora, gi, exp = plain10k
    w = synth.WORKLOADS["plain-10k"]
    G, r = w["G"], w["r"]
    u = synth.uniforms(G, 12345).numpy()
    gi16 = hntl.Index.build(torch.from_numpy(X).cuda(), G, r, u=u, n_train=len(X), n_seed=len(X), max_iter=25,
                            seed=3, precision=hntl.PREC_INT16)
    e16 = gi16.export()
    np.testing.assert_array_equal(e16["ids"], exp["ids"])  # the same partition and order
    f = O.int16_form(exp)
    np.testing.assert_array_equal(e16["Z"], f["Zf32"])
    np.testing.assert_array_equal(e16["rho"], f["rhof32"])
    Q, _ = synth.sample_queries(synth.make_cluster_model(w["n"], w["d"], w["n_clusters"], sizes=w["sizes"],
                                                         seed=w["seed"]), 200, 77)
    Q = Q.numpy()
    ids, dist = gi16.search(torch.from_numpy(Q).cuda(), 10, 20, 4)
    ref = O.search(exp, X, Q, 10, 20, 4, precision="int16")
    agree = np.mean([len(set(a.tolist()) & set(b.tolist())) / 10 for a, b in zip(ids.cpu().numpy(), ref["out_id"])])
    assert agree > 0.99, agree


def test_basis_spans_the_oracle_eigenvectors_above_the_gap(plain10k):
    """Principal angles against the oracle's eigendecomposition of the same
    members: the workload's rows vary along 8 directions per cluster (stds
    0.8^i) above an isotropic floor (0.05^2), so the top 8 eigenvectors are
    well separated from the rest; each must lie in the GPU basis's span (its
    projection keeps 1 - 1e-6 of its length)."""
    X, ora, gi, exp = plain10k
    off = exp["grain_off"]
    for g in range(exp["G"]):
        rows = exp["ids"][off[g]:off[g + 1]]
        U = exp["U"][g].astype(np.float64)
        E, _ = O.grain_pca(X, rows, exp["M"][g], 8)
        for j in range(8):
            e = E[j]
            kept = np.linalg.norm(U @ e)
            assert kept >= 1 - 1e-6, (g, j, kept)


def test_capacity_bounded_grains_match_oracle(hntl):
    """Zipf clusters (the largest far above N / G rows) into grains of at most
    ceil(1.05 N / G) rows: the GPU's deferred acceptance (top-8 lists on the
    GPU, proposals on the host) against the oracle's, from the same k-means++
    draws and Lloyd iterations."""
    n, d, G = 12000, 48, 96
    m = synth.make_cluster_model(n, d, 12, sizes="zipf", seed=321)
    X, _ = synth.sample_points(m, 322)
    X = X.numpy()
    cap = int(np.ceil(1.05 * n / G))
    u = synth.uniforms(G, 323).numpy()
    ora = O.build_index(X, G, 8, u, max_grain_rows=cap)
    plain = O.build_index(X, G, 8, u)
    assert np.bincount(plain["assign"], minlength=G).max() > cap  # the premise: plain grains overflow the cap
    gi = hntl.Index.build(torch.from_numpy(X).cuda(), G, 8, u=u, n_train=n, n_seed=n, max_iter=25, seed=3,
                          max_grain_rows=cap)
    exp = gi.export()
    off = exp["grain_off"]
    assert np.diff(off).max() <= cap
    g_assign = np.zeros(n, dtype=np.int64)
    for g in range(G):
        g_assign[exp["ids"][off[g]:off[g + 1]]] = g
    assert (g_assign == ora["assign"]).mean() >= 0.999, (g_assign == ora["assign"]).mean()
    with pytest.raises(hntl.HntlError):  # a cap below N / G cannot hold every row
        hntl.Index.build(torch.from_numpy(X).cuda(), G, 8, u=u, max_grain_rows=n // G - 1)
