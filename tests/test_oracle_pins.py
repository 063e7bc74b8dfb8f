"""Pins of the CPU oracle to things other than itself: values the paper
prints, hand-computed fixtures, closed forms, invariants and special cases
that reduce to brute force. CPU only."""
import json
import os

import numpy as np
import pytest
import torch

from oracle import hntl_oracle as O
from paper_2606_08813_b300 import synth

from cases import clustered_case, partition_index
from conftest import GOLDEN


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _clustered(n, d, nc, nq, seed, sizes="equal"):
    m = synth.make_cluster_model(n, d, nc, sizes=sizes, seed=seed)
    X, lab = synth.sample_points(m, seed + 1)
    Q, _ = synth.sample_queries(m, nq, seed + 2)
    return X.numpy(), Q.numpy(), lab.numpy()


# ---------------------------------------------------------------- k-means


def test_kmeans_hand_fixture():
    g = _load("kmeans_line.json")
    X = np.array(g["points"], dtype=np.float32)
    lib = O._c()
    chosen = np.zeros(g["G"], dtype=np.int64)
    u = np.array(g["u"], dtype=np.float64)
    lib.or_kmeanspp(O._p(X), X.shape[0], X.shape[1], g["G"], O._p(u), O._p(chosen))
    assert chosen.tolist() == g["chosen"]
    mu, assign, iters = O.kmeans(X, g["G"], u)
    assert assign.tolist() == g["assign"]
    np.testing.assert_array_equal(mu, np.array(g["means"], dtype=np.float32))
    assert iters == g["lloyd_iterations"]


def _objective(X, M, assign):
    X64 = X.astype(np.float64)
    return float(((X64 - M.astype(np.float64)[assign]) ** 2).sum())


def test_lloyd_objective_non_increasing_and_fixed_point():
    X, _, _ = _clustered(600, 12, 6, 1, 5)
    G = 6
    u = synth.uniforms(G, 9).numpy()
    objs = []
    for it in range(1, 8):
        mu, assign, iters = O.kmeans(X, G, u, max_iter=it)
        objs.append(_objective(X, mu, assign))
    for a, b in zip(objs, objs[1:]):
        assert b <= a * (1 + 1e-12)
    # converged run: centres are the means of their members, members are nearest to their centre
    mu, assign, iters = O.kmeans(X, G, u, max_iter=100)
    assert iters < 100
    for g in range(G):
        mem = X[assign == g].astype(np.float64)
        if len(mem):
            np.testing.assert_allclose(mu[g], mem.mean(0).astype(np.float32), rtol=0, atol=1e-6)
    d2 = ((X[:, None, :].astype(np.float64) - mu[None].astype(np.float64)) ** 2).sum(-1)
    best = d2.min(1)
    assert np.all(d2[np.arange(len(X)), assign] <= best + 1e-9 * (1 + best))


def test_kmeans_empty_grain_reseeded():
    # 5 distinct points, G=5 -> every grain must end non-empty (one point each)
    X = np.array([[0, 0], [0.1, 0], [5, 5], [5.1, 5], [20, 0]], dtype=np.float32)
    u = np.array([0.0, 0.1, 0.2, 0.3, 0.4])
    mu, assign, _ = O.kmeans(X, 5, u)
    assert sorted(np.bincount(assign, minlength=5).tolist()) == [1, 1, 1, 1, 1]


# ---------------------------------------------------------------- PCA


def test_pca_invariant_orthonormal_and_eigen_equation():
    X, _, _ = _clustered(3000, 48, 4, 1, 21)
    G, r = 4, 10
    idx = O.build_index(X, G, r, synth.uniforms(G, 3).numpy(), keep_fp64=True)
    off = idx["grain_off"]
    for g in range(G):
        sl = slice(off[g], off[g + 1])
        lam = idx["eig"][g]
        U = idx["U64"][g]
        # rows orthonormal
        np.testing.assert_allclose(U @ U.T, np.eye(r), atol=1e-12)
        # eigenvalues descending, trace = sum of eigenvalues
        assert np.all(np.diff(lam) <= 1e-12)
        rows = idx["ids"][sl].astype(np.int64)
        V = X[rows].astype(np.float64) - idx["M"][g].astype(np.float64)
        trace = float((V * V).sum() / len(rows))
        assert abs(lam.sum() - trace) <= 1e-10 * trace
        # eigen-equation residual of the kept directions, covariance formed row by row
        cov = np.zeros((X.shape[1], X.shape[1]))
        for v in V:
            cov += np.outer(v, v)
        cov /= len(rows)
        for j in range(r):
            res = cov @ U[j] - lam[j] * U[j]
            assert np.linalg.norm(res) <= 1e-9 * max(1.0, lam[0])
        # mean squared residual = sum of discarded eigenvalues (FP64 basis)
        disc = lam[r:].sum()
        assert abs(idx["rho64"][sl].mean() - disc) <= 1e-9 * disc
        # stored FP32 basis: same invariant within FP32 rounding of the basis
        assert abs(idx["rho"][sl].astype(np.float64).mean() - disc) <= 1e-5 * disc
        # largest-magnitude component of each basis row is positive
        for j in range(r):
            assert U[j, np.argmax(np.abs(U[j]))] > 0


def test_captured_variance_matches_generating_closed_form():
    # one cluster, many samples: sample PCA tends to the generating spectrum
    d, r = 64, 8
    m = synth.make_cluster_model(40000, d, 1, seed=31)
    X, _ = synth.sample_points(m, 32)
    idx = O.build_index(X.numpy(), 1, r, np.array([0.5]))
    lam = idx["eig"][0]
    got = lam[:r].sum() / lam.sum()
    want = synth.expected_captured_fraction(d, 8, 0.8, 0.05, r)
    assert abs(got - want) < 0.01


@pytest.mark.slow
def test_isotropic_captured_variance_table1():
    """Table 1 isotropic row: PCA at subspace dimension 32 captures 6.5% of an
    isotropic Gaussian (d=768, N=10k). Marchenko-Pastur puts it there too."""
    g = _load("paper_table1_isotropic.json")
    X = synth.isotropic(10000, 768, 11).numpy()
    idx = O.build_index(X, 1, 32, np.array([0.3]))
    lam = idx["eig"][0]
    got = lam[:32].sum() / lam.sum()
    assert abs(got - g["pca_variance_captured"]) < 0.002


@pytest.mark.slow
def test_isotropic_mode_b_recall_table1_soft():
    """Table 1 isotropic Mode B row (cand. recall 10.3%, rerank recall 49.4%
    at C=200). The paper's query set is unstated; in-sample queries are used,
    so this is a soft pin (a few points)."""
    g = _load("paper_table1_isotropic.json")
    X = synth.isotropic(10000, 768, 11).numpy()
    idx = O.build_index(X, 1, 32, np.array([0.3]))
    Q = X[np.arange(0, 10000, 10)]
    res = O.search(idx, X, Q, 10, 200, 1)
    bf, _, _ = O.brute_force(X, Q, 10)
    rer = np.mean([len(set(a.tolist()) & set(b.tolist())) / 10 for a, b in zip(res["out_id"], bf)])
    cand = np.mean([len(set(a[:10].astype(np.int64).tolist()) & set(b.tolist())) / 10
                    for a, b in zip(res["cand_id"], bf)])
    assert abs(cand - g["candidate_recall_at_10"]) < 0.02
    assert abs(rer - g["rerank_recall_at_10"]) < 0.05


# ---------------------------------------------------------------- search


def _hand_index(g):
    d, r = g["d"], g["r"]
    rows = np.array(g["rows"], dtype=np.float32)
    U = np.array(g["basis"], dtype=np.float32).reshape(1, r, d)
    mu = np.array(g["centre"], dtype=np.float32).reshape(1, d)
    Z = (rows.astype(np.float64) - mu[0]) @ U[0].T.astype(np.float64)
    E = (rows - mu[0]) - Z @ U[0]
    return dict(M=mu, U=U, grain_off=np.array([0, len(rows)]), ids=np.arange(len(rows), dtype=np.uint32),
                Z=Z.astype(np.float32), rho=(E * E).sum(1).astype(np.float32), G=1, r=r, d=d, N=len(rows)), rows


def test_eq6_hand_fixture():
    g = _load("eq6_tiny.json")
    idx, rows = _hand_index(g)
    Q = np.array([g["query"]], dtype=np.float32)
    res = O.search(idx, rows, Q, g["k"], g["C"], 1)
    assert res["cand_id"][0].tolist() == g["cand_id"]
    np.testing.assert_allclose(res["cand_d"][0], g["cand_d"], rtol=0, atol=1e-12)
    assert res["out_id"][0].tolist() == g["out_id"]
    np.testing.assert_allclose(res["out_d"][0][:g["k"]], g["out_d"], rtol=0, atol=1e-12)
    bf, bd, _ = O.brute_force(rows, Q, 3)
    assert bf[0].tolist() == g["exact_order"]


def test_bruteforce_ties_by_id():
    X = np.array([[1, 0], [0, 1], [-1, 0], [2, 0], [0, -1]], dtype=np.float32)
    Q = np.zeros((1, 2), dtype=np.float32)
    ids, dd, nxt = O.brute_force(X, Q, 4)
    assert ids[0].tolist() == [0, 1, 2, 4]
    assert dd[0].tolist() == [1.0, 1.0, 1.0, 1.0]
    assert nxt[0] == 4.0


def test_full_basis_all_probes_reduces_to_brute_force():
    """r = d makes every residual zero and Eq. 6 exact; with nprobe = G and
    C = N the pool is every row, so candidates are in exact-distance order and
    the reranked top-k equals brute-force kNN."""
    X, Q, _ = _clustered(400, 16, 4, 25, 41)
    G = 4
    idx = O.build_index(X, G, 16, synth.uniforms(G, 1).numpy())
    assert np.max(idx["rho"]) < 1e-9
    res = O.search(idx, X, Q, 10, 400, G)
    bf, bd, _ = O.brute_force(X, Q, 10)
    np.testing.assert_array_equal(res["out_id"], bf)
    np.testing.assert_allclose(res["out_d"][:, :10], bd, rtol=1e-12)
    # candidate distances are the exact distances, up to the FP32 rounding of the stored U and z
    ball, dall, _ = O.brute_force(X, Q, 400)
    for qi in range(len(Q)):
        ex = {int(i): dv for i, dv in zip(ball[qi], dall[qi])}
        for j, cid in enumerate(res["cand_id"][qi]):
            assert abs(res["cand_d"][qi, j] - ex[int(cid)]) <= 1e-6 * (1 + ex[int(cid)])


def test_eq6_error_is_twice_residual_inner_product():
    """For r < d: D - ||q - x||^2 = 2 e_q . e_i, so |D - exact| <= 2 sqrt(rho_q rho_i)
    (Cauchy-Schwarz). rho_q is taken by Pythagoras, ||v'||^2 - ||z_q||^2."""
    X, Q, _ = _clustered(500, 24, 3, 10, 51)
    G, r = 3, 5
    idx = O.build_index(X, G, r, synth.uniforms(G, 2).numpy())
    res = O.search(idx, X, Q, 5, 500, G)
    pos = {int(i): p for p, i in enumerate(idx["ids"])}
    gof = np.searchsorted(idx["grain_off"], np.arange(len(X)), side="right") - 1
    for qi in range(len(Q)):
        q = Q[qi].astype(np.float64)
        for j, cid in enumerate(res["cand_id"][qi]):
            p = pos[int(cid)]
            g = gof[p]
            v = q - idx["M"][g].astype(np.float64)
            zq = idx["U"][g].astype(np.float64) @ v
            rho_q = max(0.0, v @ v - zq @ zq)
            ex = float(((q - X[cid].astype(np.float64)) ** 2).sum())
            bound = 2 * np.sqrt(rho_q * float(idx["rho"][p])) + 1e-6 * (1 + ex)
            assert abs(res["cand_d"][qi, j] - ex) <= bound


# ---------------------------------------------------------------- Mode A


def _pos_and_grain(idx, n):
    pos = np.zeros(n, dtype=np.int64)
    pos[idx["ids"]] = np.arange(len(idx["ids"]))
    gof = np.searchsorted(idx["grain_off"], np.arange(len(idx["ids"])), side="right") - 1
    return pos, gof


def test_mode_a_is_pool_distance_minus_row_residual():
    """With orthonormal basis rows, ||v' - U^T z_i||^2 = ||z_q - z_i||^2 + rho_q
    (Pythagoras: the residual e_q is orthogonal to the basis), which is the
    pool distance of Eq. 6 minus rho_i. The oracle's Mode A reconstructs
    mu_g + U^T z_i in d dimensions; its distances must agree with the scan's,
    and the pool is the one Mode B keeps."""
    X, Q, _ = _clustered(1500, 24, 4, 20, 71)
    G, r = 4, 6
    idx = O.build_index(X, G, r, synth.uniforms(G, 3).numpy())
    a = O.search(idx, X, Q, 10, 60, 2, mode="A")
    b = O.search(idx, X, Q, 10, 60, 2, mode="B")
    np.testing.assert_array_equal(a["cand_id"], b["cand_id"])
    pos, _ = _pos_and_grain(idx, len(X))
    for qi in range(len(Q)):
        pool = {int(i): dv - float(idx["rho"][pos[int(i)]]) for i, dv in zip(a["cand_id"][qi], a["cand_d"][qi])}
        want = sorted((dv, i) for i, dv in pool.items())[:10]
        assert [i for _, i in want] == a["out_id"][qi].tolist()
        for j in range(10):
            assert abs(a["out_d"][qi, j] - want[j][0]) <= 1e-6 * (1.0 + want[j][0])


def test_mode_a_full_basis_equals_brute_force():
    """r = d: every row equals its reconstruction (zero residual), so Mode A with
    every grain probed and the whole set pooled is exact kNN."""
    X, Q, _ = _clustered(400, 16, 4, 25, 43)
    G = 4
    idx = O.build_index(X, G, 16, synth.uniforms(G, 4).numpy())
    res = O.search(idx, X, Q, 10, 400, G, mode="A")
    bf, bd, _ = O.brute_force(X, Q, 10)
    np.testing.assert_array_equal(res["out_id"], bf)
    np.testing.assert_allclose(res["out_d"][:, :10], bd, rtol=1e-6)


def test_mode_a_precision_form_gram_expansion():
    """Precision form: BF16 bases are not orthonormal, so Pythagoras no longer
    applies; the reconstruction distance must still equal its expansion
    ||v'||^2 - 2 z_i . (U_b v') + z_i^T (U_b U_b^T) z_i with v' = q_b - mu_b and
    the decoded FP8 coordinates z_i."""
    X, Q, _ = _clustered(1200, 32, 4, 12, 81)
    G, r = 4, 8
    idx = O.build_index(X, G, r, synth.uniforms(G, 5).numpy())
    res = O.search(idx, X, Q, 10, 40, 2, mode="A", precision="bf16-fp8")
    M = O.bf16_to_f32(O.bf16_round(idx["M"])).reshape(idx["M"].shape).astype(np.float64)
    U = O.bf16_to_f32(O.bf16_round(idx["U"])).reshape(idx["U"].shape).astype(np.float64)
    Zd = O.fp8_decoded(idx).astype(np.float64)
    Qb = O.bf16_to_f32(O.bf16_round(Q)).reshape(Q.shape).astype(np.float64)
    pos, gof = _pos_and_grain(idx, len(X))
    for qi in range(len(Q)):
        for j, i in enumerate(res["out_id"][qi]):
            p = pos[int(i)]
            g = gof[p]
            v = Qb[qi] - M[g]
            z = Zd[p]
            want = v @ v - 2.0 * z @ (U[g] @ v) + z @ (U[g] @ U[g].T) @ z
            assert abs(res["out_d"][qi, j] - want) <= 1e-9 * (1.0 + v @ v)


# ---------------------------------------------------------------- 16-bit form (Eq. 5)


def test_int16_codes_round_trip():
    """Per grain the rows use half of each 16-bit range, the largest |z| of a
    grain maps to +-16383 and the largest residual to 32767, and every value
    the scan uses is within half a step (plus FP32 rounding) of the stored one."""
    X, Q, _ = _clustered(2000, 24, 5, 5, 91)
    idx = O.build_index(X, 5, 6, synth.uniforms(5, 6).numpy())
    f = O.int16_form(idx)
    off = idx["grain_off"]
    for g in range(5):
        a, b = off[g], off[g + 1]
        c = f["codes"][a:b].astype(np.int64)
        assert np.abs(c).max() == 16383 and f["rcodes"][a:b].max() == 32767
        z = idx["Z"][a:b].astype(np.float64)
        err = np.abs(f["Zf32"][a:b].astype(np.float64) - z)
        assert np.all(err <= 0.5 * float(f["delta"][g]) * (1 + 1e-6) + 1e-6 * np.abs(z))
        rr = np.abs(f["rhof32"][a:b].astype(np.float64) - idx["rho"][a:b])
        assert np.all(rr <= 0.5 * float(f["dres"][g]) * (1 + 1e-6) + 1e-6 * idx["rho"][a:b])


def test_int16_envelope_filter_drops_a_far_grain():
    """Grain B is tight and far from a query that sits in grain A: in B's frame
    the query's coordinates are far beyond twice B's extent, every one
    saturates, and the envelope filter keeps B's rows out of the pool, which
    the FP32 form (no filter) fills with them."""
    rng = np.random.default_rng(17)
    A = rng.standard_normal((50, 8))
    B = 60.0 + 0.01 * rng.standard_normal((50, 8))
    X = np.concatenate([A, B]).astype(np.float32)
    assign = np.repeat([0, 1], 50)
    idx = partition_index(X, assign, 2, 4)
    Q = (0.1 * rng.standard_normal((3, 8))).astype(np.float32)
    f32 = O.search(idx, X, Q, 10, 80, 2, precision="fp32")
    i16 = O.search(idx, X, Q, 10, 80, 2, precision="int16")
    for qi in range(3):
        assert (f32["cand_id"][qi] >= 50).sum() == 30  # B's rows fill the rest of the FP32 pool
        ids = i16["cand_id"][qi]
        assert set(ids[ids != 0xFFFFFFFF].tolist()) == set(range(50))  # only A's rows
        assert (ids == 0xFFFFFFFF).sum() == 30


def _int16_query_side(idx, f, q, g):
    """The 16-bit form's query side written out in numpy float32 (Eq. 5):
    codes rint(fl32(z / delta)) saturating at +-32767 (count of saturated
    ones) and the residual code rint(fl32(rho / dres)) before any clipping."""
    v = q.astype(np.float64) - idx["M"][g].astype(np.float64)
    U = idx["U"][g].astype(np.float64)
    zq = U @ v
    rq = float(((v - U.T @ zq) ** 2).sum())
    t = np.rint(np.float32(zq.astype(np.float32)) / np.float32(f["delta"][g])).astype(np.float64)
    sat = int((np.abs(t) > 32767).sum())
    codes = np.clip(t, -32767, 32767).astype(np.int64)
    rcode = float(np.rint(np.float32(rq) / np.float32(f["dres"][g])))
    return codes, rcode, sat


def _int16_D(f, g, codes_q, rcode_q, row_codes, rho_grid_i):
    """Eq. 6 on the codes: exact integer S, then fl32(fl32(delta^2) fl32(S)) + fl32(rho_q + rho_i)."""
    S = int(sum((int(a) - int(b)) ** 2 for a, b in zip(codes_q, row_codes)))
    dl = np.float32(f["delta"][g])
    rq = np.float32(np.float32(rcode_q) * np.float32(f["dres"][g]))
    return float(np.float32(np.float32(dl * dl) * np.float32(S)) + np.float32(rq + np.float32(rho_grid_i)))


def test_int16_distance_is_integer_eq6_on_the_codes():
    """Pool distances of the 16-bit form are Eq. 6 on the integer codes,
    bit for bit: the integer sum written out with Python integers and the
    scale-back with numpy float32 operations; giving the oracle the same query
    codes reproduces its own quantisation's result exactly."""
    X, Q, _ = _clustered(1200, 16, 3, 8, 95)
    idx = O.build_index(X, 3, 5, synth.uniforms(3, 9).numpy())
    f = O.int16_form(idx)
    res = O.search(idx, X, Q, 5, 60, 2, precision="int16")
    pos = np.zeros(len(X), dtype=np.int64)
    pos[idx["ids"]] = np.arange(len(X))
    gof = np.repeat(np.arange(3), np.diff(idx["grain_off"]))
    qcodes = np.zeros((len(Q), 2, 5), dtype=np.int16)
    qr = np.zeros((len(Q), 2), dtype=np.int32)
    n = 0
    for qi in range(len(Q)):
        per = {}
        for p, g in enumerate(res["probe"][qi]):
            c, rc, sat = _int16_query_side(idx, f, Q[qi], int(g))
            assert 4 * sat <= 5  # the premise: no grain is left out here
            per[int(g)] = (c, min(rc, 65535.0))
            qcodes[qi, p] = c
            qr[qi, p] = int(min(rc, 65535.0))
        for i, d in zip(res["cand_id"][qi].tolist(), res["cand_d"][qi].tolist()):
            if i == 0xFFFFFFFF:
                continue
            g = int(gof[pos[i]])
            c, rc = per[g]
            want = _int16_D(f, g, c, rc, f["codes"][pos[i]], f["rhof32"][pos[i]])
            assert d == want, (qi, i, d, want)
            n += 1
    assert n > 400
    again = O.search(idx, X, Q, 5, 60, 2, precision="int16", query_codes=(qcodes, qr))
    assert np.array_equal(again["cand_id"], res["cand_id"])
    assert np.array_equal(again["cand_d"], res["cand_d"]) and np.array_equal(again["out_id"], res["out_id"])


def test_int16_residual_is_clipped_not_pruned_by_default():
    """Grain B varies only inside its own 4-dimensional subspace; a query near
    grain A projects into B's frame with coordinates inside B's range (no
    coordinate saturates) but with a residual norm far beyond any of B's rows.
    The paper's filter counts coordinates only, so B stays in the scan with the
    query's residual code clipped at 65535 (Eq. 5, unsigned 16 bits): B's rows
    enter the pool at exactly the distances of that clipped residual. With the
    residual-saturation option (the build's own rule) B is left out."""
    rng = np.random.default_rng(19)
    A = rng.standard_normal((50, 8))
    B = np.zeros((50, 8))
    B[:, :4] = rng.standard_normal((50, 4))
    B[:, 4:] = 20.0 + 1e-3 * rng.standard_normal((50, 4))
    X = np.concatenate([A, B]).astype(np.float32)
    idx = partition_index(X, np.repeat([0, 1], 50), 2, 4)
    Q = (0.1 * rng.standard_normal((3, 8))).astype(np.float32)
    f = O.int16_form(idx)
    pos = np.zeros(len(X), dtype=np.int64)
    pos[idx["ids"]] = np.arange(len(X))
    i16 = O.search(idx, X, Q, 10, 80, 2, precision="int16")
    for qi in range(3):
        c, rc, sat = _int16_query_side(idx, f, Q[qi], 1)
        assert sat == 0 and rc > 65535  # the premise
        ids = i16["cand_id"][qi]
        b_rows = [(i, d) for i, d in zip(ids.tolist(), i16["cand_d"][qi].tolist()) if 50 <= i < 100]
        # the clipped residual is tiny on B's fine grid, so B's rows look close and crowd the pool
        assert len(b_rows) >= 30
        for i, d in b_rows:
            assert d == _int16_D(f, 1, c, 65535.0, f["codes"][pos[i]], f["rhof32"][pos[i]])


def test_int16_residual_prune_option_drops_the_grain():
    """The build's own option: with residual-saturation pruning on, the same
    grain B (query residual beyond 65535 steps) is left out of the pool."""
    rng = np.random.default_rng(19)
    A = rng.standard_normal((50, 8))
    B = np.zeros((50, 8))
    B[:, :4] = rng.standard_normal((50, 4))
    B[:, 4:] = 20.0 + 1e-3 * rng.standard_normal((50, 4))
    X = np.concatenate([A, B]).astype(np.float32)
    idx = partition_index(X, np.repeat([0, 1], 50), 2, 4)
    Q = (0.1 * rng.standard_normal((3, 8))).astype(np.float32)
    f = O.int16_form(idx)
    for q in Q:  # the premise: no coordinate of the query saturates in B's frame
        zq = idx["U"][1].astype(np.float64) @ (q - idx["M"][1].astype(np.float64))
        assert np.abs(zq).max() < 32767 * float(f["delta"][1])
    f32 = O.search(idx, X, Q, 10, 80, 2, precision="fp32")
    i16 = O.search(idx, X, Q, 10, 80, 2, precision="int16", resid_prune=True)
    for qi in range(3):
        assert (f32["cand_id"][qi] >= 50).sum() == 30
        ids = i16["cand_id"][qi]
        assert set(ids[ids != 0xFFFFFFFF].tolist()) == set(range(50))


def test_int16_distances_within_quantisation_bound():
    """Each coordinate of a query or row moves by at most half a step, so a
    pool distance of the 16-bit form differs from the FP32 form's by at most
    sum_j (2 |z_qj - z_ij| delta + delta^2) + dres (the two residuals), for
    every pair whose query residual is inside the grain's residual range."""
    X, Q, _ = _clustered(2000, 24, 4, 20, 93)
    idx = O.build_index(X, 4, 6, synth.uniforms(4, 8).numpy())
    f = O.int16_form(idx)
    a = O.search(idx, X, Q, 10, 40, 1, precision="int16")
    b = O.search(idx, X, Q, 10, 40, 1, precision="fp32")
    pos = np.zeros(len(X), dtype=np.int64)
    pos[idx["ids"]] = np.arange(len(X))
    checked = 0
    for qi in range(len(Q)):
        g = int(b["probe"][qi, 0])
        v = Q[qi].astype(np.float64) - idx["M"][g].astype(np.float64)
        U = idx["U"][g].astype(np.float64)
        zq = U @ v
        rho_q = float(((v - U.T @ zq) ** 2).sum())
        dl, dr = float(f["delta"][g]), float(f["dres"][g])
        if rho_q > 65535 * dr or np.abs(zq).max() > 32767 * dl:
            continue  # clipped: outside the bound's premise
        d32 = dict(zip(b["cand_id"][qi].tolist(), b["cand_d"][qi].tolist()))
        for i, d16 in zip(a["cand_id"][qi].tolist(), a["cand_d"][qi].tolist()):
            if i in d32:
                dz = np.abs(zq - idx["Z"][pos[i]].astype(np.float64))
                bound = float(np.sum(2 * dz * dl + dl * dl)) + dr + 1e-6 * d32[i]
                assert abs(d16 - d32[i]) <= bound
                checked += 1
    assert checked > 100


def test_basis_sign_and_rotation_invariance():
    X, Q, _ = _clustered(300, 20, 2, 8, 61)
    G, r = 2, 6
    idx = O.build_index(X, G, r, synth.uniforms(G, 3).numpy())
    base = O.search(idx, X, Q, 5, 40, G)
    rng = np.random.default_rng(0)
    R = np.linalg.qr(rng.standard_normal((r, r)))[0]
    idx2 = dict(idx)
    idx2["U"] = np.einsum("ij,gjd->gid", R, idx["U"].astype(np.float64)).astype(np.float64)
    # keep the coordinates exactly consistent with the rotated basis, in FP64
    idx2["Z"] = (idx["Z"].astype(np.float64) @ R.T)
    idx2["U"] = idx2["U"].astype(np.float32)
    idx2["Z"] = idx2["Z"].astype(np.float32)
    rot = O.search(idx2, X, Q, 5, 40, G)
    np.testing.assert_allclose(rot["cand_d"], base["cand_d"], rtol=2e-5)
    idx3 = dict(idx)
    idx3["U"] = -idx["U"]
    idx3["Z"] = -idx["Z"]
    flip = O.search(idx3, X, Q, 5, 40, G)
    np.testing.assert_array_equal(flip["cand_id"], base["cand_id"])
    np.testing.assert_array_equal(flip["cand_d"], base["cand_d"])


def test_routing_order_and_ties():
    # centres at distance 1, 1, 4 from the query -> probes by (dist, grain)
    M = np.array([[0, 2], [1, 0], [0, 1], [-1, 0]], dtype=np.float32)
    idx = dict(M=M, U=np.zeros((4, 1, 2), dtype=np.float32) + np.array([1, 0], dtype=np.float32),
               grain_off=np.array([0, 0, 0, 0, 0]), ids=np.zeros(0, dtype=np.uint32),
               Z=np.zeros((0, 1), dtype=np.float32), rho=np.zeros(0, dtype=np.float32), G=4, r=1, d=2, N=0)
    Q = np.zeros((1, 2), dtype=np.float32)
    res = O.search(idx, np.zeros((0, 2), dtype=np.float32), Q, 1, 1, 3)
    assert res["probe"][0].tolist() == [1, 2, 3]
    assert res["probe_d"][0].tolist() == [1.0, 1.0, 1.0, 4.0]
    assert res["out_id"][0].tolist() == [-1]
    assert res["cand_id"][0].tolist() == [0xFFFFFFFF]


def test_filter_equals_search_on_filtered_subset():
    """An in-scan range filter returns what the unfiltered path returns on the
    rows that pass (r = d, all probes, C = N makes both exact)."""
    X, Q, _ = _clustered(300, 8, 3, 12, 71)
    attr = synth.attributes(300, 5, span=1000).numpy()
    ranges = synth.range_filters(12, 6, span=1000, selectivity=0.3, frac_filtered=0.6).numpy()
    idx = O.build_index(X, 3, 8, synth.uniforms(3, 1).numpy())
    res = O.search(idx, X, Q, 5, 300, 3, attr=attr, ranges=ranges)
    for qi in range(len(Q)):
        keep = np.nonzero((attr >= ranges[qi, 0]) & (attr <= ranges[qi, 1]))[0]
        sub_ids, sub_d, _ = O.brute_force(X[keep], Q[qi:qi + 1], 5)
        want = [int(keep[i]) if i >= 0 else -1 for i in sub_ids[0]]
        assert res["out_id"][qi].tolist() == want


def test_mode_a_filter_full_basis_equals_filtered_brute_force():
    """Mode A with range filters: with r = d the reconstruction mu + U^T z is
    the row itself, so with every grain probed and C = N the filtered Mode A
    answer is brute force over the rows that pass."""
    X, Q, _ = _clustered(300, 8, 3, 12, 73)
    attr = synth.attributes(300, 7, span=1000).numpy()
    ranges = synth.range_filters(12, 8, span=1000, selectivity=0.3, frac_filtered=0.6).numpy()
    idx = O.build_index(X, 3, 8, synth.uniforms(3, 2).numpy())
    res = O.search(idx, X, Q, 5, 300, 3, attr=attr, ranges=ranges, mode="A")
    for qi in range(len(Q)):
        keep = np.nonzero((attr >= ranges[qi, 0]) & (attr <= ranges[qi, 1]))[0]
        sub_ids, sub_d, _ = O.brute_force(X[keep], Q[qi:qi + 1], 5)
        want = [int(keep[i]) if i >= 0 else -1 for i in sub_ids[0]]
        assert res["out_id"][qi].tolist() == want
        ok = sub_ids[0] >= 0
        np.testing.assert_allclose(res["out_d"][qi][:5][ok], sub_d[0][ok], rtol=1e-5, atol=1e-5)  # k + 1 kept


def test_nprobe_all_c_all_recall_one():
    X, Q, _ = _clustered(800, 32, 8, 30, 81)
    G = 8
    idx = O.build_index(X, G, 4, synth.uniforms(G, 7).numpy())
    res = O.search(idx, X, Q, 10, 800, G)
    bf, _, _ = O.brute_force(X, Q, 10)
    np.testing.assert_array_equal(res["out_id"], bf)


def test_short_results_are_padded():
    X, Q, _ = _clustered(50, 8, 2, 3, 91)
    idx = O.build_index(X, 2, 4, synth.uniforms(2, 1).numpy())
    res = O.search(idx, X, Q, 100, 200, 2)
    assert np.all(res["out_id"][:, 50:] == -1)
    assert np.all(np.isinf(res["out_d"][:, 50:]))
    assert np.all(res["cand_id"][:, 50:] == 0xFFFFFFFF)


# ---------------------------------------------------------------- number formats


def test_e4m3_spec_values_and_exhaustive_round_trip():
    g = _load("e4m3_values.json")
    for code, val in g["codes"].items():
        assert O.e4m3_value(np.uint8(int(code, 16))) == val
    for code in g["nan_codes"]:
        assert np.isnan(O.e4m3_value(np.uint8(int(code, 16))))
    codes = np.arange(256, dtype=np.uint8)
    vals = O.e4m3_value(codes)
    fin = ~np.isnan(vals) & (codes != 0x80)
    np.testing.assert_array_equal(O.e4m3_encode(vals[fin]), codes[fin])


def test_e4m3_matches_torch_cast_and_ties_to_even():
    # torch's float8_e4m3fn cast is an independent implementation (RNE); compare inside the finite range
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(20000) * s for s in (1e-3, 0.1, 1, 30, 200)])
    x = x[np.abs(x) <= 448]
    ours = O.e4m3_value(O.e4m3_encode(x))
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(ours, ref)
    # exact midpoints between neighbours go to the even code
    pos = O.e4m3_value(np.arange(0, 0x7F, dtype=np.uint8))
    mids = (pos[:-1] + pos[1:]) / 2
    enc = O.e4m3_encode(mids)
    assert np.all(enc % 2 == 0)
    # saturation to the largest finite value
    assert O.e4m3_value(O.e4m3_encode(np.array([1000.0, -5000.0]))).tolist() == [448.0, -448.0]


def test_bf16_matches_torch_cast():
    rng = np.random.default_rng(4)
    x = (rng.standard_normal(100000) * 10).astype(np.float32)
    x[:4] = [0.0, -0.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8]  # exact ties: to even
    ours = O.bf16_to_f32(O.bf16_round(x))
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(ours, ref)


def test_index_file_header_and_checksum_round_trip(tmp_path):
    X, Q, _ = _clustered(200, 8, 2, 2, 95)
    idx = O.build_index(X, 2, 4, synth.uniforms(2, 1).numpy())
    p = str(tmp_path / "a.hntl")
    O.write_index(p, idx, X)
    h = O.read_index_header(p)
    assert (h["N"], h["d"], h["G"], h["r"], h["version"]) == (200, 8, 2, 4, 1)
    data = open(p, "rb").read()
    body, tail = data[:-8], data[-8:]
    s, _ = O._wsum(body, (0, 0))
    assert s == int(np.frombuffer(tail, dtype="<u8")[0])


# ---------------------------------------------------------------- precision form


def _grid_index():
    """One grain, centre 0, basis = the first two axes; every row, query and
    coordinate lies on a grid that BF16 holds exactly and whose coordinates
    FP8-E4M3 holds exactly after the grain scale 2/448 (|z| in {0, 1/4, 1/2, 1, 2})."""
    rng = np.random.default_rng(9)
    d, r, n = 8, 2, 200
    vals = np.array([0, 0.25, 0.5, 1.0, 2.0, -0.25, -0.5, -1.0, -2.0], dtype=np.float32)
    X = vals[rng.integers(0, len(vals), (n, d))]
    X[0, :2] = [2.0, -2.0]  # max |z| = 2
    U = np.zeros((1, r, d), dtype=np.float32)
    U[0, 0, 0] = U[0, 1, 1] = 1.0
    Z = X[:, :2].copy()
    rho = (X[:, 2:].astype(np.float64) ** 2).sum(1).astype(np.float32)
    idx = dict(M=np.zeros((1, d), dtype=np.float32), U=U, grain_off=np.array([0, n]),
               ids=np.arange(n, dtype=np.uint32), Z=Z, rho=rho, G=1, r=r, d=d, N=n)
    Q = vals[rng.integers(0, len(vals), (12, d))].astype(np.float32)
    return idx, X, Q


def test_precision_form_reduces_to_plain_on_representable_inputs():
    idx, X, Q = _grid_index()
    z8, scale = O.fp8_coords(idx)
    np.testing.assert_allclose(O.fp8_decoded(idx), idx["Z"], rtol=1e-6, atol=0)
    plain = O.search(idx, X, Q, 5, 40, 1)
    prec = O.search(idx, X, Q, 5, 40, 1, precision="bf16-fp8")
    np.testing.assert_allclose(prec["cand_d"], plain["cand_d"], rtol=1e-6)
    np.testing.assert_allclose(prec["out_d"], plain["out_d"], rtol=1e-12)


def test_precision_form_recall_close_to_plain():
    m = synth.make_cluster_model(4000, 128, 8, seed=41)
    X, _ = synth.sample_points(m, 42)
    Q, _ = synth.sample_queries(m, 60, 43)
    X, Q = X.numpy(), Q.numpy()
    idx = O.build_index(X, 8, 16, synth.uniforms(8, 44).numpy())
    bf, _, _ = O.brute_force(X, Q, 10)
    rec = lambda res: np.mean([len(set(a.tolist()) & set(b.tolist())) / 10 for a, b in zip(res["out_id"], bf)])
    plain = O.search(idx, X, Q, 10, 50, 2)
    prec = O.search(idx, X, Q, 10, 50, 2, precision="bf16-fp8")
    assert rec(prec) >= rec(plain) - 0.02
    assert rec(prec) >= 0.95


def test_given_probes_equal_routing_when_they_are_the_routed_ones():
    """Step 1 replaced by the probes routing itself picks (in any order)
    leaves the pool and the top k unchanged: the pool is a global (D, id)
    order over the probed rows, whatever order the grains are visited in."""
    X, Q, idx = clustered_case(1500, 16, 6, 6, 4, 25, seed=31)
    ref = O.search(idx, X, Q, 5, 30, 3)
    rev = np.ascontiguousarray(ref["probe"][:, ::-1])
    got = O.search(idx, X, Q, 5, 30, 3, probes=rev)
    assert np.array_equal(got["cand_id"], ref["cand_id"]) and np.array_equal(got["out_id"], ref["out_id"])
    np.testing.assert_array_equal(got["out_d"][:, :5], ref["out_d"][:, :5])
    assert np.isinf(got["probe_d"][:, 3]).all()
    # a probe set that leaves out the nearest grain changes the pool
    far = np.ascontiguousarray(np.stack([ref["probe"][:, 1], ref["probe"][:, 2]], 1))
    got2 = O.search(idx, X, Q, 5, 30, 2, probes=far)
    assert not np.array_equal(got2["cand_id"], ref["cand_id"][:, :30])


# ---------------------------------------------------------------- capacity-bounded grains


def _blocking_pairs(X, M, assign, cap):
    """(row, centre) pairs that block stability: the row ranks the centre above
    its own grain, and the centre has room or holds a row it ranks below it."""
    D = ((X.astype(np.float64)[:, None, :] - M.astype(np.float64)[None]) ** 2).sum(-1)
    G = M.shape[0]
    held = [np.flatnonzero(assign == g) for g in range(G)]
    out = []
    for i in range(len(X)):
        a = assign[i]
        for g in range(G):
            if (D[i, g], g) >= (D[i, a], a):
                continue
            if len(held[g]) < cap or any((D[j, g], j) > (D[i, g], i) for j in held[g]):
                out.append((i, g))
    return out


def test_balanced_assignment_is_stable_and_capped():
    rng = np.random.default_rng(41)
    X = np.concatenate([rng.standard_normal((150, 6)) + 3, rng.standard_normal((50, 6)) - 3]).astype(np.float32)
    M = np.concatenate([rng.standard_normal((3, 6)) + 3, rng.standard_normal((2, 6)) - 3])
    cap = 45
    a = O.balanced_assign(X, M, cap)
    assert (a >= 0).all() and np.bincount(a, minlength=5).max() <= cap
    assert _blocking_pairs(X, M, a, cap) == []
    # with room for every row the grains are the nearest-centre (Voronoi) cells
    D = ((X.astype(np.float64)[:, None, :] - M[None]) ** 2).sum(-1)
    np.testing.assert_array_equal(O.balanced_assign(X, M, len(X)), D.argmin(1))


def test_balanced_assignment_is_the_row_optimal_stable_one():
    """Brute force over every capacity-respecting assignment of 7 rows to 3
    centres (cap 3): among the stable ones, the oracle's gives every row a
    centre it ranks at least as high as in any other."""
    import itertools

    rng = np.random.default_rng(43)
    X = rng.standard_normal((7, 2)).astype(np.float32)
    M = rng.standard_normal((3, 2))
    cap = 3
    D = ((X.astype(np.float64)[:, None, :] - M[None]) ** 2).sum(-1)
    rank = np.argsort(np.argsort(D, 1, kind="stable"), 1)  # rank of each centre for each row
    stable = []
    for a in itertools.product(range(3), repeat=7):
        a = np.array(a)
        if np.bincount(a, minlength=3).max() <= cap and not _blocking_pairs(X, M, a, cap):
            stable.append(a)
    got = O.balanced_assign(X, M, cap)
    assert any(np.array_equal(got, s) for s in stable)
    for s in stable:
        assert np.all(rank[np.arange(7), got] <= rank[np.arange(7), s])


def test_given_projection_reproduces_the_oracle_own():
    """Feeding the oracle its own projection values (rounded to FP32, as another
    implementation would hand them over) leaves every pool and top k id
    unchanged where the ranking has gaps well above FP32 rounding, and moves
    distances by no more than that rounding."""
    X, Q, idx = clustered_case(1500, 16, 6, 6, 4, 25, seed=33)
    ref = O.search(idx, X, Q, 5, 30, 3)
    M, U = idx["M"].astype(np.float64), idx["U"].astype(np.float64)
    z = np.zeros((len(Q), 3, 4), np.float32)
    rho = np.zeros((len(Q), 3), np.float32)
    for qi in range(len(Q)):
        for p, g in enumerate(ref["probe"][qi]):
            v = Q[qi].astype(np.float64) - M[g]
            z[qi, p] = U[g] @ v
            rho[qi, p] = ((v - U[g].T @ (U[g] @ v)) ** 2).sum()
    got = O.search(idx, X, Q, 5, 30, 3, probes=ref["probe"], pair_proj=(z, rho))
    assert np.array_equal(got["out_id"], ref["out_id"])
    np.testing.assert_allclose(got["cand_d"][:, :30], ref["cand_d"][:, :30], rtol=1e-6)


# ---------------------------------------------------------------- per-stage FP64 values


def test_stage_values_hand_fixture():
    """The hand-derived fixture: z_q = 1, rho_q = 1, row coordinates [1, 2, 0]
    with residuals [0.25, 0, 1], D = [1.25, 2, 3], exact [0.25, 2, 1], and the
    centre distance ||q||^2 = 2; rows are given out of order and with a gap."""
    g = _load("eq6_tiny.json")
    idx, rows = _hand_index(g)
    Q = np.array([g["query"]], dtype=np.float32)
    sv = O.stage_values(idx, rows, Q, [[0]], [[2, -1, 0, 1]])
    assert sv["route_d"][0, 0] == 2.0
    assert sv["z"][0, 0, 0] == 1.0 and sv["rho"][0, 0] == 1.0
    np.testing.assert_allclose(sv["zi"][0, [0, 2, 3], 0], [0, 1, 2], atol=1e-12)
    np.testing.assert_allclose(sv["rhoi"][0, [0, 2, 3]], [1, 0.25, 0], atol=1e-12)
    D = [g["cand_d"][2], g["cand_d"][0], g["cand_d"][1]]
    np.testing.assert_allclose(sv["D"][0, [0, 2, 3]], D, atol=1e-12)
    np.testing.assert_allclose(sv["exact"][0, [0, 2, 3]], [1.0, 0.25, 2.0], atol=1e-12)
    assert np.isnan(sv["D"][0, 1]) and np.isnan(sv["exact"][0, 1])


def test_stage_values_full_basis_is_exact_and_overrides_enter_eq6():
    """r = d: every residual is zero and Eq. 6 equals the exact distance for
    rows of probed grains (up to the FP32 rounding of the stored basis, whose
    rows are orthonormal to about 1e-7); rows of unprobed grains stay NaN. Given query
    terms shifted by +1 in one coordinate move D_pair by (dz + 1)^2 - dz^2,
    and given row residuals raised by 0.5 move D_row by 0.5."""
    X, Q, _ = _clustered(300, 8, 3, 4, 77)
    idx = O.build_index(X, 3, 8, synth.uniforms(3, 5).numpy())
    probes = np.array([[0, 2]] * len(Q))
    rows = np.tile(np.arange(0, 300, 7), (len(Q), 1))
    sv = O.stage_values(idx, X, Q, probes, rows)
    gid = np.zeros(300, dtype=np.int64)
    gid[idx["ids"]] = np.repeat(np.arange(3), np.diff(idx["grain_off"]))
    probed = np.isin(gid[rows[0]], [0, 2])
    assert probed.any() and (~probed).any()
    np.testing.assert_allclose(sv["D"][:, probed], sv["exact"][:, probed], rtol=1e-6)
    assert np.isnan(sv["D"][:, ~probed]).all()
    assert (sv["rho"] <= 1e-6 * sv["route_d"]).all()
    zq = sv["z"].copy()
    zq[:, :, 0] += 1.0
    rz = sv["zi"].copy()
    rr = sv["rhoi"] + 0.5
    sv2 = O.stage_values(idx, X, Q, probes, rows, pair_proj=(zq, sv["rho"]), row_terms=(rz, rr))
    slot = np.where(gid[rows[0]] == 0, 0, 1)
    dz = sv["z"][:, slot, 0] - sv["zi"][:, :, 0]
    want = sv["D"] + (dz + 1.0) ** 2 - dz ** 2
    np.testing.assert_allclose(sv2["D_pair"][:, probed], want[:, probed], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(sv2["D_row"][:, probed], sv["D"][:, probed] + 0.5, rtol=1e-9)


def test_stage_values_route_distances_are_brute_force_over_centres():
    """The routing distances of the probes brute force picks over the centres
    are brute force's own distances."""
    X, Q, _ = _clustered(400, 16, 4, 20, 91)
    idx = O.build_index(X, 8, 4, synth.uniforms(8, 6).numpy())
    bid, bd, _ = O.brute_force(idx["M"], Q, 3)
    sv = O.stage_values(idx, X, Q, bid, np.full((len(Q), 1), -1))
    np.testing.assert_allclose(sv["route_d"], bd, rtol=1e-12)


# ---------------------------------------------------------------- grain shards


def test_shard_assign_hand_fixture_and_balance_bound():
    """Rows [5, 4, 3, 3, 2, 1] into 2 shards, longest first to the lighter
    shard: 5 -> s0, 4 -> s1, 3 -> s1 (4 < 5), 3 -> s0 (5 < 7), 2 -> s1
    (7 < 8), 1 -> s0 (8 < 9); loads 9 and 9. On random sizes every shard
    stays within the greedy rule's bound: mean load + largest grain."""
    assert O.shard_assign([5, 4, 3, 3, 2, 1], 2).tolist() == [0, 1, 1, 0, 1, 0]
    rows = np.random.default_rng(3).integers(0, 500, 97)
    for S in (1, 3, 8):
        sog = O.shard_assign(rows, S)
        load = np.bincount(sog, weights=rows, minlength=S)
        assert load.sum() == rows.sum()
        assert load.max() <= rows.sum() / S + rows.max()


def test_sharded_search_reduces_to_plain_and_to_brute_force():
    """One shard is the plain search. With every grain probed and C = N each
    shard's pool is all its rows, so its top k is its exact top k and the
    merge is brute force. In between, the shards' pools together contain the
    single index's pool, so the merged distances are at most the single
    index's, position by position."""
    X, Q, _ = _clustered(1200, 16, 6, 30, 57)
    G = 12
    idx = O.build_index(X, G, 4, synth.uniforms(G, 2).numpy())
    rows = np.diff(idx["grain_off"])
    plain = O.search(idx, X, Q, 10, 40, 4)
    i1, d1, _ = O.sharded_search(idx, X, Q, 10, 40, 4, np.zeros(G, dtype=np.int64))
    np.testing.assert_array_equal(i1, plain["out_id"])
    np.testing.assert_allclose(d1, plain["out_d"][:, :10])
    sog = O.shard_assign(rows, 3)
    ia, da, _ = O.sharded_search(idx, X, Q, 10, 1200, G, sog)
    bf, bd, _ = O.brute_force(X, Q, 10)
    np.testing.assert_array_equal(ia, bf)
    np.testing.assert_allclose(da, bd, rtol=1e-12)
    ib, db, _ = O.sharded_search(idx, X, Q, 10, 40, 4, sog)
    assert (db <= plain["out_d"][:, :10] + 1e-12).all()
    assert (db < plain["out_d"][:, :10] - 1e-9).any() or np.array_equal(ib, plain["out_id"])


# ---------------------------------------------------------------- refined rerank (precision form)


def _one_grain_index(X, r):
    return partition_index(X, np.zeros(len(X), dtype=np.int64), 1, r)


def test_refined_rerank_hand_fixture():
    """Rows (1 + 3 2^-10, 0) and (1 + 2^-10, 0), query at the origin: both round
    to (1, 0) in BF16, so the BF16 rerank ties them at distance 1 and keeps
    the lower id (row 0). Their second BF16 parts are 3 2^-10 and 2^-10
    exactly, so the refined stage (min(C, 2k) = 2 rows) orders them by their
    exact distances and returns row 1 at (1 + 2^-10)^2."""
    X = np.array([[1 + 3 * 2.0 ** -10, 0.0], [1 + 2.0 ** -10, 0.0]], dtype=np.float32)
    Q = np.zeros((1, 2), dtype=np.float32)
    idx = _one_grain_index(X, 1)
    plain = O.search(idx, X, Q, 1, 2, 1, precision="bf16-fp8")
    ref = O.search(idx, X, Q, 1, 2, 1, precision="bf16-fp8", refine=True)
    assert plain["out_id"][0].tolist() == [0] and plain["out_d"][0, 0] == 1.0
    assert ref["out_id"][0].tolist() == [1] and ref["out_d"][0, 0] == (1 + 2.0 ** -10) ** 2


def test_refined_rerank_reduces_to_plain_and_to_brute_force():
    """Rows exactly representable in BF16 have a zero second part: the refined
    rerank returns the BF16 rerank's ids and distances. Rows of 16 significant
    bits are exactly the sum of their two parts; with C = N <= 2k the refined
    stage sees every row and returns brute force's ids and distances."""
    rng = np.random.default_rng(21)
    Xb = O.bf16_to_f32(O.bf16_round(rng.standard_normal((300, 16)).astype(np.float32))).reshape(300, 16)
    Q = rng.standard_normal((5, 16)).astype(np.float32)
    idx = _one_grain_index(Xb, 4)
    a = O.search(idx, Xb, Q, 10, 40, 1, precision="bf16-fp8")
    b = O.search(idx, Xb, Q, 10, 40, 1, precision="bf16-fp8", refine=True)
    np.testing.assert_array_equal(a["out_id"], b["out_id"])
    np.testing.assert_array_equal(a["out_d"][:, :10], b["out_d"][:, :10])
    # 16 significant bits: the sign, the exponent and the top 15 of the 23 stored mantissa bits
    X16 = (rng.standard_normal((16, 8)).astype(np.float32).view(np.uint32) & np.uint32(0xFFFFFF00)).view(np.float32)
    Q16 = rng.standard_normal((4, 8)).astype(np.float32)
    idx16 = _one_grain_index(X16, 2)
    c = O.search(idx16, X16, Q16, 8, 16, 1, precision="bf16-fp8", refine=True)
    bf, bd, _ = O.brute_force(X16, Q16, 8)
    np.testing.assert_array_equal(c["out_id"], bf)
    np.testing.assert_allclose(c["out_d"][:, :8], bd, rtol=1e-12)
