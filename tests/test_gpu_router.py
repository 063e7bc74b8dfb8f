"""Learned grain router on the GPU against the FP64 router oracle (same BF16
roundings), and what training it gains over centroid routing."""
import numpy as np
import pytest
import torch

from oracle import hntl_oracle as O
from oracle import router_oracle as R
from paper_2606_08813_b300 import synth

from cases import write
from parity import compare_search

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hntl():
    from paper_2606_08813_b300 import build_lib

    build_lib.build()
    from paper_2606_08813_b300 import hntl as h

    return h


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def test_gradients_and_logits_match_oracle(hntl):
    d, h1, h2, G, B = 64, 128, 96, 64, 32
    params = R.init_params(d, h1, h2, G, seed=3)
    rng = np.random.default_rng(4)
    params[1] = (0.1 * rng.standard_normal(h1)).astype(np.float32)
    params[5] = (0.1 * rng.standard_normal(G)).astype(np.float32)
    X = rng.standard_normal((B, d)).astype(np.float32)
    T = rng.random((B, G))
    T = (T / T.sum(1, keepdims=True)).astype(np.float32)
    rt = hntl.Router(params, max_batch=64)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    loss = torch.zeros(1, device="cuda")
    logits = rt.logits(Xd).cpu().numpy()
    rt.step(Xd, Td, update=False, loss=loss)
    torch.cuda.synchronize()
    f = R.forward(params, X, round_bf16=True)
    # At these widths an activation's FP32 sum (GPU) and FP64 sum (oracle)
    # straddle a BF16 rounding boundary for about one in 10^3 elements; such an
    # activation then differs by one BF16 step (2^-8 relative) on the two sides
    # and moves every downstream product by |w| 2^-8 |h|. Over the 1024 inputs
    # of a layer that is ~1e-4 of the logits' norm (measured 1.2e-4), so the
    # logits are held to 1e-3, the gradients (two more rounding points) to 1e-2,
    # and the loss, a mean over the batch, to 1e-4.
    assert _rel(logits, f["L"]) < 1e-3, _rel(logits, f["L"])
    grads, ref_loss = R.backward(params, X, T.astype(np.float64), round_bf16=True)
    assert abs(float(loss.item()) - ref_loss) <= 1e-4 * abs(ref_loss)
    for name, g, ref in zip(("dW1", "db1", "dW2", "db2", "dW3", "db3"), rt.grads(), grads):
        assert _rel(g, ref) < 1e-2, (name, _rel(g, ref))


def test_adamw_step_matches_oracle(hntl):
    d, h1, h2, G, B = 32, 64, 64, 32, 16
    params = R.init_params(d, h1, h2, G, seed=5)
    rng = np.random.default_rng(6)
    X = rng.standard_normal((B, d)).astype(np.float32)
    T = np.zeros((B, G), dtype=np.float32)
    T[np.arange(B), rng.integers(0, G, B)] = 1.0
    rt = hntl.Router(params, max_batch=16)
    rt.step(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda(), lr=1e-2, wd=0.01, update=True)
    torch.cuda.synchronize()
    grads = rt.grads()  # the gradients the GPU stepped with (checked against the oracle above)
    zeros = [np.zeros_like(p, dtype=np.float64) for p in params]
    wd = [0.01 if i % 2 == 0 else 0.0 for i in range(6)]
    want = []
    for i, (p, g) in enumerate(zip(params, grads)):
        np_, _, _ = R.adamw([p], [np.asarray(g, np.float64)], [zeros[i]], [zeros[i]], step=1, lr=1e-2, wd=wd[i])
        want.append(np_[0])
    for got, ref in zip(rt.params(), want):
        np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-7)


def test_step_graph_replays_direct_launches_bit_for_bit(hntl):
    """The captured training step against the same step launched kernel by
    kernel: new input buffers (graph updated in place), another lr, a smaller
    batch (new grid sizes) and a gradient-only step in between."""
    d, h1, h2, G = 32, 64, 64, 48
    params = R.init_params(d, h1, h2, G, seed=9)
    rng = np.random.default_rng(10)
    routers = [hntl.Router(params, max_batch=32) for _ in range(2)]
    routers[1].set_graphs(False)
    bufs = []
    for B in (32, 32, 16):
        X = torch.from_numpy(rng.standard_normal((B, d)).astype(np.float32)).cuda()
        T = torch.zeros(B, G, device="cuda")
        T[torch.arange(B), torch.from_numpy(rng.integers(0, G, B)).cuda()] = 1.0
        bufs.append((X, T))
    plan = [(0, 1e-3, True), (1, 1e-3, True), (0, 1e-3, True), (0, 5e-4, True), (2, 5e-4, True), (1, 5e-4, False),
            (1, 5e-4, True)]
    losses = [torch.zeros(1, device="cuda") for _ in routers]
    for b, lr, upd in plan:
        for rt, lo in zip(routers, losses):
            rt.step(bufs[b][0], bufs[b][1], lr=lr, wd=0.01, update=upd, loss=lo)
    torch.cuda.synchronize()
    for a, b in zip(routers[0].params() + routers[0].grads(), routers[1].params() + routers[1].grads()):
        np.testing.assert_array_equal(a, b)
    # the loss is a sum of per-row atomic adds, in whatever order the blocks
    # finish (on either path): n adds to a running sum below 2^5 differ by at
    # most n ulp(2^5) = n 2^-18 between two orders
    n_adds = sum(bufs[b][0].shape[0] for b, _, _ in plan)
    assert abs(float(losses[0].item()) - float(losses[1].item())) <= n_adds * 2.0 ** -18
    assert float(losses[0].item()) < 32
    assert routers[0].status() == 0 and routers[1].status() == 0
    # the steps did move the parameters
    assert any(not np.array_equal(a, b) for a, b in zip(routers[0].params(), params))


def test_router_route_fallback_and_search_with_probes(hntl, tmp_path):
    m = synth.make_cluster_model(4000, 64, 8, seed=71)
    X, _ = synth.sample_points(m, 72)
    Q, _ = synth.sample_queries(m, 40, 73)
    X, Q = X.numpy(), Q.numpy()
    idx = O.build_index(X, 8, 8, synth.uniforms(8, 74).numpy())
    gi = hntl.Index.load(write(tmp_path, "rt", idx, X), 0)
    rt = hntl.Router(R.init_params(64, 64, 64, 8, seed=1), max_batch=64)
    Qd = torch.from_numpy(Q).cuda()
    # tau > 1: every query falls back to centroid routing -> identical to the plain search
    probes, nfb = rt.route(gi, Qd, 3, tau=2.0)
    assert int(nfb.item()) == len(Q)
    cprobe, _ = gi.route(Qd, 3)
    assert torch.equal(probes.cpu(), cprobe.cpu())
    ids, dist = hntl.search_probes(gi, Qd, probes, 10, 40)
    ids2, dist2 = gi.search(Qd, 10, 40, 3)
    assert torch.equal(ids, ids2) and torch.equal(dist, dist2)
    # the router's own probes (tau = 0: no fallback) searched on both sides:
    # the oracle takes the same probe lists in place of its routing
    probes0, nfb0 = rt.route(gi, Qd, 3, tau=0.0)
    assert int(nfb0.item()) == 0
    ids3, dist3 = hntl.search_probes(gi, Qd, probes0, 10, 40)
    p0 = probes0.cpu().numpy()
    ora = O.search(idx, X, Q, 10, 40, 3, probes=p0)
    gpu = dict(ids=ids3.cpu().numpy(), dist=dist3.cpu().numpy())
    st = compare_search(gpu, ora, 10, 40, 3)
    assert st["route_excluded"] == 0 and st["checked"] >= 0.8 * len(Q), st
    assert hntl.device_status(gi) == 0


def _route_against_oracle(hntl, gi, rt, params, Q, idx, X, nprobe, tau_mid=None):
    """Route Q at tau 0, tau_mid (default: the median of the oracle's softmax
    masses, so that about half the queries fall back) and 2, and compare with
    the router oracle: probe
    sets must agree unless the nprobe-th and next logits are within the
    logits' FP32 error, the fallback decision unless the probes' softmax mass
    is within that error of tau; fallen-back queries carry the oracle's
    centroid probes."""
    Qd = torch.from_numpy(Q).cuda()
    cent = O.search(idx, X, Q, 1, 1, nprobe)
    if tau_mid is None:
        tau_mid = float(np.median(R.route(params, Q, nprobe, 0.0, cent["probe"])[2]))
    for tau in (0.0, tau_mid, 2.0):
        probes, nfb = rt.route(gi, Qd, nprobe, tau=tau)
        got = probes.cpu().numpy()
        want, fell, mass, L = R.route(params, Q, nprobe, tau, cent["probe"])
        Ls = -np.sort(-L, axis=1)
        tol = 1e-4 * np.maximum(1.0, np.abs(L).max(1))  # FP32 logits: ~1e-5 of their scale
        n_cmp = n_fb = 0
        for i in range(len(Q)):
            if abs(mass[i] - tau) <= 1e-4 * max(1.0, tau):
                continue  # fallback decision within rounding
            rd = cent["probe_d"][i]
            if fell[i]:
                n_fb += 1
                if (rd[nprobe] - rd[nprobe - 1]) <= 1e-4 * rd[nprobe - 1]:
                    continue  # centroid routing boundary is a near tie
                assert set(got[i].tolist()) == set(want[i].tolist()), (tau, i, "fallback")
            else:
                if Ls[i, nprobe - 1] - Ls[i, nprobe] <= tol[i]:
                    continue
                assert set(got[i].tolist()) == set(want[i].tolist()), (tau, i)
            n_cmp += 1
        assert n_cmp >= 0.9 * len(Q), (tau, n_cmp)
        assert abs(int(nfb.item()) - int(fell.sum())) <= len(Q) - n_cmp, (tau, int(nfb.item()), int(fell.sum()))
        if tau == 0.0:
            assert not fell.any() and int(nfb.item()) == 0
        if tau == 2.0:
            assert fell.all()
        if tau == tau_mid:
            assert 0 < n_fb < len(Q), n_fb  # a mix of kept and fallen-back queries


def test_learned_probes_and_fallback_match_oracle(hntl, tmp_path):
    """Top-nprobe of the GPU's logits and the tau fallback against the router
    oracle (FP64 with the same BF16 roundings), over three query chunks of
    the router's batch."""
    d, G, nprobe = 64, 48, 4
    m = synth.make_cluster_model(6000, d, 12, seed=91)
    X, _ = synth.sample_points(m, 92)
    Q, _ = synth.sample_queries(m, 300, 93)
    X, Q = X.numpy(), Q.numpy()
    idx = O.build_index(X, G, 8, synth.uniforms(G, 94).numpy())
    gi = hntl.Index.load(write(tmp_path, "lp", idx, X), 0)
    params = R.init_params(d, 128, 128, G, seed=95)
    rng = np.random.default_rng(96)
    params[4] = (params[4] * 6.0).astype(np.float32)  # spread the logits so the masses vary by query
    params[5] = rng.standard_normal(G).astype(np.float32)
    rt = hntl.Router(params, max_batch=128)
    _route_against_oracle(hntl, gi, rt, params, Q, idx, X, nprobe, tau_mid=0.35)


@pytest.mark.parametrize("G,nprobe", [(4096, 64), (5000, 32), (304, 65)])
def test_learned_selection_paths_match_oracle(hntl, tmp_path, G, nprobe):
    """The fused per-query selection at its edges (4096 grains, 16 logits a
    thread, the largest nprobe it takes; 5000 grains, 32 logits a thread) and
    the general path beyond 64 probes, against the router oracle."""
    from cases import partition_index

    d = 32
    m = synth.make_cluster_model(4 * G, d, G, seed=970 + G)  # one grain per cluster: separated centres
    X, lab = synth.sample_points(m, 971 + G)
    Q, _ = synth.sample_queries(m, 160, 972 + G)
    X, Q = X.numpy(), Q.numpy()
    idx = partition_index(X, lab.numpy(), G, 4)
    gi = hntl.Index.load(write(tmp_path, f"sel{G}", idx, X), 0)
    params = R.init_params(d, 64, 64, G, seed=973 + G)
    rng = np.random.default_rng(974 + G)
    params[4] = (params[4] * 6.0).astype(np.float32)
    params[5] = rng.standard_normal(G).astype(np.float32)
    rt = hntl.Router(params, max_batch=128)
    _route_against_oracle(hntl, gi, rt, params, Q, idx, X, nprobe)


def test_gradients_at_full_router_widths(hntl):
    """The config-sized router (768 -> 1024 -> 1024 -> 4096, batch 1024):
    the 128-wide GEMM tiles, K loops of up to 64 blocks that wrap the TMA
    ring many times, against the FP64 oracle with the same BF16 roundings."""
    d, h1, h2, G, B = 768, 1024, 1024, 4096, 1024
    params = R.init_params(d, h1, h2, G, seed=13)
    rng = np.random.default_rng(14)
    params[1] = (0.1 * rng.standard_normal(h1)).astype(np.float32)
    params[5] = (0.1 * rng.standard_normal(G)).astype(np.float32)
    X = rng.standard_normal((B, d)).astype(np.float32)
    T = np.zeros((B, G), dtype=np.float32)
    for i in range(B):  # ten neighbours spread over up to ten grains, like the method's labels
        for g in rng.integers(0, G, 10):
            T[i, g] += 0.1
    rt = hntl.Router(params, max_batch=B)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    loss = torch.zeros(1, device="cuda")
    logits = rt.logits(Xd).cpu().numpy()
    rt.step(Xd, Td, update=False, loss=loss)
    torch.cuda.synchronize()
    assert rt.status() == 0
    f = R.forward(params, X, round_bf16=True)
    # At these widths an activation's FP32 sum (GPU) and FP64 sum (oracle)
    # straddle a BF16 rounding boundary for about one in 10^3 elements; such an
    # activation then differs by one BF16 step (2^-8 relative) on the two sides
    # and moves every downstream product by |w| 2^-8 |h|. Over the 1024 inputs
    # of a layer that is ~1e-4 of the logits' norm (measured 1.2e-4), so the
    # logits are held to 1e-3, the gradients (two more rounding points) to 1e-2,
    # and the loss, a mean over the batch, to 1e-4.
    assert _rel(logits, f["L"]) < 1e-3, _rel(logits, f["L"])
    grads, ref_loss = R.backward(params, X, T.astype(np.float64), round_bf16=True)
    assert abs(float(loss.item()) - ref_loss) <= 1e-4 * abs(ref_loss)
    for name, g, ref in zip(("dW1", "db1", "dW2", "db2", "dW3", "db3"), rt.grads(), grads):
        assert _rel(g, ref) < 1e-2, (name, _rel(g, ref))


def _labels(X, Q, assign, G, k=10):
    nb, _, _ = O.brute_force(X, Q, k)
    return R.soft_targets(nb, assign, G).astype(np.float32)


def test_training_gain_over_centroid_routing(hntl, tmp_path):
    """What the trained router gains over the method without it (centroid
    routing) at the same nprobe. Grains are capacity-bounded (at most N / G
    rows each, by deferred acceptance): Zipf-sized clusters overflow their
    nearest centres, so a grain is no longer the Voronoi cell of its centre and
    the nearest centres often do not hold a query's neighbours. The router,
    trained on the grains that hold each training query's brute-force top 10,
    learns where the rows actually went. Measured on 1000 held-out queries:
    recall@10 of the same search (C = 100, k = 10) with learned against
    centroid probes, at nprobe 2, 4 and 8. Training also brings the loss close
    to its floor (the targets' entropy)."""
    d, n_clusters, n, G, r = 64, 16, 40000, 256, 8
    m = synth.make_cluster_model(n, d, n_clusters, sizes="zipf", seed=5)
    X, _ = synth.sample_points(m, 6)
    Qtr, _ = synth.sample_queries(m, 20000, 7)
    Qev, _ = synth.sample_queries(m, 1000, 8)
    X, Qtr, Qev = X.numpy(), Qtr.numpy(), Qev.numpy()
    cap = n // G + (n % G > 0)
    idx = O.build_index(X, G, r, synth.uniforms(G, 9).numpy(), max_grain_rows=cap)
    assert np.bincount(idx["assign"], minlength=G).max() <= cap
    gi = hntl.Index.load(write(tmp_path, "train", idx, X), 0)
    T = _labels(X, Qtr, idx["assign"], G)
    init = R.init_params(d, 256, 256, G, seed=86)
    untrained = hntl.Router(init, max_batch=256)
    rt = hntl.Router(init, max_batch=256)
    Xtr, Ttr = torch.from_numpy(Qtr).cuda(), torch.from_numpy(T).cuda()
    gen = torch.Generator().manual_seed(87)
    losses = []
    for epoch in range(30):
        perm = torch.randperm(len(Qtr), generator=gen).cuda()
        lo = torch.zeros(1, device="cuda")
        for s in range(0, len(Qtr), 256):
            b = perm[s:s + 256]
            rt.step(Xtr[b].contiguous(), Ttr[b].contiguous(), lr=2e-3, wd=0.01, loss=lo)
        losses.append(float(lo.item()) * 256 / len(Qtr))
    floor = float(-(T * np.log(np.maximum(T, 1e-12))).sum(1).mean())
    bf, _, _ = O.brute_force(X, Qev, 10)
    Qd = torch.from_numpy(Qev).cuda()

    def recall(ids):
        return np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ids.cpu().numpy().tolist(), bf.tolist())])

    report = {}
    for nprobe in (2, 4, 8):
        ids_c, _ = gi.search(Qd, 10, 100, nprobe)
        out = []
        for router in (rt, untrained):
            probes, _ = router.route(gi, Qd, nprobe, tau=0.0)
            ids_r, _ = hntl.search_probes(gi, Qd, probes, 10, 100)
            out.append(recall(ids_r))
        report[nprobe] = dict(centroid=recall(ids_c), learned=out[0], untrained=out[1],
                              gain=out[0] - recall(ids_c))
    print("router loss first/last/floor", losses[0], losses[-1], floor)
    print("router recall by nprobe:", report)
    assert losses[-1] < 0.5 * losses[0] and losses[-1] < floor + 0.5
    for nprobe, rep in report.items():
        assert rep["learned"] >= rep["untrained"] + 0.2, (nprobe, rep)
    assert report[4]["gain"] >= 0.05 and report[8]["gain"] >= 0.05, report
