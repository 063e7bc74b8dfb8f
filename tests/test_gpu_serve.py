"""Continuous-batching server: a request's answer must not depend on the
batch it rides in. Each request served in a mixed stream (mixed k, C and
range filters, submitted in uneven chunks so batches mix them differently)
is compared with the same query searched alone with its own k, C and filter.
The library's open-loop replay gives the same answers. Also: memory
admission refuses requests beyond the free slots, polling an
unknown ticket is an error, and the bounded device waits report a timeout
without losing the context."""
import numpy as np
import pytest
import torch

from paper_2606_08813_b300 import synth

from cases import clustered_case, write

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hntl():
    from paper_2606_08813_b300 import build_lib

    build_lib.build()
    from paper_2606_08813_b300 import hntl as h

    return h


@pytest.fixture(scope="module", params=["fp32", "bf16-fp8"])
def served(hntl, tmp_path_factory, request):
    X, Q, idx = clustered_case(20000, 128, 48, 64, 16, 400, seed=301, sizes="zipf")
    attr = synth.attributes(len(X), 302, span=1000).numpy()
    p = write(tmp_path_factory.mktemp("serve"), "serve", idx, X, attr=attr, precision=request.param)
    prec = hntl.PREC_BF16_FP8 if request.param == "bf16-fp8" else hntl.PREC_FP32
    return hntl.Index.load(p, 0, prec), Q, attr


def _mix(nq, seed):
    rng = np.random.default_rng(seed)
    k = rng.choice([10, 100], nq).astype(np.uint32)
    C = rng.choice([20, 200, 1000], nq).astype(np.uint32)
    C = np.maximum(C, k)
    lo = rng.integers(0, 800, nq)
    ranges = np.stack([lo, lo + 199], 1).astype(np.int64)  # 20% of the attribute span
    filt = rng.random(nq) < 0.5
    ranges[~filt, 0] = np.iinfo(np.int64).min
    ranges[~filt, 1] = np.iinfo(np.int64).max
    return k, C, ranges, filt


def test_mixed_stream_equals_alone(hntl, served):
    gi, Q, _ = served
    nq, nprobe = len(Q), 4
    k, C, ranges, filt = _mix(nq, 303)
    srv = hntl.Server(gi, mem_budget=1 << 30, max_slots=4096, batch=64, nprobe=nprobe, k_max=100, C_max=1000)
    tickets = []
    s = 0
    for chunk in (1, 7, 64, 3, 100, 33, 192):
        t = srv.submit(Q[s:s + chunk], k[s:s + chunk], C[s:s + chunk], ranges[s:s + chunk])
        assert len(t) == chunk
        tickets.extend(t.tolist())
        s += chunk
    assert s == nq
    half = nq // 2
    got = [srv.poll(t, int(k[i])) for i, t in enumerate(tickets[:half])]
    # the rest in bulk
    tk = np.asarray(tickets[half:], dtype=np.uint64)
    done = np.zeros(len(tk), dtype=np.uint8)
    ids_b = np.zeros((len(tk), 100), dtype=np.int64)
    dist_b = np.zeros((len(tk), 100), dtype=np.float32)
    for _ in range(100):
        srv.poll_many(tk, done, ids_b, dist_b, timeout_ms=100)
        if done.all():
            break
    assert done.all()
    got += [(ids_b[j, :k[half + j]], dist_b[j, :k[half + j]]) for j in range(len(tk))]
    with pytest.raises(hntl.HntlError):  # released tickets are unknown now
        srv.poll(int(tk[0]), 10, timeout_ms=0)
    st = srv.stats()
    srv.close()
    assert all(g is not None for g in got)
    assert st["completed"] == nq and st["batches"] >= nq // 64
    # the latency's parts: caller lag, queueing, service (each per request, so none exceeds the whole)
    for part in ("lag", "upload", "queue", "service"):
        assert 0 <= st[f"{part}_p50_us"] <= st[f"{part}_p99_us"] <= st["max_us"] + 1e-6
    assert st["service_p50_us"] > 0
    assert hntl.device_status(gi) == 0
    for i in range(nq):
        q = torch.from_numpy(Q[i:i + 1]).cuda()
        F = torch.from_numpy(ranges[i:i + 1]).cuda() if filt[i] else None
        ids, dist = gi.search(q, int(k[i]), int(C[i]), nprobe, filters=F)
        np.testing.assert_array_equal(got[i][0], ids.cpu().numpy()[0], err_msg=f"query {i}")
        np.testing.assert_array_equal(got[i][1], dist.cpu().numpy()[0], err_msg=f"query {i}")


def test_replay_equals_alone(hntl, served):
    """The library's open-loop replay: every request finishes, the wanted rows
    carry the same ids as the query searched alone, and the latency record
    covers exactly the replayed requests. 96 slots for 400 requests that all
    arrive within a few milliseconds, so admission runs out of slots and the
    replay has to wait for completions before it submits the rest."""
    gi, Q, _ = served
    nq, nprobe = len(Q), 4
    k, C, ranges, filt = _mix(nq, 304)
    rng = np.random.default_rng(305)
    arrival = np.cumsum(rng.exponential(10_000, nq)).astype(np.int64)  # 100k requests/s
    want = np.zeros(nq, dtype=np.uint8)
    want[rng.choice(nq, 120, replace=False)] = 1
    srv = hntl.Server(gi, mem_budget=1 << 30, max_slots=96, batch=32, nprobe=nprobe, k_max=100, C_max=1000)
    n_done, ids = srv.replay(Q, k, C, arrival, ranges=ranges, want=want, timeout_ms=60000)
    st = srv.stats()
    srv.close()
    assert n_done == nq
    assert st["completed"] == nq
    assert (ids[want == 0] == 0).all()
    for i in np.flatnonzero(want):
        q = torch.from_numpy(Q[i:i + 1]).cuda()
        F = torch.from_numpy(ranges[i:i + 1]).cuda() if filt[i] else None
        ref, _ = gi.search(q, int(k[i]), int(C[i]), nprobe, filters=F)
        np.testing.assert_array_equal(ids[i, :k[i]], ref.cpu().numpy()[0], err_msg=f"query {i}")
    with pytest.raises(ValueError):  # arrival times must not decrease
        srv2 = hntl.Server(gi, mem_budget=1 << 30, max_slots=16, batch=8, nprobe=2, k_max=100, C_max=1000)
        try:
            srv2.replay(Q[:2], k[:2], C[:2], np.array([5, 1], np.int64))
        finally:
            srv2.close()


def test_admission_refuses_beyond_free_slots(hntl, served):
    gi, Q, _ = served
    n = 40
    k = np.full(n, 10, np.uint32)
    C = np.full(n, 20, np.uint32)
    srv = hntl.Server(gi, mem_budget=1 << 30, max_slots=16, batch=8, nprobe=2, k_max=10, C_max=20)
    assert srv.stats()["slots"] == 16
    t = srv.submit(Q[:n], k, C)
    assert len(t) == 16  # the rest is refused until slots free up
    for x in t:
        assert srv.poll(x, 10) is not None
    t2 = srv.submit(Q[16:n], k[16:], C[16:])
    assert len(t2) == 16
    with pytest.raises(hntl.HntlError) as e:
        srv.poll(10 ** 9, 10)
    assert e.value.code == hntl.EINVAL
    for x in t2:
        assert srv.poll(x, 10) is not None
    with pytest.raises(hntl.HntlError) as e:
        srv.submit(Q[:1], np.array([11], np.uint32), np.array([20], np.uint32))  # k beyond k_max
    assert e.value.code == hntl.EINVAL
    srv.close()
    # a budget that cannot hold the lanes is refused at creation
    with pytest.raises(hntl.HntlError) as e:
        hntl.Server(gi, mem_budget=1 << 16, max_slots=16, batch=8, nprobe=2, k_max=10, C_max=20)
    assert e.value.code == hntl.ENOMEM


def test_bounded_wait_reports_timeout(hntl, served):
    gi, Q, _ = served
    assert hntl.device_status(gi) == 0
    hntl.selftest_wait_timeout(gi, polls=256)
    torch.cuda.synchronize()
    assert hntl.device_status(gi) & 1  # bit 0: a bounded wait gave up
    assert hntl.device_status(gi) == 0  # cleared by the read
    ids, _ = gi.search(torch.from_numpy(Q[:8]).cuda(), 10, 20, 2)  # the context is still usable
    assert (ids.cpu().numpy() >= 0).all()
