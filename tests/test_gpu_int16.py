"""The paper's 16-bit form (Eq. 5, with the Quantization Envelope Filter of
sec. 2.3) on the GPU, loaded from an FP32 index file, against the oracle's
16-bit form on the same file, element by element.

Rows are quantised the same way on both sides (IEEE single-precision steps
and codes), so their values agree exactly. The query's coordinates are
quantised from z_q, which the GPU forms in FP32 and the oracle in FP64: near
a rounding boundary the two can pick neighbouring codes, which moves D by at
most 2 |z_qj - z_ij| delta + delta^2 in that coordinate, and the query's
residual by one step dres. A pool distance is therefore checked to
1e-5 D + 4 delta_g sqrt(D) + 2 delta_g^2 + dres_g (two coordinates and the
residual on a neighbouring code; |z_qj - z_ij| <= sqrt(D)), with g the
member's grain; id sets are compared wherever the oracle's gap exceeds twice
that. The final top k are exact L2 distances to the raw rows (1e-5)."""
import numpy as np
import pytest
import torch

from oracle import hntl_oracle as O
from paper_2606_08813_b300 import synth

from cases import clustered_case, partition_index, write
from parity import GAP, _rel_gap, check_ranked

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hntl():
    from paper_2606_08813_b300 import build_lib

    build_lib.build()
    from paper_2606_08813_b300 import hntl as h

    return h


def run(h, path, Q, k, C, nprobe, filters=None, precision=None):
    gi = h.Index.load(path, 0, h.PREC_INT16 if precision is None else precision)
    F = None if filters is None else torch.from_numpy(filters).cuda()
    ids, dist, pid, pd, probe = gi.search(torch.from_numpy(np.ascontiguousarray(Q)).cuda(), k, C, nprobe, filters=F,
                                          return_pool=True, return_probe=True)
    torch.cuda.synchronize()
    return gi, dict(ids=ids.cpu().numpy(), dist=dist.cpu().numpy(), pool_ids=pid.cpu().numpy().view(np.uint32),
                    pool_d=pd.cpu().numpy(), probe=probe.cpu().numpy())


def _grain_of_id(idx, n):
    pos = np.zeros(n, dtype=np.int64)
    pos[idx["ids"]] = np.arange(len(idx["ids"]))
    gof = np.searchsorted(idx["grain_off"], np.arange(len(idx["ids"])), side="right") - 1
    return gof[pos]


def compare_int16(gpu, ora, ora_next, idx, n, k, C, nprobe):
    """ora_next: the oracle's pool with C + 1 members (the id past the edge)."""
    f = O.int16_form(idx)
    gof = _grain_of_id(idx, n)

    def tol(i, dv):
        g = gof[int(i)]
        dl, dr = float(f["delta"][g]), float(f["dres"][g])
        return 1e-5 * dv + 4 * dl * np.sqrt(max(dv, 0.0)) + 2 * dl * dl + dr

    Ce = max(C, k)
    stats = dict(route_excluded=0, topk_excluded=0, checked=0)
    for qi in range(len(ora["out_id"])):
        pd = ora["probe_d"][qi]
        if _rel_gap(pd[nprobe - 1], pd[nprobe]) <= GAP and np.isfinite(pd[nprobe]):
            stats["route_excluded"] += 1
            continue
        assert set(gpu["probe"][qi].tolist()) == set(ora["probe"][qi].tolist()), f"probe set q{qi}"
        o_ids = [int(x) for x in ora["cand_id"][qi]]
        g_ids = [int(x) for x in gpu["pool_ids"][qi]]
        od, gd = ora["cand_d"][qi], gpu["pool_d"][qi]
        nv = sum(1 for x in o_ids if x != 0xFFFFFFFF)
        assert nv == sum(1 for x in g_ids if x != 0xFFFFFFFF), f"pool q{qi}: valid entries"
        assert np.all(np.diff(gd[:nv].astype(np.float64)) >= 0), f"pool q{qi}: not sorted"
        nxt = [int(x) for x in ora_next["cand_id"][qi]]
        for m in range(1, nv + 1):
            nid = o_ids[m] if m < nv else nxt[m] if m < len(nxt) else 0xFFFFFFFF
            t = tol(o_ids[m - 1], od[m - 1])
            if nid != 0xFFFFFFFF:
                t = max(t, tol(nid, od[m]))
            if not np.isfinite(od[m]) or od[m] - od[m - 1] > 2 * t:
                assert set(g_ids[:m]) == set(o_ids[:m]), f"pool q{qi}: first {m} ids differ"
        ref = {i: od[j] for j, i in enumerate(o_ids) if i != 0xFFFFFFFF}
        for j, i in enumerate(g_ids):
            if i in ref:
                assert abs(float(gd[j]) - ref[i]) <= tol(i, ref[i]), f"pool q{qi} id {i}: {gd[j]} vs {ref[i]}"
        # the pool's edge: within the error its members may differ, and so may the top k
        if np.isfinite(od[Ce]):
            t = max(tol(o_ids[Ce - 1], od[Ce - 1]), tol(nxt[Ce], od[Ce]))
            if od[Ce] - od[Ce - 1] <= 2 * t:
                stats["topk_excluded"] += 1
                continue
        check_ranked(gpu["ids"][qi], gpu["dist"][qi], ora["out_id"][qi], ora["out_d"][qi], "topk", qi, invalid=-1)
        stats["checked"] += 1
    return stats


def oracle_pair(idx, X, Q, k, C, nprobe, **kw):
    return (O.search(idx, X, Q, k, C, nprobe, precision="int16", **kw),
            O.search(idx, X, Q, k, C + 1, nprobe, precision="int16", **kw))


def test_int16_clustered(hntl, tmp_path):
    X, Q, idx = clustered_case(8000, 64, 8, 8, 16, 300, seed=221, sizes="zipf")
    p = write(tmp_path, "i16", idx, X)
    ora, nxt = oracle_pair(idx, X, Q, 10, 50, 3)
    gi, gpu = run(hntl, p, Q, 10, 50, 3)
    st = compare_int16(gpu, ora, nxt, idx, len(X), 10, 50, 3)
    # dense pools: about a fifth of the pool edges lie within the quantisation error
    assert st["checked"] >= 0.75 * len(Q), st
    assert hntl.device_status(gi) == 0
    with pytest.raises(hntl.HntlError):  # no Mode A on the 16-bit form
        gi.search(torch.from_numpy(Q[:4]).cuda(), 10, 50, 3, mode="A")


@pytest.mark.parametrize("d,r", [(24, 5), (16, 16), (64, 8)])
def test_int16_edge_shapes(hntl, tmp_path, d, r):
    """Grains of 0, 1, 127, 128, 129 and 300 rows; r padded to the 8-code lane
    (r = 5); a full basis (r = d)."""
    sizes = [0, 1, 127, 128, 129, 300]
    rng = np.random.default_rng(d * 11 + r)
    centres = rng.standard_normal((len(sizes), d)) * 3
    assign = np.repeat(np.arange(len(sizes)), sizes)
    X = (centres[assign] + rng.standard_normal((len(assign), d)) * 0.7).astype(np.float32)
    idx = partition_index(X, assign, len(sizes), r)
    Q = (centres[rng.integers(0, len(sizes), 30)] + rng.standard_normal((30, d)) * 0.7).astype(np.float32)
    p = write(tmp_path, f"i16e{d}_{r}", idx, X)
    for k, C, nprobe in [(10, 20, 2), (5, 200, 3), (10, 685, 6)]:
        ora, nxt = oracle_pair(idx, X, Q, k, C, nprobe)
        _, gpu = run(hntl, p, Q, k, C, nprobe)
        st = compare_int16(gpu, ora, nxt, idx, len(X), k, C, nprobe)
        assert st["checked"] >= len(Q) // 2, (k, C, nprobe, st)


def test_int16_envelope_filter_drops_a_far_grain(hntl, tmp_path):
    """A tight grain far from the queries: every query coordinate saturates in
    its frame, so its rows never reach the pool (they would without the filter)."""
    rng = np.random.default_rng(17)
    A = rng.standard_normal((50, 8))
    B = 60.0 + 0.01 * rng.standard_normal((50, 8))
    X = np.concatenate([A, B]).astype(np.float32)
    idx = partition_index(X, np.repeat([0, 1], 50), 2, 4)
    Q = (0.1 * rng.standard_normal((3, 8))).astype(np.float32)
    p = write(tmp_path, "i16qef", idx, X)
    ora = O.search(idx, X, Q, 10, 80, 2, precision="int16")
    _, gpu = run(hntl, p, Q, 10, 80, 2)
    for qi in range(3):
        ids = gpu["pool_ids"][qi]
        assert set(ids[ids != 0xFFFFFFFF].tolist()) == set(range(50)) == set(
            ora["cand_id"][qi][ora["cand_id"][qi] != 0xFFFFFFFF].tolist())
        np.testing.assert_array_equal(gpu["ids"][qi], ora["out_id"][qi])
    # the FP32 form of the same file does take the far grain's rows
    gf = hntl.Index.load(p, 0, hntl.PREC_FP32)
    _, _, pid, _ = gf.search(torch.from_numpy(Q).cuda(), 10, 80, 2, return_pool=True)
    assert (pid.cpu().numpy().view(np.uint32) >= 50).sum() == 3 * 30


def test_int16_filters(hntl, tmp_path):
    X, Q, idx = clustered_case(3000, 32, 8, 8, 8, 60, seed=197)
    attr = synth.attributes(len(X), 9, span=1 << 40).numpy()
    ranges = synth.range_filters(len(Q), 10, span=1 << 40, selectivity=0.2, frac_filtered=0.5).numpy()
    p = write(tmp_path, "i16filt", idx, X, attr=attr)
    ora, nxt = oracle_pair(idx, X, Q, 10, 50, 3, attr=attr, ranges=ranges)
    _, gpu = run(hntl, p, Q, 10, 50, 3, filters=ranges)
    st = compare_int16(gpu, ora, nxt, idx, len(X), 10, 50, 3)
    assert st["checked"] >= 0.85 * len(Q), st


def _resid_case(tmp_path):
    rng = np.random.default_rng(19)
    A = rng.standard_normal((50, 8))
    B = np.zeros((50, 8))
    B[:, :4] = rng.standard_normal((50, 4))
    B[:, 4:] = 20.0 + 1e-3 * rng.standard_normal((50, 4))
    X = np.concatenate([A, B]).astype(np.float32)
    idx = partition_index(X, np.repeat([0, 1], 50), 2, 4)
    Q = (0.1 * rng.standard_normal((3, 8))).astype(np.float32)
    return X, Q, idx, write(tmp_path, "i16res", idx, X)


def test_int16_residual_clipped_by_default_and_pruned_by_option(hntl, tmp_path):
    """Grain B varies only inside its own subspace; the queries sit off it:
    their coordinates in B's frame stay in range but the residual code exceeds
    65535. Under the paper's rule (Eq. 5, the filter of sec. 2.3 counts
    coordinates) the residual is clipped and B's rows enter the pool, on both
    sides alike; with the library's residual-saturation option B stays out."""
    X, Q, idx, p = _resid_case(tmp_path)
    ws_nq, k, C, nprobe = len(Q), 10, 80, 2
    gi = hntl.Index.load(p, 0, hntl.PREC_INT16)
    ws = gi.workspace(gi.workspace_bytes(ws_nq, k, C, nprobe))
    ids, dist, pid, pd = gi.search(torch.from_numpy(Q).cuda(), k, C, nprobe, return_pool=True, ws=ws)
    codes, rc = hntl.search_pair_codes(gi, ws, ws_nq, C, nprobe)
    torch.cuda.synchronize()
    ora = O.search(idx, X, Q, k, C, nprobe, precision="int16",
                   query_codes=(codes.cpu().numpy(), rc.cpu().numpy()), probes=np.tile([0, 1], (len(Q), 1)))
    assert (rc.cpu().numpy() == 65535).any()  # the premise: a clipped residual
    pid = pid.cpu().numpy().view(np.uint32)
    for qi in range(len(Q)):
        assert (pid[qi] >= 50).sum() >= 30  # B's rows crowd in with the clipped residual
        np.testing.assert_array_equal(pid[qi], ora["cand_id"][qi])
        np.testing.assert_array_equal(pd.cpu().numpy()[qi].astype(np.float64), ora["cand_d"][qi][:C])
    ora_p = O.search(idx, X, Q, k, C, nprobe, precision="int16", resid_prune=True)
    _, gp = run(hntl, p, Q, k, C, nprobe, precision=hntl.PREC_INT16 | hntl.INT16_RESID_PRUNE)
    for qi in range(len(Q)):
        got = gp["pool_ids"][qi]
        assert set(got[got != 0xFFFFFFFF].tolist()) == set(range(50)) == set(
            ora_p["cand_id"][qi][ora_p["cand_id"][qi] != 0xFFFFFFFF].tolist())
        np.testing.assert_array_equal(gp["ids"][qi], ora_p["out_id"][qi])
    with pytest.raises(hntl.HntlError):  # the option belongs to the 16-bit form
        hntl.Index.load(p, 0, hntl.PREC_FP32 | hntl.INT16_RESID_PRUNE)


@pytest.mark.parametrize("case", ["clustered", "edge"])
def test_int16_integer_scan_bit_exact_on_the_same_codes(hntl, tmp_path, case):
    """The integer scan against the oracle's integer Eq. 6 on the same integer
    inputs: the GPU's quantised query codes (read back from the workspace) go
    to the oracle in place of its own quantisation, and then every pool id and
    pool distance must be equal bit for bit (the same integer sums, the same
    single-precision scale-back), the top k to the parity tolerance. Covers
    dp2a sums over r = 5 (padded lane), 16 and 64 codes, grains of 0 .. 300
    rows, and pools that overflow into the recomputing fallback (C = 685)."""
    if case == "clustered":
        X, Q, idx = clustered_case(8000, 64, 8, 8, 16, 200, seed=231, sizes="zipf")
        shapes = [(10, 50, 3), (10, 685, 8)]
    else:
        sizes = [0, 1, 127, 128, 129, 300]
        rng = np.random.default_rng(77)
        d = 64
        centres = rng.standard_normal((len(sizes), d)) * 3
        assign = np.repeat(np.arange(len(sizes)), sizes)
        X = (centres[assign] + rng.standard_normal((len(assign), d)) * 0.7).astype(np.float32)
        Q = (centres[rng.integers(0, len(sizes), 40)] + rng.standard_normal((40, d)) * 0.7).astype(np.float32)
        shapes = []
        for r in (5, 64):
            idx_r = partition_index(X, assign, len(sizes), r)
            shapes.append((idx_r, (10, 200, 3)))
    runs = [(idx, sh) for sh in shapes] if case == "clustered" else shapes
    for n_run, (ix, (k, C, nprobe)) in enumerate(runs):
        p = write(tmp_path, f"i16x{case}{n_run}", ix, X)
        gi = hntl.Index.load(p, 0, hntl.PREC_INT16)
        nq = len(Q)
        ws = gi.workspace(gi.workspace_bytes(nq, k, C, nprobe))
        ids, dist, pid, pd, probe = gi.search(torch.from_numpy(Q).cuda(), k, C, nprobe, return_pool=True,
                                              return_probe=True, ws=ws)
        codes, rc = hntl.search_pair_codes(gi, ws, nq, C, nprobe)
        torch.cuda.synchronize()
        codes, rc = codes.cpu().numpy(), rc.cpu().numpy()
        # the codes belong to the GPU's probe list, so the oracle takes that list too
        ora = O.search(ix, X, Q, k, max(C, k), nprobe, precision="int16", query_codes=(codes, rc),
                       probes=probe.cpu().numpy())
        pidn = pid.cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(pidn, ora["cand_id"])
        np.testing.assert_array_equal(pd.cpu().numpy().astype(np.float64), ora["cand_d"][:, :C])
        for qi in range(nq):
            check_ranked(ids.cpu().numpy()[qi], dist.cpu().numpy()[qi], ora["out_id"][qi], ora["out_d"][qi], "topk",
                         qi, invalid=-1)
        assert hntl.device_status(gi) == 0
