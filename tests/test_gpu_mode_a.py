"""Mode A (the pool reranked by L2 to each row's reconstruction mu_g + W_g z_i,
no raw row read) on the GPU against the oracle's Mode A, element by element,
in both forms (routing and pool under the Mode B rules; the reranked
distances under the tolerance derived below); and the pool Mode A reranks is
bit for bit the one Mode B reranks."""
import numpy as np
import pytest
import torch

from oracle import hntl_oracle as O
from paper_2606_08813_b300 import synth

from cases import clustered_case, partition_index, write
from parity import GAP, _rel_gap, check_ranked

pytestmark = pytest.mark.gpu

# The GPU forms a Mode A distance as ||v'||^2 - 2 z_i . z_q + z_i^T G z_i in
# FP32, with v' = q - mu_g of the member's grain g: every term is of the size
# of ||v'||^2, the result can be far smaller, and FP32 rounding of about
# (d / 32 + r + 10) 2^-24 of those terms (under 1e-5 of them for d <= 768,
# r <= 32) is what separates it from the oracle's FP64 reconstruction. The
# pool distances of the precision form carry the same kind of error, since
# their rho_q comes from ||v'||^2 - 2 ||z_q||^2 + z_q^T G z_q. So such a
# distance is checked to 1e-5 (d + 2 ||v'_g||^2) with g the member's grain,
# and sets of ids are compared wherever the oracle's gap exceeds twice that.
ATOL_SCALE = 1e-5


def _grain_of_id(idx, n):
    pos = np.zeros(n, dtype=np.int64)
    pos[idx["ids"]] = np.arange(len(idx["ids"]))
    gof = np.searchsorted(idx["grain_off"], np.arange(len(idx["ids"])), side="right") - 1
    return gof[pos]


def _check_abs(g_ids, g_d, o_ids, o_d_ext, vn_of, vn_max, what, qi, invalid):
    g_ids, o_ids = [int(x) for x in g_ids], [int(x) for x in o_ids]
    n_valid = sum(1 for x in o_ids if x != invalid)
    assert n_valid == sum(1 for x in g_ids if x != invalid), f"{what} q{qi}: valid entries"
    assert np.all(np.diff(np.asarray(g_d, dtype=np.float64)[:n_valid]) >= 0), f"{what} q{qi}: not sorted"

    def tol(j):  # bound of the oracle's j-th entry; past the listed ones the grain is unknown
        vn = vn_of(o_ids[j]) if j < n_valid else vn_max
        return ATOL_SCALE * (o_d_ext[j] + 2 * vn)

    for m in range(1, n_valid + 1):
        if not np.isfinite(o_d_ext[m]) or o_d_ext[m] - o_d_ext[m - 1] > 2 * max(tol(m - 1), tol(m)):
            assert set(g_ids[:m]) == set(o_ids[:m]), f"{what} q{qi}: first {m} ids differ"
    ref = {i: o_d_ext[j] for j, i in enumerate(o_ids) if i != invalid}
    for j, i in enumerate(g_ids):
        if i in ref:
            d = float(g_d[j])
            assert abs(d - ref[i]) <= ATOL_SCALE * (ref[i] + 2 * vn_of(i)), f"{what} q{qi} id {i}: {d} vs {ref[i]}"


def compare_mode_a(gpu, ora, ora_next, grain_of, k, C, nprobe, precision):
    """ora: the oracle's Mode A; ora_next: its pool with C + 1 members (the id
    just past the pool's edge); grain_of: grain of every id."""
    nq = ora["out_id"].shape[0]
    Ce = max(C, k)
    stats = dict(route_excluded=0, topk_excluded=0, checked=0)
    for qi in range(nq):
        pd = ora["probe_d"][qi]
        if _rel_gap(pd[nprobe - 1], pd[nprobe]) <= GAP and np.isfinite(pd[nprobe]):
            stats["route_excluded"] += 1
            continue
        vmap = {int(g): float(pd[p]) for p, g in enumerate(ora["probe"][qi])}

        def vn_of(i):
            return vmap[int(grain_of[i])]

        cd = ora["cand_d"][qi]
        # pool distances: both forms form rho_q as the explicit residual, so the Mode B rules hold
        check_ranked(gpu["pool_ids"][qi].astype(np.uint32), gpu["pool_d"][qi], ora["cand_id"][qi], cd, "pool",
                     qi, invalid=0xFFFFFFFF)
        edge_tie = _rel_gap(cd[Ce - 1], cd[Ce]) <= GAP and np.isfinite(cd[Ce])
        if edge_tie:
            stats["topk_excluded"] += 1  # the pool's edge is within the error: its members may differ
            continue
        _check_abs(gpu["ids"][qi], gpu["dist"][qi], ora["out_id"][qi], ora["out_d"][qi], vn_of, max(vmap.values()),
                   "topk", qi, -1)
        stats["checked"] += 1
    return stats


def oracle_pair(idx, X, Q, k, C, nprobe, precision, **kw):
    ora = O.search(idx, X, Q, k, C, nprobe, mode="A", precision=precision, **kw)
    ora_next = O.search(idx, X, Q, k, C + 1, nprobe, mode="A", precision=precision, **kw)
    return ora, ora_next, _grain_of_id(idx, len(X))


@pytest.fixture(scope="module")
def hntl():
    from paper_2606_08813_b300 import build_lib

    build_lib.build()
    from paper_2606_08813_b300 import hntl as h

    return h


def run(h, path, Q, k, C, nprobe, precision, filters=None):
    gi = h.Index.load(path, 0, h.PREC_BF16_FP8 if precision == "bf16-fp8" else h.PREC_FP32)
    F = None if filters is None else torch.from_numpy(filters).cuda()
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    ids, dist, pid, pd = gi.search(Qd, k, C, nprobe, filters=F, return_pool=True, mode="A")
    torch.cuda.synchronize()
    return gi, dict(ids=ids.cpu().numpy(), dist=dist.cpu().numpy(), pool_ids=pid.cpu().numpy().view(np.uint32),
                    pool_d=pd.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp32", "bf16-fp8"])
def test_mode_a_clustered(hntl, tmp_path, precision):
    X, Q, idx = clustered_case(8000, 64, 8, 8, 16, 300, seed=211, sizes="zipf")
    p = write(tmp_path, "ma" + precision, idx, X, precision=precision)
    ora, ora_next, gof = oracle_pair(idx, X, Q, 10, 50, 3, precision)
    gi, gpu = run(hntl, p, Q, 10, 50, 3, precision)
    st = compare_mode_a(gpu, ora, ora_next, gof, 10, 50, 3, precision)
    assert st["checked"] >= 0.9 * len(Q), st
    # the pool is Mode B's, bit for bit
    Qd = torch.from_numpy(Q).cuda()
    _, _, pid_b, pd_b = gi.search(Qd, 10, 50, 3, return_pool=True)
    np.testing.assert_array_equal(pid_b.cpu().numpy().view(np.uint32), gpu["pool_ids"])
    np.testing.assert_array_equal(pd_b.cpu().numpy(), gpu["pool_d"])
    assert hntl.device_status(gi) == 0


@pytest.mark.parametrize("precision", ["fp32", "bf16-fp8"])
@pytest.mark.parametrize("d,r", [(24, 5), (16, 16), (64, 8)])
def test_mode_a_edge_shapes(hntl, tmp_path, precision, d, r):
    """Grains of 0, 1, 127, 128, 129 and 300 rows (empty, single row, a ragged
    last block, an exact block); a full basis (r = d); short results."""
    sizes = [0, 1, 127, 128, 129, 300]
    rng = np.random.default_rng(d * 7 + r)
    centres = rng.standard_normal((len(sizes), d)) * 3
    assign = np.repeat(np.arange(len(sizes)), sizes)
    X = (centres[assign] + rng.standard_normal((len(assign), d)) * 0.7).astype(np.float32)
    idx = partition_index(X, assign, len(sizes), r)
    Q = (centres[rng.integers(0, len(sizes), 30)] + rng.standard_normal((30, d)) * 0.7).astype(np.float32)
    p = write(tmp_path, f"mae{precision}{d}_{r}", idx, X, precision=precision)
    for k, C, nprobe in [(10, 20, 2), (5, 200, 3), (10, 685, 6)]:
        ora, ora_next, gof = oracle_pair(idx, X, Q, k, C, nprobe, precision)
        _, gpu = run(hntl, p, Q, k, C, nprobe, precision)
        st = compare_mode_a(gpu, ora, ora_next, gof, k, C, nprobe, precision)
        assert st["checked"] >= len(Q) // 2, (k, C, nprobe, st)


def test_mode_a_filters(hntl, tmp_path):
    X, Q, idx = clustered_case(3000, 32, 8, 8, 6, 60, seed=187)
    attr = synth.attributes(len(X), 7, span=1 << 40).numpy()
    ranges = synth.range_filters(len(Q), 8, span=1 << 40, selectivity=0.2, frac_filtered=0.5).numpy()
    p = write(tmp_path, "mafilt", idx, X, attr=attr, precision="bf16-fp8")
    ora, ora_next, gof = oracle_pair(idx, X, Q, 10, 50, 3, "bf16-fp8", attr=attr, ranges=ranges)
    _, gpu = run(hntl, p, Q, 10, 50, 3, "bf16-fp8", filters=ranges)
    st = compare_mode_a(gpu, ora, ora_next, gof, 10, 50, 3, "bf16-fp8")
    assert st["checked"] >= 0.9 * len(Q), st


@pytest.mark.parametrize("precision", ["fp32", "bf16-fp8"])
def test_mode_a_without_raw_rows(hntl, tmp_path, precision):
    """An index loaded without its raw rows (HNTL_LOAD_NO_RAW) holds less device
    memory, answers Mode A exactly as the full index does, and refuses Mode B
    and the server, which rerank raw rows."""
    X, Q, idx = clustered_case(4000, 64, 8, 8, 16, 50, seed=231)
    p = write(tmp_path, "nr" + precision, idx, X, precision=precision)
    prec = hntl.PREC_BF16_FP8 if precision == "bf16-fp8" else hntl.PREC_FP32
    full = hntl.Index.load(p, 0, prec)
    lean = hntl.Index.load(p, 0, prec | hntl.LOAD_NO_RAW)
    raw_bytes = X.shape[0] * X.shape[1] * (2 if precision == "bf16-fp8" else 4)
    assert full.info()["device_bytes"] - lean.info()["device_bytes"] >= raw_bytes
    Qd = torch.from_numpy(Q).cuda()
    a = [t.cpu() for t in full.search(Qd, 10, 50, 3, mode="A")]
    b = [t.cpu() for t in lean.search(Qd, 10, 50, 3, mode="A")]
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    with pytest.raises(hntl.HntlError) as e:
        lean.search(Qd, 10, 50, 3)
    assert e.value.code == hntl.EINVAL
    with pytest.raises(hntl.HntlError):
        hntl.Server(lean, mem_budget=1 << 28, max_slots=64, batch=32, nprobe=3, k_max=10, C_max=50)
