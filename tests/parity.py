"""Comparison of the CUDA path with the oracle.

Gap rule: let the oracle's ranking be d_1 <= ... <= d_n <= d_{n+1} (the
(n+1)-th value is also reported by the oracle). For every m with
(d_{m+1} - d_m) / d_m > GAP, the GPU's first m ids must be the oracle's first
m ids as a set. Distances of ids present in both must agree within RTOL
relative. Queries whose routing boundary (nprobe-th vs next centre distance)
is closer than GAP relative have no fixed probe set and are excluded from the
pool/top-k comparison (counted); where the pool boundary (C-th vs (C+1)-th)
is closer than GAP, the top k is still compared when the members only one
pool holds are in neither top k (both are then the top k of the common
members), and the query is excluded (counted) otherwise.
"""
import numpy as np

GAP = 1e-4
RTOL = 1e-5


def _rel_gap(a, b):
    if not np.isfinite(a):
        return 0.0
    if not np.isfinite(b):
        return np.inf
    return (b - a) / max(abs(a), 1e-30)


def check_ranked(gpu_ids, gpu_d, ora_ids, ora_d_ext, what, qi, rtol=RTOL, gap=GAP, invalid=None):
    """ora_d_ext has one more value than ora_ids (the next distance)."""
    n = len(ora_ids)
    g_ids = [int(x) for x in gpu_ids]
    o_ids = [int(x) for x in ora_ids]
    # padding must agree exactly where the oracle ran out of rows
    n_valid = sum(1 for x in o_ids if x != invalid)
    g_valid = sum(1 for x in g_ids if x != invalid)
    assert n_valid == g_valid, f"{what} q{qi}: {g_valid} valid entries, oracle {n_valid}"
    # sorted
    gd = np.asarray(gpu_d, dtype=np.float64)[:g_valid]
    assert np.all(np.diff(gd) >= 0), f"{what} q{qi}: GPU distances not sorted"
    for m in range(1, n_valid + 1):
        if _rel_gap(ora_d_ext[m - 1], ora_d_ext[m]) > gap:
            assert set(g_ids[:m]) == set(o_ids[:m]), f"{what} q{qi}: first {m} ids differ"
    od = {i: float(d) for i, d in zip(o_ids, ora_d_ext[:n])}
    for i, d in zip(g_ids[:g_valid], gd):
        if i in od:
            ref = od[i]
            assert abs(d - ref) <= rtol * max(abs(ref), 1e-30) + 1e-30, f"{what} q{qi} id {i}: {d} vs {ref}"


def compare_search(gpu, ora, k, C, nprobe, rtol=RTOL, gap=GAP):
    """gpu: dict of numpy arrays ids, dist, pool_ids (uint32), pool_d, probe.
    ora: oracle search dict. Returns counts of checked / excluded queries."""
    nq = ora["out_id"].shape[0]
    Ce = max(C, k)
    stats = dict(route_excluded=0, topk_excluded=0, checked=0)
    for qi in range(nq):
        # routing: probe set must agree unless the boundary is a near tie
        pd = ora["probe_d"][qi]
        if _rel_gap(pd[nprobe - 1], pd[nprobe]) <= gap and np.isfinite(pd[nprobe]):
            stats["route_excluded"] += 1
            continue
        if "probe" in gpu:
            assert set(gpu["probe"][qi].tolist()) == set(ora["probe"][qi].tolist()), f"probe set q{qi}"
        if "pool_ids" in gpu:
            check_ranked(gpu["pool_ids"][qi].astype(np.uint32), gpu["pool_d"][qi], ora["cand_id"][qi],
                         ora["cand_d"][qi], "pool", qi, rtol, gap, invalid=0xFFFFFFFF)
        cd = ora["cand_d"][qi]
        if _rel_gap(cd[Ce - 1], cd[Ce]) <= gap and np.isfinite(cd[Ce]):
            # the pool's edge is a near tie, so the two pools may hold different
            # members there. Each top k is the k smallest exact distances of its
            # pool; when no member that only one pool holds is in that pool's
            # top k, both are the top k of the common members and must agree.
            if "pool_ids" not in gpu:
                stats["topk_excluded"] += 1
                continue
            gp = set(int(x) for x in gpu["pool_ids"][qi].astype(np.uint32).tolist()) - {0xFFFFFFFF}
            op = set(int(x) for x in ora["cand_id"][qi].tolist()) - {0xFFFFFFFF}
            if (gp - op) & set(int(x) for x in gpu["ids"][qi].tolist()) or \
                    (op - gp) & set(int(x) for x in ora["out_id"][qi].tolist()):
                stats["topk_excluded"] += 1
                continue
        check_ranked(gpu["ids"][qi], gpu["dist"][qi], ora["out_id"][qi], ora["out_d"][qi], "topk", qi, rtol, gap,
                     invalid=-1)
        stats["checked"] += 1
    return stats
