"""Throughput benchmark of the HNTL batched query path on B300.

A step is one hntl_search call over one batch of queries: routing, bucketing,
projection, Block-SoA scan, pool selection and exact rerank, all in the
library's CUDA kernels, with the index and the queries resident in HBM. The
index is built once on the GPU by the library's builder (not timed).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Multi-GPU (torchrun): every rank holds a replica of the index and searches
its own query stream; no data-path collective (weak scaling). value = all
ranks' queries / max over ranks of the timed seconds.

--impl reference times the CPU oracle (the plain FP64 program the tests use
as ground truth) on the host cores, on a bounded sample of the same
workload's queries against the same index, and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_08813_b300 import synth  # noqa: E402

METRIC = "QPS at Recall@10>=0.95"
L2_BYTES = 126 * 1024 * 1024


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), "measured"
    except Exception:
        return 6400.0, 1800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.out.close()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.remove(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows), "power_w_max": max(power) if power else None}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        if torch.cuda.is_available():
            dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
        else:  # host-only runs (the multi-process tests): same collectives over gloo
            dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_qps(world: int, steps: int, batch: int, total_ms_max: float) -> float:
    """Whole-job queries/s of replicas that each searched `steps` batches of
    `batch` queries: every rank's queries over the slowest rank's time."""
    return world * steps * batch / (total_ms_max / 1e3)


def make_workload(name: str, device, rank: int = 0):
    w = dict(synth.WORKLOADS[name])
    sd = synth.seeds(w["seed"])
    model = synth.make_cluster_model(w["n"], w["d"], w["n_clusters"], sizes=w["sizes"], seed=sd["data"])
    X, _ = synth.sample_points(model, sd["data"] + 11, device=device, chunk=65536)
    Q, _ = synth.sample_queries(model, w["nq"], sd["queries"] + 7919 * rank, device=device, chunk=65536)
    return w, sd, X, Q


def exact_topk(X: torch.Tensor, Q: torch.Tensor, k: int, shortlist: int = 64, qblock: int = 512,
               chunk: int = 1 << 20, attr: torch.Tensor | None = None, ranges: torch.Tensor | None = None):
    """Ground-truth kNN for recall (evaluation only, not the search path): an
    FP32 matmul shortlist per row chunk, then the shortlist re-ranked by FP64
    direct-form distances with ties broken by id. With attr [N] and ranges
    [nq, 2] (device int64), only rows with lo <= attr <= hi count; missing
    neighbours are -1."""
    out = []
    for q0 in range(0, Q.shape[0], qblock):
        Qb = Q[q0:q0 + qblock]
        nq = Qb.shape[0]
        Rb = None if ranges is None else ranges[q0:q0 + qblock]
        best_d = torch.full((nq, shortlist), float("inf"), device=Q.device)
        best_i = torch.zeros((nq, shortlist), dtype=torch.int64, device=Q.device)
        qn = (Qb * Qb).sum(1, keepdim=True)
        for s in range(0, X.shape[0], chunk):
            Xc = X[s:s + chunk]
            dd = qn + (Xc * Xc).sum(1)[None] - 2.0 * (Qb @ Xc.T)
            if Rb is not None:
                a = attr[s:s + chunk][None]
                dd = torch.where((a >= Rb[:, :1]) & (a <= Rb[:, 1:]), dd, float("inf"))
            v, i = torch.topk(dd, min(shortlist, Xc.shape[0]), dim=1, largest=False)
            cat_d = torch.cat([best_d, v], 1)
            cat_i = torch.cat([best_i, i + s], 1)
            best_d, j = torch.topk(cat_d, shortlist, dim=1, largest=False)
            best_i = torch.gather(cat_i, 1, j)
        exact = ((X[best_i].double() - Qb.double()[:, None, :]) ** 2).sum(-1)
        exact = torch.where(torch.isinf(best_d), float("inf"), exact).cpu().numpy()
        ids = best_i.cpu().numpy()
        for qi in range(nq):
            order = np.lexsort((ids[qi], exact[qi]))[:k]
            row = ids[qi][order]
            row[np.isinf(exact[qi][order])] = -1
            out.append(row)
    return torch.from_numpy(np.stack(out))


def recall_at_k(found, truth) -> float:
    """Mean share of each query's true neighbours (ids >= 0) found among its first k results."""
    f = found.cpu().numpy() if torch.is_tensor(found) else np.asarray(found)
    t = truth.cpu().numpy() if torch.is_tensor(truth) else np.asarray(truth)
    k = t.shape[1]
    out = []
    for a, b in zip(f, t):
        want = set(b[b >= 0].tolist())
        if want:
            out.append(len(set(a[:k].tolist()) & want) / len(want))
    return float(np.mean(out)) if out else float("nan")


def stage_bytes(idx, rows_g, probe: np.ndarray, w: dict, batch: int):
    """Algorithmic bytes per launch of each stage for one batch, from the
    batch's probes (grains hit at least once are read once per batch). FP32
    form: 4-byte coordinates, bases and rows; precision form: 1-byte FP8
    coordinates, BF16 bases, centres and rows."""
    r, d, G = w["r"], w["d"], w["G"]
    p8 = w.get("precision", "fp32") == "bf16-fp8"
    cb, eb = (1, 2) if p8 else (4, 4)
    hit = np.zeros(G, dtype=bool)
    hit[np.unique(probe)] = True
    union_rows = int(rows_g[hit].sum())
    return {
        "scan": union_rows * (cb * r + 4),               # coordinates + FP32 residual norm per row
        "project": int(hit.sum()) * (r + 1) * d * eb,    # probed bases + centres
        "rerank": batch * w["C"] * d * eb,               # gathered raw rows
        "route": G * d * eb + batch * d * 4,
    }


def traffic_from_profiles(workload: str, stage: str, batch: int):
    """DRAM bytes per launch of the kernels of `stage` on `workload`, from the
    committed ncu summary (profiles/ncu_traffic.json), when it was taken on the
    current source of those kernels; else None. Entries captured on a smaller
    case either grow with the queries of a launch (captured_queries) or carry
    the factor that scales them to a full launch of the batch they name."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        rec = json.load(open(p))[workload][stage]
        for src, sha in rec["source_sha"].items():
            data = open(os.path.join(ROOT, "paper_2606_08813_b300", "csrc", src), "rb").read()
            if hashlib.sha256(data).hexdigest()[:16] != sha:
                return None
        if "captured_queries" in rec:  # traffic in proportion to the queries of a launch
            return int(rec["dram_bytes_per_launch"] * batch / rec["captured_queries"])
        if rec.get("captured_batch", batch) != batch:
            return None
        return int(rec["dram_bytes_per_launch"] * rec.get("scale_to_full_launch", 1.0))
    except Exception:
        return None


def _gap_sets_agree(g_ids, o_ids, o_ext, invalid, gap=1e-4):
    """Gap rule: wherever the oracle's ranking has a relative gap above `gap`
    after position m, the first m ids agree as sets."""
    n_valid = sum(1 for x in o_ids if x != invalid)
    if n_valid != sum(1 for x in g_ids if x != invalid):
        return False
    for m in range(1, n_valid + 1):
        a, b = o_ext[m - 1], o_ext[m]
        if np.isfinite(b) and (b - a) <= gap * max(abs(a), 1e-30):
            continue
        if set(g_ids[:m]) != set(o_ids[:m]):
            return False
    return True


def parity_vs_oracle(gpu, ora, k, C, nprobe, gap=1e-4):
    """Headline-batch rows against the oracle's search of the same queries:
    probe sets, pools and top k under the gap rule (near ties at the routing
    or pool boundary excluded and counted) and the largest relative distance
    error of ids both sides hold."""
    nq = ora["out_id"].shape[0]
    Ce = max(C, k)
    out = dict(queries=int(nq), route_excluded=0, topk_excluded=0, probe_sets_equal=0, pools_equal=0,
               topk_equal=0, max_rel_err_pool=0.0, max_rel_err_topk=0.0)
    for qi in range(nq):
        pd = ora["probe_d"][qi]
        if np.isfinite(pd[nprobe]) and (pd[nprobe] - pd[nprobe - 1]) <= gap * pd[nprobe - 1]:
            out["route_excluded"] += 1
            continue
        out["probe_sets_equal"] += int(set(gpu["probe"][qi].tolist()) == set(ora["probe"][qi].tolist()))
        for kind, gi_, gd_, oi_, od_, inv in (
                ("pool", gpu["pool_ids"][qi], gpu["pool_d"][qi], ora["cand_id"][qi], ora["cand_d"][qi], 0xFFFFFFFF),
                ("topk", gpu["ids"][qi], gpu["dist"][qi], ora["out_id"][qi], ora["out_d"][qi], -1)):
            if kind == "topk":
                cd = ora["cand_d"][qi]
                if np.isfinite(cd[Ce]) and (cd[Ce] - cd[Ce - 1]) <= gap * cd[Ce - 1]:
                    out["topk_excluded"] += 1
                    continue
            g_ids, o_ids = [int(x) for x in gi_], [int(x) for x in oi_]
            out["pools_equal" if kind == "pool" else "topk_equal"] += int(_gap_sets_agree(g_ids, o_ids, od_, inv))
            ref = {i: float(d) for i, d in zip(o_ids, od_) if i != inv}
            errs = [abs(float(d) - ref[i]) / max(ref[i], 1e-30) for i, d in zip(g_ids, gd_) if i in ref]
            key = "max_rel_err_pool" if kind == "pool" else "max_rel_err_topk"
            if errs:
                out[key] = max(out[key], max(errs))
    out["max_rel_err_pool"] = float(f"{out['max_rel_err_pool']:.3g}")
    out["max_rel_err_topk"] = float(f"{out['max_rel_err_topk']:.3g}")
    return out


def cpu_oracle_qps(idx_host, X_np, Q_np, k, C, nprobe, budget_s: float = 15.0, precision="fp32", first=None):
    """The oracle's QPS on a bounded sample of the workload's queries. With
    `first` (row indices), those queries are searched first (timed with the
    rest) and their results returned for the parity sample."""
    from oracle import hntl_oracle as O

    O.build_c()
    if precision == "bf16-fp8":  # exported coordinates are already the decoded FP8 values
        X_np = O.bf16_to_f32(O.bf16_round(X_np)).reshape(X_np.shape)
    oprec = "bf16-fp8-decoded" if precision == "bf16-fp8" else "fp32"
    n = 16
    t = 0.0
    done = 0
    first_out = None
    if first is not None:
        t0 = time.perf_counter()
        first_out = O.search(idx_host, X_np, Q_np[first], k, C, nprobe, precision=oprec)
        t += time.perf_counter() - t0
        done += len(first)
    while t < budget_s and done < Q_np.shape[0]:
        m = min(n, Q_np.shape[0] - done)
        t0 = time.perf_counter()
        O.search(idx_host, X_np, Q_np[done:done + m], k, C, nprobe, precision=oprec)
        t += time.perf_counter() - t0
        done += m
        n = min(4 * n, 4096)
    return done / t, done, O.threads(), first_out


def _err_stats(a):
    a = np.asarray(a, dtype=np.float64).ravel()
    a = a[np.isfinite(a)]
    if a.size == 0:
        return None
    return {"p50": float(f"{np.percentile(a, 50):.3g}"), "p99": float(f"{np.percentile(a, 99):.3g}"),
            "max": float(f"{a.max():.3g}"), "n": int(a.size)}


def precision_error(host, X_np, Q_np, gpu, zq, rq, route_d, k, C, nprobe, n_e2e, threads=16):
    """Error of each stage of the GPU's search against FP64 on the same index
    (the plain method on its FP32 rows, centres and bases): `gpu` holds one
    batch's probes, pool and top k for the queries Q_np, zq/rq its projections
    of those queries into their probes, route_d its routing distances.
    Relative errors are |gpu - fp64| / fp64 of each stage's own output and,
    for the projection and the coordinates, of the distance (Eq. 6) they
    feed. The first n_e2e queries are also searched end to end by the
    oracle's FP64 plain method on exact coordinates (computed for the grains
    its routing probes), for the id agreement of pool and top k."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import hntl_oracle as O

    nq = Q_np.shape[0]
    t0 = time.perf_counter()
    pool = gpu["pool_ids"].astype(np.int64)
    pool[gpu["pool_ids"] == 0xFFFFFFFF] = -1
    # the stored coordinates of each pool row (FP8 decoded and scaled) and its stored residual norm
    pos = np.zeros(len(host["ids"]), dtype=np.int64)
    pos[host["ids"].astype(np.int64)] = np.arange(len(host["ids"]))
    pp = pos[np.maximum(pool, 0)]
    sv = O.stage_values(host, X_np, Q_np, gpu["probe"], pool, pair_proj=(zq, rq),
                        row_terms=(host["Z"][pp], host["rho"][pp]))
    rel = lambda g, f: np.abs(np.asarray(g, np.float64) - f) / np.maximum(np.abs(f), 1e-30)
    ref_route = O.brute_force(host["M"], Q_np, nprobe)[0]
    g_sets = [set(x.tolist()) for x in gpu["probe"]]
    shared = np.array([len(g & set(o.tolist())) / nprobe for g, o in zip(g_sets, ref_route)])
    zerr = np.linalg.norm(zq - sv["z"], axis=2) / np.maximum(np.linalg.norm(sv["z"], axis=2), 1e-30)
    # the rerank: output distances, and the top k of the GPU's own pool by FP64 exact distance
    ex = np.where(pool >= 0, sv["exact"], np.inf)
    order = np.lexsort((np.where(pool >= 0, pool, np.iinfo(np.int64).max), ex), axis=1)[:, :k]
    exact_topk = np.take_along_axis(pool, order, axis=1)
    ids_pos = {}
    for qi in range(nq):
        for j, i in enumerate(pool[qi].tolist()):
            ids_pos[(qi, i)] = j
    out_ex = np.array([[sv["exact"][qi, ids_pos[(qi, int(i))]] if (qi, int(i)) in ids_pos else np.nan
                        for i in gpu["ids"][qi]] for qi in range(nq)])
    exs = np.sort(ex, axis=1)
    clear = (exs[:, k] - exs[:, k - 1]) > 1e-4 * exs[:, k - 1]
    same = np.array([set(a.tolist()) == set(b.tolist()) for a, b in zip(gpu["ids"], exact_topk)])
    res = {
        "queries": int(nq), "reference": "FP64 on the FP32 rows, centres and bases of the same index (oracle)",
        "route": {"probe_sets_equal": round(float(np.mean([g == set(o.tolist()) for g, o in zip(g_sets, ref_route)])), 4),
                  "probes_shared": round(float(shared.mean()), 4),
                  "dist_rel_err": _err_stats(rel(route_d, sv["route_d"]))},
        "project": {"z_rel_err": _err_stats(zerr), "rho_rel_err": _err_stats(rel(rq, sv["rho"])),
                    "D_rel_err": _err_stats(rel(sv["D_pair"], sv["D"]))},
        "coordinates": {"D_rel_err": _err_stats(rel(sv["D_row"], sv["D"]))},
        "scan": {"pool_D_rel_err": _err_stats(rel(np.where(pool >= 0, gpu["pool_d"], np.nan), sv["D"]))},
        "rerank": {"dist_rel_err": _err_stats(rel(gpu["dist"], out_ex)),
                   "topk_equal_fp64_rerank_of_pool": round(float(same[clear].mean()), 4) if clear.any() else None,
                   "queries_without_near_tie_at_k": int(clear.sum())},
    }
    # end to end: the oracle's FP64 plain search on exact coordinates of the grains its routing probes
    if n_e2e:
        Qe = Q_np[:n_e2e]
        grains = np.unique(ref_route[:n_e2e])
        off = host["grain_off"]
        Zx = np.zeros_like(host["Z"])
        rx = np.zeros_like(host["rho"])

        def one(g):
            a_, b_ = int(off[g]), int(off[g + 1])
            if b_ > a_:
                z, rh = O.tangent(X_np, host["ids"][a_:b_].astype(np.int64), host["M"][g], host["U"][g].astype(np.float64))
                Zx[a_:b_] = z
                rx[a_:b_] = rh

        with ThreadPoolExecutor(threads) as ex_:
            list(ex_.map(one, grains.tolist()))
        ora = O.search(host, X_np, Qe, k, C, nprobe, precision="fp32", Z=Zx, rho=rx)
        pool_shared = [len(set(int(x) for x in p if x >= 0) & set(int(x) for x in o if x != 0xFFFFFFFF)) /
                       max(1, sum(1 for x in o if x != 0xFFFFFFFF)) for p, o in zip(pool[:n_e2e], ora["cand_id"])]
        topk_shared = [len(set(a.tolist()) & set(b.tolist())) / k for a, b in zip(gpu["ids"][:n_e2e], ora["out_id"])]
        res["end_to_end"] = {"queries": int(n_e2e), "grains_with_exact_coordinates": int(len(grains)),
                             "pool_ids_shared": round(float(np.mean(pool_shared)), 4),
                             "topk_ids_shared": round(float(np.mean(topk_shared)), 4)}
    res["cpu_s"] = round(time.perf_counter() - t0, 1)
    return res


ATTR_SPAN = 1 << 40


def run_serving(a, hntl, gi, X, Q, attr, w, sd):
    """Continuous batching over the same index (the library's server): open-loop
    Poisson arrivals at each offered rate, k in {10, 100} and C in {20, 200,
    1000} drawn uniformly (C raised to k), half of the requests carrying a
    20%-selectivity range on the int64 attribute column. The library's own
    replay submits each request when its arrival time comes (with the others
    that have arrived by then), stamped with that time, so a slow submitter
    shows up as latency, not as a lower offered rate. Latency is from
    scheduled arrival to completion (the server's clock)."""
    rng = np.random.default_rng(sd["serve"])
    Qh = Q.cpu().numpy()
    nQ = len(Qh)
    dev = Q.device
    budget = min(int(a.serve_budget_gb * (1 << 30)), int(0.8 * torch.cuda.mem_get_info(dev)[0]))
    t0 = time.perf_counter()
    srv = hntl.Server(gi, mem_budget=budget, max_slots=a.serve_slots, batch=a.serve_batch, nprobe=w["nprobe"],
                      k_max=100, C_max=1000)
    create_s = time.perf_counter() - t0
    slots = srv.stats()["slots"]
    samples = []  # (query row, range, C, first 10 ids)

    # warm-up, untimed: bursts that make the server launch each of its graph
    # sizes once (a graph's first launch uploads it), then a clean record
    for burst in (a.serve_batch, a.serve_batch // 2, a.serve_batch // 4, a.serve_batch // 8, 128, 64, 8):
        nb_ = max(1, min(burst, nQ))
        kk = np.full(nb_, 100, np.uint32)
        tk = srv.submit(Qh[:nb_], kk, np.full(nb_, 1000, np.uint32))
        dn = np.zeros(len(tk), dtype=np.uint8)
        for _ in range(200):
            srv.poll_many(tk, dn, None, None, 50)
            if dn.all():
                break
    srv.reset_stats()
    rates_out = []
    ceiling_rates = [int(x) for x in a.serve_ceiling_rates.split(",") if x]
    n_rates = len([x for x in a.serve_rates.split(",") if x]) + len(ceiling_rates)
    for R in [int(x) for x in a.serve_rates.split(",") if x] + ceiling_rates:
        n = max(1, int(R * a.serve_seconds))
        qi = rng.integers(0, nQ, n)
        k = rng.choice(np.array([10, 100], np.uint32), n)
        C = np.maximum(rng.choice(np.array([20, 200, 1000], np.uint32), n), k)
        ranges = synth.range_filters(n, sd["serve"] + R, span=ATTR_SPAN, selectivity=0.2,
                                     frac_filtered=0.5).numpy()
        want = np.zeros(n, dtype=bool)
        want[rng.choice(n, min(n, a.serve_recall // max(1, n_rates)), replace=False)] = True
        srv.reset_stats()
        Qr = Qh[qi]
        off = 2_000_000 + np.cumsum(rng.exponential(1e9 / R, n)).astype(np.int64)
        t_call = time.monotonic_ns()
        n_done, ids_all = srv.replay(Qr, k, C, off, ranges=ranges, want=want, timeout_ms=120_000)
        end = time.monotonic_ns()
        start = t_call + 2_000_000
        del Qr
        rec = [(int(i_), ids_all[i_, :10].copy()) for i_ in np.flatnonzero(want)] if n_done == n else []
        st = srv.stats()
        achieved = n_done / ((end - start) / 1e9)
        for idx, ids in rec:
            samples.append((int(qi[idx]), ranges[idx], int(C[idx]), ids))
        rec_R = None
        if rec and X is not None:
            rows = torch.tensor([qi[idx_] for idx_, _ in rec], device=dev)
            rg = torch.from_numpy(np.stack([ranges[idx_] for idx_, _ in rec])).to(dev)
            truth_R = exact_topk(X, Q[rows].contiguous(), 10, attr=attr, ranges=rg).numpy()
            rec_R = round(recall_at_k(np.stack([ids_ for _, ids_ in rec]), truth_R), 4)
        rates_out.append({"offered_qps": R, "achieved_qps": round(achieved, 1), "completed": n_done,
                          "p50_ms": round(st["p50_us"] / 1e3, 3), "p99_ms": round(st["p99_us"] / 1e3, 3),
                          "max_ms": round(st["max_us"] / 1e3, 3), "mean_batch": round(st["mean_batch"], 1),
                          "recall_at_10": rec_R,
                          "parts_p50_p99_ms": {part: [round(st[f"{part}_p50_us"] / 1e3, 3),
                                                      round(st[f"{part}_p99_us"] / 1e3, 3)]
                                               for part in ("lag", "upload", "queue", "service")}})
        print(f"serving {R} q/s: {rates_out[-1]}", file=sys.stderr)
        if R in ceiling_rates and not (rates_out[-1]["achieved_qps"] >= 0.97 * R
                                       and rates_out[-1]["p99_ms"] <= a.serve_ceiling_p99_ms):
            break  # the ceiling search stops at the first rate it misses
    srv.close()
    # stage times of one search at each graph size the server captures (k_max, C_max, unfiltered)
    sizes = []
    rows_ = a.serve_batch
    while rows_ >= 32:
        sizes.insert(0, rows_)
        if rows_ // 2 < 32:
            break
        rows_ //= 2
    batch_profile = {}
    for rows_ in sizes:
        Qb = Q[:rows_].contiguous()
        for _ in range(3):
            gi.search(Qb, 100, 1000, w["nprobe"])
        torch.cuda.synchronize()
        hntl.profile_read()
        hntl.profile_enable(True)
        for _ in range(5):
            gi.search(Qb, 100, 1000, w["nprobe"])
        torch.cuda.synchronize()
        hntl.profile_enable(False)
        sm, calls = hntl.profile_read()
        batch_profile[rows_] = {k_: round(v_ / max(calls, 1), 3) for k_, v_ in sm.items()}
        batch_profile[rows_]["total"] = round(sum(sm.values()) / max(calls, 1), 3)
        sv = hntl.search_survivors(gi, gi.workspace(0), rows_, 1000, w["nprobe"]).cpu().numpy()
        batch_profile[rows_]["survivors_mean_max_overflow"] = [round(float(sv.mean()), 1), int(sv.max()),
                                                               int((sv > 32000).sum())]
    print(f"serving batch stage ms (k=100, C=1000): {batch_profile}", file=sys.stderr)
    recall = {}
    if samples and X is not None:
        rows = torch.tensor([s[0] for s in samples], device=dev)
        rg = torch.from_numpy(np.stack([s[1] for s in samples])).to(dev)
        truth = exact_topk(X, Q[rows].contiguous(), 10, attr=attr, ranges=rg).numpy()
        got = np.stack([s[3] for s in samples])
        Cs = np.array([s[2] for s in samples])
        filt = np.array([s[1][0] != np.iinfo(np.int64).min for s in samples])
        recall["all"] = round(recall_at_k(got, truth), 4)
        for c in (20, 200, 1000):
            m = Cs == c
            if m.any():
                recall[f"C={c}"] = round(recall_at_k(got[m], truth[m]), 4)
        recall["filtered"] = round(recall_at_k(got[filt], truth[filt]), 4)
        recall["unfiltered"] = round(recall_at_k(got[~filt], truth[~filt]), 4)
        recall["queries"] = len(samples)
    ok = [r for r in rates_out if r["achieved_qps"] >= 0.97 * r["offered_qps"] and r["p99_ms"] <= a.serve_p99_ms]
    ceil_ok = [r for r in rates_out if r["achieved_qps"] >= 0.97 * r["offered_qps"]
               and r["p99_ms"] <= a.serve_ceiling_p99_ms and (r["recall_at_10"] or 0) >= 0.95]
    return {"sustained_qps": max((r["offered_qps"] for r in ok), default=None),
            "sustained_rule": f"highest offered rate served at >= 97% with p99 <= {a.serve_p99_ms} ms",
            "ceiling_qps": max((r["offered_qps"] for r in ceil_ok), default=None),
            "ceiling_rule": f"highest offered rate served at >= 97% with p99 <= {a.serve_ceiling_p99_ms} ms and "
                            "recall@10 >= 0.95 on that rate's sampled requests (rates above the listed ones are "
                            "tried in order until one misses)",
            "rates": rates_out, "recall_at_10": recall, "batch": a.serve_batch, "slots": slots,
            "batch_stage_ms_k100_C1000": batch_profile,
            "mem_budget_gb": round(budget / (1 << 30), 1), "create_s": round(create_s, 2),
            "mix": "k in {10,100}, C in {20,200,1000} uniform (C >= k), 50% with a 20%-selectivity attribute range",
            "seconds_per_rate": a.serve_seconds}


class MultiStream:
    """Batches of one search call alternate over S streams, each with its own
    workspace and outputs, so one batch's small kernels and tails overlap the
    next batch's work (the server's two lanes do the same)."""

    def __init__(self, gi, B, k, C, nprobe, S, dev, mode="B"):
        self.gi, self.k, self.C, self.nprobe, self.mode = gi, k, C, nprobe, mode
        self.streams = [torch.cuda.Stream(device=dev) for _ in range(S)]
        nb = gi.workspace_bytes(B, k, C, nprobe)
        self.ws = [torch.empty(nb, dtype=torch.uint8, device=dev) for _ in range(S)]
        self.outs = [(torch.empty(B, k, dtype=torch.int64, device=dev), torch.empty(B, k, dtype=torch.float32,
                                                                                   device=dev)) for _ in range(S)]

    def run(self, batches, steps, events=None):
        """Launch `steps` searches; with events, record (start, end) per batch and
        bracket the whole on the current stream: returns the bracket's ms."""
        st = torch.cuda.current_stream()
        S = len(self.streams)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for s_ in self.streams:
            s_.wait_stream(st)
        for i in range(steps):
            j = i % S
            if events is not None:
                events[i][0].record(self.streams[j])
            self.gi.search(batches[i % len(batches)], self.k, self.C, self.nprobe, out=self.outs[j],
                           ws=self.ws[j], stream=self.streams[j], mode=self.mode)
            if events is not None:
                events[i][1].record(self.streams[j])
        for s_ in self.streams:
            st.wait_stream(s_)
        e1.record(st)
        return e0, e1


def run_fp32_compare(a, hntl, X, Q, w, sd, B, n_recall, truth, line):
    """The plain FP32 method (FP32 rows, coordinates, bases; TF32 routing with
    an exact refine; direct-form FP32 scan) on the same data, k-means draws,
    batch and parameters: its QPS and recall beside the precision form's."""
    t0 = time.perf_counter()
    gf = hntl.Index.build(X, w["G"], w["r"], u=synth.uniforms(w["G"], sd["kmeans"]).numpy(), seed=sd["kmeans"],
                          precision=hntl.PREC_FP32)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    k, C, nprobe = w["k"], w["C"], w["nprobe"]
    nb = w["nq"] // B
    batches = [Q[i * B:(i + 1) * B].contiguous() for i in range(nb)]
    found = [gf.search(batches[i], k, C, nprobe)[0] for i in range(max(1, (n_recall + B - 1) // B))]
    rec = recall_at_k(torch.cat(found)[:n_recall], truth) if n_recall else None
    ms_ = MultiStream(gf, B, k, C, nprobe, a.streams, Q.device)
    ms_.run(batches, a.warmup)
    torch.cuda.synchronize()
    steps = max(10, a.steps // 2)
    hntl.profile_read()
    hntl.profile_enable(True)  # stage times: one stream
    out = ms_.outs[0]
    for i in range(steps):
        gf.search(batches[i % nb], k, C, nprobe, out=out, ws=ms_.ws[0])
    torch.cuda.synchronize()
    hntl.profile_enable(False)
    sm, calls = hntl.profile_read()
    e0, e1 = ms_.run(batches, steps)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    qps = B / (ms / 1e3)
    del gf
    torch.cuda.empty_cache()
    return {"value": round(qps, 1), "unit": "queries/s", "ms_per_step": round(ms, 4),
            "recall_at_10": None if rec is None else round(rec, 4), "index_build_s": round(build_s, 2),
            "stages_ms": {k_: round(v_ / max(calls, 1), 4) for k_, v_ in sm.items()},
            "precision_form_gain": round(line["value"] / qps, 3),
            "streams": a.streams,
            "note": "same rows, k-means draws, batch, nprobe, C, k and streams; FP32 rows, coordinates and bases"}


def run_refined(a, hntl, X, Q, w, sd, B, n_recall, truth, line):
    """The precision form with the refined rerank (HNTL_RERANK_REFINE: second
    BF16 parts of the rows, the min(C, 2k) best of the BF16 rerank ranked
    again on both parts) on the same rows, k-means draws, batch and streams:
    its QPS, recall and stage times beside the headline's."""
    t0 = time.perf_counter()
    gr = hntl.Index.build(X, w["G"], w["r"], u=synth.uniforms(w["G"], sd["kmeans"]).numpy(), seed=sd["kmeans"],
                          precision=hntl.PREC_BF16_FP8 | hntl.RERANK_REFINE)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    k, C, nprobe = w["k"], w["C"], w["nprobe"]
    nb = w["nq"] // B
    batches = [Q[i * B:(i + 1) * B].contiguous() for i in range(nb)]
    found = [gr.search(batches[i], k, C, nprobe)[0] for i in range(max(1, (n_recall + B - 1) // B))]
    rec = recall_at_k(torch.cat(found)[:n_recall], truth) if n_recall else None
    ms_ = MultiStream(gr, B, k, C, nprobe, a.streams, Q.device)
    ms_.run(batches, a.warmup)
    torch.cuda.synchronize()
    steps = max(10, a.steps // 2)
    hntl.profile_read()
    hntl.profile_enable(True)
    for i in range(steps):
        gr.search(batches[i % nb], k, C, nprobe, out=ms_.outs[0], ws=ms_.ws[0])
    torch.cuda.synchronize()
    hntl.profile_enable(False)
    sm, calls = hntl.profile_read()
    e0, e1 = ms_.run(batches, steps)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    del gr
    torch.cuda.empty_cache()
    return {"value": round(B / (ms / 1e3), 1), "unit": "queries/s", "ms_per_step": round(ms, 4),
            "recall_at_10": None if rec is None else round(rec, 4), "index_build_s": round(build_s, 2),
            "stages_ms": {k_: round(v_ / max(calls, 1), 4) for k_, v_ in sm.items()},
            "note": "same rows, k-means draws, batch, nprobe, C, k and streams; the rerank's second stage "
                    f"re-scores min(C, 2k) = {min(C, 2 * k)} rows a query on both BF16 parts"}


def run_int16(a, hntl, X, Q, w, sd, B, n_recall, truth):
    """The paper's 16-bit form (Eq. 5, with the envelope filter) built from the
    same rows and k-means draws: QPS over the same batches and streams, recall."""
    t0 = time.perf_counter()
    g16 = hntl.Index.build(X, w["G"], w["r"], u=synth.uniforms(w["G"], sd["kmeans"]).numpy(), seed=sd["kmeans"],
                           precision=hntl.PREC_INT16)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    k, C, nprobe = w["k"], w["C"], w["nprobe"]
    nb = w["nq"] // B
    batches = [Q[i * B:(i + 1) * B].contiguous() for i in range(nb)]
    found = [g16.search(batches[i], k, C, nprobe)[0] for i in range(max(1, (n_recall + B - 1) // B))]
    rec = recall_at_k(torch.cat(found)[:n_recall], truth) if n_recall else None
    ms_ = MultiStream(g16, B, k, C, nprobe, a.streams, Q.device)
    ms_.run(batches, a.warmup)
    torch.cuda.synchronize()
    hntl.profile_read()
    hntl.profile_enable(True)  # stage times: one stream
    for i in range(a.steps):
        g16.search(batches[i % nb], k, C, nprobe, out=ms_.outs[0], ws=ms_.ws[0])
    torch.cuda.synchronize()
    hntl.profile_enable(False)
    sm, calls = hntl.profile_read()
    e0, e1 = ms_.run(batches, a.steps)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    del ms_, g16
    torch.cuda.empty_cache()
    return {"value": round(B / (ms / 1e3), 1), "unit": "queries/s", "ms_per_step": round(ms, 4),
            "recall_at_10": None if rec is None else round(rec, 4), "index_build_s": round(build_s, 2),
            "streams": a.streams, "stages_ms": {k_: round(v_ / max(calls, 1), 4) for k_, v_ in sm.items()},
            "note": "same rows, k-means draws, batches, nprobe, C, k and streams; int16 coordinates with per-grain "
                    "steps, uint16 residuals, quantised queries and the envelope filter; FP32 raw rows"}


def run_mode_a(a, hntl, gi, Q, w, B, n_recall, truth):
    """Mode A on the same index, batches, parameters and streams: the pool
    reranked by L2 to each row's reconstruction (no raw row read)."""
    k, C, nprobe = w["k"], w["C"], w["nprobe"]
    nb = w["nq"] // B
    batches = [Q[i * B:(i + 1) * B].contiguous() for i in range(nb)]
    found = [gi.search(batches[i], k, C, nprobe, mode="A")[0] for i in range(max(1, (n_recall + B - 1) // B))]
    rec = recall_at_k(torch.cat(found)[:n_recall], truth) if n_recall else None
    ms_ = MultiStream(gi, B, k, C, nprobe, a.streams, Q.device, mode="A")
    ms_.run(batches, a.warmup)
    torch.cuda.synchronize()
    hntl.profile_read()
    hntl.profile_enable(True)  # stage times: one stream
    for i in range(a.steps):
        gi.search(batches[i % nb], k, C, nprobe, out=ms_.outs[0], ws=ms_.ws[0], mode="A")
    torch.cuda.synchronize()
    hntl.profile_enable(False)
    sm, calls = hntl.profile_read()
    e0, e1 = ms_.run(batches, a.steps)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    return {"value": round(B / (ms / 1e3), 1), "unit": "queries/s", "ms_per_step": round(ms, 4),
            "recall_at_10": None if rec is None else round(rec, 4), "streams": a.streams,
            "stages_ms": {k_: round(v_ / max(calls, 1), 4) for k_, v_ in sm.items()},
            "note": "same index, batches, nprobe, C, k and streams; rerank by L2 to mu_g + W_g z_i"}


def run_ours(a, world, rank, local):
    from paper_2606_08813_b300 import build_lib

    build_lib.build()
    from paper_2606_08813_b300 import hntl

    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    w, sd, X, Q = make_workload(a.workload, dev, rank)
    B = a.batch or w.get("batch", w["nq"])
    k, C, nprobe = w["k"], w["C"], w["nprobe"]
    t0 = time.perf_counter()
    prec = w.get("precision", "fp32")
    serve = bool(a.serve_rates) and not a.profile_mode
    attr = synth.attributes(w["n"], sd["serve"], span=ATTR_SPAN, device=dev) if serve else None
    gi = hntl.Index.build(X, w["G"], w["r"], u=synth.uniforms(w["G"], sd["kmeans"]).numpy(), seed=sd["kmeans"],
                          precision=hntl.PREC_BF16_FP8 if prec == "bf16-fp8" else hntl.PREC_FP32, attr=attr)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    if a.profile_mode:
        del X
        torch.cuda.empty_cache()
        X = None
    rows_g = gi.grain_rows().astype(np.int64)
    print(f"index: build {build_s:.2f} s, grain rows max {rows_g.max()} median {int(np.median(rows_g))} "
          f"min {rows_g.min()}", file=sys.stderr)
    nb = w["nq"] // B
    batches = [Q[i * B:(i + 1) * B].contiguous() for i in range(nb)]
    out = (torch.empty(B, k, dtype=torch.int64, device=dev), torch.empty(B, k, dtype=torch.float32, device=dev))
    # probes of every batch (untimed) for algorithmic bytes; results of batch 0 for recall
    probes = []
    found = []
    surv = []
    for b in batches:
        ids, dist, probe = gi.search(b, k, C, nprobe, return_probe=True)
        probes.append(probe.cpu().numpy())
        found.append(ids)
        if len(surv) < 4:  # pool survivors per query (rows that passed the pilot bound)
            surv.append(hntl.search_survivors(gi, gi.workspace(0), B, C, nprobe).cpu().numpy())
    torch.cuda.synchronize()
    surv = np.concatenate(surv).astype(np.int64)
    cap = max(16384, 32 * C)
    surv_stats = {"mean": round(float(surv.mean()), 1), "p50": int(np.percentile(surv, 50)),
                  "p99": int(np.percentile(surv, 99)), "max": int(surv.max()),
                  "overflowed": int((surv > cap).sum()), "queries": int(len(surv))}
    n_recall = 0 if a.profile_mode else min(w["nq"], a.recall_queries)
    rec = float("nan")
    truth = None
    if n_recall:
        truth = exact_topk(X, Q[:n_recall], 10)
        rec = recall_at_k(torch.cat(found)[:n_recall], truth)
    sbytes = [stage_bytes(gi, rows_g, p, w, B) for p in probes]

    st = torch.cuda.current_stream()
    ms_ = MultiStream(gi, B, k, C, nprobe, a.streams, dev)
    ms_.run(batches, a.warmup)
    torch.cuda.synchronize()
    # stage times for the roofline: the same K batches on one stream, CUDA
    # events between stages on that stream (under two streams a kernel's
    # bracket would also hold the other stream's kernels)
    hntl.profile_read()  # discard warm-up records
    hntl.profile_enable(True)
    for i in range(a.steps):
        gi.search(batches[i % nb], k, C, nprobe, out=out, ws=ms_.ws[0])
    torch.cuda.synchronize()
    hntl.profile_enable(False)
    stage_ms, calls = hntl.profile_read()
    # the timed region: K batches over the streams
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = ms_.run(batches, a.steps, ev)
        torch.cuda.synchronize()
        barrier(world)
    step_ms = [x.elapsed_time(y) for x, y in ev]
    total_ms = e0.elapsed_time(e1)
    total_ms_max = max_over_ranks(total_ms, world)
    qps = aggregate_qps(world, a.steps, B, total_ms_max)
    clocks = clk.summary()

    # e2e: host queries (pinned) -> device -> search -> host results, per step;
    # one host thread per stream, each with its own workspace
    e2e_steps = 0 if a.profile_mode else a.steps
    hq = [b.cpu().pin_memory() for b in batches]
    hnb = int(hntl.lib.hntl_search_host_workspace_bytes(gi.handle, B, k, C, nprobe, 0))
    hws = [torch.empty(hnb, dtype=torch.uint8, device=dev) for _ in range(a.streams)]

    def e2e_worker(j, n):
        torch.cuda.set_device(local)
        for i in range(j, n, a.streams):
            gi.search_host(hq[i % nb], k, C, nprobe, stream=ms_.streams[j], ws=hws[j])

    def e2e_run(n):
        th = [threading.Thread(target=e2e_worker, args=(j, n)) for j in range(a.streams)]
        for t in th:
            t.start()
        for t in th:
            t.join()

    e2e_run(min(3, a.warmup) * a.streams)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    e2e_run(e2e_steps)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_qps = world * e2e_steps * B / e2e_s if e2e_steps else None

    # roofline of the dominant stage
    hbm, bf16, src = _peaks()
    per_launch_ms = {s: stage_ms[s] / max(calls, 1) for s in stage_ms}
    used = [sbytes[i % nb] for i in range(a.steps)]
    mean_bytes = {s: float(np.mean([u[s] for u in used])) for s in used[0]}
    dom = max(("scan", "rerank", "project", "select", "route", "pilot"), key=lambda s: per_launch_ms.get(s, 0.0))
    if dom in mean_bytes:
        ach = mean_bytes[dom] / (per_launch_ms[dom] / 1e3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(ach / hbm, 4), "traffic": traffic_from_profiles(a.workload, dom, B), "peak_source": src,
                "algorithmic_bytes_per_launch": int(mean_bytes[dom])}
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None,
                "traffic": None, "peak_source": src, "note": "no algorithmic byte model for this stage"}
    others = {s: {"ms_per_launch": round(per_launch_ms[s], 4),
                  "GBps": (round(mean_bytes[s] / (per_launch_ms[s] / 1e3) / 1e9, 1)
                           if s in mean_bytes and per_launch_ms[s] > 0 else None)} for s in per_launch_ms}

    line = {
        "metric": METRIC, "value": round(qps, 1), "unit": "queries/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(total_ms_max / a.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16/fp8" if prec == "bf16-fp8" else "f32",
        "data": "synthetic",
        "config": {"workload": a.workload, "precision": prec, "N": w["n"], "d": w["d"], "G": w["G"], "r": w["r"], "batch": B,
                   "nprobe": nprobe, "C": C, "k": k, "recall_at_10": None if rec != rec else round(rec, 4), "recall_queries": n_recall,
                   "recall_note": "skipped in profile mode" if a.profile_mode else "brute force, FP64 re-rank",
                   "sizes": w["sizes"], "l2": "no flush; per-step working set (probed coordinates, bases and "
                   "gathered rows: about 8 GB a 16384-query batch at 10M rows) exceeds the 126 MB L2", "index_build_s": round(build_s, 2),
                   "parallelism": f"replicas x{world}", "streams": a.streams,
                   "stage_timing": "CUDA events between stages, the same K batches on one stream",
                   "pool_survivors": surv_stats, "batch_latency_ms_p50": round(float(np.percentile(step_ms, 50)), 4),
                   "batch_latency_ms_p99": round(float(np.percentile(step_ms, 99)), 4)},
        "roofline": roof, "stages": others,
        "e2e": {"value": round(e2e_qps, 1) if e2e_qps else None, "unit": "queries/s",
                "h2d_bytes_per_step": B * w["d"] * 4,
                "d2h_bytes_per_step": B * k * 12},
        # our kernels per search: precision form = row norms, BF16 queries, route (TC + refine), bucket (3),
        # projection, pilot, live pairs, classify, scan (sparse + TC), pool select (2), rerank;
        # FP32 form = row norms, route (2), bucket (3), projection, pilot, scan, pool select (2), rerank
        "gpu_launches": (16 if prec == "bf16-fp8" else 12) * a.steps, "clocks": clocks,
    }
    if serve:
        line["serving"] = run_serving(a, hntl, gi, X, Q, attr, w, sd)
    if a.mode_a and not a.profile_mode:
        line["mode_a_same_data"] = run_mode_a(a, hntl, gi, Q, w, B, n_recall, truth)
        print(f"mode A: {line['mode_a_same_data']}", file=sys.stderr)
    if a.int16 and X is not None and not a.profile_mode:
        line["int16_form_same_data"] = run_int16(a, hntl, X, Q, w, sd, B, n_recall, truth)
        print(f"16-bit form: {line['int16_form_same_data']}", file=sys.stderr)
    if prec == "bf16-fp8" and a.fp32_compare and X is not None:
        line["plain_fp32_same_data"] = run_fp32_compare(a, hntl, X, Q, w, sd, B, n_recall, truth, line)
    if prec == "bf16-fp8" and a.refined and X is not None and not a.profile_mode:
        line["precision_refined_same_data"] = run_refined(a, hntl, X, Q, w, sd, B, n_recall, truth, line)
        print(f"refined rerank: {line['precision_refined_same_data']}", file=sys.stderr)
    if a.router and world == 1 and not a.profile_mode:
        line["learned_router"] = router_leg(a, hntl, dev)
    if rank == 0 and world == 1 and not a.no_cpu_baseline and not a.profile_mode:
        # the headline batch 0 searched once more (untimed) with its pool and
        # probes; 64 of its rows, spread over the batch, are the parity sample
        # the oracle searches first inside its timed baseline
        ids0, d0, pid0, pd0, pr0 = gi.search(batches[0], k, C, nprobe, return_pool=True, return_probe=True)
        zq0, rq0 = hntl.search_pair_proj(gi, gi.workspace(0), B, C, nprobe)
        ne = min(a.err_queries, B) if prec == "bf16-fp8" else 0
        rp0, rd0 = gi.route(batches[0][:max(ne, 1)], nprobe)
        torch.cuda.synchronize()
        rows = np.arange(0, B, max(1, B // 64))[:64]
        gpu0 = dict(ids=ids0.cpu().numpy()[rows], dist=d0.cpu().numpy()[rows],
                    pool_ids=pid0.cpu().numpy().view(np.uint32)[rows], pool_d=pd0.cpu().numpy()[rows],
                    probe=pr0.cpu().numpy()[rows])
        host = gi.export()
        Xn = X.cpu().numpy()
        Qn = Q[:max(4096, B)].cpu().numpy()
        q, nq_done, cores, ora0 = cpu_oracle_qps(host, Xn, Qn, k, C, nprobe, budget_s=a.cpu_budget,
                                                  precision=prec, first=rows)
        line["cpu_baseline"] = {"value": round(q, 2), "unit": "queries/s", "cores": cores, "kind": "oracle",
                                "sample": f"{nq_done} queries of the same workload against the same index "
                                          f"(FP64 oracle search, OpenMP over queries)"}
        if a.cpu_budget_1core > 0:  # the same oracle on one host core
            from oracle import hntl_oracle as O

            O.set_threads(1)
            try:
                q1, n1, _, _ = cpu_oracle_qps(host, Xn, Qn, k, C, nprobe, budget_s=a.cpu_budget_1core,
                                              precision=prec)
            finally:
                O.set_threads(cores)
            line["cpu_baseline"]["one_core"] = {"value": round(q1, 2), "unit": "queries/s", "cores": 1,
                                                "sample": f"{n1} queries, the same search on one thread"}
        line["parity_sample"] = dict(parity_vs_oracle(gpu0, ora0, k, C, nprobe),
                                     rows="64 rows of headline batch 0 (every B/64-th), as searched in the "
                                          "timed launch configuration, against the oracle on the exported index",
                                     rule="ids equal as sets wherever the oracle's ranking has a gap > 1e-4 "
                                          "relative; near ties at the routing or pool boundary excluded")
        if ne:
            # per-stage error of the precision form against FP64, the first `ne` queries of batch 0
            pr_np = pr0.cpu().numpy()[:ne]
            rp, rd = rp0.cpu().numpy(), rd0.cpu().numpy()
            route_d = np.full((ne, nprobe), np.nan)
            for qi in range(ne):
                at = {int(g): float(x) for g, x in zip(rp[qi], rd[qi])}
                route_d[qi] = [at.get(int(g), np.nan) for g in pr_np[qi]]
            gpu_e = dict(ids=ids0.cpu().numpy()[:ne], dist=d0.cpu().numpy()[:ne],
                         pool_ids=pid0.cpu().numpy().view(np.uint32)[:ne], pool_d=pd0.cpu().numpy()[:ne],
                         probe=pr_np)
            line["precision_error"] = precision_error(host, Xn, batches[0][:ne].cpu().numpy(), gpu_e,
                                                      zq0.cpu().numpy()[:ne], rq0.cpu().numpy()[:ne], route_d,
                                                      k, C, nprobe, min(a.err_e2e, ne))
            print(f"precision error: {line['precision_error']}", file=sys.stderr)
    if rank == 0:
        print(json.dumps(line), flush=True)


def knn_ids_bf16(X: torch.Tensor, Q: torch.Tensor, k: int, qblock: int = 2048, chunk: int = 1 << 20):
    """Approximate top-k neighbour ids by a BF16 matmul (training labels only)."""
    Xb = X.to(torch.bfloat16)
    xn = (X * X).sum(1)
    out = []
    for q0 in range(0, Q.shape[0], qblock):
        Qb = Q[q0:q0 + qblock]
        best_d = torch.full((Qb.shape[0], k), float("inf"), device=Q.device)
        best_i = torch.zeros((Qb.shape[0], k), dtype=torch.int64, device=Q.device)
        for s in range(0, X.shape[0], chunk):
            dd = xn[s:s + chunk][None] - 2.0 * (Qb.to(torch.bfloat16) @ Xb[s:s + chunk].T).float()
            v, i = torch.topk(dd, k, dim=1, largest=False)
            cd, ci = torch.cat([best_d, v], 1), torch.cat([best_i, i + s], 1)
            best_d, j = torch.topk(cd, k, dim=1, largest=False)
            best_i = torch.gather(ci, 1, j)
        out.append(best_i)
    return torch.cat(out)


def router_leg(a, hntl, dev):
    """Learned grain router at its full configuration (router-5m: 5M rows,
    G = 4096 capacity-bounded grains over 1024 equal clusters): train the MLP with
    the library's BF16 kernels on labels the method generates (the grains
    holding each training query's top-10), compare recall@10 with centroid
    routing at equal nprobe (equal grain sizes: equal probed rows), and state
    the QPS at Recall@10 >= 0.95 of the plain FP32 method with centroid routing
    against the learned-router, BF16/FP8, batched form on the same partition
    (both indices built from the same rows and k-means draws)."""
    w = dict(synth.WORKLOADS["router-5m"])
    sd = synth.seeds(w["seed"])
    model = synth.make_cluster_model(w["n"], w["d"], w["n_clusters"], sizes=w["sizes"], seed=sd["data"])
    X, _ = synth.sample_points(model, sd["data"] + 11, device=dev, chunk=65536)
    Qtr, _ = synth.sample_queries(model, a.router_train, sd["router"], device=dev, chunk=65536)
    Qev, _ = synth.sample_queries(model, w["nq"], sd["queries"], device=dev, chunk=65536)
    G, d = w["G"], w["d"]
    u = synth.uniforms(G, sd["kmeans"]).numpy()
    t0 = time.perf_counter()
    gi = hntl.Index.build(X, G, w["r"], u=u, seed=sd["kmeans"], max_grain_rows=w["max_grain_rows"])
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    # the low-precision form with the refined rerank (second BF16 parts of the rows): BF16 rows alone
    # cap recall@10 near 0.94 on this data
    gp = hntl.Index.build(X, G, w["r"], u=u, seed=sd["kmeans"], max_grain_rows=w["max_grain_rows"],
                          precision=hntl.PREC_BF16_FP8 | hntl.RERANK_REFINE)
    exp = gi.export()
    assign_np = np.empty(w["n"], dtype=np.int64)
    assign_np[exp["ids"].astype(np.int64)] = np.repeat(np.arange(G), np.diff(exp["grain_off"]))
    rows_g = np.diff(exp["grain_off"])
    same_partition = bool(np.array_equal(exp["grain_off"], gp.export()["grain_off"]))
    assign = torch.from_numpy(assign_np).to(dev)
    del exp
    t0 = time.perf_counter()
    nb_tr = knn_ids_bf16(X, Qtr, 10)
    torch.cuda.synchronize()
    label_s = time.perf_counter() - t0
    lab = assign[nb_tr]  # [n_train, 10] grain of each neighbour
    # MLP d -> 1024 -> 1024 -> G, uniform(+-1/sqrt(fan_in)) weights, zero biases
    rng = np.random.default_rng(sd["router"])
    params = []
    for fo, fi in ((a.router_hidden, d), (a.router_hidden, a.router_hidden), (G, a.router_hidden)):
        lim = 1.0 / np.sqrt(fi)
        params += [rng.uniform(-lim, lim, (fo, fi)).astype(np.float32), np.zeros(fo, np.float32)]
    B = a.router_batch
    rt = hntl.Router(params, max_batch=max(B, 4096))
    flop_per_sample = 6 * (d * a.router_hidden + a.router_hidden * a.router_hidden + a.router_hidden * G)
    gen = torch.Generator(device=dev).manual_seed(sd["router"])
    T = torch.empty(B, G, device=dev)
    ones = torch.full((B, 10), 0.1, device=dev)
    losses = []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    steps = 0
    ev[0].record()
    for ep in range(a.router_epochs):
        perm = torch.randperm(Qtr.shape[0], generator=gen, device=dev)
        lo = torch.zeros(1, device=dev)
        for s0 in range(0, Qtr.shape[0] - B + 1, B):
            idx = perm[s0:s0 + B]
            T.zero_()
            T.scatter_add_(1, lab[idx], ones)
            rt.step(Qtr[idx].contiguous(), T, lr=a.router_lr, wd=0.01, loss=lo)
            steps += 1
        losses.append(float(lo.item()) * B / (Qtr.shape[0] // B * B))
    ev[1].record()
    torch.cuda.synchronize()
    train_ms = ev[0].elapsed_time(ev[1])
    del Qtr, nb_tr, lab
    # evaluation: exact ground truth on batches of 4096, centroid vs learned routing
    QB = 4096
    nev = (Qev.shape[0] // QB) * QB
    batches = [Qev[i:i + QB].contiguous() for i in range(0, nev, QB)]
    truth = exact_topk(X, Qev[:nev], 10)
    reps = 3

    def timed(fn):
        """recall@10 over the evaluation batches and QPS of `reps` passes over them (one stream)."""
        found = [fn(b)[0] for b in batches]
        torch.cuda.synchronize()
        rec = recall_at_k(torch.cat(found), truth)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            for b in batches:
                fn(b)
        e1.record()
        torch.cuda.synchronize()
        return rec, reps * nev / (e0.elapsed_time(e1) / 1e3)

    out = []
    C2 = 2 * w["C"]  # the 8-bit coordinates' pool error is won back by a larger pool
    for nprobe in (2, 4, 8, 16, 32, 64):
        rc, qc = timed(lambda b: gi.search(b, 10, w["C"], nprobe))
        rcp, qcp = timed(lambda b: gp.search(b, 10, w["C"], nprobe))
        rl, ql = timed(lambda b: hntl.search_probes(gi, b, rt.route(gi, b, nprobe, tau=0.0)[0], 10, w["C"]))
        rp, qp = timed(lambda b: hntl.search_probes(gp, b, rt.route(gp, b, nprobe, tau=0.0)[0], 10, w["C"]))
        rp2, qp2 = timed(lambda b: hntl.search_probes(gp, b, rt.route(gp, b, nprobe, tau=0.0)[0], 10, C2))
        out.append({"nprobe": nprobe, "recall_centroid_fp32": round(rc, 4), "recall_learned_fp32": round(rl, 4),
                    "recall_centroid_bf16_fp8": round(rcp, 4), "qps_centroid_bf16_fp8": round(qcp, 1),
                    "recall_learned_bf16_fp8": round(rp, 4), f"recall_learned_bf16_fp8_C{C2}": round(rp2, 4),
                    "qps_centroid_fp32": round(qc, 1), "qps_learned_fp32": round(ql, 1),
                    "qps_learned_bf16_fp8": round(qp, 1), f"qps_learned_bf16_fp8_C{C2}": round(qp2, 1),
                    "gain": round(rl - rc, 4)})
        print(f"router nprobe {nprobe}: {out[-1]}", file=sys.stderr)

    # training throughput at a batch whose GEMM tiles fill every SM (after the
    # evaluation, on evaluation queries with random soft targets: a timing of
    # the same step, not a training run)
    B4 = 4096
    T4 = torch.zeros(B4, G, device=dev)
    T4.scatter_add_(1, torch.randint(0, G, (B4, 10), device=dev, generator=gen), torch.full((B4, 10), 0.1, device=dev))
    X4 = Qev[:B4].contiguous()
    for _ in range(3):
        rt.step(X4, T4, lr=a.router_lr, wd=0.01)
    torch.cuda.synchronize()
    e4 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e4[0].record()
    for _ in range(20):
        rt.step(X4, T4, lr=a.router_lr, wd=0.01)
    e4[1].record()
    torch.cuda.synchronize()
    ms4 = e4[0].elapsed_time(e4[1]) / 20

    def at_target(rk, qk):
        ok = [(o[qk], o["nprobe"]) for o in out if o[rk] >= 0.95]
        return (max(ok)[1], max(ok)[0]) if ok else (None, None)

    npc, qpc = at_target("recall_centroid_fp32", "qps_centroid_fp32")
    cands = [(at_target("recall_learned_bf16_fp8", "qps_learned_bf16_fp8"), w["C"]),
             (at_target(f"recall_learned_bf16_fp8_C{C2}", f"qps_learned_bf16_fp8_C{C2}"), C2)]
    cands = [(q, n_, c) for (n_, q), c in cands if q]
    qpl, npl, cl = max(cands) if cands else (None, None, None)
    npf, qpf = at_target("recall_learned_fp32", "qps_learned_fp32")
    samples = steps * B
    _, bf16, src = _peaks()
    tflops = samples * flop_per_sample / (train_ms / 1e3) / 1e12
    res = {"workload": "router-5m", "N": w["n"], "d": d, "G": G, "r": w["r"], "C": w["C"], "k": 10,
           "clusters": f"{w['n_clusters']} {w['sizes']}", "max_grain_rows": w["max_grain_rows"],
           "grain_rows_min_max": [int(rows_g.min()), int(rows_g.max())], "same_partition_both_forms": same_partition,
           "mlp": f"{d}-{a.router_hidden}-{a.router_hidden}-{G}", "train_queries": int(samples / max(a.router_epochs, 1)),
           "eval_queries": nev, "epochs": a.router_epochs, "batch": B, "lr": a.router_lr,
           "index_build_s": round(build_s, 2), "label_s": round(label_s, 2),
           "by_nprobe": out, "loss_by_epoch": [round(x, 4) for x in losses],
           "qps_at_recall_0.95": {"plain_fp32_centroid": {"nprobe": npc, "C": w["C"], "qps": qpc},
                                  "learned_fp32": {"nprobe": npf, "C": w["C"], "qps": qpf},
                                  "learned_bf16_fp8_batched": {"nprobe": npl, "C": cl, "qps": qpl},
                                  "gain": round(qpl / qpc, 3) if (qpl and qpc) else None,
                                  "centroid_bf16_fp8": dict(zip(("nprobe", "qps"), at_target(
                                      "recall_centroid_bf16_fp8", "qps_centroid_bf16_fp8"))),
                                  "note": "each method's fastest setting of the sweep with recall@10 >= 0.95; "
                                          "batches of 4096 on one stream; the learned forms' time includes "
                                          "the router's forward pass and top-nprobe selection; the BF16/FP8 "
                                          "index reranks in two stages (HNTL_RERANK_REFINE)"},
           "train": {"samples_per_s": round(samples / (train_ms / 1e3), 1), "ms_per_step": round(train_ms / steps, 4),
                     "achieved_tflops": round(tflops, 1), "peak_tflops": bf16, "frac": round(tflops / bf16, 4),
                     "peak_source": src,
                     "note": "forward + backward + AdamW, 6 flops per weight per sample (GEMMs only)",
                     "at_batch_4096": {"ms_per_step": round(ms4, 4), "samples_per_s": round(B4 / (ms4 / 1e3), 1),
                                       "achieved_tflops": round(B4 * flop_per_sample / (ms4 / 1e3) / 1e12, 1),
                                       "frac": round(B4 * flop_per_sample / (ms4 / 1e3) / 1e12 / bf16, 4),
                                       "note": "the same step timed at 4096 samples after the evaluation"}}}
    del gi, gp, rt, X, Qev, batches, truth
    torch.cuda.empty_cache()
    return res


def run_router(a, world, rank, local):
    """--workload router-5m: the router leg alone, as its own JSON line."""
    from paper_2606_08813_b300 import build_lib

    build_lib.build()
    from paper_2606_08813_b300 import hntl

    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    res = router_leg(a, hntl, dev)
    best = max(o["gain"] for o in res["by_nprobe"])
    line = {"metric": "learned-router recall@10 gain over centroid routing at equal nprobe", "value": best,
            "unit": "recall points", "n_gpus": 1, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
            "config": {k: v for k, v in res.items() if k not in ("by_nprobe", "loss_by_epoch", "train")},
            "by_nprobe": res["by_nprobe"], "loss_by_epoch": res["loss_by_epoch"], "train": res["train"]}
    print(json.dumps(line), flush=True)


def run_reference(a, world, rank, local):
    if rank != 0:
        return
    from paper_2606_08813_b300 import build_lib

    build_lib.build()
    from oracle import hntl_oracle as O
    from paper_2606_08813_b300 import hntl

    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    w, sd, X, Q = make_workload(a.workload, dev, 0)
    k, C, nprobe = w["k"], w["C"], w["nprobe"]
    prec = w.get("precision", "fp32")
    gi = hntl.Index.build(X, w["G"], w["r"], u=synth.uniforms(w["G"], sd["kmeans"]).numpy(), seed=sd["kmeans"],
                          precision=hntl.PREC_BF16_FP8 if prec == "bf16-fp8" else hntl.PREC_FP32)
    host = gi.export()
    Xn = X.cpu().numpy()
    if prec == "bf16-fp8":
        Xn = O.bf16_to_f32(O.bf16_round(Xn)).reshape(Xn.shape)
    Qn = Q.cpu().numpy()
    del gi
    oprec = "bf16-fp8-decoded" if prec == "bf16-fp8" else "fp32"
    O.build_c()
    per_step = a.ref_queries
    for i in range(a.warmup):
        O.search(host, Xn, Qn[(i * per_step) % len(Qn):][:per_step], k, C, nprobe, precision=oprec)
    t0 = time.perf_counter()
    for i in range(a.steps):
        s = (i * per_step) % max(1, len(Qn) - per_step)
        O.search(host, Xn, Qn[s:s + per_step], k, C, nprobe, precision=oprec)
    el = time.perf_counter() - t0
    qps = a.steps * per_step / el
    line = {"metric": METRIC, "value": round(qps, 2), "unit": "queries/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": round(el / a.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": a.workload, "N": w["n"], "d": w["d"], "G": w["G"], "r": w["r"],
                       "batch": per_step, "nprobe": nprobe, "C": C, "k": k},
            "cpu_baseline": {"value": round(qps, 2), "unit": "queries/s", "cores": O.threads(), "kind": "oracle",
                             "sample": f"{per_step} queries per step against the GPU-built index of the same "
                                       f"workload"},
            "e2e": {"value": round(qps, 2), "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="precision-10m", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--streams", type=int, default=3, help="CUDA streams the timed batches alternate over")
    ap.add_argument("--recall-queries", type=int, default=2048)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-queries", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--err-queries", type=int, default=512,
                    help="precision form: queries of batch 0 whose per-stage error against FP64 is reported")
    ap.add_argument("--err-e2e", type=int, default=64,
                    help="of those, queries also searched end to end by the oracle's FP64 plain method")
    ap.add_argument("--serve-rates", default="25000,100000,200000",
                    help="offered Poisson rates (q/s) of the serving run; empty to skip it")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--cpu-budget-1core", type=float, default=4.0,
                    help="seconds of the oracle on one host core beside the all-core cpu_baseline (0: skip)")
    ap.add_argument("--serve-batch", type=int, default=2048)
    ap.add_argument("--serve-slots", type=int, default=1 << 18)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-recall", type=int, default=1536, help="served requests checked against brute force")
    ap.add_argument("--serve-p99-ms", type=float, default=50.0)
    ap.add_argument("--serve-ceiling-rates", default="300000,350000,400000,600000,800000,1200000",
                    help="rates tried after --serve-rates, in order, until one misses the ceiling rule")
    ap.add_argument("--serve-ceiling-p99-ms", type=float, default=5.0)
    ap.add_argument("--no-int16", dest="int16", action="store_false",
                    help="skip timing the paper's 16-bit form built from the same rows")
    ap.add_argument("--no-mode-a", dest="mode_a", action="store_false",
                    help="skip timing Mode A (rerank on reconstructions) on the same index")
    ap.add_argument("--no-fp32-compare", dest="fp32_compare", action="store_false",
                    help="skip timing the plain FP32 method on the same data (precision workloads)")
    ap.add_argument("--no-refined", dest="refined", action="store_false",
                    help="skip the refined-rerank precision form on the same data")
    ap.add_argument("--no-router", dest="router", action="store_false",
                    help="skip the learned-router leg (router-5m) of the default run")
    ap.add_argument("--router-train", type=int, default=400_000)
    ap.add_argument("--router-epochs", type=int, default=24)
    ap.add_argument("--router-batch", type=int, default=1024)
    ap.add_argument("--router-hidden", type=int, default=1024)
    ap.add_argument("--router-lr", type=float, default=1e-3)
    ap.add_argument("--profile-mode", action="store_true",
                    help="for ncu captures: free the raw rows after the build; no recall, CPU baseline or e2e")
    a = ap.parse_args()
    if a.warmup < 3:
        a.warmup = 3
    world, rank, local = dist_setup()
    try:
        if a.impl == "reference":
            run_reference(a, world, rank, local)
        elif a.workload == "router-5m":
            if rank == 0:
                run_router(a, world, rank, local)
        else:
            run_ours(a, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
