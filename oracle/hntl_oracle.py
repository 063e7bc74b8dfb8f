"""Plain, slow CPU oracle of the HNTL batched query path (FP64).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users. The product library neither imports nor
links anything here, and this module imports nothing from the product package.

What it computes, in the paper's order (HNTL technical report):
  * grain partitioning (unspecified in the paper; k-means++ seeding with the
    uniform draws passed in, then Lloyd iterations, sec. 2.2 "spatial grains");
  * per-grain local PCA basis W_g (sec. 2.2), here U_g = W_g^T, r x d, from an
    FP64 covariance centred on the stored FP32 centre and numpy's symmetric
    eigensolver (a library primitive), eigenvalues descending;
  * database tangent coordinates and residual norms, Eq. 1-4;
  * the Mode B query path: routing (sec. 2.1 step 1, sec. 2.3), projection
    (Eq. 1-4), scan with the approximate distance of Eq. 6, the pool of the C
    best (Table 1, "Pool C"), exact L2 rerank to top k (sec. 2.1 step 4);
  * Mode A: the same pool reranked by L2 to each row's reconstruction
    mu_g + W_g z_i (sec. 2.1 step 4, sec. 1, the reconstruction of Eq. 3);
  * the brute-force exact kNN used as ground truth.
The loops live in hntl_oracle.c; the covariance, the tangent coordinates of
the database rows and the eigendecomposition are written as numpy matmuls and
`numpy.linalg.eigh`.

Readings where the paper is silent are listed in the design notes: ties are
broken by (distance, id) and routing by (distance, grain); the pool is global
per query across probes; a grain with fewer rows than the basis size keeps an
orthonormal completion (any eigenvectors of its covariance); each basis row is
signed so that its largest-magnitude component is positive.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hntl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# ---------------------------------------------------------------------------
# C core
# ---------------------------------------------------------------------------


def build_c(force: bool = False) -> str:
    """Compile the C core with gcc (-O2, OpenMP, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _c():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_c())
            P = ctypes.c_void_p
            I = ctypes.c_int64
            lib.or_bruteforce.argtypes = [P, I, I, P, I, I, P, P, P, P, P]
            lib.or_kmeanspp.argtypes = [P, I, I, I, P, P]
            lib.or_assign.argtypes = [P, I, I, P, I, P, P]
            lib.or_means.argtypes = [P, I, I, P, I, P, P]
            lib.or_means.restype = I
            lib.or_lloyd.argtypes = [P, I, I, I, P, I, P]
            lib.or_lloyd.restype = I
            lib.or_balanced_assign.argtypes = [P, I, I, P, I, I, P]
            lib.or_search.argtypes = [P, P, I, I, I, P, P, P, P, P, P, P, P, I, I, I, I, P,
                                      P, P, P, P, P, P, I, P, P, P, P, P, P, I, P, P, P, P, P, I]
            lib.or_threads.restype = ctypes.c_int
            lib.or_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(np.asarray(a), dtype=np.float32)


def threads() -> int:
    return int(_c().or_threads())


def set_threads(n: int) -> None:
    _c().or_set_threads(int(n))


# ---------------------------------------------------------------------------
# index build
# ---------------------------------------------------------------------------


def balanced_assign(X, M, cap: int):
    """Capacity-bounded grains (see or_balanced_assign in hntl_oracle.c): the
    row-proposing stable assignment of the rows of X to the centres M with at
    most `cap` rows per grain. Returns assign i32 [N]."""
    X = _f32(X)
    M = np.ascontiguousarray(M, dtype=np.float64)
    n, d = X.shape
    G = M.shape[0]
    if cap * G < n:
        raise ValueError("cap * G must be at least N")
    out = np.full(n, -1, dtype=np.int32)
    _c().or_balanced_assign(_p(X), n, d, _p(M), G, int(cap), _p(out))
    return out


def kmeans(X, G: int, u, train_idx=None, max_iter: int = 25, max_grain_rows: int = 0):
    """Grain partition of X: k-means++ seeding (draws `u`, one per centre) on
    the training rows, Lloyd iterations there, one assignment pass of all rows
    to the trained centres (with max_grain_rows > 0, the capacity-bounded
    assignment of balanced_assign instead), then each centre is the exact FP64
    mean of its final members rounded once to FP32 (an empty final grain keeps
    its trained centre). Returns (mu f32 [G, d], assign i32 [N],
    lloyd_iterations)."""
    X = _f32(X)
    n, d = X.shape
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert u.shape[0] >= G
    Xt = X if train_idx is None else np.ascontiguousarray(X[np.asarray(train_idx)])
    nt = Xt.shape[0]
    if nt < G:
        raise ValueError("fewer training rows than grains")
    lib = _c()
    chosen = np.zeros(G, dtype=np.int64)
    lib.or_kmeanspp(_p(Xt), nt, d, G, _p(u), _p(chosen))
    M = Xt[chosen].astype(np.float64)
    at = np.zeros(nt, dtype=np.int32)
    iters = lib.or_lloyd(_p(Xt), nt, d, G, _p(M), max_iter, _p(at))
    assign = np.zeros(n, dtype=np.int32)
    if max_grain_rows:
        assign = balanced_assign(X, M, max_grain_rows)
    else:
        lib.or_assign(_p(X), n, d, _p(M), G, _p(assign), None)
    count = np.zeros(G, dtype=np.int64)
    Mf = M.copy()
    lib.or_means(_p(X), n, d, _p(assign), G, _p(Mf), _p(count))
    return Mf.astype(np.float32), assign, int(iters)


def grain_pca(X, rows, mu32, r: int):
    """Local PCA of one grain (sec. 2.2): FP64 covariance (1/n_g) V^T V with
    V = X[rows] - mu (stored FP32 centre), eigenvalues descending, basis
    U = top-r eigenvectors as rows, each signed so that its largest-magnitude
    component is positive. Returns (U f64 [r, d], eigenvalues f64 [d])."""
    d = mu32.shape[0]
    if len(rows) > 0:
        V = X[rows].astype(np.float64) - mu32.astype(np.float64)
        cov = (V.T @ V) / float(len(rows))
    else:
        cov = np.zeros((d, d), dtype=np.float64)
    w, E = np.linalg.eigh(cov)
    order = np.argsort(-w, kind="stable")
    w = w[order]
    E = E[:, order]
    U = E[:, :r].T.copy()
    for j in range(r):
        m = int(np.argmax(np.abs(U[j])))
        if U[j, m] < 0:
            U[j] = -U[j]
    return U, w


def tangent(X, rows, mu32, U):
    """z = U (x - mu) (Eq. 1-2) and rho = ||(x - mu) - U^T z||^2 (Eq. 3-4), FP64."""
    V = X[rows].astype(np.float64) - mu32.astype(np.float64)
    Z = V @ U.T
    E = V - Z @ U
    return Z, np.einsum("ij,ij->i", E, E)


def build_index(X, G: int, r: int, u, train_idx=None, max_iter: int = 25, keep_fp64: bool = False,
                max_grain_rows: int = 0):
    """Oracle index build: partition, per-grain PCA, database coordinates.

    Rows are stored in grain order (ascending original id inside a grain).
    Returned arrays: M f32 [G, d], U f32 [G, r, d], eig f64 [G, d],
    grain_off i64 [G+1], ids u32 [N], Z f32 [N, r], rho f32 [N], assign i32 [N].
    z and rho are computed from the stored FP32 basis, so database rows and
    queries use the same basis. With keep_fp64, also Z64/rho64 computed with
    the FP64 eigenvectors (for the PCA invariant)."""
    X = _f32(X)
    n, d = X.shape
    if not (1 <= r <= d):
        raise ValueError("need 1 <= r <= d")
    mu, assign, iters = kmeans(X, G, u, train_idx, max_iter, max_grain_rows)
    order = np.argsort(assign, kind="stable")
    counts = np.bincount(assign, minlength=G)
    grain_off = np.zeros(G + 1, dtype=np.int64)
    grain_off[1:] = np.cumsum(counts)
    U32 = np.zeros((G, r, d), dtype=np.float32)
    eig = np.zeros((G, d), dtype=np.float64)
    Z = np.zeros((n, r), dtype=np.float32)
    rho = np.zeros(n, dtype=np.float32)
    out = {}
    if keep_fp64:
        out["U64"] = np.zeros((G, r, d))
        out["Z64"] = np.zeros((n, r))
        out["rho64"] = np.zeros(n)
    for g in range(G):
        rows = order[grain_off[g]:grain_off[g + 1]]
        U, w = grain_pca(X, rows, mu[g], r)
        U32[g] = U.astype(np.float32)
        eig[g] = w
        if len(rows):
            z, rh = tangent(X, rows, mu[g], U32[g].astype(np.float64))
            Z[grain_off[g]:grain_off[g + 1]] = z.astype(np.float32)
            rho[grain_off[g]:grain_off[g + 1]] = rh.astype(np.float32)
            if keep_fp64:
                z64, rh64 = tangent(X, rows, mu[g], U)
                out["Z64"][grain_off[g]:grain_off[g + 1]] = z64
                out["rho64"][grain_off[g]:grain_off[g + 1]] = rh64
        if keep_fp64:
            out["U64"][g] = U
    out.update(dict(M=mu, U=U32, eig=eig, grain_off=grain_off, ids=order.astype(np.uint32), Z=Z, rho=rho,
                    assign=assign, lloyd_iters=iters, N=n, d=d, G=G, r=r))
    return out


# ---------------------------------------------------------------------------
# search and brute force
# ---------------------------------------------------------------------------


def search(idx, X, Q, k: int, C: int, nprobe: int, attr=None, ranges=None, Z=None, rho=None, precision="fp32",
           mode: str = "B", probes=None, resid_prune: bool = False, query_codes=None, pair_proj=None,
           refine: bool = False):
    """Mode B (default) or Mode A search of every query (see hntl_oracle.c or_search).

    probes (optional, [nq, nprobe] grain ids): replaces the centroid routing
    of step 1 (a learned router's probes); the rest of the path is unchanged.
    pair_proj (optional, (z [nq, nprobe, r], rho [nq, nprobe]) with probes):
    replaces the projection step (Eq. 1-4) by given values, so that the scan,
    pool and rerank can be compared on the same inputs as another
    implementation's.

    mode="B": the pool is reranked by exact L2 to the raw rows (sec. 2.1 step 4).
    mode="A": the pool is reranked by L2 to each row's reconstruction
    mu_g + U_g^T z_i (its grain's centre and basis, its stored coordinates),
    against the query as routed and projected; no raw row is read (sec. 2.1
    step 4, sec. 1). Routing, projection, scan and pool are the same.

    precision="fp32": the plain method on the stored FP32 values.
    precision="int16": the paper's 16-bit form (Eq. 5): rows on their grain's
    16-bit grids (int16_form), the query's coordinates quantised with the same
    steps (saturating at +-32767) and its residual norm clipped at 65535
    steps, and a grain left out of a query's scan when more than a quarter of
    its coordinates saturate (sec. 2.3). Eq. 6 is then evaluated on the codes:
    the exact integer sum of squared code differences, scaled back by the
    squared step in IEEE single precision (see hntl_oracle.c). resid_prune
    (the build's own option, not the paper's): also leave the grain out when
    the residual code would exceed 65535. query_codes (codes, rcodes) with
    codes [nq, nprobe, r] int16 and rcodes [nq, nprobe] int32 (-1 = pair left
    out) replace the query-side quantisation (to compare the scan on the same
    integer inputs).
    precision="bf16-fp8": the precision form, defined on rounded inputs: the
    query, centres and bases are rounded to BF16 for routing and projection,
    the scan reads the FP8 coordinates decoded and scaled (fp8_coords), and the
    rerank compares the FP32 query with BF16-rounded rows. X is the FP32 rows
    in original id order; Z/rho override the index's coordinates.

    refine (precision form, Mode B): a second rerank stage. Each row also
    has a second BF16 part, xl = bf16(x - bf16(x)); the min(C, 2k) smallest
    (distance, id) of the BF16 rerank are ranked again by the distance to
    bf16(x) + xl, and the k smallest of those are returned."""
    X = _f32(X)
    Q = _f32(Q)
    nq, d = Q.shape
    G, r = idx["G"], idx["r"]
    if not (1 <= nprobe <= G) or k < 1 or C < 1:
        raise ValueError("bad search parameters")
    M = _f32(idx["M"])
    U = _f32(idx["U"])
    Qp = None
    Xlo = None
    kref = 0
    if refine:
        if precision != "bf16-fp8" or mode != "B":  # X must be the FP32 rows
            raise ValueError("refine applies to the precision form's Mode B rerank (precision='bf16-fp8')")
        Xf = _f32(X)
        # second BF16 part of each row, from the FP32 rows (X must be FP32 here)
        Xlo = np.ascontiguousarray(bf16_to_f32(bf16_round(Xf - bf16_to_f32(bf16_round(Xf)).reshape(Xf.shape)))
                                   .reshape(Xf.shape))
        kref = min(C, 2 * k)
    if precision in ("bf16-fp8", "bf16-fp8-decoded"):
        # "bf16-fp8-decoded": idx["Z"] already holds decoded FP8 values and X BF16-rounded values
        M = bf16_to_f32(bf16_round(M)).reshape(M.shape)
        U = bf16_to_f32(bf16_round(U)).reshape(U.shape)
        if precision == "bf16-fp8":
            X = bf16_to_f32(bf16_round(X)).reshape(X.shape)
            if Z is None:
                Z = fp8_decoded(idx)
        Qp = np.ascontiguousarray(bf16_to_f32(bf16_round(Q)).reshape(Q.shape))
    elif precision not in ("fp32", "int16"):
        raise ValueError(precision)
    qdelta = qdres = None
    Zs = _f32(idx["Z"] if Z is None else Z)
    rhos = _f32(idx["rho"] if rho is None else rho)
    Zc = qc_in = qr_in = None
    if precision == "int16":  # rows and queries on the grains' 16-bit grids (Eq. 5)
        q16 = int16_form(idx)
        Zs = q16["Zf32"]
        rhos = q16["rhof32"]
        Zc = np.ascontiguousarray(q16["codes"], dtype=np.int16)
        qdelta, qdres = q16["delta"].astype(np.float64), q16["dres"].astype(np.float64)
        if query_codes is not None:
            qc_in = np.ascontiguousarray(query_codes[0], dtype=np.int16)
            qr_in = np.ascontiguousarray(query_codes[1], dtype=np.int32)
            if qc_in.shape != (nq, nprobe, r) or qr_in.shape != (nq, nprobe):
                raise ValueError("query_codes must be ([nq, nprobe, r] int16, [nq, nprobe] int32)")
    elif query_codes is not None or resid_prune:
        raise ValueError("query_codes and resid_prune apply to the 16-bit form")
    off = np.ascontiguousarray(idx["grain_off"], dtype=np.int64)
    ids = np.ascontiguousarray(idx["ids"], dtype=np.uint32)
    attr_a = None if attr is None else np.ascontiguousarray(attr, dtype=np.int64)
    rng = None if ranges is None else np.ascontiguousarray(ranges, dtype=np.int64)
    if rng is not None and attr_a is None:
        raise ValueError("ranges need attr")
    probe = np.zeros((nq, nprobe), dtype=np.int32)
    probe_d = np.zeros((nq, nprobe + 1), dtype=np.float64)
    cand_id = np.zeros((nq, C), dtype=np.uint32)
    cand_d = np.zeros((nq, C + 1), dtype=np.float64)
    out_id = np.zeros((nq, k), dtype=np.int64)
    out_d = np.zeros((nq, k + 1), dtype=np.float64)
    if mode not in ("A", "B"):
        raise ValueError(mode)
    pos_of_id = grain_of_pos = None
    if mode == "A":  # the stored position of each id, and the grain of each position
        pos_of_id = np.zeros(len(ids), dtype=np.int64)
        pos_of_id[ids] = np.arange(len(ids), dtype=np.int64)
        grain_of_pos = np.repeat(np.arange(G, dtype=np.int32), np.diff(off)).astype(np.int32)
    pz = prho = None
    if pair_proj is not None:
        if probes is None:
            raise ValueError("pair_proj needs the probes it belongs to")
        pz = np.ascontiguousarray(pair_proj[0], dtype=np.float32)
        prho = np.ascontiguousarray(pair_proj[1], dtype=np.float32)
        if pz.shape != (nq, nprobe, r) or prho.shape != (nq, nprobe):
            raise ValueError("pair_proj must be ([nq, nprobe, r], [nq, nprobe])")
    pin = None
    if probes is not None:
        pin = np.ascontiguousarray(probes, dtype=np.int32)
        if pin.shape != (nq, nprobe) or pin.min() < 0 or pin.max() >= G:
            raise ValueError("probes must be [nq, nprobe] grain ids")
    _c().or_search(_p(M), _p(U), G, d, r, _p(off), _p(ids), _p(Zs), _p(rhos), _p(X), _p(attr_a), _p(Q), _p(Qp), nq,
                   k, C, nprobe, _p(rng), _p(probe), _p(probe_d), _p(cand_id), _p(cand_d), _p(out_id), _p(out_d),
                   1 if mode == "A" else 0, _p(pos_of_id), _p(grain_of_pos), _p(qdelta), _p(qdres), _p(pin),
                   _p(Zc), 1 if resid_prune else 0, _p(qc_in), _p(qr_in), _p(pz), _p(prho), _p(Xlo), kref)
    return dict(probe=probe, probe_d=probe_d, cand_id=cand_id, cand_d=cand_d, out_id=out_id, out_d=out_d)


def int16_form(idx):
    """The paper's 16-bit form of the stored rows (Eq. 5), per grain g:
    delta_g = fl32(max |z| / 16383) and dres_g = fl32(R / 32767) with
    R = max(max rho, fl32(max|z|^2) 2^-20) (a residual grid no finer than FP32
    can resolve next to the coordinates' energy; 1 for a grain whose values
    are all zero), so the rows use at most half of the signed and
    unsigned 16-bit ranges and a query's values up to twice the grain's extent
    stay representable (the paper leaves the steps open; saturation, which the
    envelope filter counts, then means a query well outside the grain); codes
    rint(fl32(z / delta_g)) and rint(fl32(rho / dres_g)) (round half to even),
    all in IEEE single precision so that any implementation of these steps
    gets the same codes. Returns the codes, the steps and the values the scan
    uses, fl32(code * step)."""
    Z = _f32(idx["Z"])
    rho = _f32(idx["rho"])
    off = np.asarray(idx["grain_off"], dtype=np.int64)
    G = len(off) - 1
    delta = np.ones(G, dtype=np.float32)
    dres = np.ones(G, dtype=np.float32)
    codes = np.zeros(Z.shape, dtype=np.int16)
    rcodes = np.zeros(rho.shape, dtype=np.uint16)
    for g in range(G):
        a, b = off[g], off[g + 1]
        if b > a:
            m = np.max(np.abs(Z[a:b])) if Z.shape[1] else np.float32(0)
            if m > 0:
                delta[g] = np.float32(m) / np.float32(16383)
            mr = max(np.float32(np.max(rho[a:b])), np.float32(np.float32(m) * np.float32(m)) * np.float32(2.0 ** -20))
            if mr > 0:
                dres[g] = np.float32(mr) / np.float32(32767)
            codes[a:b] = np.clip(np.rint(Z[a:b] / delta[g]), -32767, 32767).astype(np.int16)
            rcodes[a:b] = np.clip(np.rint(rho[a:b] / dres[g]), 0, 65535).astype(np.uint16)
    gof = np.repeat(np.arange(G), np.diff(off))
    Zf32 = np.ascontiguousarray(codes.astype(np.float32) * delta[gof][:, None])
    rhof32 = np.ascontiguousarray(rcodes.astype(np.float32) * dres[gof])
    return dict(codes=codes, rcodes=rcodes, delta=delta, dres=dres, Zf32=Zf32, rhof32=rhof32)


def shard_assign(grain_rows, S: int):
    """Grains to S shards by rows: grains in order of (rows descending, grain
    ascending), each to the shard holding the fewest rows so far, the lowest
    such shard on ties (the greedy longest-first rule). Returns int [G]."""
    rows = [int(x) for x in grain_rows]
    if not (1 <= S <= len(rows)):
        raise ValueError("need 1 <= S <= G")
    load = [0] * S
    out = np.zeros(len(rows), dtype=np.int64)
    for g in sorted(range(len(rows)), key=lambda g: (-rows[g], g)):
        s = min(range(S), key=lambda j: (load[j], j))
        out[g] = s
        load[s] += rows[g]
    return out


def sharded_search(idx, X, Q, k: int, C: int, nprobe: int, shard_of_grain, precision="fp32"):
    """The query path split by grains: shard s is the index with every grain
    of another shard emptied (all centres and bases kept, so routing is
    unchanged); each shard searches on its own (its own pool of C, its own
    rerank to k), then per query the k best (distance, id) over all shards'
    lists are kept. Returns (out_id [nq, k] int64, out_d [nq, k] float64,
    per-shard results)."""
    sog = np.asarray(shard_of_grain)
    off = np.asarray(idx["grain_off"], dtype=np.int64)
    G = int(idx["G"])
    per = []
    for s in sorted(set(sog.tolist())):
        keep = np.concatenate([np.arange(off[g], off[g + 1]) for g in range(G) if sog[g] == s] or [np.zeros(0, np.int64)])
        cnt = np.array([off[g + 1] - off[g] if sog[g] == s else 0 for g in range(G)], dtype=np.int64)
        sub = dict(idx)
        sub["grain_off"] = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
        sub["ids"] = np.asarray(idx["ids"])[keep]
        sub["Z"] = np.asarray(idx["Z"])[keep]
        sub["rho"] = np.asarray(idx["rho"])[keep]
        per.append(search(sub, X, Q, k, C, nprobe, precision=precision))
    nq = Q.shape[0]
    out_id = np.full((nq, k), -1, dtype=np.int64)
    out_d = np.full((nq, k), np.inf)
    for qi in range(nq):
        cand = [(float(r["out_d"][qi, j]), int(r["out_id"][qi, j])) for r in per for j in range(k)
                if r["out_id"][qi, j] >= 0]
        cand.sort()
        for j, (dd, ii) in enumerate(cand[:k]):
            out_id[qi, j] = ii
            out_d[qi, j] = dd
    return out_id, out_d, per


def stage_values(idx, X, Q, probes, rows, pair_proj=None, row_terms=None):
    """FP64 values of the plain method's stages at given probes and rows, on
    the FP32 query, rows, centres and bases (X in original id order), so that
    another implementation's stage outputs can be held against them.

    probes [nq, p] grain ids; rows [nq, m] original row ids (negative = none).
    Returns (FP64):
      route_d [nq, p]: ||q - mu_g||^2 for each given grain (sec. 2.1 step 1);
      z [nq, p, r], rho [nq, p]: the query in each given grain (Eq. 1-4);
      zi [nq, m, r], rhoi [nq, m]: each row's coordinates and residual norm in
        its own grain (Eq. 1-4);
      D [nq, m]: Eq. 6 with both sides as above (NaN where the row is absent
        or its grain is not among the query's probes);
      exact [nq, m]: ||q - x||^2 (sec. 2.1 step 4).
    pair_proj (z [nq, p, r], rho [nq, p]) adds D_pair: Eq. 6 with the given
    query side and the rows' own FP64 side. row_terms (Z [nq, m, r], rho
    [nq, m]) adds D_row: the query's FP64 side and the given row side."""
    X = _f32(X)
    Q = _f32(Q)
    probes = np.asarray(probes, dtype=np.int64)
    rows = np.asarray(rows, dtype=np.int64)
    nq, p = probes.shape
    m = rows.shape[1]
    r = int(idx["r"])
    M = _f32(idx["M"]).astype(np.float64)
    U = _f32(idx["U"])
    off = np.asarray(idx["grain_off"], dtype=np.int64)
    ids = np.asarray(idx["ids"], dtype=np.int64)
    grain_of_id = np.zeros(len(ids), dtype=np.int64)
    grain_of_id[ids] = np.repeat(np.arange(int(idx["G"])), np.diff(off))
    out = dict(route_d=np.zeros((nq, p)), z=np.zeros((nq, p, r)), rho=np.zeros((nq, p)),
               zi=np.full((nq, m, r), np.nan), rhoi=np.full((nq, m), np.nan), D=np.full((nq, m), np.nan),
               exact=np.full((nq, m), np.nan))
    if pair_proj is not None:
        out["D_pair"] = np.full((nq, m), np.nan)
    if row_terms is not None:
        out["D_row"] = np.full((nq, m), np.nan)

    def eq6(zq, rq, zi, ri):
        return ((zq - zi) ** 2).sum(-1) + rq + ri

    for qi in range(nq):
        q = Q[qi].astype(np.float64)
        g = probes[qi]
        Ug = U[g].astype(np.float64)
        v = q[None, :] - M[g]
        out["route_d"][qi] = (v * v).sum(1)
        z = np.einsum("prd,pd->pr", Ug, v)
        e = v - np.einsum("pr,prd->pd", z, Ug)
        out["z"][qi] = z
        out["rho"][qi] = (e * e).sum(1)
        have = rows[qi] >= 0
        if not have.any():
            continue
        rid = rows[qi][have]
        gi = grain_of_id[rid]
        x = X[rid].astype(np.float64)
        Ui = U[gi].astype(np.float64)
        w = x - M[gi]
        zi = np.einsum("mrd,md->mr", Ui, w)
        ei = w - np.einsum("mr,mrd->md", zi, Ui)
        ri = (ei * ei).sum(1)
        cols = np.nonzero(have)[0]
        out["zi"][qi, cols] = zi
        out["rhoi"][qi, cols] = ri
        dq = q[None, :] - x
        out["exact"][qi, cols] = (dq * dq).sum(1)
        # the probe slot of each row's grain (rows of unprobed grains keep NaN)
        slot = {int(gg): s for s, gg in enumerate(g)}
        sl = np.array([slot.get(int(gg), -1) for gg in gi])
        ok = sl >= 0
        c, s = cols[ok], sl[ok]
        out["D"][qi, c] = eq6(z[s], out["rho"][qi, s], zi[ok], ri[ok])
        if pair_proj is not None:
            zq_in = np.asarray(pair_proj[0][qi], dtype=np.float64)
            rq_in = np.asarray(pair_proj[1][qi], dtype=np.float64)
            out["D_pair"][qi, c] = eq6(zq_in[s], rq_in[s], zi[ok], ri[ok])
        if row_terms is not None:
            zr = np.asarray(row_terms[0][qi], dtype=np.float64)[c]
            rr = np.asarray(row_terms[1][qi], dtype=np.float64)[c]
            out["D_row"][qi, c] = eq6(z[s], out["rho"][qi, s], zr, rr)
    return out


def brute_force(X, Q, k: int, attr=None, ranges=None):
    """Exact kNN by (dist, id), FP64. Returns (ids i64 [nq,k], d f64 [nq,k], next f64 [nq])."""
    X = _f32(X)
    Q = _f32(Q)
    nq = Q.shape[0]
    ids = np.zeros((nq, k), dtype=np.int64)
    dd = np.zeros((nq, k), dtype=np.float64)
    nxt = np.zeros(nq, dtype=np.float64)
    attr_a = None if attr is None else np.ascontiguousarray(attr, dtype=np.int64)
    rng = None if ranges is None else np.ascontiguousarray(ranges, dtype=np.int64)
    _c().or_bruteforce(_p(X), X.shape[0], X.shape[1], _p(Q), nq, k, _p(attr_a), _p(rng), _p(ids), _p(dd),
                       _p(nxt))
    return ids, dd, nxt


# ---------------------------------------------------------------------------
# number formats (precision form)
# ---------------------------------------------------------------------------


def bf16_round(x, chunk: int = 1 << 24):
    """FP32 -> BF16 (round to nearest, ties to even), returned as the 16-bit
    codes: add 0x7FFF plus the lowest kept bit, keep the top 16 bits (NaN ->
    quiet NaN). Works in chunks with 32-bit arithmetic (finite inputs cannot
    overflow it), so large arrays need no wide temporaries."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    flat = a.reshape(-1)
    out = np.empty(flat.shape, dtype=np.uint16)
    for s in range(0, flat.size, chunk):
        f = flat[s:s + chunk]
        b = f.view(np.uint32)
        lsb = (b >> np.uint32(16)) & np.uint32(1)
        with np.errstate(over="ignore"):
            r = (b + np.uint32(0x7FFF) + lsb) >> np.uint32(16)
        o = r.astype(np.uint16)
        o[np.isnan(f)] = 0x7FC0
        out[s:s + chunk] = o
    return out.reshape(a.shape)


def bf16_to_f32(h):
    return (np.ascontiguousarray(h, dtype=np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32)


def e4m3_value(code):
    """Value of OCP FP8 E4M3 codes: sign bit, 4 exponent bits (bias 7), 3
    mantissa bits; exponent field 0 is subnormal (m/8 * 2^-6); S.1111.111 is
    NaN; no infinities; largest finite 448."""
    c = np.asarray(code, dtype=np.uint8).astype(np.int64)
    s = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = c & 0x7
    val = np.where(e == 0, (m / 8.0) * 2.0 ** -6, (1.0 + m / 8.0) * np.exp2(e - 7.0))
    val = np.where((e == 0xF) & (m == 0x7), np.nan, val)
    return s * val


def e4m3_encode(x):
    """Round each value to the nearest E4M3 number (ties to the even code),
    saturating to +-448 (satfinite). Returns the 8-bit codes. Written as a
    search over the 127 non-negative finite codes, which is the plain
    definition of round-to-nearest."""
    x = np.asarray(x, dtype=np.float64)
    codes = np.arange(0, 0x7F, dtype=np.uint8)  # 0x00..0x7E, non-negative finite
    vals = e4m3_value(codes)
    a = np.minimum(np.abs(x), 448.0)
    # index of the largest value <= a
    hi = np.searchsorted(vals, a, side="right") - 1
    hi = np.clip(hi, 0, len(vals) - 1)
    lo_v = vals[hi]
    nxt = np.clip(hi + 1, 0, len(vals) - 1)
    up_v = vals[nxt]
    dlo = a - lo_v
    dup = up_v - a
    pick_up = (dup < dlo) | ((dup == dlo) & (nxt != hi) & ((hi & 1) == 1))
    idx = np.where(pick_up, nxt, hi)
    out = codes[idx]
    neg = (x < 0) & (out != 0)
    out = np.where(neg, out | 0x80, out).astype(np.uint8)
    out = np.where(np.isnan(x), np.uint8(0x7F), out).astype(np.uint8)
    return out


# ---------------------------------------------------------------------------
# index file (format shared with the library's loader by specification only)
# ---------------------------------------------------------------------------

MAGIC = b"HNTLIDX\0"
VERSION = 1
F_EIG, F_FP8, F_XBF16, F_ATTR = 1, 2, 4, 8


def _wsum(buf: bytes, state):
    """Position-weighted 64-bit word sum: sum of w_i * (2 i + 1) mod 2^64 over
    little-endian u64 words (zero padded). state = (sum, next_word_index)."""
    s, pos = state
    a = np.frombuffer(buf + b"\0" * ((-len(buf)) % 8), dtype="<u8")
    w = (np.arange(a.size, dtype=np.uint64) + np.uint64(pos)) * np.uint64(2) + np.uint64(1)
    with np.errstate(over="ignore"):
        s = np.uint64(s) + np.sum(a * w, dtype=np.uint64)
    return int(s), pos + a.size


def write_index(path, idx, X, attr=None, precision: str = "fp32", include_eig: bool = True):
    """Write the index file. precision="fp32": FP32 X. precision="bf16-fp8":
    BF16 X plus FP8-E4M3 coordinates with a per-grain FP32 scale
    s_g = max|z| / 448 over the grain (1 for an all-zero grain)."""
    N, d, G, r = idx["N"], idx["d"], idx["G"], idx["r"]
    flags = (F_EIG if include_eig else 0) | (F_ATTR if attr is not None else 0)
    sections = [_f32(idx["M"]).tobytes(), _f32(idx["U"]).tobytes()]
    if include_eig:
        sections.append(np.ascontiguousarray(idx["eig"], dtype="<f8").tobytes())
    sections += [np.ascontiguousarray(idx["grain_off"], dtype="<u8").tobytes(),
                 np.ascontiguousarray(idx["ids"], dtype="<u4").tobytes(),
                 _f32(idx["Z"]).tobytes(), _f32(idx["rho"]).tobytes()]
    if precision == "bf16-fp8":
        flags |= F_FP8 | F_XBF16
        z8, scale = fp8_coords(idx)
        sections += [z8.tobytes(), scale.astype("<f4").tobytes(), bf16_round(X).tobytes()]
    elif precision == "fp32":
        sections.append(_f32(X).tobytes())
    else:
        raise ValueError(precision)
    if attr is not None:
        sections.append(np.ascontiguousarray(attr, dtype="<i8").tobytes())
    head = MAGIC + np.array([VERSION, flags], dtype="<u4").tobytes() + np.array([N], dtype="<u8").tobytes() \
        + np.array([d, G, r, 0], dtype="<u4").tobytes()
    state = (0, 0)
    with open(path, "wb") as f:
        for blob in [head] + sections:
            f.write(blob)
        f.flush()
    # checksum over the whole file so far, in 8-byte words (chunks are multiples of 8 bytes)
    with open(path, "rb") as f:
        while True:
            data = f.read(1 << 26)
            if not data:
                break
            state = _wsum(data, state)
    with open(path, "ab") as f:
        f.write(np.array([state[0]], dtype="<u8").tobytes())


def fp8_coords(idx):
    """Per-grain FP8 coordinates: s_g = max|z_ij| / 448 over grain g (1.0 if
    that is zero), code = E4M3(z / s_g) rounded to nearest even, saturating."""
    G = idx["G"]
    off = idx["grain_off"]
    Z = np.asarray(idx["Z"], dtype=np.float32)
    scale = np.ones(G, dtype=np.float32)
    z8 = np.zeros(Z.shape, dtype=np.uint8)
    for g in range(G):
        blk = Z[off[g]:off[g + 1]]
        if blk.size == 0:
            continue
        m = float(np.max(np.abs(blk)))
        s = np.float32(m / 448.0) if m > 0 else np.float32(1.0)
        scale[g] = s
        z8[off[g]:off[g + 1]] = e4m3_encode(blk.astype(np.float64) / np.float64(s))
    return z8, scale


def fp8_decoded(idx):
    """FP8 coordinates decoded and scaled back, as FP32 (what the FP8 scan sees)."""
    z8, scale = fp8_coords(idx)
    off = idx["grain_off"]
    vals = e4m3_value(z8).astype(np.float64)
    out = np.zeros(vals.shape, dtype=np.float32)
    for g in range(idx["G"]):
        out[off[g]:off[g + 1]] = (vals[off[g]:off[g + 1]] * np.float64(scale[g])).astype(np.float32)
    return out


def read_index_header(path):
    with open(path, "rb") as f:
        h = f.read(40)
    if h[:8] != MAGIC:
        raise ValueError("bad magic")
    ver, flags = np.frombuffer(h[8:16], dtype="<u4")
    N = int(np.frombuffer(h[16:24], dtype="<u8")[0])
    d, G, r, _ = (int(v) for v in np.frombuffer(h[24:40], dtype="<u4"))
    return dict(version=int(ver), flags=int(flags), N=N, d=d, G=G, r=r)
