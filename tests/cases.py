"""Seeded test cases: data from the input generator, index built by the oracle."""
import os

import numpy as np

from oracle import hntl_oracle as O
from paper_2606_08813_b300 import synth


def clustered_case(n, d, n_clusters, G, r, nq, seed, sizes="equal", train=None):
    m = synth.make_cluster_model(n, d, n_clusters, sizes=sizes, seed=seed)
    X, _ = synth.sample_points(m, seed + 1)
    Q, _ = synth.sample_queries(m, nq, seed + 2)
    X, Q = X.numpy(), Q.numpy()
    tr = None if train is None else synth.train_subset(n, train, seed + 3).numpy()
    idx = O.build_index(X, G, r, synth.uniforms(G, seed + 4).numpy(), train_idx=tr)
    return X, Q, idx


def partition_index(X, assign, G, r):
    """Oracle index over a GIVEN partition (to force grain sizes such as 0,
    1, 127, 128, 129): centre = FP64 mean of the members rounded to FP32,
    basis and coordinates by the oracle's PCA and Eq. 1-4."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    n, d = X.shape
    order = np.argsort(assign, kind="stable")
    counts = np.bincount(assign, minlength=G)
    off = np.zeros(G + 1, dtype=np.int64)
    off[1:] = np.cumsum(counts)
    M = np.zeros((G, d), dtype=np.float32)
    U32 = np.zeros((G, r, d), dtype=np.float32)
    eig = np.zeros((G, d))
    Z = np.zeros((n, r), dtype=np.float32)
    rho = np.zeros(n, dtype=np.float32)
    for g in range(G):
        rows = order[off[g]:off[g + 1]]
        if len(rows):
            M[g] = X[rows].astype(np.float64).mean(0).astype(np.float32)
        U, w = O.grain_pca(X, rows, M[g], r)
        U32[g] = U.astype(np.float32)
        eig[g] = w
        if len(rows):
            z, rh = O.tangent(X, rows, M[g], U32[g].astype(np.float64))
            Z[off[g]:off[g + 1]] = z
            rho[off[g]:off[g + 1]] = rh
    return dict(M=M, U=U32, eig=eig, grain_off=off, ids=order.astype(np.uint32), Z=Z, rho=rho,
                assign=np.asarray(assign, dtype=np.int32), N=n, d=d, G=G, r=r)


def write(tmpdir, name, idx, X, attr=None, precision="fp32"):
    p = os.path.join(str(tmpdir), name + ".hntl")
    O.write_index(p, idx, X, attr=attr, precision=precision)
    return p
