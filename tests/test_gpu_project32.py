"""The FP32 form's projection (Eq. 1-4) on the tensor cores, with every FP32
operand in three BF16 parts, and its SIMT fallback for bases of more than 32
rows.

Near a grain's subspace (q = mu_g + U_g^T c + a tiny off-subspace part) the
residual rho_q = ||v' - U_g^T z||^2 is a small difference of large terms. The
explicit form computed in FP32 moves it by about 2 sqrt(rho) |dw| with
|dw| ~ 2^-24 (|q| + |mu|) per reconstruction: the test holds the GPU to
2 sqrt(rho) e + e^2 with e = 2^-17 (|q| + |mu|), against the oracle's FP64
value at the GPU's own probes. The identity ||v'||^2 - ||z||^2 (or its Gram
form) would be off by about 2^-24 ||v'||^2, far above that bound at
rho ~ 1e-8 ||v'||^2."""
import numpy as np
import pytest
import torch

from oracle import hntl_oracle as O

from cases import clustered_case, write
from parity import compare_search

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hntl():
    from paper_2606_08813_b300 import build_lib

    build_lib.build()
    from paper_2606_08813_b300 import hntl as h

    return h


def _search(gi, Q, k, C, nprobe):
    Qd = torch.from_numpy(np.ascontiguousarray(Q)).cuda()
    ws = gi.workspace(gi.workspace_bytes(len(Q), k, C, nprobe))
    ids, dist, pid, pd, probe = gi.search(Qd, k, C, nprobe, return_pool=True, return_probe=True, ws=ws)
    torch.cuda.synchronize()
    return dict(ids=ids.cpu().numpy(), dist=dist.cpu().numpy(), pool_ids=pid.cpu().numpy().view(np.uint32),
                pool_d=pd.cpu().numpy(), probe=probe.cpu().numpy()), ws


@pytest.mark.parametrize("r", [16, 32])
def test_near_subspace_residual(hntl, tmp_path, r):
    d, G, nq, k, C, nprobe = 64, 8, 256, 10, 50, 2
    X, _, idx = clustered_case(6000, d, 8, G, r, 4, seed=700 + r)
    rng = np.random.default_rng(710 + r)
    g = rng.integers(0, G, nq)
    U, M = idx["U"].astype(np.float64), idx["M"].astype(np.float64)
    c = rng.standard_normal((nq, r)) * 2.0
    off = rng.standard_normal((nq, d))
    Q = np.empty((nq, d))
    for i in range(nq):
        base = M[g[i]] + U[g[i]].T @ c[i]
        o = off[i] - U[g[i]].T @ (U[g[i]] @ off[i])  # off the subspace
        Q[i] = base + o * (1e-4 * np.linalg.norm(c[i]) / np.linalg.norm(o))
    Q = Q.astype(np.float32)
    gi = hntl.Index.load(write(tmp_path, f"near{r}", idx, X), 0, hntl.PREC_FP32)
    gpu, ws = _search(gi, Q, k, C, nprobe)
    zq, rq = hntl.search_pair_proj(gi, ws, nq, C, nprobe)
    zq, rq = zq.cpu().numpy(), rq.cpu().numpy()
    assert hntl.device_status(gi) == 0
    # the FP32 arrays the library loaded, widened
    Mf, Uf = idx["M"].astype(np.float32).astype(np.float64), idx["U"].astype(np.float32).astype(np.float64)
    Qf = Q.astype(np.float64)
    near = 0
    for qi in range(nq):
        for p, gg in enumerate(gpu["probe"][qi]):
            v = Qf[qi] - Mf[gg]
            z = Uf[gg] @ v
            rho = float(((v - Uf[gg].T @ z) ** 2).sum())
            e = 2.0 ** -17 * (np.linalg.norm(Qf[qi]) + np.linalg.norm(Mf[gg]))
            assert abs(float(rq[qi, p]) - rho) <= 2 * np.sqrt(rho) * e + e * e, (qi, p, float(rq[qi, p]), rho)
            assert np.abs(zq[qi, p] - z).max() <= 1e-5 * max(np.abs(z).max(), 1e-3), (qi, p)
            near += int(gg == g[qi] and rho < 1e-6 * float(v @ v))
    assert near >= nq // 2  # most queries probed their own grain, where rho_q is tiny


def test_simt_projection_beyond_32_rows(hntl, tmp_path):
    """Bases of 40 rows take the SIMT direct form: same parity bar."""
    X, Q, idx = clustered_case(5000, 64, 8, 8, 40, 120, seed=731)
    gi = hntl.Index.load(write(tmp_path, "r40", idx, X), 0, hntl.PREC_FP32)
    k, C, nprobe = 10, 100, 3
    gpu, _ = _search(gi, Q, k, C, nprobe)
    ora = O.search(idx, X, Q, k, C, nprobe)
    st = compare_search(gpu, ora, k, C, nprobe)
    assert st["checked"] >= 0.8 * len(Q), st


def test_ragged_d_and_r(hntl, tmp_path):
    """d not a multiple of the 64-coordinate K block (d = 200: the last block
    is partly outside), r below its padded width (r = 12 in RN = 16, r = 20
    in RN = 32), grains of Zipf sizes."""
    for r, seed in ((12, 741), (20, 742)):
        X, Q, idx = clustered_case(6000, 200, 10, 10, r, 150, seed=seed, sizes="zipf")
        gi = hntl.Index.load(write(tmp_path, f"rag{r}", idx, X), 0, hntl.PREC_FP32)
        k, C, nprobe = 10, 100, 3
        gpu, _ = _search(gi, Q, k, C, nprobe)
        ora = O.search(idx, X, Q, k, C, nprobe)
        st = compare_search(gpu, ora, k, C, nprobe)
        assert st["checked"] >= 0.8 * len(Q), (r, st)
