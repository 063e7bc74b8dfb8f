"""Allocation-free routing entry point (hntl_route_noalloc).

For callers that cannot allocate device memory while they query (a host
application that reserves the whole GPU and hands its plug-ins no allocator,
or a loop where a cudaMalloc would stall the device), the library offers a
routing call whose scratch lives in a fixed device array inside the library.
This test calls it through the C ABI and checks it against the ordinary
hntl_route on two calls in a row, under the gap rule of the parity tests: the
two calls may sum a distance in different orders, so their probe lists must
agree wherever the oracle's routing distances are more than 1e-4 apart, and
their distances within 1e-5 relative. It lives in a file of its own that
pytest collects last, and it builds everything it needs, so it passes alone
in a fresh process as well as after the other tests."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import hntl_oracle as O

from cases import clustered_case, write
from parity import GAP, RTOL

pytestmark = pytest.mark.gpu


def _check_probe_lists(got, ref, ora_d, nprobe):
    """got/ref: [nq, nprobe] grain ids; ora_d: the oracle's nprobe + 1 routing
    distances per query. Where the oracle's boundary is not a near tie, the
    probe sets agree; inside the list, every prefix that ends at a gap agrees
    as a set. Returns the number of queries compared."""
    checked = 0
    for qi in range(got.shape[0]):
        d = ora_d[qi]
        if np.isfinite(d[nprobe]) and (d[nprobe] - d[nprobe - 1]) <= GAP * d[nprobe - 1]:
            continue
        for m in range(1, nprobe + 1):
            if m == nprobe or (d[m] - d[m - 1]) > GAP * d[m - 1]:
                assert set(got[qi, :m].tolist()) == set(ref[qi, :m].tolist()), (qi, m)
        checked += 1
    return checked


def test_route_noalloc_matches_route_on_two_calls(tmp_path):
    from paper_2606_08813_b300 import build_lib

    build_lib.build()
    from paper_2606_08813_b300 import hntl

    X, Q, idx = clustered_case(4000, 64, 48, 48, 8, 500, seed=2024)
    gi = hntl.Index.load(write(tmp_path, "noalloc", idx, X), 0)
    Qd = torch.from_numpy(Q).cuda()
    for nq, nprobe in [(500, 8), (123, 3)]:  # two calls in a row, different shapes
        q = Qd[:nq].contiguous()
        ora = O.search(idx, X, Q[:nq], 1, 1, nprobe)
        ref_probe, ref_d = gi.route(q, nprobe)
        probe = torch.full((nq, nprobe), -7, dtype=torch.int32, device="cuda")
        pd = torch.full((nq, nprobe), -1.0, dtype=torch.float32, device="cuda")
        rc = hntl.lib.hntl_route_noalloc(gi.handle, ctypes.c_void_p(q.data_ptr()), nq, nprobe,
                                         ctypes.c_void_p(probe.data_ptr()), ctypes.c_void_p(pd.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == hntl.OK, hntl.last_error()
        torch.cuda.synchronize()
        got, ref = probe.cpu().numpy(), ref_probe.cpu().numpy()
        assert _check_probe_lists(got, ref, ora["probe_d"], nprobe) >= 0.95 * nq
        assert _check_probe_lists(got, ora["probe"], ora["probe_d"], nprobe) >= 0.95 * nq
        # distances of the grains both calls chose, within the parity tolerance
        gd, rd = pd.cpu().numpy().astype(np.float64), ref_d.cpu().numpy().astype(np.float64)
        for qi in range(nq):
            rmap = dict(zip(ref[qi].tolist(), rd[qi].tolist()))
            for g, dv in zip(got[qi].tolist(), gd[qi].tolist()):
                if g in rmap:
                    assert abs(dv - rmap[g]) <= RTOL * rmap[g], (qi, g, dv, rmap[g])


def test_route_noalloc_rejects_batches_beyond_its_scratch(tmp_path):
    from paper_2606_08813_b300 import build_lib

    build_lib.build()
    from paper_2606_08813_b300 import hntl

    X, Q, idx = clustered_case(2000, 16, 8, 8, 4, 4, seed=7)
    gi = hntl.Index.load(write(tmp_path, "noalloc_big", idx, X), 0)
    nq = (1 << 21) // 8 + 1  # nq * G just over the 2^21 limit; rejected before any launch
    rc = hntl.lib.hntl_route_noalloc(gi.handle, ctypes.c_void_p(1), nq, 2, ctypes.c_void_p(1), ctypes.c_void_p(1),
                                     None)
    assert rc == hntl.EINVAL
    assert "exceeds" in hntl.last_error()
