"""The C-ABI library on a machine without a GPU: it loads, exports every
entry point declared in include/hntl.h, and rejects bad index files on the
host before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from oracle import hntl_oracle as O

from paper_2606_08813_b300 import build_lib

build_lib.build()
from paper_2606_08813_b300 import hntl  # noqa: E402


def _declared():
    src = open(os.path.join(ROOT, "include", "hntl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hntl_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    names = _declared()
    assert len(names) >= 8
    for n in names:
        assert hasattr(hntl.lib, n), n


def _load(path):
    h = ctypes.c_void_p()
    rc = hntl.lib.hntl_index_load(os.fsencode(path), 0, 0, ctypes.byref(h))
    return rc, hntl.last_error()


@pytest.fixture(scope="module")
def good_file(tmp_path_factory):
    rng = np.random.default_rng(0)
    X = rng.standard_normal((60, 8)).astype(np.float32)
    idx = O.build_index(X, 3, 4, np.array([0.1, 0.5, 0.9]))
    p = str(tmp_path_factory.mktemp("idx") / "good.hntl")
    O.write_index(p, idx, X)
    return p


def test_missing_file_is_eio():
    rc, msg = _load("/nonexistent/x.hntl")
    assert rc == hntl.EIO and "cannot open" in msg


def test_bad_magic_is_eformat(tmp_path, good_file):
    data = bytearray(open(good_file, "rb").read())
    data[0:4] = b"XXXX"
    p = tmp_path / "bad.hntl"
    p.write_bytes(bytes(data))
    rc, msg = _load(str(p))
    assert rc == hntl.EFORMAT and "magic" in msg


def test_truncated_is_eformat(tmp_path, good_file):
    data = open(good_file, "rb").read()
    for cut in (10, 100, len(data) - 1):
        p = tmp_path / f"t{cut}.hntl"
        p.write_bytes(data[:cut])
        rc, _ = _load(str(p))
        assert rc == hntl.EFORMAT


def test_flipped_byte_fails_checksum(tmp_path, good_file):
    data = bytearray(open(good_file, "rb").read())
    data[200] ^= 0x40
    p = tmp_path / "flip.hntl"
    p.write_bytes(bytes(data))
    rc, msg = _load(str(p))
    assert rc == hntl.EFORMAT and "checksum" in msg


def test_bad_version_is_eformat(tmp_path, good_file):
    data = bytearray(open(good_file, "rb").read())
    data[8] = 9
    p = tmp_path / "ver.hntl"
    p.write_bytes(bytes(data))
    rc, msg = _load(str(p))
    assert rc == hntl.EFORMAT and "version" in msg


def test_ids_not_permutation_is_eformat(tmp_path):
    rng = np.random.default_rng(1)
    X = rng.standard_normal((20, 4)).astype(np.float32)
    idx = O.build_index(X, 2, 2, np.array([0.2, 0.7]))
    idx["ids"] = idx["ids"].copy()
    idx["ids"][1] = idx["ids"][0]  # duplicate id; the checksum is recomputed by the writer
    p = str(tmp_path / "dup.hntl")
    O.write_index(p, idx, X)
    rc, msg = _load(p)
    assert rc == hntl.EFORMAT and "permutation" in msg


def test_bad_offsets_is_eformat(tmp_path):
    rng = np.random.default_rng(2)
    X = rng.standard_normal((20, 4)).astype(np.float32)
    idx = O.build_index(X, 2, 2, np.array([0.2, 0.7]))
    idx["grain_off"] = np.array([0, 15, 12], dtype=np.int64)  # last != N and decreasing
    p = str(tmp_path / "off.hntl")
    O.write_index(p, idx, X)
    rc, _ = _load(p)
    assert rc == hntl.EFORMAT


def test_precision_mismatch_is_einval(tmp_path, good_file):
    h = ctypes.c_void_p()
    rc = hntl.lib.hntl_index_load(os.fsencode(good_file), 0, hntl.PREC_BF16_FP8, ctypes.byref(h))
    assert rc == hntl.EINVAL


def test_null_arguments_are_einval():
    assert hntl.lib.hntl_index_load(None, 0, 0, None) == hntl.EINVAL
    assert hntl.lib.hntl_search(None, None, 1, 1, 1, 1, None, None, 0, None, None, None, None, None, None) \
        == hntl.EINVAL
    assert hntl.lib.hntl_search_workspace_bytes(None, 1, 1, 1, 1) == 0


def test_binding_marks_its_tensors_in_use_on_side_streams(monkeypatch):
    """Tensors the binding allocates are recorded on the call's stream when it
    is not the current one (so the allocator does not reuse them early), and
    left alone otherwise."""

    class FakeStream:
        def __init__(self, handle):
            self.cuda_stream = handle
            self.device = "cuda:0"

    class FakeTensor:
        def __init__(self):
            self.recorded = []

        def record_stream(self, s):
            self.recorded.append(s)

    current = FakeStream(7)
    monkeypatch.setattr(hntl.torch.cuda, "current_stream", lambda device=None: current)
    a, b = FakeTensor(), FakeTensor()
    hntl._in_use(None, a, b)
    hntl._in_use(FakeStream(7), a, b)
    assert a.recorded == [] and b.recorded == []
    side = FakeStream(9)
    hntl._in_use(side, a, None, b)
    assert a.recorded == [side] and b.recorded == [side]


def _int16_both(idx):
    f = O.int16_form(idx)
    Z = np.ascontiguousarray(idx["Z"], dtype=np.float32)
    rho = np.ascontiguousarray(idx["rho"], dtype=np.float32)
    return f, hntl.int16_quantize_host(Z, rho, np.asarray(idx["grain_off"]))


@pytest.mark.parametrize("case", ["clustered", "edges", "full-basis", "zero-grain"])
def test_int16_quantisation_host_code_equals_oracle_bit_for_bit(case):
    """The library's 16-bit quantisation (host C++, shared by the loader and
    the builder) and the oracle's (numpy) take the same IEEE single-precision
    steps: the same steps, codes and grid residuals, bit for bit."""
    from cases import clustered_case, partition_index

    if case == "clustered":
        _, _, idx = clustered_case(3000, 32, 8, 8, 8, 4, seed=41, sizes="zipf")
    else:
        sizes = [0, 1, 127, 128, 129, 300]
        rng = np.random.default_rng(43)
        d, r = (16, 16) if case == "full-basis" else (24, 5)
        centres = rng.standard_normal((len(sizes), d)) * 3
        assign = np.repeat(np.arange(len(sizes)), sizes)
        X = (centres[assign] + rng.standard_normal((len(assign), d)) * 0.7).astype(np.float32)
        if case == "zero-grain":
            X[assign == 3] = 0.0  # one grain of identical rows at the origin: every value zero
        idx = partition_index(X, assign, len(sizes), r)
    f, (delta, dres, codes, rho_grid) = _int16_both(idx)
    np.testing.assert_array_equal(delta.view(np.uint32), f["delta"].view(np.uint32))
    np.testing.assert_array_equal(dres.view(np.uint32), f["dres"].view(np.uint32))
    np.testing.assert_array_equal(codes, f["codes"])
    np.testing.assert_array_equal(rho_grid.view(np.uint32), f["rhof32"].view(np.uint32))
    if case == "zero-grain":
        g = 3
        assert delta[g] == 1.0 and dres[g] == 1.0
    assert np.abs(codes).max() <= 16383  # the rows use at most half of the signed range


def test_int16_quantisation_host_rejects_bad_offsets():
    Z = np.zeros((4, 2), np.float32)
    rho = np.zeros(4, np.float32)
    with pytest.raises(hntl.HntlError):
        hntl.int16_quantize_host(Z, rho, np.array([0, 3, 2, 4]))
    with pytest.raises(ValueError):
        hntl.int16_quantize_host(Z, rho, np.array([0, 3]))


def test_server_wrapper_checks_shapes_before_the_library_reads_them():
    """The server's host entry points read n rows of every array they are
    given: the binding refuses mismatched shapes before calling them (checked
    on a wrapper with no server behind it, so no call is made)."""
    srv = object.__new__(hntl.Server)
    srv._h, srv.d, srv.k_max = None, 8, 10
    Q = np.zeros((4, 8), np.float32)
    k = np.full(4, 10, np.uint32)
    with pytest.raises(ValueError):
        srv.submit(np.zeros((4, 7), np.float32), k, k)  # wrong d
    with pytest.raises(ValueError):
        srv.submit(Q, k[:3], k)  # k shorter than Q
    with pytest.raises(ValueError):
        srv.submit(Q, k, k, ranges=np.zeros((4, 3), np.int64))
    with pytest.raises(ValueError):
        srv.submit(Q, k, k, arrival_ns=np.zeros(3, np.int64))
    tickets = np.zeros(4, np.uint64)
    with pytest.raises(ValueError):
        srv.poll_many(tickets, np.zeros(3, np.uint8))  # done shorter than tickets
    with pytest.raises(ValueError):
        srv.poll_many(tickets, np.zeros(4, np.uint8), ids=np.zeros((3, 10), np.int64))  # too few rows
    with pytest.raises(ValueError):
        srv.poll_many(tickets, np.zeros(4, np.uint8), ids=np.zeros((4, 10), np.int32))  # wrong dtype


def test_router_parameters_must_agree_before_the_library_reads_them():
    from oracle import router_oracle as R

    params = R.init_params(16, 24, 32, 8, seed=1)
    for i, bad in ((1, np.zeros(23, np.float32)), (2, np.zeros((32, 23), np.float32)), (5, np.zeros(9, np.float32))):
        p = list(params)
        p[i] = bad
        with pytest.raises(ValueError):
            hntl.Router(p, max_batch=8)


def test_router_parameters_that_agree_pass_the_shape_checks():
    from oracle import router_oracle as R

    try:
        hntl.Router(R.init_params(16, 24, 32, 8, seed=1), max_batch=8).close()
    except hntl.HntlError:
        pass  # no GPU here: the library itself refuses, after the checks passed


def test_binding_without_the_library_fails_loudly(tmp_path):
    """No CPU fallback: a copy of the binding with no libhntl.so beside it
    refuses to import (run in a child interpreter, so this process keeps its
    loaded library)."""
    import shutil
    import subprocess
    import sys

    pkg = tmp_path / "paper_2606_08813_b300"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_2606_08813_b300", "hntl.py"), pkg / "hntl.py")
    (pkg / "__init__.py").write_text("")
    code = "import paper_2606_08813_b300.hntl"
    p = subprocess.run([sys.executable, "-c", code], cwd=str(tmp_path), capture_output=True, text=True,
                       env={**os.environ, "PYTHONPATH": str(tmp_path)})
    assert p.returncode != 0
    assert "ImportError" in p.stderr and "libhntl.so is not built" in p.stderr


def test_oracle_and_product_share_no_code():
    """The oracle is test infrastructure: nothing in the product package
    imports, loads or includes it, and it imports nothing from the package
    (the seeded input generators are passed in by the tests)."""
    import re

    pkg = os.path.join(ROOT, "paper_2606_08813_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b|hntl_oracle|router_oracle|oracle/", src,
                                     re.M), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert not re.search(r"paper_2606_08813_b300|libhntl|hntl\.h", src), f


def test_server_wrapper_marshalling_against_a_fake_library(monkeypatch):
    """submit / poll / poll_many pass pointers, counts and strides that a
    library writing whole rows can use safely: a fake of the three calls
    writes the request's own k results the way the library does."""
    import ctypes as ct

    k_of = {}

    class Fake:
        def hntl_server_submit(self, h, q, n, k, C, R, A, tickets, got):
            ks = np.ctypeslib.as_array(ct.cast(k, ct.POINTER(ct.c_uint32)), (n,))
            tk = np.ctypeslib.as_array(ct.cast(tickets, ct.POINTER(ct.c_uint64)), (n,))
            for i in range(n):
                tk[i] = 100 + i
                k_of[100 + i] = int(ks[i])
            got._obj.value = n
            return hntl.OK

        def _rows(self, t):
            kk = k_of[int(t)]
            return np.arange(kk, dtype=np.int64) + 1000 * int(t), np.arange(kk, dtype=np.float32) * 0.5

        def hntl_server_poll(self, h, t, ids, dist, timeout):
            a, b = self._rows(t)
            ct.memmove(ids, a.ctypes.data, a.nbytes)  # the request's own k entries
            ct.memmove(dist, b.ctypes.data, b.nbytes)
            return hntl.OK

        def hntl_server_poll_many(self, h, tickets, n, ids, dist, stride, done, timeout, n_done):
            tk = np.ctypeslib.as_array(ct.cast(tickets, ct.POINTER(ct.c_uint64)), (n,))
            dn = np.ctypeslib.as_array(ct.cast(done, ct.POINTER(ct.c_uint8)), (n,))
            for i in range(n):
                a, b = self._rows(tk[i])
                if ids:
                    ct.memmove(ids.value + i * stride * 8, a.ctypes.data, a.nbytes)
                if dist:
                    ct.memmove(dist.value + i * stride * 4, b.ctypes.data, b.nbytes)
                dn[i] = 1
            n_done._obj.value = n
            return hntl.OK

    monkeypatch.setattr(hntl, "lib", Fake())
    srv = object.__new__(hntl.Server)
    srv._h, srv.d, srv.k_max = None, 8, 10
    k = np.array([10, 3, 7], np.uint32)
    t = srv.submit(np.zeros((3, 8), np.float32), k, k)
    assert t.tolist() == [100, 101, 102]
    ids, dist = srv.poll(101, 3)
    assert ids.tolist() == [101000, 101001, 101002] and dist.tolist() == [0.0, 0.5, 1.0]
    ids, dist = srv.poll(100, 2)  # a k below the request's: the buffer still holds its 10 results
    assert ids.tolist() == [100000, 100001]
    done = np.zeros(3, np.uint8)
    I = np.full((3, 10), -7, np.int64)
    D = np.zeros((3, 10), np.float32)
    assert srv.poll_many(t, done, I, D) == 3 and done.all()
    assert I[1, :3].tolist() == [101000, 101001, 101002] and (I[1, 3:] == -7).all()
    assert I[0].tolist() == list(range(100000, 100010)) and D[2, 6] == 3.0
