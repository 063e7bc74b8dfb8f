"""Thin ctypes binding of libhntl.so (the C ABI in include/hntl.h).

Argument marshalling only: every step of the search runs in the library's
CUDA kernels. PyTorch supplies device memory (outputs and workspace) and the
current CUDA stream. There is no CPU fallback: if the library is missing or
fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhntl.so")

OK, EINVAL, ENOMEM, ECUDA, EIO, EFORMAT, ETIMEOUT, EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
PREC_FP32, PREC_BF16_FP8, PREC_INT16 = 0, 1, 2  # INT16: the 16-bit form, built at load from an FP32 file
INT16_RESID_PRUNE = 0x200  # OR into PREC_INT16: the library's residual-saturation pruning option
RERANK_REFINE = 0x400  # OR into PREC_BF16_FP8 at build: second BF16 parts of the rows, two-stage rerank
LOAD_NO_RAW = 0x100  # OR into the precision of Index.load: no raw rows on the device (Mode A only)
INVALID_ID = 0xFFFFFFFF
_NAMES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", EIO: "EIO", EFORMAT: "EFORMAT",
          ETIMEOUT: "ETIMEOUT", EBUSY: "EBUSY"}


class HntlError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libhntl.so is not built ({LIB_PATH}); run paper_2606_08813_b300/build_lib.py")

lib = ctypes.CDLL(LIB_PATH)


class IndexDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("d", ctypes.c_uint32), ("G", ctypes.c_uint32), ("r", ctypes.c_uint32),
                ("precision", ctypes.c_uint32), ("has_attr", ctypes.c_uint32), ("block_rows", ctypes.c_uint32),
                ("n_blocks", ctypes.c_uint64), ("max_grain_rows", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("device", ctypes.c_int)]


_P = ctypes.c_void_p
_U32 = ctypes.c_uint32
_SZ = ctypes.c_size_t
lib.hntl_version.restype = ctypes.c_char_p
lib.hntl_last_error.restype = ctypes.c_char_p
lib.hntl_index_load.argtypes = [ctypes.c_char_p, ctypes.c_int, _U32, ctypes.POINTER(_P)]
lib.hntl_index_info.argtypes = [_P, ctypes.POINTER(IndexDesc)]
lib.hntl_index_free.argtypes = [_P]
lib.hntl_index_free.restype = None
lib.hntl_search_workspace_bytes.argtypes = [_P, _U32, _U32, _U32, _U32]
lib.hntl_search_workspace_bytes.restype = _SZ
lib.hntl_search_host_workspace_bytes.argtypes = [_P, _U32, _U32, _U32, _U32, ctypes.c_int]
lib.hntl_search_host_workspace_bytes.restype = _SZ
lib.hntl_search.argtypes = [_P, _P, _U32, _U32, _U32, _U32, _P, _P, _SZ, _P, _P, _P, _P, _P, _P]
lib.hntl_search_host.argtypes = [_P, _P, _U32, _U32, _U32, _U32, _P, _P, _SZ, _P, _P, _P]
lib.hntl_route.argtypes = [_P, _P, _U32, _U32, _P, _SZ, _P, _P, _P]
lib.hntl_route_noalloc.argtypes = [_P, _P, _U32, _U32, _P, _P, _P]
lib.hntl_index_build.argtypes = [_P, ctypes.c_uint64, _U32, _U32, _U32, _P, ctypes.c_int, _P, ctypes.POINTER(_P)]
lib.hntl_index_grain_rows.argtypes = [_P, _P]
lib.hntl_index_export.argtypes = [_P, _P, _P, _P, _P, _P, _P]
lib.hntl_profile_enable.argtypes = [ctypes.c_int]
lib.hntl_profile_read.argtypes = [_P, _P]
lib.hntl_int16_quantize_host.argtypes = [_P, _P, _P, _U32, _U32, _P, _P, _P, _P]
NSTAGES = 7
STAGES = ("route", "bucket", "project", "pilot", "scan", "select", "rerank")


class BuildParams(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_uint32), ("max_iter", ctypes.c_uint32), ("n_train", ctypes.c_uint64),
                ("n_seed", ctypes.c_uint64), ("pca_iters", ctypes.c_uint32), ("max_grain_rows", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("u", _P), ("d_attr", _P)]


def profile_enable(on: bool = True):
    _check(lib.hntl_profile_enable(int(on)))


def profile_read():
    """(per-stage milliseconds summed over the covered searches, number of searches)."""
    ms = (ctypes.c_double * NSTAGES)()
    calls = ctypes.c_uint64()
    _check(lib.hntl_profile_read(ms, ctypes.byref(calls)))
    return dict(zip(STAGES, list(ms))), int(calls.value)


def int16_quantize_host(Z, rho, grain_off):
    """The 16-bit form's row quantisation as the loader and builder apply it
    (hntl_int16_quantize_host), on host arrays: Z [N, r] and rho [N] float32
    in grain order, grain_off [G + 1]. Returns (delta [G], dres [G],
    codes [N, r] int16, rho_grid [N] float32)."""
    import numpy as np

    Z = np.ascontiguousarray(Z, dtype=np.float32)
    rho = np.ascontiguousarray(rho, dtype=np.float32)
    off = np.ascontiguousarray(grain_off, dtype=np.uint64)
    N, r = Z.shape
    G = len(off) - 1
    if rho.shape != (N,) or G < 1 or int(off[-1]) != N:
        raise ValueError("Z [N, r], rho [N] and grain_off [G + 1] ending at N are required")
    delta = np.empty(G, np.float32)
    dres = np.empty(G, np.float32)
    codes = np.empty((N, r), np.int16)
    rho_grid = np.empty(N, np.float32)
    _check(lib.hntl_int16_quantize_host(Z.ctypes.data, rho.ctypes.data, off.ctypes.data, G, r, delta.ctypes.data,
                                        dres.ctypes.data, codes.ctypes.data, rho_grid.ctypes.data))
    return delta, dres, codes, rho_grid


def last_error() -> str:
    return lib.hntl_last_error().decode()


def _check(rc: int):
    if rc != OK:
        raise HntlError(rc, last_error())


def version() -> str:
    return lib.hntl_version().decode()


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _in_use(stream, *tensors):
    """Mark tensors that this binding allocated (or caches) as used by `stream`
    when the call runs on a stream other than the current one, so that the
    caching allocator does not hand their memory to other work (a cached
    workspace replaced by a larger one, an output the caller drops) before
    that stream's queued kernels are done with it."""
    if stream is None:
        return
    if stream.cuda_stream == torch.cuda.current_stream(getattr(stream, "device", None)).cuda_stream:
        return
    for t in tensors:
        if t is not None:
            t.record_stream(stream)


def _dev_tensor(t, dtype, shape, device, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)}")
    if t.device.index != device:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the index is on cuda:{device}")
    return t


class Index:
    """A device-resident HNTL index (owned by the library)."""

    def __init__(self, handle):
        self._h = handle
        d = IndexDesc()
        _check(lib.hntl_index_info(self._h, ctypes.byref(d)))
        self.desc = d
        self._ws = None

    @classmethod
    def load(cls, path: str, device: int = 0, precision: int = PREC_FP32) -> "Index":
        h = _P()
        _check(lib.hntl_index_load(os.fsencode(path), int(device), int(precision), ctypes.byref(h)))
        return cls(h)

    @classmethod
    def build(cls, X: torch.Tensor, G: int, r: int, precision: int = PREC_FP32, u=None, seed: int = 0,
              attr: torch.Tensor | None = None, max_iter: int = 0, n_train: int = 0, n_seed: int = 0,
              pca_iters: int = 0, max_grain_rows: int = 0, stream=None) -> "Index":
        """Build an index on the GPU from CUDA rows X [N, d] f32 (see hntl_index_build)."""
        if not X.is_cuda or X.dtype != torch.float32 or X.dim() != 2 or not X.is_contiguous():
            raise ValueError("X must be a contiguous CUDA float32 tensor [N, d]")
        N, d = X.shape
        dev = X.device.index
        if attr is not None:
            _dev_tensor(attr, torch.int64, (N,), dev, "attr")
        u_arr = None
        if u is not None:
            import numpy as np

            u_np = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
            if u_np.shape[0] < G:
                raise ValueError("need G uniform draws")
            u_arr = u_np
        prm = BuildParams(precision=precision, max_iter=max_iter, n_train=n_train, n_seed=n_seed,
                          pca_iters=pca_iters, max_grain_rows=max_grain_rows, seed=seed,
                          u=None if u_arr is None else u_arr.ctypes.data_as(_P),
                          d_attr=None if attr is None else attr.data_ptr())
        h = _P()
        _check(lib.hntl_index_build(_ptr(X), N, d, G, r, ctypes.byref(prm), dev, _stream(stream), ctypes.byref(h)))
        return cls(h)

    def grain_rows(self):
        import numpy as np

        out = np.zeros(int(self.desc.G), dtype=np.uint32)
        _check(lib.hntl_index_grain_rows(self._h, out.ctypes.data_as(_P)))
        return out

    def export(self):
        """Index arrays on the host, grain order (numpy): M, U, grain_off, ids, Z, rho."""
        import numpy as np

        d = self.desc
        M = np.zeros((d.G, d.d), dtype=np.float32)
        U = np.zeros((d.G, d.r, d.d), dtype=np.float32)
        off = np.zeros(d.G + 1, dtype=np.uint64)
        ids = np.zeros(d.n, dtype=np.uint32)
        Z = np.zeros((d.n, d.r), dtype=np.float32)
        rho = np.zeros(d.n, dtype=np.float32)
        _check(lib.hntl_index_export(self._h, *(a.ctypes.data_as(_P) for a in (M, U, off, ids, Z, rho))))
        return dict(M=M, U=U, grain_off=off.astype(np.int64), ids=ids, Z=Z, rho=rho, N=int(d.n), d=int(d.d),
                    G=int(d.G), r=int(d.r))

    @property
    def handle(self):
        return self._h

    @property
    def device(self) -> int:
        return int(self.desc.device)

    def close(self):
        if self._h is not None and self._h.value:
            lib.hntl_index_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        d = self.desc
        return {f: getattr(d, f) for f, _ in IndexDesc._fields_}

    def workspace_bytes(self, nq: int, k: int, C: int, nprobe: int) -> int:
        n = lib.hntl_search_workspace_bytes(self._h, nq, k, C, nprobe)
        if n == 0:
            raise HntlError(EINVAL, last_error())
        return int(n)

    def workspace(self, nbytes: int) -> torch.Tensor:
        """A cached device workspace of at least nbytes (256-byte aligned)."""
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=f"cuda:{self.device}")
        return self._ws

    def _caller_ws(self, ws, nbytes: int) -> torch.Tensor:
        if ws is None:
            return self.workspace(nbytes)
        if not ws.is_cuda or ws.dtype != torch.uint8 or ws.numel() < nbytes or not ws.is_contiguous():
            raise ValueError(f"ws must be a contiguous CUDA uint8 tensor of at least {nbytes} bytes")
        return ws

    def search(self, Q: torch.Tensor, k: int, C: int, nprobe: int, filters: torch.Tensor | None = None,
               return_pool: bool = False, return_probe: bool = False, stream=None, out=None, ws=None,
               mode: str = "B"):
        """Batched search of CUDA queries Q [nq, d] f32: mode "B" reranks the
        pool by exact L2 to the raw rows (hntl_search), mode "A" by L2 to the
        rows' reconstructions (hntl_search_mode_a; no probe output).

        Returns (ids i64 [nq, k], dist f32 [nq, k]); with return_pool also the
        pool (ids as int32 [nq, max(C, k)] holding the uint32 ids, so the
        0xFFFFFFFF pad reads as -1, and approximate distances f32); with
        return_probe also the probed grains int32 [nq, nprobe]. `ws` is a
        caller-owned uint8 device workspace (for concurrent searches on
        several streams, each with its own); by default the index's cached
        one is used, which searches on different streams must not share."""
        nq = int(Q.shape[0])
        d = int(self.desc.d)
        _dev_tensor(Q, torch.float32, (nq, d), self.device, "Q")
        if filters is not None:
            _dev_tensor(filters, torch.int64, (nq, 2), self.device, "filters")
        Ce = max(C, k)
        dev = Q.device
        if out is None:
            ids = torch.empty(nq, k, dtype=torch.int64, device=dev)
            dist = torch.empty(nq, k, dtype=torch.float32, device=dev)
        else:
            ids, dist = out
        pool_ids = torch.empty(nq, Ce, dtype=torch.int32, device=dev) if return_pool else None
        pool_d = torch.empty(nq, Ce, dtype=torch.float32, device=dev) if return_pool else None
        probe = torch.empty(nq, nprobe, dtype=torch.int32, device=dev) if return_probe else None
        nb = self.workspace_bytes(max(nq, 1), k, C, nprobe)
        own_ws = ws is None
        ws = self._caller_ws(ws, nb)
        _in_use(stream, ws if own_ws else None, *((ids, dist) if out is None else ()), pool_ids, pool_d, probe)
        if mode == "A":
            if return_probe:
                raise ValueError("mode A has no probe output")
            _check(lib.hntl_search_mode_a(self._h, _ptr(Q), nq, k, C, nprobe, _ptr(filters), _ptr(ws), ws.numel(),
                                          _ptr(ids), _ptr(dist), _ptr(pool_ids), _ptr(pool_d), _stream(stream)))
        elif mode == "B":
            _check(lib.hntl_search(self._h, _ptr(Q), nq, k, C, nprobe, _ptr(filters), _ptr(ws), ws.numel(),
                                   _ptr(ids), _ptr(dist), _ptr(pool_ids), _ptr(pool_d), _ptr(probe), _stream(stream)))
        else:
            raise ValueError("mode must be 'A' or 'B'")
        res = [ids, dist]
        if return_pool:
            res += [pool_ids, pool_d]
        if return_probe:
            res.append(probe)
        return tuple(res)

    def search_host(self, Q, k: int, C: int, nprobe: int, filters=None, stream=None, ws=None):
        """Host-buffer form: Q is a CPU float32 tensor (pinned for async copies);
        returns CPU (ids i64, dist f32). Copies happen inside the call. `ws`
        as for search (sized by hntl_search_host_workspace_bytes)."""
        nq, d = int(Q.shape[0]), int(self.desc.d)
        if Q.is_cuda or Q.dtype != torch.float32 or tuple(Q.shape) != (nq, d) or not Q.is_contiguous():
            raise ValueError("Q must be a contiguous CPU float32 tensor [nq, d]")
        if filters is not None and (filters.is_cuda or filters.dtype != torch.int64 or
                                    tuple(filters.shape) != (nq, 2) or not filters.is_contiguous()):
            raise ValueError("filters must be a contiguous CPU int64 tensor [nq, 2]")
        ids = torch.empty(nq, k, dtype=torch.int64, pin_memory=Q.is_pinned())
        dist = torch.empty(nq, k, dtype=torch.float32, pin_memory=Q.is_pinned())
        nb = int(lib.hntl_search_host_workspace_bytes(self._h, max(nq, 1), k, C, nprobe, int(filters is not None)))
        if nb == 0:
            raise HntlError(EINVAL, last_error())
        ws = self._caller_ws(ws, nb)
        _check(lib.hntl_search_host(self._h, _ptr(Q), nq, k, C, nprobe, _ptr(filters), _ptr(ws), ws.numel(),
                                    _ptr(ids), _ptr(dist), _stream(stream)))
        return ids, dist

    def route_noalloc(self, Q: torch.Tensor, nprobe: int, probe: torch.Tensor, probe_d: torch.Tensor,
                      stream=None):
        """Routing into caller-provided outputs with no workspace and no
        allocation inside the library (see hntl_route_noalloc)."""
        nq = int(Q.shape[0])
        _dev_tensor(Q, torch.float32, (nq, int(self.desc.d)), self.device, "Q")
        _dev_tensor(probe, torch.int32, (nq, nprobe), self.device, "probe")
        _dev_tensor(probe_d, torch.float32, (nq, nprobe), self.device, "probe_d")
        _check(lib.hntl_route_noalloc(self._h, _ptr(Q), nq, nprobe, _ptr(probe), _ptr(probe_d), _stream(stream)))
        return probe, probe_d

    def route(self, Q: torch.Tensor, nprobe: int, stream=None):
        nq = int(Q.shape[0])
        _dev_tensor(Q, torch.float32, (nq, int(self.desc.d)), self.device, "Q")
        probe = torch.empty(nq, nprobe, dtype=torch.int32, device=Q.device)
        pd = torch.empty(nq, nprobe, dtype=torch.float32, device=Q.device)
        nb = self.workspace_bytes(max(nq, 1), 1, 1, nprobe)
        ws = self.workspace(nb)
        _in_use(stream, ws, probe, pd)
        _check(lib.hntl_route(self._h, _ptr(Q), nq, nprobe, _ptr(ws), ws.numel(), _ptr(probe), _ptr(pd),
                              _stream(stream)))
        return probe, pd


lib.hntl_search_probes.argtypes = [_P, _P, _U32, _U32, _U32, _U32, _P, _P, _P, _SZ, _P, _P, _P, _P, _P]
lib.hntl_search_mode_a.argtypes = [_P, _P, _U32, _U32, _U32, _U32, _P, _P, _SZ, _P, _P, _P, _P, _P]
lib.hntl_device_status.argtypes = [_P, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
lib.hntl_router_create.argtypes = [ctypes.c_int, _U32, _U32, _U32, _U32, _U32, _P, _P, _P, _P, _P, _P,
                                   ctypes.POINTER(_P)]
lib.hntl_router_free.argtypes = [_P]
lib.hntl_router_free.restype = None
lib.hntl_router_params.argtypes = [_P] + [_P] * 6
lib.hntl_router_grads.argtypes = [_P] + [_P] * 6
lib.hntl_router_step.argtypes = [_P, _P, _P, _U32, ctypes.c_float, ctypes.c_float, ctypes.c_int, _P, _P]
lib.hntl_router_logits.argtypes = [_P, _P, _U32, _P, _P]
lib.hntl_router_set_graphs.argtypes = [_P, ctypes.c_int]
lib.hntl_router_status.argtypes = [_P]
lib.hntl_router_route_workspace_bytes.argtypes = [_P, _P, _U32, _U32]
lib.hntl_router_route_workspace_bytes.restype = _SZ
lib.hntl_router_route.argtypes = [_P, _P, _P, _U32, _U32, ctypes.c_float, _P, _SZ, _P, _P, _P]


def search_probes(index: Index, Q: torch.Tensor, probes: torch.Tensor, k: int, C: int, filters=None,
                  return_pool: bool = False, stream=None):
    """Mode B search with the given probed grains (int32 CUDA [nq, nprobe])."""
    nq, nprobe = int(probes.shape[0]), int(probes.shape[1])
    _dev_tensor(Q, torch.float32, (nq, int(index.desc.d)), index.device, "Q")
    _dev_tensor(probes, torch.int32, (nq, nprobe), index.device, "probes")
    if filters is not None:
        _dev_tensor(filters, torch.int64, (nq, 2), index.device, "filters")
    Ce = max(C, k)
    ids = torch.empty(nq, k, dtype=torch.int64, device=Q.device)
    dist = torch.empty(nq, k, dtype=torch.float32, device=Q.device)
    pid = torch.empty(nq, Ce, dtype=torch.int32, device=Q.device) if return_pool else None
    pd = torch.empty(nq, Ce, dtype=torch.float32, device=Q.device) if return_pool else None
    ws = index.workspace(index.workspace_bytes(max(nq, 1), k, C, nprobe))
    _in_use(stream, ws, ids, dist, pid, pd)
    _check(lib.hntl_search_probes(index.handle, _ptr(Q), nq, k, C, nprobe, _ptr(probes), _ptr(filters), _ptr(ws),
                                  ws.numel(), _ptr(ids), _ptr(dist), _ptr(pid), _ptr(pd), _stream(stream)))
    return (ids, dist, pid, pd) if return_pool else (ids, dist)


def device_status(index: Index, clear: bool = True) -> int:
    st = ctypes.c_int(0)
    lib.hntl_device_status(index.handle, ctypes.byref(st), int(clear))
    return int(st.value)


class Router:
    """Learned grain router (see hntl_router_* in include/hntl.h)."""

    def __init__(self, params, max_batch: int, device: int = 0):
        import numpy as np

        W1, b1, W2, b2, W3, b3 = [np.ascontiguousarray(p, dtype=np.float32) for p in params]
        if W1.ndim != 2 or W2.ndim != 2 or W3.ndim != 2:
            raise ValueError("W1, W2, W3 must be matrices")
        self.h1, self.d = W1.shape
        self.h2 = W2.shape[0]
        self.G = W3.shape[0]
        # the library reads each array at the sizes these imply
        if (W2.shape != (self.h2, self.h1) or W3.shape != (self.G, self.h2) or b1.shape != (self.h1,) or
                b2.shape != (self.h2,) or b3.shape != (self.G,)):
            raise ValueError("parameters must be W1 [h1, d], b1 [h1], W2 [h2, h1], b2 [h2], W3 [G, h2], b3 [G]")
        self.max_batch = int(max_batch)
        self.device = device
        self._keep = (W1, b1, W2, b2, W3, b3)
        h = _P()
        _check(lib.hntl_router_create(device, self.d, self.h1, self.h2, self.G, self.max_batch,
                                      *(a.ctypes.data_as(_P) for a in self._keep), ctypes.byref(h)))
        self._h = h
        self._ws = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.hntl_router_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _host(self, fn):
        import numpy as np

        shapes = [(self.h1, self.d), (self.h1,), (self.h2, self.h1), (self.h2,), (self.G, self.h2), (self.G,)]
        out = [np.zeros(s, dtype=np.float32) for s in shapes]
        _check(fn(self._h, *(a.ctypes.data_as(_P) for a in out)))
        return out

    def params(self):
        return self._host(lib.hntl_router_params)

    def grads(self):
        return self._host(lib.hntl_router_grads)

    def step(self, X: torch.Tensor, T: torch.Tensor, lr: float = 1e-3, wd: float = 0.01, update: bool = True,
             loss: torch.Tensor | None = None, stream=None):
        B = int(X.shape[0])
        _dev_tensor(X, torch.float32, (B, self.d), self.device, "X")
        _dev_tensor(T, torch.float32, (B, self.G), self.device, "T")
        if loss is not None:  # the loss kernel adds into loss[0] on the device
            _dev_tensor(loss, torch.float32, tuple(loss.shape), self.device, "loss")
            if loss.numel() < 1:
                raise ValueError("loss must hold at least one element")
        _check(lib.hntl_router_step(self._h, _ptr(X), _ptr(T), B, float(lr), float(wd), int(update), _ptr(loss),
                                    _stream(stream)))

    def set_graphs(self, enable: bool):
        """Run training steps through the captured CUDA graph (default) or as direct launches."""
        _check(lib.hntl_router_set_graphs(self._h, int(bool(enable))))

    def status(self) -> int:
        """0, or the error code of a GEMM pipeline wait that timed out (blocking)."""
        return lib.hntl_router_status(self._h)

    def logits(self, X: torch.Tensor, stream=None) -> torch.Tensor:
        B = int(X.shape[0])
        _dev_tensor(X, torch.float32, (B, self.d), self.device, "X")
        out = torch.empty(B, self.G, dtype=torch.float32, device=X.device)
        _in_use(stream, out)
        _check(lib.hntl_router_logits(self._h, _ptr(X), B, _ptr(out), _stream(stream)))
        return out

    def route(self, index: Index, Q: torch.Tensor, nprobe: int, tau: float = 0.5, stream=None):
        """(probes int32 [nq, nprobe], number of queries that fell back to centroid routing)."""
        nq = int(Q.shape[0])
        _dev_tensor(Q, torch.float32, (nq, self.d), self.device, "Q")
        nb = int(lib.hntl_router_route_workspace_bytes(self._h, index.handle, max(nq, 1), nprobe))
        if nb == 0:
            raise HntlError(EINVAL, last_error())
        if self._ws is None or self._ws.numel() < nb:
            self._ws = torch.empty(nb, dtype=torch.uint8, device=Q.device)
        probe = torch.empty(nq, nprobe, dtype=torch.int32, device=Q.device)
        nfb = torch.zeros(1, dtype=torch.int32, device=Q.device)
        _in_use(stream, self._ws, probe, nfb)
        _check(lib.hntl_router_route(self._h, index.handle, _ptr(Q), nq, nprobe, float(tau), _ptr(self._ws),
                                     self._ws.numel(), _ptr(probe), _ptr(nfb), _stream(stream)))
        return probe, nfb


lib.hntl_selftest_wait_timeout.argtypes = [_P, _U32, _P]
lib.hntl_server_create.argtypes = [_P, _SZ, _U32, _U32, _U32, _U32, _U32, ctypes.POINTER(_P)]
lib.hntl_server_free.argtypes = [_P]
lib.hntl_server_free.restype = None
lib.hntl_server_submit.argtypes = [_P, _P, _U32, _P, _P, _P, _P, _P, ctypes.POINTER(_U32)]
lib.hntl_server_poll.argtypes = [_P, ctypes.c_uint64, _P, _P, _U32]
lib.hntl_server_reset_stats.argtypes = [_P]
lib.hntl_server_poll_many.argtypes = [_P, _P, _U32, _P, _P, _U32, _P, _U32, ctypes.POINTER(_U32)]
lib.hntl_server_replay.argtypes = [_P, _P, _U32, _P, _P, _P, _P, _P, _P, _U32, ctypes.POINTER(_U32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64), ("mean_batch", ctypes.c_double),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("max_us", ctypes.c_double),
                ("slots", ctypes.c_uint32), ("lag_p50_us", ctypes.c_double), ("lag_p99_us", ctypes.c_double),
                ("queue_p50_us", ctypes.c_double), ("queue_p99_us", ctypes.c_double),
                ("service_p50_us", ctypes.c_double), ("service_p99_us", ctypes.c_double),
                ("upload_p50_us", ctypes.c_double), ("upload_p99_us", ctypes.c_double)]


lib.hntl_server_get_stats.argtypes = [_P, ctypes.POINTER(ServerStats)]


lib.hntl_search_survivors.argtypes = [_P, _P, _SZ, _U32, _U32, _U32, _P, _P]


def search_survivors(index: Index, ws: torch.Tensor, nq: int, C: int, nprobe: int) -> torch.Tensor:
    """Pool survivors per query of the last search run in workspace `ws` (see hntl_search_survivors)."""
    out = torch.empty(nq, dtype=torch.int32, device=ws.device)
    _check(lib.hntl_search_survivors(index.handle, _ptr(ws), ws.numel(), nq, C, nprobe, _ptr(out), None))
    return out


lib.hntl_search_scan_stats.argtypes = [_P, _P, _SZ, _U32, _U32, _U32, _P, _P]
lib.hntl_debug_set_persistent_cap.argtypes = [_U32]
lib.hntl_search_pair_codes.argtypes = [_P, _P, _SZ, _U32, _U32, _U32, _P, _P, _P]
lib.hntl_search_pair_proj.argtypes = [_P, _P, _SZ, _U32, _U32, _U32, _P, _P, _P]


def search_pair_proj(index: Index, ws: torch.Tensor, nq: int, C: int, nprobe: int):
    """Projection output z_q [nq, nprobe, r] and rho_q [nq, nprobe] (FP32) of the last search run in workspace
    `ws`, in query order (see hntl_search_pair_proj)."""
    r = int(index.desc.r)
    z = torch.zeros(nq, nprobe, r, dtype=torch.float32, device=ws.device)
    rho = torch.zeros(nq, nprobe, dtype=torch.float32, device=ws.device)
    _check(lib.hntl_search_pair_proj(index.handle, _ptr(ws), ws.numel(), nq, C, nprobe, _ptr(z), _ptr(rho), None))
    return z, rho


def search_pair_codes(index: Index, ws: torch.Tensor, nq: int, C: int, nprobe: int):
    """16-bit form: query codes [nq, nprobe, r] int16 and residual codes [nq, nprobe] int32 (-1 = left out) of
    the last search run in workspace `ws` (see hntl_search_pair_codes)."""
    r = int(index.desc.r)
    codes = torch.zeros(nq, nprobe, r, dtype=torch.int16, device=ws.device)
    rc = torch.zeros(nq, nprobe, dtype=torch.int32, device=ws.device)
    _check(lib.hntl_search_pair_codes(index.handle, _ptr(ws), ws.numel(), nq, C, nprobe, _ptr(codes), _ptr(rc), None))
    return codes, rc


def search_scan_stats(index: Index, ws: torch.Tensor, nq: int, C: int, nprobe: int) -> dict:
    """Scan work-item counters of the last search run in workspace `ws` (see hntl_search_scan_stats)."""
    out = torch.zeros(5, dtype=torch.int32, device=ws.device)
    _check(lib.hntl_search_scan_stats(index.handle, _ptr(ws), ws.numel(), nq, C, nprobe, _ptr(out), None))
    v = [int(x) for x in out.cpu().tolist()]
    return dict(dense_claimed=v[0], dense=v[1], sparse_light=v[2], sparse_claimed=v[3], sparse_heavy=v[4])


def set_persistent_cap(ctas: int):
    """Cap every persistent kernel's grid at `ctas` CTAs (0 = default); a test hook."""
    _check(lib.hntl_debug_set_persistent_cap(int(ctas)))


def selftest_wait_timeout(index: Index, polls: int = 64):
    _check(lib.hntl_selftest_wait_timeout(index.handle, int(polls), None))


class Server:
    """Continuous-batching server over an index (see hntl_server_* in include/hntl.h)."""

    def __init__(self, index: Index, mem_budget: int, max_slots: int, batch: int, nprobe: int, k_max: int,
                 C_max: int):
        h = _P()
        _check(lib.hntl_server_create(index.handle, int(mem_budget), max_slots, batch, nprobe, k_max, C_max,
                                      ctypes.byref(h)))
        self._h = h
        self.index = index
        self.d = int(index.desc.d)
        self.k_max = int(k_max)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.hntl_server_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, Q, k, C, ranges=None, arrival_ns=None):
        """Admit requests (numpy: Q [n, d] f32, k [n], C [n] uint32, ranges [n, 2] int64, arrival_ns [n]
        int64). Returns the tickets of the admitted prefix (length < n when slots ran out)."""
        import numpy as np

        Q = np.ascontiguousarray(Q, dtype=np.float32)
        n = Q.shape[0]
        k = np.ascontiguousarray(k, dtype=np.uint32)
        C = np.ascontiguousarray(C, dtype=np.uint32)
        R = None if ranges is None else np.ascontiguousarray(ranges, dtype=np.int64)
        A = None if arrival_ns is None else np.ascontiguousarray(arrival_ns, dtype=np.int64)
        # the library reads n rows of each: shapes are checked here
        if Q.shape != (n, self.d) or k.shape != (n,) or C.shape != (n,):
            raise ValueError(f"Q must be [n, {self.d}] and k, C [n]")
        if (R is not None and R.shape != (n, 2)) or (A is not None and A.shape != (n,)):
            raise ValueError("ranges must be [n, 2] and arrival_ns [n]")
        tickets = np.zeros(n, dtype=np.uint64)
        got = ctypes.c_uint32(0)
        rc = lib.hntl_server_submit(self._h, Q.ctypes.data_as(_P), n, k.ctypes.data_as(_P), C.ctypes.data_as(_P),
                                    None if R is None else R.ctypes.data_as(_P),
                                    None if A is None else A.ctypes.data_as(_P), tickets.ctypes.data_as(_P),
                                    ctypes.byref(got))
        if rc not in (OK, EBUSY):
            raise HntlError(rc, last_error())
        return tickets[: got.value]

    def replay(self, Q, k, C, arrival_ns, ranges=None, want=None, timeout_ms=600000):
        """Open-loop replay inside the library: request i is submitted at
        arrival_ns[i] nanoseconds after the call starts (non-decreasing).
        Returns (n_done, ids): ids int64 [n, k_max] holds the results of the
        rows with want[i] != 0 (zeros elsewhere), or None when want is None.
        Raises on a submission error; n_done < n after a timeout."""
        import numpy as np

        Q = np.ascontiguousarray(Q, dtype=np.float32)
        n = Q.shape[0]
        k = np.ascontiguousarray(k, dtype=np.uint32)
        C = np.ascontiguousarray(C, dtype=np.uint32)
        A = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        R = None if ranges is None else np.ascontiguousarray(ranges, dtype=np.int64)
        W = None if want is None else np.ascontiguousarray(want, dtype=np.uint8)
        if Q.shape != (n, self.d) or k.shape != (n,) or C.shape != (n,) or A.shape != (n,):
            raise ValueError(f"Q must be [n, {self.d}] and k, C, arrival_ns [n]")
        if (R is not None and R.shape != (n, 2)) or (W is not None and W.shape != (n,)):
            raise ValueError("ranges must be [n, 2] and want [n]")
        if n > 1 and np.any(np.diff(A) < 0):
            raise ValueError("arrival_ns must not decrease")
        ids = None if W is None else np.zeros((n, self.k_max), dtype=np.int64)
        got = ctypes.c_uint32(0)
        rc = lib.hntl_server_replay(self._h, Q.ctypes.data_as(_P), n, k.ctypes.data_as(_P), C.ctypes.data_as(_P),
                                    None if R is None else R.ctypes.data_as(_P), A.ctypes.data_as(_P),
                                    None if W is None else W.ctypes.data_as(_P),
                                    None if ids is None else ids.ctypes.data_as(_P), int(timeout_ms),
                                    ctypes.byref(got))
        if rc not in (OK, ETIMEOUT):
            raise HntlError(rc, last_error())
        return got.value, ids

    def poll(self, ticket, k, timeout_ms=10000):
        """(ids int64 [k], dist f32 [k]) of a request submitted with this k,
        or None on timeout."""
        import numpy as np

        # room for the request's own k (up to k_max), whatever k the caller passes
        ids = np.zeros(max(int(k), self.k_max), dtype=np.int64)
        dist = np.zeros(max(int(k), self.k_max), dtype=np.float32)
        rc = lib.hntl_server_poll(self._h, int(ticket), ids.ctypes.data_as(_P), dist.ctypes.data_as(_P),
                                  int(timeout_ms))
        if rc == ETIMEOUT:
            return None
        _check(rc)
        return ids[:k], dist[:k]

    def poll_many(self, tickets, done, ids=None, dist=None, timeout_ms=0):
        """Collect every completed request among `tickets` (numpy uint64) whose
        `done` flag (numpy uint8, updated in place) is 0; ids / dist (numpy
        [n, k_max] int64 / float32) receive the rows, or None to discard.
        Returns the number collected by this call."""
        import numpy as np

        n = len(tickets)
        if tickets.dtype != np.uint64 or not tickets.flags.c_contiguous or tickets.ndim != 1:
            raise ValueError("tickets must be a contiguous uint64 vector")
        if done.dtype != np.uint8 or not done.flags.c_contiguous or done.shape != (n,):
            raise ValueError("done must be a contiguous uint8 vector as long as tickets")
        stride = 0 if ids is None and dist is None else (ids if ids is not None else dist).shape[1]
        for a, dt in ((ids, np.int64), (dist, np.float32)):
            if a is not None and (a.dtype != dt or not a.flags.c_contiguous or a.ndim != 2 or a.shape[0] < n or
                                  a.shape[1] != stride):
                raise ValueError("ids / dist must be contiguous [len(tickets), stride] int64 / float32")
        got = ctypes.c_uint32(0)
        rc = lib.hntl_server_poll_many(self._h, tickets.ctypes.data_as(_P), len(tickets),
                                       None if ids is None else ids.ctypes.data_as(_P),
                                       None if dist is None else dist.ctypes.data_as(_P), stride,
                                       done.ctypes.data_as(_P), int(timeout_ms), ctypes.byref(got))
        if rc not in (OK, ETIMEOUT):
            raise HntlError(rc, last_error())
        return got.value

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib.hntl_server_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def reset_stats(self):
        _check(lib.hntl_server_reset_stats(self._h))


# ---------------------------------------------------------------- grain shards

lib.hntl_shard_assign.argtypes = [_P, _U32, _U32, _P]
lib.hntl_index_shard.argtypes = [_P, _P, _U32, ctypes.c_int, ctypes.POINTER(_P)]
lib.hntl_shard_global_ids.argtypes = [_P, _P, ctypes.c_uint64, _P]
lib.hntl_merge_topk.argtypes = [_P, _P, _U32, _U32, _U32, _P, _P, _P]
lib.hntl_merge_topk_host.argtypes = [_P, _P, _U32, _U32, _U32, _P, _P]


def shard_assign(grain_rows, S: int):
    """Shard of every grain, size-balanced by rows (see hntl_shard_assign): uint32 [G]."""
    import numpy as np

    rows = np.ascontiguousarray(np.asarray(grain_rows, dtype=np.uint32))
    out = np.zeros(len(rows), dtype=np.uint32)
    _check(lib.hntl_shard_assign(rows.ctypes.data_as(_P), len(rows), int(S), out.ctypes.data_as(_P)))
    return out


def index_shard(index: Index, shard_of_grain, shard: int, device: int | None = None) -> Index:
    """Shard `shard` of `index` on `device` (default: the index's device); see hntl_index_shard."""
    import numpy as np

    sog = np.ascontiguousarray(np.asarray(shard_of_grain, dtype=np.uint32))
    if sog.shape != (int(index.desc.G),):
        raise ValueError("shard_of_grain must hold one shard per grain")
    h = _P()
    dev = index.device if device is None else int(device)
    _check(lib.hntl_index_shard(index.handle, sog.ctypes.data_as(_P), int(shard), dev, ctypes.byref(h)))
    return Index(h)


def shard_global_ids(shard: Index, ids: torch.Tensor, stream=None) -> torch.Tensor:
    """Replace a shard's local ids (CUDA int64, any shape, on the shard's device) by original ids, in place."""
    if not ids.is_cuda or ids.dtype != torch.int64 or not ids.is_contiguous() or ids.device.index != shard.device:
        raise ValueError("ids must be a contiguous CUDA int64 tensor on the shard's device")
    with torch.cuda.device(ids.device):
        _in_use(stream, ids)
        _check(lib.hntl_shard_global_ids(shard.handle, _ptr(ids), ids.numel(), _stream(stream)))
    return ids


def merge_topk(ids: torch.Tensor, dist: torch.Tensor, stream=None):
    """The k best by (distance, id) over S lists per query: ids int64 / dist f32 [S, nq, k] (CUDA, one
    device) -> ([nq, k], [nq, k]); see hntl_merge_topk."""
    if ids.dim() != 3 or ids.shape != dist.shape:
        raise ValueError("ids and dist must both be [S, nq, k]")
    S, nq, k = (int(x) for x in ids.shape)
    _dev_tensor(ids, torch.int64, (S, nq, k), ids.device.index, "ids")
    _dev_tensor(dist, torch.float32, (S, nq, k), ids.device.index, "dist")
    oi = torch.empty(nq, k, dtype=torch.int64, device=ids.device)
    od = torch.empty(nq, k, dtype=torch.float32, device=ids.device)
    _in_use(stream, ids, dist, oi, od)
    with torch.cuda.device(ids.device):
        _check(lib.hntl_merge_topk(_ptr(ids), _ptr(dist), S, nq, k, _ptr(oi), _ptr(od), _stream(stream)))
    return oi, od


def merge_topk_host(ids, dist):
    """hntl_merge_topk_host on host arrays [S, nq, k] (numpy or CPU tensors) -> numpy ([nq, k], [nq, k])."""
    import numpy as np

    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.int64))
    dist = np.ascontiguousarray(np.asarray(dist, dtype=np.float32))
    if ids.ndim != 3 or ids.shape != dist.shape:
        raise ValueError("ids and dist must both be [S, nq, k]")
    S, nq, k = ids.shape
    oi = np.zeros((nq, k), dtype=np.int64)
    od = np.zeros((nq, k), dtype=np.float32)
    _check(lib.hntl_merge_topk_host(ids.ctypes.data_as(_P), dist.ctypes.data_as(_P), S, nq, k,
                                    oi.ctypes.data_as(_P), od.ctypes.data_as(_P)))
    return oi, od


def exchange_merge(ids: torch.Tensor, dist: torch.Tensor, group=None):
    """One rank's top k (original ids, [nq, k]) against every rank's: one all-gather of k (id, distance)
    per query over the process group, then the merge (hntl_merge_topk for CUDA tensors,
    hntl_merge_topk_host for CPU tensors). Every rank returns the merged [nq, k]."""
    import torch.distributed as dist_

    W = dist_.get_world_size(group)
    gi = [torch.empty_like(ids) for _ in range(W)]
    gd = [torch.empty_like(dist) for _ in range(W)]
    dist_.all_gather(gi, ids.contiguous(), group=group)
    dist_.all_gather(gd, dist.contiguous(), group=group)
    si, sd = torch.stack(gi), torch.stack(gd)
    if si.is_cuda:
        return merge_topk(si, sd)
    oi, od = merge_topk_host(si.numpy(), sd.numpy())
    return torch.from_numpy(oi), torch.from_numpy(od)


class ShardedIndex:
    """An index split into S grain shards (hntl_index_shard), each on its own device (or all on one).
    search() runs every shard's search on its device, maps its ids back and merges on the first
    shard's device."""

    def __init__(self, index: Index, S: int, devices=None):
        self.shard_of_grain = shard_assign(index.grain_rows(), S)
        devices = [index.device] * S if devices is None else list(devices)
        if len(devices) != S:
            raise ValueError("one device per shard")
        self.shards = [index_shard(index, self.shard_of_grain, s, devices[s]) for s in range(S)]

    def search(self, Q: torch.Tensor, k: int, C: int, nprobe: int, return_local: bool = False):
        dev0 = torch.device(f"cuda:{self.shards[0].device}")
        loc = []
        for sh in self.shards:
            with torch.cuda.device(sh.device):
                q = Q.to(f"cuda:{sh.device}")
                i, d = sh.search(q, k, C, nprobe)
                shard_global_ids(sh, i)
                torch.cuda.current_stream().synchronize()
            loc.append((i.to(dev0), d.to(dev0)))
        si = torch.stack([a for a, _ in loc])
        sd = torch.stack([b for _, b in loc])
        with torch.cuda.device(dev0):
            out = merge_topk(si, sd)
        return (out, (si, sd)) if return_local else out
