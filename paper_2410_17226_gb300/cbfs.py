"""Python binding of libcbfs.so (include/cbfs.h): argument marshalling only.

Every step of the traversal and of the query runs in the CUDA library; this
module only converts arrays and tensors into pointers and sizes.  PyTorch
supplies device memory and streams.  There is no CPU fallback: when
libcbfs.so is missing or CUDA is unavailable, every entry point raises.

Device buffers are torch tensors.  64-bit subset words are stored in
``torch.int64`` tensors (same bits as the C ABI's uint64_t) and query answers
in ``torch.int16`` tensors (same bits as uint16_t); ``as_numpy_u64`` /
``as_numpy_u16`` reinterpret them on the host.
"""
from __future__ import annotations

import ctypes
import os
import weakref
from typing import Sequence

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcbfs.so")

OK = 0
E_INVALID, E_DIAMETER, E_DEPTH, E_NOMEM, E_TIMEOUT, E_CUDA, E_GRAPH = -1, -2, -3, -4, -5, -6, -7
NO_PATH = 0xFFFF
UNREACHED = 0xFF


class CbfsError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().cbfs_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg}")
        self.code = code


class Tune(ctypes.Structure):
    _fields_ = [("pull_alpha", ctypes.c_float), ("slots", ctypes.c_int), ("dense_div", ctypes.c_int),
                ("host_loop", ctypes.c_int), ("small_deg", ctypes.c_int), ("mid_deg", ctypes.c_int),
                ("sparse_mid_deg", ctypes.c_int), ("wave_order", ctypes.c_int), ("fused_pull", ctypes.c_int),
                ("stage_rounds", ctypes.c_int), ("pack", ctypes.c_int)]


class KernelTimes(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64 * 3), ("ms", ctypes.c_double * 3), ("total_launches", ctypes.c_uint64)]


KERNEL_KINDS = ("setup", "vertex_phase", "edge_phase")


class ClusterStats(ctypes.Structure):
    _fields_ = [("frontier_appearances", ctypes.c_uint64), ("arcs_scanned", ctypes.c_uint64),
                ("reached_arcs", ctypes.c_uint64), ("rounds", ctypes.c_uint64)]


_lib = None

# name -> (restype, argtypes) for every symbol declared in include/cbfs.h
_P, _I, _I64, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
SIGNATURES = {
    "cbfs_graph_create": (_I, [_I64, _P, _I, _P, _I64, _I, _I, _P, _P]),
    "cbfs_graph_destroy": (_I, [_P]),
    "cbfs_graph_info": (_I, [_P, _P, _P]),
    "cbfs_run": (_I, [_P, _P, _I, _I, _P, _P, _P]),
    "cbfs_run_batched": (_I, [_P, _P, _P, _I, _I, _P, _P, _P, _P]),
    "cbfs_run_batched_labels": (_I, [_P, _P, _P, _I, _I, _P, _P, _P, _P, _P]),
    "cbfs_run_noalloc": (_I, [_I64, _P, _P, _I64, _P, _I, _I, _P, _P, _P]),
    "cbfs_output_stats": (_I, [_P, _P, _P, _P, _I, _I, _P, _P]),
    "cbfs_profile": (_I, [_P, _I, _P]),
    "cbfs_labels_create": (_I, [_I64, _I, _I, _SZ, _P]),
    "cbfs_labels_create_w": (_I, [_I64, _I, _I, _I, _SZ, _P]),
    "cbfs_labels_destroy": (_I, [_P]),
    "cbfs_labels_append": (_I, [_P, _P, _P, _P, _I, _P]),
    "cbfs_labels_reset": (_I, [_P]),
    "cbfs_labels_count": (_I, [_P, _P]),
    "cbfs_labels_rows": (_I, [_P, _P, _P]),
    "cbfs_query_distance": (_I, [_P, _P, _I64, _P, _P]),
    "cbfs_query_local": (_I, [_P, _P, _P, _I64, _I, _P, _P]),
    "cbfs_labels_status": (_I, [_P, _P]),
    "cbfs_graph_status": (_I, [_P, _P]),
    "cbfs_sync_status": (_I, [_P]),
    "cbfs_status_string": (ctypes.c_char_p, [_I]),
    "cbfs_server_create": (_I, [_P, _I64, _I, _SZ, _P]),
    "cbfs_server_submit": (_I, [_P, _P, _I64, _P, _P]),
    "cbfs_server_wait": (_I, [_P, ctypes.c_uint64, ctypes.c_double]),
    "cbfs_server_stats": (_I, [_P, _P, _P, _I64, _P]),
    "cbfs_server_destroy": (_I, [_P]),
    "cbfs_host_alloc": (_I, [_SZ, _P]),
    "cbfs_host_free": (_I, [_P]),
}


def lib():
    """Loads libcbfs.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != OK:
        raise CbfsError(rc, where)


def _require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("the C-BFS library needs a CUDA GPU; there is no CPU path")


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t: torch.Tensor) -> int:
    return int(t.data_ptr())


def _host_i32(a) -> np.ndarray:
    if isinstance(a, torch.Tensor):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def pinned_empty(shape, dtype: torch.dtype) -> torch.Tensor:
    """Uninitialised page-locked host tensor from ``cbfs_host_alloc``; the
    memory is returned with ``cbfs_host_free`` once no tensor uses it."""
    count = 1
    for x in (shape if isinstance(shape, (tuple, list)) else (shape,)):
        count *= int(x)
    nbytes = max(count * torch.empty((), dtype=dtype).element_size(), 1)
    p = ctypes.c_void_p()
    _check(lib().cbfs_host_alloc(nbytes, ctypes.byref(p)), "cbfs_host_alloc")
    buf = (ctypes.c_uint8 * nbytes).from_address(p.value)
    weakref.finalize(buf, lib().cbfs_host_free, ctypes.c_void_p(p.value))
    return torch.frombuffer(buf, dtype=torch.uint8)[:count * torch.empty((), dtype=dtype).element_size()].view(
        dtype).view(*(shape if isinstance(shape, (tuple, list)) else (shape,)))


def as_numpy_u64(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64)


def as_numpy_u16(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint16)


class Graph:
    """A CSR graph resident on the GPU (``cbfs_graph_create``).

    ``off``/``adj`` may be NumPy arrays or CPU tensors (copied from host) or
    CUDA tensors (copied device to device).  ``off`` int64 or int32, ``adj``
    int32.
    """

    def __init__(self, off, adj, validate: bool = True, stream=None):
        _require_cuda()
        self._h = ctypes.c_void_p()
        on_dev = isinstance(off, torch.Tensor) and off.is_cuda
        if on_dev:
            off_t = off.contiguous()
            adj_t = adj.to(torch.int32).contiguous()
            is64 = off_t.dtype == torch.int64
            if not is64:
                off_t = off_t.to(torch.int32)
            n, nnz = off_t.numel() - 1, adj_t.numel()
            keep = (off_t, adj_t)
            p_off, p_adj = _ptr(off_t), _ptr(adj_t) if nnz else None
        else:
            if isinstance(off, torch.Tensor):
                off, adj = off.numpy(), adj.numpy()
            off_a = np.ascontiguousarray(off)
            is64 = off_a.dtype == np.int64
            off_a = off_a.astype(np.int64 if is64 else np.int32, copy=False)
            adj_a = np.ascontiguousarray(adj, dtype=np.int32)
            n, nnz = off_a.size - 1, adj_a.size
            keep = (off_a, adj_a)
            p_off = off_a.ctypes.data
            p_adj = adj_a.ctypes.data if nnz else None
        rc = lib().cbfs_graph_create(n, p_off, int(is64), p_adj, nnz, int(on_dev), int(validate),
                                     _stream_ptr(stream), ctypes.byref(self._h))
        del keep
        _check(rc, "cbfs_graph_create")
        self.n, self.nnz = int(n), int(nnz)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().cbfs_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- traversal -----------------------------------------------------------
    # The traversal calls are stream-ordered in the C ABI.  With check=True
    # (the default) the binding then waits for the stream and raises on an
    # error the kernels detected (cbfs_graph_status); with check=False it
    # returns at once and such errors come from status() or sync_status().
    def _checked(self, rc: int, where: str, check: bool, stream):
        _check(rc, where)
        if check:
            _check(lib().cbfs_graph_status(self._h, _stream_ptr(stream)), where)

    def status(self, stream=None) -> int:
        """``cbfs_graph_status``: waits for ``stream``, returns and clears the
        handle's device status word."""
        return int(lib().cbfs_graph_status(self._h, _stream_ptr(stream)))

    def run(self, sources, d: int, dist: torch.Tensor | None = None, masks: torch.Tensor | None = None,
            stream=None, check: bool = True):
        """One C-BFS (``cbfs_run``).  Returns ``(dist uint8[n], masks int64[d, n])``."""
        S = _host_i32(sources)
        dev = torch.device("cuda", torch.cuda.current_device())
        if dist is None:
            dist = torch.empty(self.n, dtype=torch.uint8, device=dev)
        if masks is None:
            masks = torch.empty((max(d, 0), self.n), dtype=torch.int64, device=dev)
        rc = lib().cbfs_run(self._h, S.ctypes.data, int(S.size), int(d), _ptr(dist),
                            _ptr(masks) if d > 0 else None, _stream_ptr(stream))
        self._checked(rc, "cbfs_run", check, stream)
        return dist, masks

    @staticmethod
    def _cluster_layout(clusters, sources_concat, cluster_off):
        if clusters is None:
            return _host_i32(sources_concat), _host_i32(cluster_off)
        arrs = [_host_i32(c) for c in clusters]
        coff = np.zeros(len(arrs) + 1, dtype=np.int32)
        np.cumsum([a.size for a in arrs], out=coff[1:])
        src = np.concatenate(arrs).astype(np.int32) if arrs else np.zeros(0, np.int32)
        return src, coff

    @staticmethod
    def _tune(tune: dict | None) -> "Tune":
        t = Tune()
        if tune:
            t.pull_alpha = float(tune.get("pull_alpha", 0.0))
            t.slots = int(tune.get("slots", 0))
            t.dense_div = int(tune.get("dense_div", 0))
            t.host_loop = int(tune.get("host_loop", 0))
            t.small_deg = int(tune.get("small_deg", 0))
            t.mid_deg = int(tune.get("mid_deg", 0))
            t.sparse_mid_deg = int(tune.get("sparse_mid_deg", 0))
            t.wave_order = int(tune.get("wave_order", 0))
            t.fused_pull = int(tune.get("fused_pull", 0))
            t.stage_rounds = int(tune.get("stage_rounds", 0))
            t.pack = int(tune.get("pack", 0))
        return t

    def run_batched(self, clusters: Sequence | None, d: int, dist: torch.Tensor | None = None,
                    masks: torch.Tensor | None = None, tune: dict | None = None, stream=None,
                    sources_concat=None, cluster_off=None, check: bool = True):
        """C clusters in one call (``cbfs_run_batched``).  ``clusters`` is a list
        of source arrays; alternatively pass ``sources_concat`` and
        ``cluster_off`` (the C ABI's layout) with ``clusters=None``.  ``dist``
        and ``masks`` may be CUDA tensors or host tensors (pinned ones let the
        copies overlap the traversal).  Returns ``(dist uint8[C, n],
        masks int64[C, d, n])``, allocated on the GPU when not given."""
        src, coff = self._cluster_layout(clusters, sources_concat, cluster_off)
        C = coff.size - 1
        dev = torch.device("cuda", torch.cuda.current_device())
        if dist is None:
            dist = torch.empty((C, self.n), dtype=torch.uint8, device=dev)
        if masks is None:
            masks = torch.empty((C, max(d, 0), self.n), dtype=torch.int64, device=dev)
        t = self._tune(tune)
        src_p = src.ctypes.data if src.size else np.zeros(1, np.int32).ctypes.data
        rc = lib().cbfs_run_batched(self._h, src_p, coff.ctypes.data, int(C), int(d), _ptr(dist),
                                    _ptr(masks) if d > 0 else None, ctypes.byref(t), _stream_ptr(stream))
        self._checked(rc, "cbfs_run_batched", check, stream)
        return dist, masks

    def run_batched_labels(self, clusters: Sequence | None, d: int, labels: "Labels", dist: torch.Tensor | None = None,
                           masks: torch.Tensor | None = None, tune: dict | None = None, stream=None,
                           sources_concat=None, cluster_off=None):
        """``cbfs_run_batched_labels``: the batched traversal that also appends
        every cluster to ``labels`` from the device-side wave outputs.
        ``dist``/``masks`` are optional (None = labels only) and may be CUDA
        or host tensors."""
        src, coff = self._cluster_layout(clusters, sources_concat, cluster_off)
        C = coff.size - 1
        t = self._tune(tune)
        src_p = src.ctypes.data if src.size else np.zeros(1, np.int32).ctypes.data
        rc = lib().cbfs_run_batched_labels(self._h, src_p, coff.ctypes.data, int(C), int(d),
                                           _ptr(dist) if dist is not None else None,
                                           _ptr(masks) if (masks is not None and d > 0) else None, labels._h,
                                           ctypes.byref(t), _stream_ptr(stream))
        _check(rc, "cbfs_run_batched_labels")
        return dist, masks

    def query_local(self, pairs: torch.Tensor, tau: int, labels: "Labels | None" = None,
                    out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """``cbfs_query_local``: the bounded bidirectional search of Appendix B
        (balls of at most ``tau`` vertices, whole BFS levels) fused with the
        label query of ``labels`` when given.  pairs: CUDA int32 [q, 2];
        returns int16 [q] holding the uint16 answers."""
        q = pairs.shape[0] if pairs.dim() == 2 else pairs.numel() // 2
        if out is None:
            out = torch.empty(q, dtype=torch.int16, device=pairs.device)
        rc = lib().cbfs_query_local(labels._h if labels is not None else None, self._h, _ptr(pairs) if q else None,
                                    int(q), int(tau), _ptr(out) if q else None, _stream_ptr(stream))
        _check(rc, "cbfs_query_local")
        return out

    def profile(self, enable: bool) -> dict:
        """Reads and resets the kernel accounting (``cbfs_profile``); ``enable``
        switches CUDA-event timing of each traversal kernel on or off."""
        kt = KernelTimes()
        _check(lib().cbfs_profile(self._h, int(enable), ctypes.byref(kt)), "cbfs_profile")
        out = {k: {"launches": int(kt.launches[i]), "ms": float(kt.ms[i])} for i, k in enumerate(KERNEL_KINDS)}
        out["total_launches"] = int(kt.total_launches)
        return out

    def output_stats(self, dist: torch.Tensor, masks: torch.Tensor, ks, d: int, stream=None) -> np.ndarray:
        """Work counters per cluster (``cbfs_output_stats``): int64 [C, 4] =
        (frontier appearances V, arcs scanned A, reached arcs, rounds)."""
        ks = _host_i32(ks)
        C = ks.size
        out = (ClusterStats * max(C, 1))()
        rc = lib().cbfs_output_stats(self._h, _ptr(dist), _ptr(masks) if d > 0 else None, ks.ctypes.data, C, int(d),
                                     ctypes.cast(out, ctypes.c_void_p), _stream_ptr(stream))
        _check(rc, "cbfs_output_stats")
        return np.array([[o.frontier_appearances, o.arcs_scanned, o.reached_arcs, o.rounds] for o in out[:C]],
                        dtype=np.int64).reshape(C, 4)


def _check_noalloc_args(off, adj, d, dist, masks):
    """Types, sizes and devices of run_noalloc's tensors (ValueError)."""
    named = {"off": off, "adj": adj, "dist": dist}
    if d > 0:
        named["masks"] = masks
    want = {"off": torch.int64, "adj": torch.int32, "dist": torch.uint8, "masks": torch.int64}
    for name, t in named.items():
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"run_noalloc: {name} must be a torch.Tensor")
        if t.dtype != want[name]:
            raise ValueError(f"run_noalloc: {name} must be {want[name]}, got {t.dtype}")
    if off.dim() != 1 or off.numel() < 2:
        raise ValueError("run_noalloc: off must be 1-D with n + 1 >= 2 entries")
    if adj.dim() != 1:
        raise ValueError("run_noalloc: adj must be 1-D")
    n = off.numel() - 1
    if dist.numel() != n:
        raise ValueError(f"run_noalloc: dist has {dist.numel()} entries, the graph {n} vertices")
    if d > 0 and tuple(masks.shape) != (d, n):
        raise ValueError(f"run_noalloc: masks has shape {tuple(masks.shape)}, expected {(d, n)}")
    for name, t in named.items():
        if not t.is_cuda:
            raise ValueError(f"run_noalloc: {name} must be a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError(f"run_noalloc: {name} must be contiguous")
        if t.device != off.device:
            raise ValueError(f"run_noalloc: {name} is on {t.device}, off on {off.device}")


def run_noalloc(off: torch.Tensor, adj: torch.Tensor, sources, d: int, dist: torch.Tensor, masks: torch.Tensor,
                stream=None):
    """``cbfs_run_noalloc``: one C-BFS for callers that cannot allocate device
    memory.  ``off`` (int64, n+1) and ``adj`` (int32) are CUDA tensors the
    caller owns; ``dist`` (uint8, n) and ``masks`` (int64, d x n) are
    preallocated CUDA tensors that receive the outputs.  The library uses a
    fixed scratch array (n <= 131072, nnz <= 4194304) shared by all calls, so
    calls must not overlap on the GPU.  Tensors of another type, shape or
    device raise ValueError before the library is called: the C entry point
    takes raw pointers and would read or write past a wrong-sized buffer."""
    _check_noalloc_args(off, adj, d, dist, masks)
    S = _host_i32(sources)
    n = off.numel() - 1
    rc = lib().cbfs_run_noalloc(int(n), _ptr(off), _ptr(adj) if adj.numel() else None, int(adj.numel()),
                                S.ctypes.data, int(S.size), int(d), _ptr(dist), _ptr(masks) if d > 0 else None,
                                _stream_ptr(stream))
    _check(rc, "cbfs_run_noalloc")
    return dist, masks


class Labels:
    """Vertex-major landmark labels on the GPU and the distance query.
    ``w`` (8, 16, 32, 64) is the subset word width: clusters of at most w
    sources, 1 + d * w / 8 bytes per cluster and vertex."""

    def __init__(self, n: int, capacity: int, d: int, budget_bytes: int = 0, w: int = 64):
        _require_cuda()
        self._h = ctypes.c_void_p()
        _check(lib().cbfs_labels_create_w(int(n), int(capacity), int(d), int(w), int(budget_bytes),
                                          ctypes.byref(self._h)), "cbfs_labels_create_w")
        self.n, self.capacity, self.d, self.w = int(n), int(capacity), int(d), int(w)

    @staticmethod
    def bytes_per_vertex(capacity: int, d: int, w: int = 64) -> int:
        """Row size of a store (the layout of ``cbfs_labels_create_w``)."""
        return (capacity + 7) // 8 * 8 + d * ((capacity * w // 8 + 7) // 8 * 8)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().cbfs_labels_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        """Forgets the stored clusters (``cbfs_labels_reset``); memory is kept."""
        _check(lib().cbfs_labels_reset(self._h), "cbfs_labels_reset")

    @property
    def count(self) -> int:
        c = ctypes.c_int()
        _check(lib().cbfs_labels_count(self._h, ctypes.byref(c)), "cbfs_labels_count")
        return c.value

    def rows(self):
        """(device pointer, stride in bytes) of the row store."""
        p, s = ctypes.c_void_p(), ctypes.c_int64()
        _check(lib().cbfs_labels_rows(self._h, ctypes.byref(p), ctypes.byref(s)), "cbfs_labels_rows")
        return p.value, s.value

    def append(self, dist: torch.Tensor, masks: torch.Tensor, ks, stream=None):
        ks = _host_i32(ks)
        rc = lib().cbfs_labels_append(self._h, _ptr(dist), _ptr(masks) if self.d > 0 else None, ks.ctypes.data,
                                      int(ks.size), _stream_ptr(stream))
        _check(rc, "cbfs_labels_append")

    def query(self, pairs: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """pairs: CUDA int32 [q, 2].  Returns int16 [q] holding the uint16 answers."""
        q = pairs.shape[0] if pairs.dim() == 2 else pairs.numel() // 2
        if out is None:
            out = torch.empty(q, dtype=torch.int16, device=pairs.device)
        rc = lib().cbfs_query_distance(self._h, _ptr(pairs) if q else None, int(q), _ptr(out) if q else None,
                                       _stream_ptr(stream))
        _check(rc, "cbfs_query_distance")
        return out

    def status(self, stream=None) -> int:
        return int(lib().cbfs_labels_status(self._h, _stream_ptr(stream)))


def status_string(code: int) -> str:
    return lib().cbfs_status_string(int(code)).decode()


def sync_status(stream=None) -> int:
    """``cbfs_sync_status``: waits for ``stream`` and returns (then clears) the
    first error left by stream-ordered calls of any handle or label store on
    it (``OK`` when none)."""
    return int(lib().cbfs_sync_status(_stream_ptr(stream)))
