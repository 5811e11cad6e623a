"""Oracle for Cluster-BFS and the landmark-label query -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it.

Everything here is a thin ctypes wrapper around ``cbfs_oracle.c``: a plain,
sequential C restatement of the paper's definitions (Section 3.1), of
Algorithm 1 (Section 3.2), of an exact certificate checker, of the
landmark-labeling query (Section 4.2) and of the bounded bidirectional search
added to queries (Appendix B).  See the C file for the readings taken
where the paper is ambiguous.

Every function is pinned by ``tests/test_oracle_pins.py`` against the
paper's worked example (Figure 2 / Section 3.1), closed forms on paths,
cycles and grids, textbook BFS from SciPy and NetworkX, and brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cbfs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

OK, INVALID, DIAMETER, DEPTH, NOMEM = 0, -1, -2, -3, -4


def build(force: bool = False) -> str:
    """Compile ``cbfs_oracle.c`` into ``liboracle.so`` next to it (gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int
        lib.oracle_bfs.argtypes = [i64, P, P, ctypes.c_int32, P]
        lib.oracle_bfs.restype = i32
        lib.oracle_cbfs_definition.argtypes = [i64, P, P, P, i32, i32, P, P]
        lib.oracle_cbfs_definition.restype = i32
        lib.oracle_cbfs_alg1.argtypes = [i64, P, P, P, i32, i32, P, P, P]
        lib.oracle_cbfs_alg1.restype = i32
        lib.oracle_certify.argtypes = [i64, P, P, P, i32, i32, P, P]
        lib.oracle_certify.restype = i64
        lib.oracle_query.argtypes = [i64, i32, i32, P, P, P, i64, P, P]
        lib.oracle_query.restype = i32
        lib.oracle_label_rows.argtypes = [i64, i32, i32, P, P, P]
        lib.oracle_label_rows.restype = i32
        lib.oracle_local_search.argtypes = [i64, P, P, i64, P, i64, P]
        lib.oracle_local_search.restype = i32
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(off, adj):
    off = np.ascontiguousarray(off, dtype=np.int64)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    if adj.size == 0:
        adj = np.zeros(1, dtype=np.int32)  # valid pointer for empty graphs
    return off, adj


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def bfs(off, adj, src: int) -> np.ndarray:
    """Textbook BFS distances from ``src`` (int32, -1 = unreachable)."""
    off, adj = _csr(off, adj)
    n = off.size - 1
    dist = np.empty(max(n, 1), dtype=np.int32)
    rc = _load().oracle_bfs(n, _p(off), _p(adj), int(src), _p(dist))
    if rc:
        raise OracleError(rc, "oracle_bfs")
    return dist[:n]


def _cbfs(fn, off, adj, sources, d, counters=None, allow=(OK,)):
    off, adj = _csr(off, adj)
    n = off.size - 1
    S = np.ascontiguousarray(sources, dtype=np.int32)
    k = int(S.size)
    dist = np.empty(max(n, 1), dtype=np.uint8)
    masks = np.zeros((max(d, 1), max(n, 1)), dtype=np.uint64)
    args = [n, _p(off), _p(adj), _p(S if k else np.zeros(1, np.int32)), k, int(d), _p(dist), _p(masks)]
    if counters is not None:
        args.append(_p(counters))
    rc = fn(*args)
    if rc not in allow:
        raise OracleError(rc, fn.__name__)
    return dist[:n].copy(), masks[:d, :n].copy(), rc


def cbfs_definition(off, adj, sources, d: int):
    """O1: cluster distance vectors from the definition (Section 3.1).

    Returns ``(dist uint8[n], masks uint64[d, n])``.  Raises ``OracleError``
    with code DIAMETER when some vertex sees a source spread wider than d.
    """
    dist, masks, _ = _cbfs(_load().oracle_cbfs_definition, off, adj, sources, d)
    return dist, masks


def cbfs_alg1(off, adj, sources, d: int, with_counters: bool = False):
    """O2: Algorithm 1 run sequentially.  Optionally returns work counters
    ``{"V": sum |F_i|, "A": arcs scanned, "rounds": ..., "reached_arcs": ...}``."""
    cnt = np.zeros(4, dtype=np.int64)
    dist, masks, _ = _cbfs(_load().oracle_cbfs_alg1, off, adj, sources, d, counters=cnt)
    if with_counters:
        return dist, masks, {"V": int(cnt[0]), "A": int(cnt[1]), "rounds": int(cnt[2]),
                             "reached_arcs": int(cnt[3])}
    return dist, masks


def certify(off, adj, sources, d: int, dist, masks) -> int:
    """-1 when (dist, masks) is the exact C-BFS output, else the first bad vertex."""
    off, adj = _csr(off, adj)
    n = off.size - 1
    S = np.ascontiguousarray(sources, dtype=np.int32)
    dist = np.ascontiguousarray(dist, dtype=np.uint8)
    masks = np.ascontiguousarray(masks, dtype=np.uint64).reshape(-1)
    if masks.size == 0:
        masks = np.zeros(1, dtype=np.uint64)
    return int(_load().oracle_certify(n, _p(off), _p(adj), _p(S), int(S.size), int(d), _p(dist), _p(masks)))


def query(dist_cn, masks_cdn, ks, pairs) -> np.ndarray:
    """Landmark-labeling query from cluster-major outputs: dist [C, n],
    masks [C, d, n], ks [C] cluster sizes, pairs [q, 2] -> uint16[q]."""
    dist_cn = np.ascontiguousarray(dist_cn, dtype=np.uint8)
    masks_cdn = np.ascontiguousarray(masks_cdn, dtype=np.uint64)
    C, n = dist_cn.shape
    d = masks_cdn.shape[1] if masks_cdn.ndim == 3 else 0
    ks = np.ascontiguousarray(ks, dtype=np.int32)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    q = pairs.shape[0]
    out = np.empty(max(q, 1), dtype=np.uint16)
    mk = masks_cdn.reshape(-1) if masks_cdn.size else np.zeros(1, np.uint64)
    rc = _load().oracle_query(n, C, d, _p(dist_cn), _p(mk), _p(ks if ks.size else np.zeros(1, np.int32)),
                              q, _p(pairs if q else np.zeros(2, np.int32)), _p(out))
    if rc:
        raise OracleError(rc, "oracle_query")
    return out[:q]


def label_rows(dist_cn, masks_cdn) -> np.ndarray:
    """Vertex-major label rows (see ``oracle_label_rows`` in the C file)."""
    dist_cn = np.ascontiguousarray(dist_cn, dtype=np.uint8)
    masks_cdn = np.ascontiguousarray(masks_cdn, dtype=np.uint64)
    C, n = dist_cn.shape
    d = masks_cdn.shape[1]
    P = (C + 7) // 8 * 8
    stride = P + 8 * d * C
    rows = np.empty((max(n, 1), stride), dtype=np.uint8)
    mk = masks_cdn.reshape(-1) if masks_cdn.size else np.zeros(1, np.uint64)
    rc = _load().oracle_label_rows(n, C, d, _p(dist_cn), _p(mk), _p(rows))
    if rc:
        raise OracleError(rc, "oracle_label_rows")
    return rows[:n]


def local_search(off, adj, pairs, tau: int) -> np.ndarray:
    """Bounded bidirectional search (Appendix B, see ``oracle_local_search``):
    uint16[q], 0xFFFF where the tau-vertex balls of the two ends do not meet."""
    off, adj = _csr(off, adj)
    n = off.size - 1
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    q = pairs.shape[0]
    out = np.empty(max(q, 1), dtype=np.uint16)
    rc = _load().oracle_local_search(n, _p(off), _p(adj), q, _p(pairs if q else np.zeros(2, np.int32)), int(tau),
                                     _p(out))
    if rc:
        raise OracleError(rc, "oracle_local_search")
    return out[:q]
