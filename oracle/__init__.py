"""CPU oracle for the exact ε-graph -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library.

The arithmetic lives in ``ctoracle.c`` (plain C, FP64, -ffp-contract=off),
compiled by :func:`build` into ``oracle/_build/liboracle.so`` and called through
ctypes.  Python here only marshals arrays.

Functions and the paper passages they follow:
  sq_l2 / brute_force   -- the ε-graph definition (Sec. III): every pair with
                           d(p, q) <= eps; L2 pinned as the FP64 sequential sum
                           of squared differences compared with fl(eps*eps)
  lev / lev_banded      -- edit distance (named in Sec. I and Sec. III), unit
                           costs; banded cutoff after Ukkonen
  hamming               -- Hamming distance of bit strings (the binary
                           datasets of Sec. V-A, Table I), bit by bit
  build_tree            -- Algorithm 1 (SplitVertex) + Algorithm 2 (BuildLevel)
  tree_query            -- Algorithm 3 (stack query with vertex-triple radii)
  check_tree            -- cover-tree invariants (Sec. III) + radius bound
                           (Sec. IV-A vertex triple)
  voronoi / landmark_graph -- Voronoi cells of landmark centres and the
                           ε-graph through ε-ghosts (Sec. IV-D, Lemma 1)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_L2, ORC_LEV, ORC_HAM = 0, 1, 2
LEVEL_NONE = -(2 ** 31)   # level of a radius-0 vertex


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags, OpenMP)."""
    src = os.path.join(_HERE, "ctoracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Space(C.Structure):
    _fields_ = [("metric", C.c_int32), ("n", C.c_int64), ("dim", C.c_int32),
                ("X", C.c_void_p), ("S", C.c_void_p), ("off", C.c_void_p)]


class _Csr(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("nnz", C.c_int64),
                ("row_ptr", C.POINTER(C.c_int64)), ("col", C.POINTER(C.c_int64)),
                ("dist", C.POINTER(C.c_double)), ("dist_evals", C.c_int64)]


class _Tree(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_points", C.c_int64),
                ("center", C.POINTER(C.c_int64)), ("radius", C.POINTER(C.c_double)),
                ("level", C.POINTER(C.c_int32)),
                ("child_begin", C.POINTER(C.c_int64)), ("child_count", C.POINTER(C.c_int64)),
                ("pts_begin", C.POINTER(C.c_int64)), ("pts_count", C.POINTER(C.c_int64)),
                ("leaf_pts", C.POINTER(C.c_int64)), ("dist_evals", C.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            lib.orc_sq_l2.restype = C.c_double
            lib.orc_sq_l2.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
            lib.orc_lev_full.restype = C.c_int32
            lib.orc_lev_full.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32]
            lib.orc_hamming.restype = C.c_int32
            lib.orc_hamming.argtypes = [C.c_void_p, C.c_void_p, C.c_int32]
            lib.orc_lev_banded.restype = C.c_int32
            lib.orc_lev_banded.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32]
            lib.orc_brute_force.restype = C.POINTER(_Csr)
            lib.orc_brute_force.argtypes = [C.POINTER(_Space), C.c_double, C.c_int32]
            lib.orc_brute_rows.restype = C.POINTER(_Csr)
            lib.orc_brute_rows.argtypes = [C.POINTER(_Space), C.c_double, C.c_int32, C.c_void_p, C.c_int64]
            lib.orc_build_tree.restype = C.POINTER(_Tree)
            lib.orc_build_tree.argtypes = [C.POINTER(_Space), C.c_int32, C.c_int64]
            lib.orc_tree_query.restype = C.POINTER(_Csr)
            lib.orc_tree_query.argtypes = [C.POINTER(_Space), C.POINTER(_Tree), C.c_double, C.c_int32]
            lib.orc_tree_query_rows.restype = C.POINTER(_Csr)
            lib.orc_tree_query_rows.argtypes = [C.POINTER(_Space), C.POINTER(_Tree), C.c_double, C.c_int32,
                                                C.c_void_p, C.c_int64]
            lib.orc_voronoi.restype = None
            lib.orc_voronoi.argtypes = [C.POINTER(_Space), C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]
            lib.orc_landmark_graph.restype = C.POINTER(_Csr)
            lib.orc_landmark_graph.argtypes = [C.POINTER(_Space), C.c_void_p, C.c_int32, C.c_double, C.c_int32,
                                               C.c_double]
            lib.orc_check_tree.restype = C.c_int32
            lib.orc_check_tree.argtypes = [C.POINTER(_Space), C.POINTER(_Tree), C.c_double,
                                           C.c_char_p, C.c_int32]
            lib.orc_csr_free.argtypes = [C.POINTER(_Csr)]
            lib.orc_tree_free.argtypes = [C.POINTER(_Tree)]
            lib.orc_num_threads.restype = C.c_int32
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().orc_num_threads())


class Space:
    """A point set with its metric: L2 over fp32 rows, Levenshtein over uint8
    strings, or Hamming over bit rows (``bits=(rows, dim)``: uint8 array of
    shape (n, ceil(dim/8)), bit j of a row = bit j % 8 of its byte j // 8).
    Keeps the numpy buffers alive for the C side."""

    def __init__(self, points=None, strings=None, bits=None):
        if sum(a is not None for a in (points, strings, bits)) != 1:
            raise ValueError("give exactly one of points=, strings= or bits=")
        if bits is not None:
            rows, dim = bits
            rows = np.ascontiguousarray(rows, dtype=np.uint8)
            if rows.ndim != 2 or rows.shape[1] != (int(dim) + 7) // 8:
                raise ValueError("bits rows must be (n, ceil(dim/8)) uint8")
            keep = rows if rows.size else np.zeros((1, 1), np.uint8)
            self.metric, self.n, self.dim = ORC_HAM, rows.shape[0], int(dim)
            self._keep = (keep,)
            self.c = _Space(ORC_HAM, self.n, self.dim, None, keep.ctypes.data, None)
            self.rows = rows
        elif points is not None:
            x = np.ascontiguousarray(points, dtype=np.float32)
            if x.ndim != 2:
                raise ValueError("points must be (n, dim)")
            self.metric, self.n, self.dim = ORC_L2, x.shape[0], x.shape[1]
            self._keep = (x,)
            self.c = _Space(ORC_L2, self.n, self.dim, x.ctypes.data, None, None)
            self.points = x
        else:
            data, off = strings
            data = np.ascontiguousarray(data, dtype=np.uint8)
            off = np.ascontiguousarray(off, dtype=np.int64)
            if data.size == 0:
                data = np.zeros(1, dtype=np.uint8)
            self.metric, self.n, self.dim = ORC_LEV, off.size - 1, 0
            self._keep = (data, off)
            self.c = _Space(ORC_LEV, self.n, 0, None, data.ctypes.data, off.ctypes.data)
            self.data, self.offsets = data, off

    def string(self, i: int) -> bytes:
        return bytes(self.data[self.offsets[i]:self.offsets[i + 1]])


def sq_l2(x, y) -> float:
    """Pinned squared L2 sum of two fp32 vectors (FP64, ascending index)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    return float(_load().orc_sq_l2(x.ctypes.data, y.ctypes.data, x.size))


def hamming(a, b, dim: int) -> int:
    """Hamming distance of two rows of `dim` bits (uint8, ceil(dim/8) bytes)."""
    x = np.ascontiguousarray(a, dtype=np.uint8)
    y = np.ascontiguousarray(b, dtype=np.uint8)
    return int(_load().orc_hamming(x.ctypes.data, y.ctypes.data, int(dim)))


def _bytes(s):
    b = np.frombuffer(bytes(s), dtype=np.uint8) if not isinstance(s, np.ndarray) else s
    return np.ascontiguousarray(b, dtype=np.uint8), int(b.size)


def lev(a, b) -> int:
    """Levenshtein distance by the full Wagner-Fischer table."""
    (x, la), (y, lb) = _bytes(a), _bytes(b)
    return int(_load().orc_lev_full(x.ctypes.data, la, y.ctypes.data, lb))


def lev_banded(a, b, k: int) -> int:
    """Edit distance if it is <= k, else k + 1."""
    (x, la), (y, lb) = _bytes(a), _bytes(b)
    return int(_load().orc_lev_banded(x.ctypes.data, la, y.ctypes.data, lb, k))


def _take_csr(p):
    c = p.contents
    n, nnz = c.n_rows, c.nnz
    row_ptr = np.ctypeslib.as_array(c.row_ptr, shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(c.col, shape=(max(nnz, 1),))[:nnz].copy()
    dist = np.ctypeslib.as_array(c.dist, shape=(max(nnz, 1),))[:nnz].copy()
    evals = int(c.dist_evals)
    _load().orc_csr_free(p)
    return {"row_ptr": row_ptr, "col": col, "dist": dist, "dist_evals": evals}


def brute_force(space: Space, eps: float, include_self: bool = False) -> dict:
    """All pairs with d <= eps.  Returns a CSR dict with int64 row_ptr/col and
    FP64 dist, rows sorted ascending."""
    return _take_csr(_load().orc_brute_force(C.byref(space.c), float(eps), int(include_self)))


def brute_rows(space: Space, eps: float, rows, include_self: bool = False) -> dict:
    """Brute force for the given query rows only (row r lists the neighbours of
    point rows[r])."""
    r = np.ascontiguousarray(rows, dtype=np.int64)
    return _take_csr(_load().orc_brute_rows(C.byref(space.c), float(eps), int(include_self),
                                            r.ctypes.data, r.size))


def voronoi(space: Space, centres):
    """(cell, dmin): index of each point's nearest centre (lowest among
    equals) and its distance, FP64 (landmark step 1, Sec. IV-D)."""
    c = np.ascontiguousarray(centres, dtype=np.int64)
    cell = np.zeros(max(space.n, 1), np.int32)
    dmin = np.zeros(max(space.n, 1), np.float64)
    _load().orc_voronoi(C.byref(space.c), c.ctypes.data, int(c.size), cell.ctypes.data, dmin.ctypes.data)
    return cell[:space.n], dmin[:space.n]


def landmark_graph(space: Space, centres, eps: float, include_self: bool = False, factor: float = 2.0) -> dict:
    """The ε-graph by Voronoi cells and ε-ghosts (Sec. IV-D, Lemma 1): each
    row by brute force over its cell's points and ghosts."""
    c = np.ascontiguousarray(centres, dtype=np.int64)
    return _take_csr(_load().orc_landmark_graph(C.byref(space.c), c.ctypes.data, int(c.size), float(eps),
                                                int(include_self), float(factor)))


class Tree:
    """A cover tree in the flat export format (node 0 is the root; children are
    contiguous node ids; leaf blocks list their points in ``leaf_pts``)."""

    FIELDS = ("center", "radius", "level", "child_begin", "child_count",
              "pts_begin", "pts_count", "leaf_pts")

    def __init__(self, **arrays):
        self.center = np.ascontiguousarray(arrays["center"], dtype=np.int64)
        self.radius = np.ascontiguousarray(arrays["radius"], dtype=np.float64)
        self.level = np.ascontiguousarray(arrays["level"], dtype=np.int32)
        self.child_begin = np.ascontiguousarray(arrays["child_begin"], dtype=np.int64)
        self.child_count = np.ascontiguousarray(arrays["child_count"], dtype=np.int64)
        self.pts_begin = np.ascontiguousarray(arrays["pts_begin"], dtype=np.int64)
        self.pts_count = np.ascontiguousarray(arrays["pts_count"], dtype=np.int64)
        self.leaf_pts = np.ascontiguousarray(arrays["leaf_pts"], dtype=np.int64)
        self.dist_evals = int(arrays.get("dist_evals", 0))

    @property
    def n_nodes(self) -> int:
        return int(self.center.size)

    def _c(self):
        P = lambda a, t: a.ctypes.data_as(C.POINTER(t))
        keep = [np.zeros(1, np.int64) if a.size == 0 else a for a in
                (self.center, self.child_begin, self.child_count, self.pts_begin,
                 self.pts_count, self.leaf_pts)]
        rad = self.radius if self.radius.size else np.zeros(1)
        lvl = self.level if self.level.size else np.zeros(1, np.int32)
        self._hold = (keep, rad, lvl)
        return _Tree(self.n_nodes, int(self.leaf_pts.size),
                     P(keep[0], C.c_int64), P(rad, C.c_double), P(lvl, C.c_int32),
                     P(keep[1], C.c_int64), P(keep[2], C.c_int64), P(keep[3], C.c_int64),
                     P(keep[4], C.c_int64), P(keep[5], C.c_int64), self.dist_evals)


def build_tree(space: Space, zeta: int = 32, root: int = 0) -> Tree:
    """Plain cover tree by vertex splitting (Algorithms 1 and 2), FP64."""
    p = _load().orc_build_tree(C.byref(space.c), int(zeta), int(root))
    c = p.contents
    N, n = c.n_nodes, c.n_points
    def take(ptr, cnt, dt):
        if cnt == 0 or not ptr:
            return np.zeros(0, dtype=dt)
        return np.ctypeslib.as_array(ptr, shape=(cnt,)).copy()
    i64, f64, i32 = np.int64, np.float64, np.int32
    t = Tree(center=take(c.center, N, i64), radius=take(c.radius, N, f64),
             level=take(c.level, N, i32), child_begin=take(c.child_begin, N, i64),
             child_count=take(c.child_count, N, i64), pts_begin=take(c.pts_begin, N, i64),
             pts_count=take(c.pts_count, N, i64), leaf_pts=take(c.leaf_pts, n, i64),
             dist_evals=c.dist_evals)
    _load().orc_tree_free(p)
    return t


def tree_query(space: Space, tree: Tree, eps: float, include_self: bool = False) -> dict:
    """ε query of every point against ``tree`` (Algorithm 3)."""
    ct = tree._c()
    return _take_csr(_load().orc_tree_query(C.byref(space.c), C.byref(ct), float(eps),
                                            int(include_self)))


def tree_query_rows(space: Space, tree: Tree, eps: float, rows, include_self: bool = False) -> dict:
    """Algorithm 3 for the given query rows only (row r lists the neighbours of
    point rows[r])."""
    ct = tree._c()
    r = np.ascontiguousarray(rows, dtype=np.int64)
    return _take_csr(_load().orc_tree_query_rows(C.byref(space.c), C.byref(ct), float(eps),
                                                 int(include_self), r.ctypes.data, r.size))


def check_tree(space: Space, tree: Tree, tol: float = 0.0):
    """(code, message): code 0 when every cover-tree invariant holds."""
    ct = tree._c()
    buf = C.create_string_buffer(512)
    code = _load().orc_check_tree(C.byref(space.c), C.byref(ct), float(tol), buf, 512)
    return int(code), buf.value.decode()


def csr_equal(a: dict, b: dict) -> bool:
    """Exact equality of row_ptr and col of two CSR dicts."""
    return (np.array_equal(np.asarray(a["row_ptr"], np.int64), np.asarray(b["row_ptr"], np.int64))
            and np.array_equal(np.asarray(a["col"], np.int64), np.asarray(b["col"], np.int64)))


def csr_symmetric(csr: dict) -> bool:
    """Column j in row i  <=>  column i in row j."""
    rp = np.asarray(csr["row_ptr"], np.int64)
    col = np.asarray(csr["col"], np.int64)
    n = rp.size - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    fwd = rows * max(n, 1) + col
    bwd = col * max(n, 1) + rows
    return np.array_equal(np.sort(fwd), np.sort(bwd))
