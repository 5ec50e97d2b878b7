"""Python binding of the C-ABI in ``include/ctgraph.h`` (ctypes; argument
marshalling only -- every step of the computation runs in the CUDA library).

PyTorch supplies device memory and streams.  Functions keep the C names:

    tree = ct_build(points)                      # torch.cuda fp32 (n, dim)
    tree = ct_build(strings=(data, offsets))     # torch.cuda uint8 / int64
    csr = eps_graph_query(tree, eps)             # CSR with torch views
    csrs = eps_graph_query_batched(trees, eps)
    csr_free(csr); ct_tree_free(tree)

There is no CPU fallback: if the library is not built, or no GPU is present,
these calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _buildmod

CT_OK, CT_EINVAL, CT_ENOMEM, CT_ECUDA, CT_ETIMEOUT, CT_EOVERFLOW, CT_EUNSUPPORTED = range(7)
STATUS_NAMES = {0: "CT_OK", 1: "CT_EINVAL", 2: "CT_ENOMEM", 3: "CT_ECUDA", 4: "CT_ETIMEOUT",
                5: "CT_EOVERFLOW", 6: "CT_EUNSUPPORTED"}
CT_L2_F32, CT_LEVENSHTEIN_U8, CT_HAMMING_B1 = 0, 1, 2

_lock = threading.Lock()
_lib = None


class CtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class ct_points(C.Structure):
    _fields_ = [("metric", C.c_int32), ("dim", C.c_int32), ("n", C.c_int64),
                ("data", C.c_void_p), ("offsets", C.c_void_p)]


class ct_build_opts(C.Structure):
    _fields_ = [("leaf_size", C.c_int32), ("root", C.c_int32)]


class ct_query_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("use_predictor", C.c_int32),
                ("include_self", C.c_int32), ("upper_triangle", C.c_int32), ("predictor", C.c_void_p)]


class ct_csr(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("dist", C.c_void_p), ("priv", C.c_void_p)]


class ct_query_stats(C.Structure):
    _fields_ = [(f, C.c_int64) for f in ("traversal_evals", "leaf_pairs", "guard_fp64",
                                           "recheck_fp32", "candidates", "overflow_rows",
                                           "kernel_launches", "emit_pairs", "reemit_rows",
                                           "leaf_rows", "guard_band", "lev_columns")]


class ct_landmark_info(C.Structure):
    _fields_ = [(f, C.c_int64) for f in ("cells", "members", "ghosts", "largest_cell")]


class ct_fit_opts(C.Structure):
    _fields_ = [("steps", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("include_self", C.c_int32),
                ("seed", C.c_uint64)]


CT_MLP_IN, CT_MLP_NPARAMS, CT_MLP_NORM = 16, 5378, 36


def library_path() -> str:
    return _buildmod.LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _buildmod.LIB
        if not os.path.exists(path):
            raise RuntimeError("CUDA library %s is not built; call paper_2510_14147_gb300.build.build()" % path)
        lib = C.CDLL(path)
        P = C.POINTER
        lib.ct_build.restype = C.c_int
        lib.ct_build.argtypes = [P(ct_points), P(ct_build_opts), C.c_void_p, P(C.c_void_p)]
        lib.eps_graph_query.restype = C.c_int
        lib.eps_graph_query.argtypes = [C.c_void_p, C.c_double, P(ct_query_opts), C.c_void_p, P(ct_csr)]
        lib.eps_graph_query_batched.restype = C.c_int
        lib.eps_graph_query_batched.argtypes = [C.c_int32, P(C.c_void_p), P(C.c_double), P(ct_query_opts),
                                                C.c_void_p, P(ct_csr)]
        lib.csr_free.restype = None
        lib.csr_free.argtypes = [P(ct_csr)]
        lib.ct_csr_stats.restype = C.c_int
        lib.ct_csr_stats.argtypes = [P(ct_csr), P(ct_query_stats)]
        lib.ct_tree_free.restype = None
        lib.ct_tree_free.argtypes = [C.c_void_p]
        lib.ct_tree_shape.restype = C.c_int
        lib.ct_tree_shape.argtypes = [C.c_void_p, P(C.c_int64), P(C.c_int64)]
        lib.ct_tree_export.restype = C.c_int
        lib.ct_tree_export.argtypes = [C.c_void_p] + [C.c_void_p] * 8
        lib.ct_last_error.restype = C.c_char_p
        lib.ct_last_error.argtypes = []
        lib.ct_version.restype = C.c_char_p
        lib.ct_version.argtypes = []
        lib.ct_profile_enable.restype = None
        lib.ct_profile_enable.argtypes = [C.c_int32]
        lib.ct_profile_reset.restype = None
        lib.ct_profile_reset.argtypes = []
        lib.ct_profile_count.restype = C.c_int32
        lib.ct_profile_count.argtypes = []
        lib.ct_profile_entry.restype = C.c_int
        lib.ct_profile_entry.argtypes = [C.c_int32, P(C.c_char_p), P(C.c_double), P(C.c_int64)]
        lib.eps_graph_degrees_noalloc.restype = C.c_int
        lib.eps_graph_degrees_noalloc.argtypes = [C.c_void_p, C.c_double, C.c_int32, C.c_void_p, C.c_void_p]
        lib.ct_selftest_tc_gemm.restype = C.c_int
        lib.ct_selftest_tc_gemm.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]
        lib.ct_kernel_launches.restype = C.c_int64
        lib.ct_kernel_launches.argtypes = []
        lib.ct_autotune.restype = C.c_int
        lib.ct_autotune.argtypes = [C.c_int32, P(C.c_void_p), P(C.c_double), P(ct_query_opts), C.c_void_p,
                                    C.c_void_p]
        lib.ct_autotune_reset.restype = None
        lib.ct_autotune_reset.argtypes = []
        lib.ct_predictor_create.restype = C.c_int
        lib.ct_predictor_create.argtypes = [C.c_uint64, P(C.c_void_p)]
        lib.ct_predictor_free.restype = None
        lib.ct_predictor_free.argtypes = [C.c_void_p]
        lib.ct_predictor_fit.restype = C.c_int
        lib.ct_predictor_fit.argtypes = [C.c_void_p, C.c_void_p, C.c_double, P(ct_fit_opts), C.c_void_p,
                                         P(C.c_double)]
        lib.ct_predictor_set_capacity.restype = C.c_int
        lib.ct_predictor_set_capacity.argtypes = [C.c_void_p, C.c_float, C.c_int32, C.c_float, C.c_int64]
        lib.ct_predictor_set_order.restype = C.c_int
        lib.ct_predictor_set_order.argtypes = [C.c_void_p, C.c_int32]
        lib.ct_predictor_get_params.restype = C.c_int
        lib.ct_predictor_get_params.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        lib.ct_predictor_set_params.restype = C.c_int
        lib.ct_predictor_set_params.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        lib.ct_predictor_features.restype = C.c_int
        lib.ct_predictor_features.argtypes = [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
        lib.ct_predictor_predict.restype = C.c_int
        lib.ct_predictor_predict.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p,
                                             C.c_void_p]
        lib.ct_mlp_loss_grad.restype = C.c_int
        lib.ct_mlp_loss_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                         P(C.c_double), C.c_void_p]
        lib.ct_mlp_forward_f16.restype = C.c_int
        lib.ct_mlp_forward_f16.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
        lib.eps_graph_query_sweep.restype = C.c_int
        lib.eps_graph_query_sweep.argtypes = [C.c_void_p, C.c_int32, P(C.c_double), P(ct_query_opts), C.c_void_p,
                                              P(ct_csr)]
        lib.ct_plan_create.restype = C.c_int
        lib.ct_plan_create.argtypes = [C.c_int32, P(C.c_void_p), P(C.c_double), P(ct_query_opts), C.c_float,
                                       C.c_int32, C.c_void_p, P(C.c_void_p)]
        lib.ct_plan_launch.restype = C.c_int
        lib.ct_plan_launch.argtypes = [C.c_void_p, C.c_void_p]
        lib.ct_plan_result.restype = C.c_int
        lib.ct_plan_result.argtypes = [C.c_void_p, C.c_void_p, P(ct_csr)]
        lib.ct_plan_set_wait.restype = C.c_int
        lib.ct_plan_set_wait.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
        lib.ct_plan_free.restype = None
        lib.ct_plan_free.argtypes = [C.c_void_p]
        lib.ct_selftest_tc_timeout.restype = C.c_int
        lib.ct_selftest_tc_timeout.argtypes = [C.c_void_p]
        lib.ct_debug_fail_alloc.restype = C.c_int
        lib.ct_debug_fail_alloc.argtypes = [C.c_int64]
        lib.ct_debug_pool_used.restype = C.c_int
        lib.ct_debug_pool_used.argtypes = [P(C.c_uint64)]
        lib.ct_debug_capacity_budget.restype = C.c_int
        lib.ct_debug_capacity_budget.argtypes = [C.c_int64]
        lib.ct_debug_guard_rows.restype = C.c_int
        lib.ct_debug_guard_rows.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
        lib.eps_graph_query_landmark.restype = C.c_int
        lib.eps_graph_query_landmark.argtypes = [P(ct_points), C.c_void_p, C.c_int32, C.c_double, P(ct_build_opts),
                                                 P(ct_query_opts), C.c_void_p, P(ct_csr), P(ct_landmark_info)]
        lib.ct_tree_save.restype = C.c_int
        lib.ct_tree_save.argtypes = [C.c_void_p, C.c_char_p]
        lib.ct_tree_load.restype = C.c_int
        lib.ct_tree_load.argtypes = [C.c_char_p, C.c_void_p, P(C.c_void_p)]
        _lib = lib
        return lib


def ct_last_error() -> str:
    return _load().ct_last_error().decode(errors="replace")


def _check(status: int):
    if status != CT_OK:
        raise CtError(status, ct_last_error())


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class _CudaArray:
    """__cuda_array_interface__ view of library-owned memory; holds `owner`."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 3,
                                         "strides": None}
        self._owner = owner


def _view(ptr, count, typestr, owner, torch_dtype):
    import torch
    if count == 0 or not ptr:
        return torch.empty(0, dtype=torch_dtype, device="cuda")
    return torch.as_tensor(_CudaArray(ptr, (count,), typestr, owner), device="cuda")


class Tree:
    """Owning handle of a device-resident cover tree."""

    def __init__(self, handle: int, n: int, metric: int):
        self.handle = C.c_void_p(handle)
        self.n = n
        self.metric = metric

    def free(self):
        if self.handle and self.handle.value:
            _load().ct_tree_free(self.handle)
            self.handle = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class _CsrOwner:
    """Holds one library CSR; releases it when the last reference goes."""

    def __init__(self, c: ct_csr):
        self.c = c

    def free(self):
        if self.c.priv:
            _load().csr_free(C.byref(self.c))

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class CSR:
    """A library-allocated CSR.  ``row_ptr``/``col``/``dist`` are zero-copy
    torch views; each keeps the memory alive until it is dropped, unless
    :meth:`free` releases it first (views taken earlier become invalid)."""

    def __init__(self, c: ct_csr):
        self._owner = _CsrOwner(c)
        self.n_rows = int(c.n_rows)
        self.nnz = int(c.nnz)

    @property
    def c(self) -> ct_csr:
        return self._owner.c

    @property
    def row_ptr(self):
        import torch
        return _view(self.c.row_ptr, self.n_rows + 1, "<i8", self._owner, torch.int64)

    @property
    def col(self):
        import torch
        return _view(self.c.col, self.nnz, "<i4", self._owner, torch.int32)

    @property
    def dist(self):
        import torch
        return _view(self.c.dist, self.nnz, "<f4", self._owner, torch.float32)

    def stats(self) -> dict:
        st = ct_query_stats()
        _check(_load().ct_csr_stats(C.byref(self.c), C.byref(st)))
        return {f: int(getattr(st, f)) for f, _ in ct_query_stats._fields_}

    def to_numpy(self) -> dict:
        return {"row_ptr": self.row_ptr.cpu().numpy(), "col": self.col.cpu().numpy(),
                "dist": self.dist.cpu().numpy()}

    def free(self):
        self._owner.free()


def ct_build(points=None, strings=None, bits=None, leaf_size: int = 32, root: int = 0, stream=None) -> Tree:
    """Cover-tree construction (Algorithms 1-2).  ``points``: CUDA fp32 tensor
    (n, dim); or ``strings=(data, offsets)``: CUDA uint8 and int64 tensors; or
    ``bits=(rows, dim)``: CUDA uint8 tensor (n, ceil(dim/8)) of bit rows (bit j
    = bit j % 8 of byte j // 8) under the Hamming distance."""
    import torch
    lib = _load()
    if sum(a is not None for a in (points, strings, bits)) != 1:
        raise ValueError("give exactly one of points=, strings= or bits=")
    p = ct_points()
    if bits is not None:
        rows, dim = bits
        if not (rows.is_cuda and rows.dtype == torch.uint8 and rows.dim() == 2
                and rows.shape[1] == (int(dim) + 7) // 8):
            raise ValueError("bits must be (CUDA uint8 tensor (n, ceil(dim/8)), dim)")
        rows = rows.contiguous()
        p.metric, p.dim, p.n = CT_HAMMING_B1, int(dim), rows.shape[0]
        p.data, p.offsets = rows.data_ptr() or None, None
        keep = (rows,)
    elif points is not None:
        if not (points.is_cuda and points.dtype == torch.float32 and points.dim() == 2):
            raise ValueError("points must be a CUDA float32 tensor of shape (n, dim)")
        points = points.contiguous()
        p.metric, p.dim, p.n = CT_L2_F32, points.shape[1], points.shape[0]
        p.data, p.offsets = points.data_ptr() or None, None
        keep = (points,)
    else:
        data, off = strings
        if not (data.is_cuda and off.is_cuda and data.dtype == torch.uint8 and off.dtype == torch.int64):
            raise ValueError("strings must be (CUDA uint8 data, CUDA int64 offsets)")
        data, off = data.contiguous(), off.contiguous()
        p.metric, p.dim, p.n = CT_LEVENSHTEIN_U8, 0, off.numel() - 1
        p.data, p.offsets = data.data_ptr() or None, off.data_ptr() or None
        keep = (data, off)
    o = ct_build_opts(leaf_size, root)
    h = C.c_void_p()
    st = lib.ct_build(C.byref(p), C.byref(o), C.c_void_p(_stream(stream)), C.byref(h))
    del keep
    _check(st)
    return Tree(h.value, int(p.n), int(p.metric))


def _opts(precision, use_predictor, include_self, predictor, upper_triangle=False):
    o = ct_query_opts()
    o.precision = int(precision)
    o.use_predictor = int(bool(use_predictor))
    o.include_self = int(bool(include_self))
    o.upper_triangle = int(bool(upper_triangle))
    o.predictor = predictor.handle.value if predictor is not None else None
    return o


def eps_graph_query(tree: Tree, eps: float, precision: int = 0, use_predictor: bool = False,
                    include_self: bool = False, predictor=None, stream=None, upper_triangle: bool = False) -> CSR:
    """The exact ε-graph of the tree's points as a CSR (rows ascending)."""
    lib = _load()
    out = ct_csr()
    o = _opts(precision, use_predictor, include_self, predictor, upper_triangle)
    _check(lib.eps_graph_query(tree.handle, float(eps), C.byref(o), C.c_void_p(_stream(stream)),
                               C.byref(out)))
    return CSR(out)


def eps_graph_query_batched(trees, eps, precision: int = 0, use_predictor: bool = False,
                            include_self: bool = False, predictor=None, stream=None, upper_triangle: bool = False):
    lib = _load()
    k = len(trees)
    arr = (C.c_void_p * max(k, 1))(*[t.handle.value for t in trees])
    ea = (C.c_double * max(k, 1))(*[float(e) for e in eps])
    outs = (ct_csr * max(k, 1))()
    o = _opts(precision, use_predictor, include_self, predictor, upper_triangle)
    _check(lib.eps_graph_query_batched(k, arr, ea, C.byref(o), C.c_void_p(_stream(stream)), outs))
    return [CSR(outs[i]) for i in range(k)]


def eps_graph_query_sweep(tree: Tree, eps, precision: int = 0, use_predictor: bool = False,
                          include_self: bool = False, predictor=None, stream=None, upper_triangle: bool = False):
    """CSRs of one tree at several radii (eps: a sequence); csrs[k] equals
    eps_graph_query(tree, eps[k], ...) bit for bit."""
    lib = _load()
    k = len(eps)
    ea = (C.c_double * max(k, 1))(*[float(e) for e in eps])
    outs = (ct_csr * max(k, 1))()
    o = _opts(precision, use_predictor, include_self, predictor, upper_triangle)
    _check(lib.eps_graph_query_sweep(tree.handle, k, ea, C.byref(o), C.c_void_p(_stream(stream)), outs))
    return [CSR(outs[i]) for i in range(k)]


class Plan:
    """Owning handle of a plan: a batch of L2 clouds with its buffers allocated
    once, run by ct_plan_launch (a CUDA-graph replay with use_graph)."""

    def __init__(self, handle: int, n_clouds: int, trees):
        self.handle = C.c_void_p(handle)
        self.n_clouds = n_clouds
        self._trees = list(trees)   # the plan borrows them

    def free(self):
        if self.handle and self.handle.value:
            _load().ct_plan_free(self.handle)
            self.handle = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def ct_plan_create(trees, eps, precision: int = 0, use_predictor: bool = False, include_self: bool = False,
                   predictor=None, margin: float = 0.1, use_graph: bool = True, stream=None, upper_triangle: bool = False) -> Plan:
    lib = _load()
    k = len(trees)
    arr = (C.c_void_p * max(k, 1))(*[t.handle.value for t in trees])
    ea = (C.c_double * max(k, 1))(*[float(e) for e in eps])
    o = _opts(precision, use_predictor, include_self, predictor, upper_triangle)
    h = C.c_void_p()
    _check(lib.ct_plan_create(k, arr, ea, C.byref(o), float(margin), int(bool(use_graph)),
                              C.c_void_p(_stream(stream)), C.byref(h)))
    return Plan(h.value, k, trees)


def ct_plan_launch(plan: Plan, stream=None):
    _check(_load().ct_plan_launch(plan.handle, C.c_void_p(_stream(stream))))


def ct_plan_result(plan: Plan, stream=None):
    """The CSRs of the last run (views into the plan's buffers, valid until the
    next launch); raises CtError with CT_EOVERFLOW / CT_ETIMEOUT on failure."""
    outs = (ct_csr * max(plan.n_clouds, 1))()
    _check(_load().ct_plan_result(plan.handle, C.c_void_p(_stream(stream)), outs))
    return [CSR(outs[i]) for i in range(plan.n_clouds)]


def ct_plan_set_wait(plan: Plan, withhold_producers: bool = False, max_polls: int = 1 << 20):
    _check(_load().ct_plan_set_wait(plan.handle, int(bool(withhold_producers)), int(max_polls)))


def ct_debug_guard_rows(rows=None, count=None):
    """Diagnostic: record the CSR rows of both ends of every pair later count
    passes decide by the FP64 sum into `rows` (CUDA int32 tensor), counting
    into `count` (CUDA int64 tensor of one zeroed entry); rows=None stops."""
    if rows is None:
        _check(_load().ct_debug_guard_rows(None, None, 0))
    else:
        _check(_load().ct_debug_guard_rows(rows.data_ptr(), count.data_ptr(), rows.numel()))


def ct_selftest_tc_timeout(stream=None):
    """The tensor-core self-test with its MMA withheld: raises CtError with
    CT_ETIMEOUT once the bounded completion wait runs out."""
    _check(_load().ct_selftest_tc_timeout(C.c_void_p(_stream(stream))))


def ct_debug_fail_alloc(k: int):
    """Test hook: the k-th next device allocation of the library fails (0: off)."""
    _check(_load().ct_debug_fail_alloc(int(k)))


def ct_debug_capacity_budget(nbytes: int):
    """Test hook: the learned form's one-pass buffers get this many bytes (0: the default)."""
    _check(_load().ct_debug_capacity_budget(int(nbytes)))


def ct_debug_pool_used() -> int:
    """Bytes in use in the device's default memory pool (after a device sync)."""
    b = C.c_uint64()
    _check(_load().ct_debug_pool_used(C.byref(b)))
    return int(b.value)


def eps_graph_query_landmark(centres, eps: float, points=None, bits=None, leaf_size: int = 32,
                             precision: int = 0, use_predictor: bool = False, include_self: bool = False,
                             predictor=None, upper_triangle: bool = False, stream=None):
    """The ε-graph through Voronoi cells of `centres` (host sequence of point
    indices) and their ε-ghosts; returns (CSR, info dict).  ``points``: CUDA
    fp32 (n, dim); or ``bits=(rows, dim)`` as for ct_build."""
    import torch
    lib = _load()
    p = ct_points()
    if points is not None:
        points = points.contiguous()
        p.metric, p.dim, p.n, p.data, p.offsets = CT_L2_F32, points.shape[1], points.shape[0], \
            points.data_ptr() or None, None
        keep = points
    else:
        rows, dim = bits
        rows = rows.contiguous()
        p.metric, p.dim, p.n, p.data, p.offsets = CT_HAMMING_B1, int(dim), rows.shape[0], rows.data_ptr() or None, None
        keep = rows
    c = np.ascontiguousarray(centres, dtype=np.int64)
    out, info = ct_csr(), ct_landmark_info()
    b = ct_build_opts(leaf_size, 0)
    o = _opts(precision, use_predictor, include_self, predictor, upper_triangle)
    _check(lib.eps_graph_query_landmark(C.byref(p), c.ctypes.data if c.size else None, int(c.size), float(eps),
                                        C.byref(b), C.byref(o), C.c_void_p(_stream(stream)), C.byref(out),
                                        C.byref(info)))
    del keep
    return CSR(out), {f: int(getattr(info, f)) for f, _ in ct_landmark_info._fields_}


def ct_tree_save(tree: Tree, path: str):
    """Writes the tree to a file (ct_tree_load reads it back)."""
    _check(_load().ct_tree_save(tree.handle, os.fsencode(path)))


def ct_tree_load(path: str, stream=None) -> Tree:
    """A tree written by ct_tree_save, on the current device."""
    lib = _load()
    h = C.c_void_p()
    _check(lib.ct_tree_load(os.fsencode(path), C.c_void_p(_stream(stream)), C.byref(h)))
    n_nodes, n_pts = C.c_int64(), C.c_int64()
    _check(lib.ct_tree_shape(h, C.byref(n_nodes), C.byref(n_pts)))
    t = Tree(h.value, int(n_pts.value), -1)
    return t


def ct_autotune(trees, eps, use_predictor: bool = False, include_self: bool = False, predictor=None,
                stream=None):
    """Tunes precision 2 on these clouds; returns each cloud's count kernel
    (1: tensor-core tiles, 0: FP32 tiles)."""
    k = len(trees)
    arr = (C.c_void_p * max(k, 1))(*[t.handle.value for t in trees])
    ea = (C.c_double * max(k, 1))(*[float(e) for e in eps])
    ch = np.zeros(max(k, 1), np.int32)
    o = _opts(2, use_predictor, include_self, predictor)
    _check(_load().ct_autotune(k, arr, ea, C.byref(o), C.c_void_p(_stream(stream)), ch.ctypes.data))
    return [int(v) for v in ch[:k]]


def ct_autotune_reset():
    _load().ct_autotune_reset()


def eps_graph_degrees_noalloc(tree: Tree, eps: float, degrees, include_self: bool = False, stream=None):
    """Writes the ε-graph degree of every point into ``degrees`` (a CUDA int32
    tensor of n entries owned by the caller) without any device allocation by
    the library; the library's temporaries live in its fixed device array."""
    import torch
    if tree.n and not (degrees.is_cuda and degrees.dtype == torch.int32 and degrees.is_contiguous()
                       and degrees.numel() >= tree.n):
        raise ValueError("degrees must be a contiguous CUDA int32 tensor with n entries")
    _check(_load().eps_graph_degrees_noalloc(tree.handle, float(eps), int(bool(include_self)),
                                             degrees.data_ptr() if tree.n else None,
                                             C.c_void_p(_stream(stream))))


def csr_free(csr: CSR):
    csr.free()


def ct_tree_free(tree: Tree):
    tree.free()


def ct_tree_export(tree: Tree) -> dict:
    """Host copy of the tree in the flat format (numpy arrays)."""
    lib = _load()
    nn, npnt = C.c_int64(), C.c_int64()
    _check(lib.ct_tree_shape(tree.handle, C.byref(nn), C.byref(npnt)))
    N, n = nn.value, npnt.value
    a = {"center": np.zeros(max(N, 1), np.int64), "radius": np.zeros(max(N, 1), np.float64),
         "level": np.zeros(max(N, 1), np.int32), "child_begin": np.zeros(max(N, 1), np.int64),
         "child_count": np.zeros(max(N, 1), np.int64), "pts_begin": np.zeros(max(N, 1), np.int64),
         "pts_count": np.zeros(max(N, 1), np.int64), "leaf_pts": np.zeros(max(n, 1), np.int64)}
    order = ("center", "radius", "level", "child_begin", "child_count", "pts_begin", "pts_count", "leaf_pts")
    _check(lib.ct_tree_export(tree.handle, *[a[k].ctypes.data for k in order]))
    for k in order:
        a[k] = a[k][:n] if k == "leaf_pts" else a[k][:N]
    return a


def ct_profile_enable(on: bool = True):
    _load().ct_profile_enable(int(bool(on)))


def ct_profile_reset():
    _load().ct_profile_reset()


def ct_profile_read() -> dict:
    """{stage: (total_ms, calls)} accumulated since the last reset."""
    lib = _load()
    out = {}
    for i in range(lib.ct_profile_count()):
        name, ms, calls = C.c_char_p(), C.c_double(), C.c_int64()
        _check(lib.ct_profile_entry(i, C.byref(name), C.byref(ms), C.byref(calls)))
        out[name.value.decode()] = (ms.value, calls.value)
    return out


def ct_kernel_launches() -> int:
    return int(_load().ct_kernel_launches())


def ct_selftest_tc_gemm(A, B, stream=None):
    """D = A @ B.T through one tcgen05 kind::f16 MMA chain: A (128, 128) and
    B (32, 128) CUDA tensors, both bfloat16 or both float16; returns D (128, 32)
    float32."""
    import torch
    if not (A.shape == (128, 128) and B.shape == (32, 128) and A.dtype == B.dtype
            and A.dtype in (torch.bfloat16, torch.float16) and A.is_cuda and B.is_cuda):
        raise ValueError("A must be (128, 128) and B (32, 128) CUDA tensors, both bfloat16 or both float16")
    A, B = A.contiguous(), B.contiguous()
    D = torch.empty(128, 32, dtype=torch.float32, device=A.device)
    f16 = 1 if A.dtype == torch.float16 else 0
    _check(_load().ct_selftest_tc_gemm(A.data_ptr(), B.data_ptr(), f16, D.data_ptr(), C.c_void_p(_stream(stream))))
    return D


class Predictor:
    """Owning handle of a degree/work predictor (the learned form's MLP)."""

    def __init__(self, seed: int = 0):
        h = C.c_void_p()
        _check(_load().ct_predictor_create(C.c_uint64(seed), C.byref(h)))
        self.handle = h

    def free(self):
        if self.handle and self.handle.value:
            _load().ct_predictor_free(self.handle)
            self.handle = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def ct_predictor_create(seed: int = 0) -> Predictor:
    return Predictor(seed)


def ct_predictor_free(p: Predictor):
    p.free()


def ct_predictor_fit(p: Predictor, tree: Tree, eps: float, steps: int = 0, batch: int = 0, lr: float = 0.0,
                     include_self: bool = False, seed: int = 0, stream=None) -> float:
    """Labels the tree's points with their exact degrees and group walk
    lengths and trains the MLP; returns the mean standardised loss of the
    last tenth of the steps."""
    o = ct_fit_opts(int(steps), int(batch), float(lr), int(bool(include_self)), int(seed))
    loss = C.c_double()
    _check(_load().ct_predictor_fit(p.handle, tree.handle, float(eps), C.byref(o), C.c_void_p(_stream(stream)),
                                    C.byref(loss)))
    return float(loss.value)


def ct_predictor_set_capacity(p: Predictor, margin: float = 0.5, pad: int = 16, arena_frac: float = 0.25,
                              arena_min: int = 65536):
    _check(_load().ct_predictor_set_capacity(p.handle, float(margin), int(pad), float(arena_frac),
                                             int(arena_min)))


def ct_predictor_set_order(p: Predictor, by_predicted_work: bool = True):
    _check(_load().ct_predictor_set_order(p.handle, int(bool(by_predicted_work))))


def ct_predictor_get_params(p: Predictor):
    """(params [5378] float32, norm [36] float32) host copies."""
    params = np.zeros(CT_MLP_NPARAMS, np.float32)
    norm = np.zeros(CT_MLP_NORM, np.float32)
    _check(_load().ct_predictor_get_params(p.handle, params.ctypes.data, norm.ctypes.data))
    return params, norm


def ct_predictor_set_params(p: Predictor, params=None, norm=None):
    a = None if params is None else np.ascontiguousarray(params, np.float32)
    b = None if norm is None else np.ascontiguousarray(norm, np.float32)
    if a is not None and a.size != CT_MLP_NPARAMS:
        raise ValueError("params must hold %d values" % CT_MLP_NPARAMS)
    if b is not None and b.size != CT_MLP_NORM:
        raise ValueError("norm must hold %d values" % CT_MLP_NORM)
    _check(_load().ct_predictor_set_params(p.handle, None if a is None else a.ctypes.data,
                                           None if b is None else b.ctypes.data))


def ct_predictor_features(tree: Tree, eps: float, stream=None):
    """Raw features (n, 16) float32 CUDA tensor, row i = tree position i."""
    import torch
    x = torch.empty(max(tree.n, 1), CT_MLP_IN, dtype=torch.float32, device="cuda")
    _check(_load().ct_predictor_features(tree.handle, float(eps), x.data_ptr(), C.c_void_p(_stream(stream))))
    return x[:tree.n]


def ct_predictor_predict(p: Predictor, tree: Tree, eps: float, stream=None):
    """(predicted degree, predicted group walk length), CUDA float32 by original id."""
    import torch
    d = torch.empty(max(tree.n, 1), dtype=torch.float32, device="cuda")
    b = torch.empty(max(tree.n, 1), dtype=torch.float32, device="cuda")
    _check(_load().ct_predictor_predict(p.handle, tree.handle, float(eps), d.data_ptr(), b.data_ptr(),
                                        C.c_void_p(_stream(stream))))
    return d[:tree.n], b[:tree.n]


def ct_mlp_loss_grad(params, x, t, stream=None):
    """(loss, grad) of the MLP for CUDA float32 params [5378], x (n, 16), t (n, 2)."""
    import torch
    params, x, t = params.contiguous(), x.contiguous(), t.contiguous()
    g = torch.empty(CT_MLP_NPARAMS, dtype=torch.float32, device="cuda")
    loss = C.c_double()
    _check(_load().ct_mlp_loss_grad(params.data_ptr(), x.data_ptr(), t.data_ptr(), x.shape[0], g.data_ptr(),
                                    C.byref(loss), C.c_void_p(_stream(stream))))
    return float(loss.value), g


def ct_mlp_forward_f16(params, x, stream=None):
    """y (n, 2): forward pass with fp16-rounded parameters, fp32 sums."""
    import torch
    params, x = params.contiguous(), x.contiguous()
    y = torch.empty(max(x.shape[0], 1), 2, dtype=torch.float32, device="cuda")
    _check(_load().ct_mlp_forward_f16(params.data_ptr(), x.data_ptr(), x.shape[0], y.data_ptr(),
                                      C.c_void_p(_stream(stream))))
    return y[:x.shape[0]]


def version() -> str:
    return _load().ct_version().decode()
