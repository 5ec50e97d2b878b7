"""Shared helpers of the tests: run the CUDA path through the C-ABI binding and
compare its CSR with the oracle's."""
import numpy as np

import oracle


def gpu_graph(points=None, strings=None, eps=0.0, leaf_size=32, root=0, precision=0,
              include_self=False, predictor=None, use_predictor=False, export=False):
    import torch
    from paper_2510_14147_gb300 import ctgraph as cg
    if points is not None:
        t = cg.ct_build(points=torch.from_numpy(np.ascontiguousarray(points, np.float32)).cuda(),
                        leaf_size=leaf_size, root=root)
    else:
        data, off = strings
        t = cg.ct_build(strings=(torch.from_numpy(np.ascontiguousarray(data, np.uint8)).cuda(),
                                 torch.from_numpy(np.ascontiguousarray(off, np.int64)).cuda()),
                        leaf_size=leaf_size, root=root)
    csr = cg.eps_graph_query(t, eps, precision=precision, include_self=include_self,
                             predictor=predictor, use_predictor=use_predictor)
    out = csr.to_numpy()
    out["stats"] = csr.stats()
    csr.free()
    if export:
        out["tree"] = cg.ct_tree_export(t)
    t.free()
    return out


def assert_csr_matches(gpu: dict, ref: dict, rtol: float = 1e-6, integer_dist: bool = False):
    """Exact row_ptr and col; dist within rtol relative of the oracle's FP64."""
    rp_g, rp_r = np.asarray(gpu["row_ptr"], np.int64), np.asarray(ref["row_ptr"], np.int64)
    assert rp_g.shape == rp_r.shape, (rp_g.shape, rp_r.shape)
    if not np.array_equal(rp_g, rp_r):
        bad = np.flatnonzero(np.diff(rp_g) != np.diff(rp_r))
        raise AssertionError("degree mismatch in %d rows, first %s: gpu %d vs oracle %d" % (
            bad.size, bad[:5], np.diff(rp_g)[bad[0]], np.diff(rp_r)[bad[0]]))
    cg_, cr = np.asarray(gpu["col"], np.int64), np.asarray(ref["col"], np.int64)
    if not np.array_equal(cg_, cr):
        i = int(np.flatnonzero(cg_ != cr)[0])
        raise AssertionError("col mismatch at entry %d: gpu %d vs oracle %d" % (i, cg_[i], cr[i]))
    dg, dr = np.asarray(gpu["dist"], np.float64), np.asarray(ref["dist"], np.float64)
    if integer_dist:
        assert np.array_equal(dg, dr)
    else:
        err = np.abs(dg - dr)
        tol = rtol * np.abs(dr)
        bad = err > tol
        assert not bad.any(), "dist off by %g relative (max)" % float(np.max(err / np.maximum(np.abs(dr), 1e-300)))


def tree_from_export(a: dict) -> oracle.Tree:
    return oracle.Tree(**a)
