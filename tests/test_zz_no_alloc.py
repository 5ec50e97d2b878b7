"""The allocation-free degree count (eps_graph_degrees_noalloc).

It exists for callers that cannot let a library allocate device memory (an
application whose allocator owns the whole device, or a latency-bound loop).
Its temporaries live in one fixed device array inside the library, so the
checks here are: the source of the call path names no allocator, and on the
GPU its degrees equal the row lengths of eps_graph_query, on two calls in a
row (the array keeps the previous call's contents), with a clear error when a
problem does not fit the array."""
import os

import numpy as np
import pytest

from paper_2510_14147_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_call_path_names_no_allocator():
    src = open(os.path.join(ROOT, "paper_2510_14147_gb300", "csrc", "query.cu")).read()
    start = src.index("void degrees_noalloc(")
    body = src[start:src.index("\n}\n", start)]
    for tok in ("dmalloc", "DBuf", "cudaMalloc", "cudaFree", "exclusive_scan_i32_to_i64(", "sort_rows("):
        assert tok not in body, tok
    assert "static __device__ __align__(256)" in src


@pytest.mark.gpu
def test_noalloc_degrees_equal_query_rows_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14147_gb300 import build
    build.build()
    from paper_2510_14147_gb300 import ctgraph as cg
    # the larger problem first, so that the smaller one runs over the array's
    # leftovers (more segments, a longer pool, spill counts); then the
    # larger one again, and both with include_self
    big = I.gmm_embedded(20000, dim=64, intrinsic=6, n_centres=4, seed=1)
    d = np.sqrt(((big[:200, None, :].astype(np.float64) - big[None, :2000, :]) ** 2).sum(-1))
    big_eps = float(np.float32(np.quantile(d, 0.01)))
    cases = [(big, big_eps, False), (I.uniform_cube(3000, 3, seed=0), 0.08, False),
             (big, big_eps, True), (I.uniform_cube(3000, 3, seed=0), 0.08, True)]
    for x, eps, include_self in cases:
        xd = torch.from_numpy(x).cuda()
        tree = cg.ct_build(points=xd)
        csr = cg.eps_graph_query(tree, eps, include_self=include_self)
        ref = np.diff(csr.row_ptr.cpu().numpy())
        csr.free()
        deg = torch.empty(x.shape[0], dtype=torch.int32, device="cuda")
        for _ in range(2):
            deg.fill_(-7)
            cg.eps_graph_degrees_noalloc(tree, eps, deg, include_self=include_self)
            torch.cuda.synchronize()
            assert np.array_equal(deg.cpu().numpy(), ref)
        tree.free()


@pytest.mark.gpu
def test_noalloc_rejects_what_does_not_fit():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14147_gb300 import build
    build.build()
    from paper_2510_14147_gb300 import ctgraph as cg
    x = I.uniform_cube(60000, 3, seed=2)
    tree = cg.ct_build(points=torch.from_numpy(x).cuda())
    deg = torch.empty(x.shape[0], dtype=torch.int32, device="cuda")
    with pytest.raises(cg.CtError) as e:
        cg.eps_graph_degrees_noalloc(tree, 10.0, deg)      # every pair: too many candidates
    assert e.value.status == cg.CT_EUNSUPPORTED and "scratch" in str(e.value)
    cg.eps_graph_degrees_noalloc(tree, 0.01, deg)          # still usable afterwards
    torch.cuda.synchronize()
    tree.free()
    data, off = I.dna_strings(n_seeds=2, per_seed=10, seed=1)
    st = cg.ct_build(strings=(torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda()))
    with pytest.raises(cg.CtError) as e:
        cg.eps_graph_degrees_noalloc(st, 3, torch.empty(20, dtype=torch.int32, device="cuda"))
    assert e.value.status == cg.CT_EUNSUPPORTED
    st.free()
