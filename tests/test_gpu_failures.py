"""Failure paths in the forms allowed on this hardware (no GPU fault, trap or
hang is ever provoked):

- host-side fault injection: the k-th device allocation of a call fails;
  every entry point returns CT_ENOMEM, zeroes its outputs and leaks nothing
  (the device pool's bytes in use are the same before and after), for every
  k up to the number of allocations the call makes;
- a bounded device wait whose producer is withheld on the host: the
  tensor-core self-test with no MMA issued returns CT_ETIMEOUT and the
  context stays usable (the plans' work-queue wait is covered in
  test_gpu_plan.py)."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2510_14147_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14147_gb300 import build
    build.build()
    oracle.build()


def _cg():
    from paper_2510_14147_gb300 import ctgraph as cg
    return cg


def _raw_query(tree, eps, **kw):
    """eps_graph_query through ctypes with an output struct full of garbage,
    so that the zeroing on failure is visible."""
    cg = _cg()
    out = cg.ct_csr()
    out.n_rows, out.nnz, out.row_ptr, out.col, out.dist, out.priv = 7, 7, 0xdead0, 0xdead0, 0xdead0, 0xdead0
    o = cg._opts(kw.get("precision", 0), kw.get("use_predictor", False), False, kw.get("predictor"),
                 kw.get("upper_triangle", False))
    st = cg._load().eps_graph_query(tree.handle, float(eps), C.byref(o), C.c_void_p(cg._stream(None)),
                                    C.byref(out))
    return st, out


def _inject_all(call, max_k=400):
    """Runs `call` with the k-th allocation failing for k = 1, 2, ... until a
    run completes; each failure must be CT_ENOMEM and leak nothing.  Returns
    the number of failing runs."""
    cg = _cg()
    fails = 0
    for k in range(1, max_k + 1):
        before = cg.ct_debug_pool_used()
        cg.ct_debug_fail_alloc(k)
        try:
            ok = call(k)
        finally:
            cg.ct_debug_fail_alloc(0)
        if ok:
            return fails
        fails += 1
        assert cg.ct_debug_pool_used() == before, "allocation %d: leaked" % k
    raise AssertionError("no complete run within %d allocations" % max_k)


def test_query_entry_points_fail_cleanly():
    import torch
    cg = _cg()
    x = I.gmm_embedded(3000, dim=32, intrinsic=6, n_centres=4, seed=1)
    eps = float(np.float32(np.quantile(oracle.brute_rows(oracle.Space(points=x), 1e30, [0, 1])["dist"], 0.03)))
    t = cg.ct_build(points=torch.from_numpy(x).cuda())
    pred = cg.ct_predictor_create(seed=1)
    cg.ct_predictor_fit(pred, t, eps, steps=50, seed=2)
    ref = cg.eps_graph_query(t, eps).to_numpy()

    for kw in (dict(), dict(precision=1), dict(precision=1, use_predictor=True, predictor=pred, upper_triangle=True)):
        def call(k, kw=kw):
            st, out = _raw_query(t, eps, **kw)
            if st == 0:
                csr = cg.CSR(out)
                got = csr.to_numpy()
                assert np.array_equal(got["col"], ref["col"])
                csr.free()
                return True
            assert st == cg.CT_ENOMEM, (k, st, cg.ct_last_error())
            assert (out.n_rows, out.nnz, out.row_ptr, out.col, out.dist, out.priv) == (0, 0, None, None, None, None)
            return False
        assert _inject_all(call) > 5

    def batched(k):
        try:
            cs = cg.eps_graph_query_batched([t, t], [eps, eps * 0.8])
        except cg.CtError as e:
            assert e.status == cg.CT_ENOMEM
            return False
        for c in cs:
            c.free()
        return True
    assert _inject_all(batched) > 5

    def sweep(k):
        try:
            cs = cg.eps_graph_query_sweep(t, [eps, eps * 0.8, eps * 0.5])
        except cg.CtError as e:
            assert e.status == cg.CT_ENOMEM
            return False
        for c in cs:
            c.free()
        return True
    assert _inject_all(sweep) > 5

    def plan(k):
        try:
            p = cg.ct_plan_create([t], [eps])
        except cg.CtError as e:
            assert e.status == cg.CT_ENOMEM
            return False
        p.free()
        return True
    assert _inject_all(plan) > 5
    t.free()


def test_build_and_load_fail_cleanly(tmp_path):
    import torch
    cg = _cg()
    x = torch.from_numpy(I.uniform_cube(2500, 8, seed=3)).cuda()
    data, off = I.dna_strings(n_seeds=3, per_seed=20, seed=4)
    sd, so = torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda()
    rows = torch.from_numpy(I.binary_codes(1500, 100, n_centres=5, flip=0.1, seed=5)).cuda()

    def builder(**kw):
        def call(k):
            try:
                t = cg.ct_build(**kw)
            except cg.CtError as e:
                assert e.status == cg.CT_ENOMEM, cg.ct_last_error()
                return False
            t.free()
            return True
        return call
    for kw in (dict(points=x), dict(strings=(sd, so)), dict(bits=(rows, 100))):
        assert _inject_all(builder(**kw)) > 5
    t = cg.ct_build(points=x)
    path = str(tmp_path / "t.cttree")
    cg.ct_tree_save(t, path)
    t.free()

    def load(k):
        try:
            t2 = cg.ct_tree_load(path)
        except cg.CtError as e:
            assert e.status == cg.CT_ENOMEM
            return False
        t2.free()
        return True
    assert _inject_all(load) > 5


def test_selftest_wait_runs_out_and_context_survives():
    import torch
    cg = _cg()
    with pytest.raises(cg.CtError) as e:
        cg.ct_selftest_tc_timeout()
    assert e.value.status == cg.CT_ETIMEOUT
    rng = np.random.default_rng(6)
    A = torch.from_numpy(rng.standard_normal((128, 128)).astype(np.float16)).cuda()
    B = torch.from_numpy(rng.standard_normal((32, 128)).astype(np.float16)).cuda()
    D = cg.ct_selftest_tc_gemm(A, B).cpu().numpy()
    ref = A.cpu().numpy().astype(np.float64) @ B.cpu().numpy().astype(np.float64).T
    assert np.allclose(D, ref, rtol=1e-5, atol=1e-3)


@pytest.mark.parametrize("dim", [3, 4, 128])
def test_build_rejects_coordinates_out_of_range(dim):
    """A NaN, an infinity or a coordinate above 2^50 anywhere in the points
    makes ct_build return CT_EUNSUPPORTED (dims 4 and 128 take the float4 row
    copy, dim 3 the padded one); 2^50 itself is accepted."""
    import torch
    cg = _cg()
    x = I.uniform_cube(257, dim, seed=3)
    for bad in (np.nan, np.inf, -np.inf, 2.0 ** 51, -(2.0 ** 51)):
        y = x.copy()
        y[200, dim - 1] = bad
        with pytest.raises(cg.CtError) as e:
            cg.ct_build(points=torch.from_numpy(y).cuda())
        assert e.value.status == cg.CT_EUNSUPPORTED
    y = x.copy()
    y[5, 0] = 2.0 ** 50
    t = cg.ct_build(points=torch.from_numpy(y).cuda())
    t.free()
