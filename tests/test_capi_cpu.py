"""The C-ABI library builds, loads and exports every declared entry point;
argument errors are reported without touching a GPU.  CPU only."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_14147_gb300 import build
    return C.CDLL(build.build())


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("ct_build", "eps_graph_query", "eps_graph_query_batched", "csr_free",
                     "ct_tree_free", "ct_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_invalid_arguments_without_gpu():
    from paper_2510_14147_gb300 import ctgraph as cg
    lib = cg._load()
    out = C.c_void_p(123)
    assert lib.ct_build(None, None, None, C.byref(out)) == cg.CT_EINVAL
    assert out.value is None
    assert "NULL" in cg.ct_last_error()
    p = cg.ct_points(cg.CT_L2_F32, 0, -5, None, None)
    assert lib.ct_build(C.byref(p), None, None, C.byref(out)) == cg.CT_EINVAL
    p = cg.ct_points(cg.CT_L2_F32, 0, 10, None, None)
    assert lib.ct_build(C.byref(p), None, None, C.byref(out)) == cg.CT_EINVAL   # dim 0
    p = cg.ct_points(7, 3, 10, None, None)
    assert lib.ct_build(C.byref(p), None, None, C.byref(out)) == cg.CT_EINVAL   # metric
    p = cg.ct_points(cg.CT_L2_F32, 3, 1 << 40, 1, None)
    assert lib.ct_build(C.byref(p), None, None, C.byref(out)) == cg.CT_EOVERFLOW
    csr = cg.ct_csr()
    assert lib.eps_graph_query(None, 1.0, None, None, C.byref(csr)) == cg.CT_EINVAL
    assert csr.row_ptr is None and csr.nnz == 0
    lib.csr_free(None)               # NULL-safe
    lib.csr_free(C.byref(csr))       # idempotent on an empty CSR
    lib.ct_tree_free(None)
    assert lib.eps_graph_query_batched(-1, None, None, None, None, None) == cg.CT_EINVAL
    assert lib.eps_graph_query_batched(0, None, None, None, None, None) == cg.CT_OK
    assert lib.ct_autotune(-1, None, None, None, None, None) == cg.CT_EINVAL
    assert lib.ct_autotune(0, None, None, None, None, None) == cg.CT_OK
    lib.ct_autotune_reset()
    st = cg.ct_query_stats()
    assert lib.ct_csr_stats(C.byref(csr), C.byref(st)) == cg.CT_EINVAL
    # predictor entry points
    assert lib.ct_predictor_create(0, None) == cg.CT_EINVAL
    lib.ct_predictor_free(None)
    assert lib.ct_predictor_fit(None, None, 1.0, None, None, None) == cg.CT_EINVAL
    assert lib.ct_predictor_set_capacity(None, 0.5, 16, 0.25, 0) == cg.CT_EINVAL
    assert lib.ct_predictor_set_order(None, 1) == cg.CT_EINVAL
    assert lib.ct_predictor_get_params(None, None, None) == cg.CT_EINVAL
    assert lib.ct_predictor_set_params(None, None, None) == cg.CT_EINVAL
    assert lib.ct_predictor_features(None, 1.0, None, None) == cg.CT_EINVAL
    assert lib.ct_predictor_predict(None, None, 1.0, None, None, None) == cg.CT_EINVAL
    assert lib.ct_mlp_loss_grad(None, None, None, 4, None, None, None) == cg.CT_EINVAL
    assert lib.ct_mlp_forward_f16(None, None, -1, None, None) == cg.CT_EINVAL


def test_product_path_has_no_cpu_fallback():
    """The binding never imports the oracle and refuses to run without the library."""
    src = open(os.path.join(ROOT, "paper_2510_14147_gb300", "ctgraph.py")).read()
    assert "oracle" not in src.replace("# ", "")
    for f in os.listdir(os.path.join(ROOT, "paper_2510_14147_gb300")):
        if f.endswith(".py"):
            assert "import oracle" not in open(os.path.join(ROOT, "paper_2510_14147_gb300", f)).read()
