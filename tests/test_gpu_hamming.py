"""Hamming ε-graphs on the GPU (the paper's binary datasets, sift-hamming and
word2bits, Sec. V-A and Table I), through the C-ABI: exact integer parity
with the oracle's brute force, GPU-built trees through the oracle's
invariant checker, and the forms that share the path (learned one-pass emit,
radius sweeps, tree files)."""
import numpy as np
import pytest

import oracle
from paper_2510_14147_gb300 import inputs as I
from helpers import assert_csr_matches, tree_from_export

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


def _tree(rows, dim, leaf_size=32, root=0):
    import torch
    return _cg().ct_build(bits=(torch.from_numpy(np.ascontiguousarray(rows)).cuda(), dim), leaf_size=leaf_size,
                          root=root)


def _graph(rows, dim, eps, **kw):
    cg = _cg()
    ts = {k: kw.pop(k) for k in ("leaf_size", "root") if k in kw}
    t = _tree(rows, dim, **ts)
    c = cg.eps_graph_query(t, eps, **kw)
    out = c.to_numpy()
    out["stats"] = c.stats()
    out["tree"] = cg.ct_tree_export(t)
    c.free()
    t.free()
    return out


@pytest.mark.parametrize("dim,n,zeta,seed", [(1, 300, 8, 0), (13, 1500, 4, 1), (64, 2500, 32, 2),
                                             (256, 3000, 32, 3), (800, 1600, 16, 4), (4096, 500, 32, 5)])
def test_hamming_parity_and_tree(dim, n, zeta, seed):
    rows = I.binary_codes(n, dim, n_centres=15, flip=0.05, seed=seed)
    sp = oracle.Space(bits=(rows, dim))
    for eps in (0, max(1, dim // 20), dim // 6 + 0.5, dim):
        out = _graph(rows, dim, eps, leaf_size=zeta)
        assert_csr_matches(out, oracle.brute_force(sp, eps), integer_dist=True)
    code, msg = oracle.check_tree(sp, tree_from_export(out["tree"]), 0.0)
    assert code == 0, msg


def test_hamming_degenerate_and_duplicates():
    for n in (0, 1, 2, 33):
        rows = I.binary_codes(n, 40, n_centres=3, flip=0.1, seed=n)
        sp = oracle.Space(bits=(rows, 40))
        for eps in (0, 5, 40):
            out = _graph(rows, 40, eps)
            assert_csr_matches(out, oracle.brute_force(sp, eps), integer_dist=True)
    rows = I.binary_codes(700, 96, n_centres=4, flip=0.0, seed=7)   # duplicate classes far above zeta
    sp = oracle.Space(bits=(rows, 96))
    for eps in (0, 30):
        for inc in (False, True):
            out = _graph(rows, 96, eps, include_self=inc)
            assert_csr_matches(out, oracle.brute_force(sp, eps, include_self=inc), integer_dist=True)


@pytest.mark.parametrize("dim", [64, 256])
def test_hamming_uniform_codes(dim):
    """Uniform random codes: all distances lie near dim / 2, above the lower
    levels' thresholds, so splits there make almost every point a child (or
    stop early as flat splits); the graph stays exact and the tree valid."""
    rng = np.random.default_rng(8)
    rows = np.packbits(rng.random((5000, dim)) < 0.5, axis=1, bitorder="little")
    sp = oracle.Space(bits=(rows, dim))
    for eps in (dim // 4, dim // 2 - 4):
        out = _graph(rows, dim, eps)
        assert_csr_matches(out, oracle.brute_force(sp, eps), integer_dist=True)
    assert oracle.check_tree(sp, tree_from_export(out["tree"]), 0.0)[0] == 0


def test_hamming_root_and_trailing_bits_ignored():
    rows = I.binary_codes(1200, 21, n_centres=5, flip=0.1, seed=9)
    noisy = rows.copy()
    noisy[:, -1] |= np.uint8(0xE0)          # bits 21..23 of the last byte are not part of the rows
    sp = oracle.Space(bits=(rows, 21))
    ref = oracle.brute_force(sp, 3)
    for r in (0, 777):
        assert_csr_matches(_graph(noisy, 21, 3, root=r), ref, integer_dist=True)


def test_hamming_learned_sweep_and_file(tmp_path):
    import torch
    cg = _cg()
    rows = I.binary_codes(4000, 256, n_centres=40, flip=0.05, seed=10)
    sp = oracle.Space(bits=(rows, 256))
    t = _tree(rows, 256)
    pred = cg.ct_predictor_create(seed=1)
    cg.ct_predictor_fit(pred, t, 20, steps=200, seed=2)
    for eps in (12, 20):
        a = cg.eps_graph_query(t, eps)
        b = cg.eps_graph_query(t, eps, use_predictor=True, predictor=pred)
        for k in ("row_ptr", "col", "dist"):
            assert torch.equal(getattr(a, k), getattr(b, k))
        assert_csr_matches(a.to_numpy(), oracle.brute_force(sp, eps), integer_dist=True)
        a.free()
        b.free()
    sw = cg.eps_graph_query_sweep(t, [20, 12, 16])
    for e, c in zip((20, 12, 16), sw):
        assert_csr_matches(c.to_numpy(), oracle.brute_force(sp, e), integer_dist=True)
        c.free()
    path = str(tmp_path / "ham.cttree")
    cg.ct_tree_save(t, path)
    t2 = cg.ct_tree_load(path)
    x, y = cg.eps_graph_query(t, 16), cg.eps_graph_query(t2, 16)
    assert torch.equal(x.col, y.col) and torch.equal(x.row_ptr, y.row_ptr)
    x.free()
    y.free()
    t2.free()
    t.free()
