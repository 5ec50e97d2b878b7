"""The GPU-built trees of the benchmark's workloads -- the 1M x 128 mixture
and every one of the 64 clouds -- pass the oracle's cover-tree invariant
checker (nesting, covering within 2^l, separation above 2^(l-1), every point
within its vertices' stored radii in FP64; Sec. III and Sec. IV-A) at the
relative tolerance the build's arithmetic allows: fp32-decided splits (their
distances err by less than 2^-17) plus the 2^-16 by which a stored radius is
rounded up (the query's pruning bound), 2^-16 + 2^-17 < 2.5e-5."""
import numpy as np
import pytest

import oracle
from paper_2510_14147_gb300 import inputs as I
from helpers import tree_from_export

pytestmark = pytest.mark.gpu

TOL = 2.5e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14147_gb300 import build
    build.build()
    oracle.build()


def _check(x):
    import torch
    from paper_2510_14147_gb300 import ctgraph as cg
    t = cg.ct_build(points=torch.from_numpy(x).cuda())
    ex = cg.ct_tree_export(t)
    t.free()
    code, msg = oracle.check_tree(oracle.Space(points=x), tree_from_export(ex), TOL)
    assert code == 0, msg


def test_tree_of_gmm_1m_within_tolerance():
    wl = I.load_workloads()["gmm_1m_k70"]
    _check(I.gmm_embedded(wl["n"], dim=wl["dim"], seed=wl["seed"]))


def test_trees_of_all_64_clouds_within_tolerance():
    for sp in I.load_workloads()["clouds_64"]["specs"]:
        _check(I.cloud_points(sp))
