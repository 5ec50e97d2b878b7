"""Pins for the FP64 predictor reference: closed-form cases and central finite
differences of the loss."""
import numpy as np

from oracle import mlp


def _theta(seed=0, scale=0.3):
    return np.random.default_rng(seed).normal(0.0, scale, mlp.N_PARAMS)


def test_layout_size():
    assert mlp.N_PARAMS == 64 * 16 + 64 + 64 * 64 + 64 + 2 * 64 + 2


def test_zero_weights_give_bias():
    theta = np.zeros(mlp.N_PARAMS)
    p = mlp.unpack(theta)
    p["b3"][:] = [1.5, -2.0]
    theta = mlp.pack(p)
    y, _ = mlp.forward(theta, np.ones((3, 16)))
    assert np.array_equal(y, np.tile([1.5, -2.0], (3, 1)))
    assert mlp.loss(theta, np.ones((3, 16)), np.tile([1.5, -2.0], (3, 1))) == 0.0


def test_linear_regime_closed_form():
    """With all pre-activations positive the network is affine; its loss
    gradient w.r.t. b3 is 2 mean(y - t)."""
    rng = np.random.default_rng(1)
    p = mlp.unpack(np.zeros(mlp.N_PARAMS))
    p["W1"][:] = np.abs(rng.normal(size=p["W1"].shape)) * 0.1
    p["b1"][:] = 1.0
    p["W2"][:] = np.abs(rng.normal(size=p["W2"].shape)) * 0.1
    p["b2"][:] = 1.0
    p["W3"][:] = rng.normal(size=p["W3"].shape)
    theta = mlp.pack(p)
    x = np.abs(rng.normal(size=(10, 16)))
    t = rng.normal(size=(10, 2))
    y, _ = mlp.forward(theta, x)
    affine = ((x @ p["W1"].T + 1.0) @ p["W2"].T + 1.0) @ p["W3"].T
    assert np.allclose(y, affine, rtol=0, atol=1e-12)
    _, g = mlp.loss_grad(theta, x, t)
    gb3 = mlp.unpack(g)["b3"]
    assert np.allclose(gb3, 2.0 * (y - t).mean(0), rtol=0, atol=1e-12)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    theta = _theta(3)
    x = rng.normal(size=(40, 16))
    t = rng.normal(size=(40, 2))
    _, g = mlp.loss_grad(theta, x, t)
    idx = rng.choice(mlp.N_PARAMS, size=60, replace=False)
    for i in idx:
        fd = mlp.finite_difference(theta, x, t, i)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_planted_mistake_in_backward_is_caught():
    """A gradient with one term dropped differs from finite differences."""
    rng = np.random.default_rng(4)
    theta = _theta(5)
    x = rng.normal(size=(20, 16))
    t = rng.normal(size=(20, 2))
    _, g = mlp.loss_grad(theta, x, t)
    bad = mlp.unpack(g)
    bad["b2"] = bad["b2"] * 0.0
    badg = mlp.pack(bad)
    i = mlp.N_PARAMS - 2 - 128 - 64 + 5       # an entry of b2
    fd = mlp.finite_difference(theta, x, t, i)
    assert abs(fd - g[i]) < 1e-6 * max(1, abs(g[i]))
    assert abs(fd) < 1e-12 or abs(fd - badg[i]) > 1e-6


def _two_leaf_tree():
    # four points on a line; root (centre p0, radius 11) with two leaf blocks
    pts = np.array([[0.0, 0.0], [1.0, 0.0], [10.0, 0.0], [11.0, 0.0]])
    tree = {"center": np.array([0, 0, 2]), "radius": np.array([11.0, 1.0, 1.0]),
            "level": np.array([4, 0, 0]), "child_begin": np.array([1, 0, 0]),
            "child_count": np.array([2, 0, 0]), "pts_begin": np.array([0, 0, 2]),
            "pts_count": np.array([0, 2, 2]), "leaf_pts": np.array([0, 1, 2, 3])}
    return tree, pts


def test_features_hand_computed():
    """Both sibling leaves form one query group (4 <= 32 points): values by hand."""
    tree, pts = _two_leaf_tree()
    gb, gc, parent = mlp.query_groups(tree)
    assert list(gb) == [0] and list(gc) == [4] and list(parent) == [-1, 0, 0]
    F = mlp.features(tree, pts, 1.0)
    L = np.log1p
    anc = [L(2), L(1), L(4), L(11), L(4), L(11), L(4), L(11)]   # leaf, root, root, root
    want1 = [L(1), L(1), L(11), 2.0] + anc + [L(2), L(4), L(4), L(4)]
    want2 = [0.0, L(10), L(11), 2.0] + anc + [L(2), L(4), L(4), L(4)]
    assert np.allclose(F[1], want1, rtol=0, atol=1e-15)
    assert np.allclose(F[2], want2, rtol=0, atol=1e-15)
    # eps = 0.5: the leaf block (radius 1) already has radius >= e and >= 2e
    F = mlp.features(tree, pts, 0.5)
    assert list(F[0, 12:16]) == [L(2), L(2), L(4), L(4)]


def test_query_groups_split_at_32_points():
    """Sibling leaves are merged while the run stays at most 32 points; a
    leaf of another parent starts a new group; a leaf block above 32 points is
    cut into groups of 32 (the last one shorter) of its own, and the sibling
    after it starts a new group."""
    # root 0 -> children 1..5 (1..4 leaf blocks of 20, 12, 5, 40 points; 5
    # internal) and 5 -> leaf block 6 of 3 points
    tree = {"center": np.zeros(7, np.int64), "radius": np.ones(7),
            "level": np.zeros(7, np.int32),
            "child_begin": np.array([1, 0, 0, 0, 0, 6, 0]), "child_count": np.array([5, 0, 0, 0, 0, 1, 0]),
            "pts_begin": np.array([0, 0, 20, 32, 37, 0, 77]), "pts_count": np.array([0, 20, 12, 5, 40, 0, 3]),
            "leaf_pts": np.arange(80)}
    gb, gc, _ = mlp.query_groups(tree)
    assert list(gb) == [0, 32, 37, 69, 77] and list(gc) == [32, 5, 32, 8, 3]
    # a small sibling after the large block does not join its last group
    tree2 = {"center": np.zeros(6, np.int64), "radius": np.ones(6), "level": np.zeros(6, np.int32),
             "child_begin": np.array([1, 0, 0, 0, 0, 0]), "child_count": np.array([5, 0, 0, 0, 0, 0]),
             "pts_begin": np.array([0, 0, 20, 32, 37, 77]), "pts_count": np.array([0, 20, 12, 5, 40, 3]),
             "leaf_pts": np.arange(80)}
    gb, gc, _ = mlp.query_groups(tree2)
    assert list(gb) == [0, 32, 37, 69, 77] and list(gc) == [32, 5, 32, 8, 3]
