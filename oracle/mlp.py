"""FP64 reference of the degree/work predictor -- TEST INFRASTRUCTURE ONLY.

The predictor has no counterpart in the paper: it is a small multilayer
perceptron, 16 inputs -> 64 -> 64 -> 2 outputs with ReLU after both hidden
layers, trained by mean squared error.  This module is the plain definition,
in float64, used to check the GPU kernels' forward pass and gradients:

    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  y = W3 h2 + b3
    loss = (1 / n) * sum over samples and outputs of (y - t)^2

Parameters are one flat vector in the order W1 (64 x 16, row-major), b1,
W2 (64 x 64), b2, W3 (2 x 64), b3 -- the library's layout.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 16, 64, 2
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape)
        o += k
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(theta, x):
    p = unpack(theta)
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (x, a1, h1, a2, h2)


def loss(theta, x, t) -> float:
    y, _ = forward(theta, x)
    n = max(len(x), 1)
    return float(np.sum((y - np.asarray(t, dtype=np.float64)) ** 2) / n)


def loss_grad(theta, x, t):
    """Loss and its analytic gradient (backpropagation), flat in the library order."""
    p = unpack(theta)
    y, (x, a1, h1, a2, h2) = forward(theta, x)
    n = max(len(x), 1)
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / n
    g = {"W3": dy.T @ h2, "b3": dy.sum(0)}
    dh2 = (dy @ p["W3"]) * (a2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(0)
    dh1 = (dh2 @ p["W2"]) * (a1 > 0)
    g["W1"] = dh1.T @ x
    g["b1"] = dh1.sum(0)
    return float(np.sum((y - t) ** 2) / n), pack(g)


def finite_difference(theta, x, t, idx, h=1e-6) -> float:
    """Central difference of the loss in parameter idx."""
    a = np.array(theta, dtype=np.float64)
    b = np.array(theta, dtype=np.float64)
    a[idx] += h
    b[idx] -= h
    return (loss(a, x, t) - loss(b, x, t)) / (2 * h)


GROUP_SIZE = 32


def query_groups(tree):
    """Query groups of a tree in the flat export format: runs of consecutive
    sibling leaf blocks (in position order) holding at most 32 points in
    total; a larger leaf block is cut into groups of 32 consecutive points
    (the last one shorter), none shared with another block.  Returns
    (begin, count) position arrays."""
    N = len(tree["center"])
    parent = np.full(N, -1, np.int64)
    for v in range(N):
        cb, cc = int(tree["child_begin"][v]), int(tree["child_count"][v])
        parent[cb:cb + cc] = v
    leaves = [v for v in range(N) if tree["child_count"][v] == 0]
    leaves.sort(key=lambda v: int(tree["pts_begin"][v]))
    gb, gc, cur = [], [], None
    for v in leaves:
        b, c, p = int(tree["pts_begin"][v]), int(tree["pts_count"][v]), int(parent[v])
        if c > GROUP_SIZE:
            for k in range(0, c, GROUP_SIZE):
                gb.append(b + k)
                gc.append(min(GROUP_SIZE, c - k))
            cur = None      # the next block starts a group of its own
        elif gc and p == cur and gc[-1] + c <= GROUP_SIZE:
            gc[-1] += c
        else:
            gb.append(b)
            gc.append(c)
            cur = p
    return np.array(gb, np.int64), np.array(gc, np.int64), parent


def features(tree, points, eps):
    """The predictor's 16 features of every tree position, in float64, from
    the definition (the library computes them in fp32), e = max(eps, 1e-20):
      0 log1p(d(q, leaf-block centre)/e)   1 log1p(d(q, group centre)/e)
      2 log1p(group radius/e)              3 log2(group size)
      4..11 leaf block and its first three ancestors (the root repeats):
            log1p(points below), log1p(radius/e)
      12..15 log1p(points below the lowest ancestor, starting at the leaf
            block, with radius >= e, 2e, 4e, 16e; the root if none)
    Group centre = its first point, group radius = the largest distance of
    its points to that centre."""
    x = np.asarray(points, dtype=np.float64)
    e = max(float(eps), 1e-20)
    N = len(tree["center"])
    pos = np.asarray(tree["leaf_pts"], np.int64)        # position -> original id
    n = len(pos)
    gb, gc, parent = query_groups(tree)
    below = np.zeros(N, np.int64)
    for v in range(N - 1, -1, -1):                      # children have larger ids
        if tree["child_count"][v] == 0:
            below[v] = tree["pts_count"][v]
        else:
            cb, cc = int(tree["child_begin"][v]), int(tree["child_count"][v])
            below[v] = below[cb:cb + cc].sum()
    leaf_of = np.zeros(n, np.int64)
    for v in range(N):
        if tree["child_count"][v] == 0:
            b, c = int(tree["pts_begin"][v]), int(tree["pts_count"][v])
            leaf_of[b:b + c] = v
    group_of = np.repeat(np.arange(len(gb)), gc)
    radius = np.asarray(tree["radius"], np.float64)
    grad_ = np.zeros(len(gb))
    for g in range(len(gb)):
        c = x[pos[gb[g]]]
        grad_[g] = np.sqrt(((x[pos[gb[g]:gb[g] + gc[g]]] - c) ** 2).sum(1)).max()
    F = np.zeros((n, N_IN))
    for i in range(n):
        q = x[pos[i]]
        v = int(leaf_of[i])
        g = int(group_of[i])
        F[i, 0] = np.log1p(np.sqrt(((q - x[tree["center"][v]]) ** 2).sum()) / e)
        F[i, 1] = np.log1p(np.sqrt(((q - x[pos[gb[g]]]) ** 2).sum()) / e)
        F[i, 2] = np.log1p(grad_[g] / e)
        F[i, 3] = np.log2(gc[g])
        a = v
        for k in range(4):
            F[i, 4 + 2 * k] = np.log1p(below[a])
            F[i, 5 + 2 * k] = np.log1p(radius[a] / e)
            if k < 3 and parent[a] >= 0:
                a = int(parent[a])
        for col, f in ((12, 1.0), (13, 2.0), (14, 4.0), (15, 16.0)):
            a = v
            while radius[a] < f * e and parent[a] >= 0:
                a = int(parent[a])
            F[i, col] = np.log1p(below[a])
    return F
