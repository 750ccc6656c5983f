"""Pins of the reference PLOC builder (oracle.ploc_f32) against facts independent of it.

PLOC (parallel locally-ordered clustering, Meister & Bittner 2018) merges
mutual nearest neighbours, by the surface area of their union, within a
window of the Morton-ordered cluster list, round after round. The pins:
hand-worked trees (boxes on a line, a tie), the balanced tree that equal boxes
give, the globally closest pair (brute force) merged into one node when the
window covers everything, the validity of the tree (every leaf once, every child box
the union of its subtree), the Morton order shared with the LBVH, and a lower
surface-area cost than the LBVH on clustered boxes. CPU only.
"""
import itertools

import numpy as np
import pytest

LEAF = 0x80000000


def _leaf(k):
    """child-array value of the leaf at sorted position k"""
    return int(np.uint32(LEAF | k).view(np.int32))


def _boxes_on_x(xs, half=0.25):
    xs = np.asarray(xs, np.float32)
    lo = np.stack([xs - half, np.zeros_like(xs), np.zeros_like(xs)], 1)
    hi = np.stack([xs + half, np.ones_like(xs), np.ones_like(xs)], 1)
    return np.concatenate([lo, hi], 1).astype(np.float32)


def _half_area(b):
    d = np.asarray(b[3:], np.float64) - np.asarray(b[:3], np.float64)
    return d[0] * d[1] + d[1] * d[2] + d[2] * d[0]


def _union(a, b):
    return np.concatenate([np.minimum(a[:3], b[:3]), np.maximum(a[3:], b[3:])])


def _check_tree(r, boxes):
    """Every leaf once, every internal node but the root once, child boxes the unions
    of their subtrees, root the union of all boxes; returns leaf depths."""
    n = len(boxes)
    perm, child, cbox = r["perm"], r["child"], r["cbox"]
    assert sorted(perm.tolist()) == list(range(n))
    seen_leaf = np.zeros(n, int)
    seen_node = np.zeros(max(n - 1, 1), int)
    depth = np.zeros(n, int)

    def visit(node, d):
        seen_node[node] += 1
        bx = []
        for side in (0, 1):
            ref = int(child[node, side])
            if ref < 0:
                k = ref & 0x7FFFFFFF
                seen_leaf[k] += 1
                depth[k] = d + 1
                b = boxes[perm[k]].astype(np.float32)
            else:
                b = visit(ref, d + 1)
            assert np.array_equal(cbox[node, 6 * side:6 * side + 6], b)
            bx.append(b)
        return _union(bx[0], bx[1]).astype(np.float32)

    root = visit(0, 0)
    assert np.array_equal(root, r["root"])
    assert (seen_leaf == 1).all() and (seen_node[: n - 1] == 1).all()
    assert np.array_equal(r["root"], np.concatenate([boxes[:, :3].min(0), boxes[:, 3:].max(0)]))
    return depth


def test_ploc_boxes_on_a_line(oracle_lib):
    # two far-apart pairs: round 1 merges (0,1) -> node 2 and (2,3) -> node 1, round 2 the root
    r = oracle_lib.ploc_f32(_boxes_on_x([0.0, 1.0, 10.0, 11.0]))
    assert r["perm"].tolist() == [0, 1, 2, 3]
    assert r["child"].tolist() == [[2, 1], [_leaf(2), _leaf(3)], [_leaf(0), _leaf(1)]]


def test_ploc_tie_goes_to_the_even_lower_pair(oracle_lib):
    # equal gaps: cluster 1 is as close to 0 as to 2; the pair {0,1} (lower index even) wins
    r = oracle_lib.ploc_f32(_boxes_on_x([0.0, 1.0, 2.0]))
    assert r["child"].tolist() == [[1, _leaf(2)], [_leaf(0), _leaf(1)]]


def test_ploc_flat_boxes_merge_by_area(oracle_lib):
    # boxes flat in z (no volume): the union areas still order the pairs, {1,2} is closest
    b = _boxes_on_x([0.0, 1.0, 1.2], half=0.05)
    b[:, 5] = b[:, 2]
    r = oracle_lib.ploc_f32(b)
    assert r["child"].tolist() == [[_leaf(0), 1], [_leaf(1), _leaf(2)]]


@pytest.mark.parametrize("n", [2, 8, 16, 64])
def test_ploc_equal_boxes_give_a_balanced_tree(oracle_lib, n):
    boxes = np.tile(np.array([[0, 0, 0, 1, 1, 1]], np.float32), (n, 1))
    r = oracle_lib.ploc_f32(boxes)
    depth = _check_tree(r, boxes)
    assert (depth == int(np.log2(n))).all()


@pytest.mark.parametrize("n", [3, 9, 40])
def test_ploc_merges_the_closest_pair(oracle_lib, n):
    """With the window covering the whole list, the least pair over all pairs (brute
    force, FP64 areas) is mutual in the first round: a node has exactly those two leaves."""
    rng = np.random.default_rng(100 + n)
    c = rng.uniform(-10, 10, (n, 3))
    e = rng.uniform(0.1, 1.5, (n, 3))
    boxes = np.concatenate([c - e, c + e], 1).astype(np.float32)
    r = oracle_lib.ploc_f32(boxes, radius=n)
    pos = {int(k): i for i, k in enumerate(r["perm"])}
    best = min(itertools.combinations(range(n), 2), key=lambda p: _half_area(_union(boxes[p[0]], boxes[p[1]])))
    want = sorted(_leaf(pos[k]) for k in best)
    assert any(sorted(int(x) for x in row) == want for row in r["child"])


@pytest.mark.parametrize("n,dups", [(2, False), (3, False), (17, False), (100, True), (1025, False), (3000, True)])
def test_ploc_tree_is_valid_and_shares_the_morton_order(oracle_lib, n, dups):
    rng = np.random.default_rng(n)
    lo = rng.uniform(-30, 30, (n, 3)).astype(np.float32)
    boxes = np.concatenate([lo, lo + rng.uniform(0, 3, (n, 3)).astype(np.float32)], 1)
    if dups:
        boxes[n // 2:] = boxes[: n - n // 2]
    r = oracle_lib.ploc_f32(boxes)
    _check_tree(r, boxes)
    l = oracle_lib.lbvh_f32(boxes)
    assert np.array_equal(r["perm"], l["perm"]) and np.array_equal(r["codes"], l["codes"])


def test_ploc_single_leaf_and_radius_zero(oracle_lib):
    box = np.array([[1, 2, 3, 4, 5, 6]], np.float32)
    r = oracle_lib.ploc_f32(box)
    assert r["perm"].tolist() == [0] and np.array_equal(r["root"], box[0])
    with pytest.raises(ValueError):
        oracle_lib.ploc_f32(_boxes_on_x([0.0, 1.0]), radius=0)


def sah_cost(r, boxes, c_node=1.0, c_leaf=1.0):
    """Surface-area cost: sum over internal nodes of area / root area, plus leaves."""
    root = _half_area(r["root"])
    cost = 0.0
    for node in range(len(r["child"])):
        b = _union(r["cbox"][node, :6], r["cbox"][node, 6:])
        cost += c_node * _half_area(b) / root
    for k in range(len(boxes)):
        cost += c_leaf * _half_area(boxes[k]) / root
    return cost


def test_ploc_sah_cost_below_lbvh(oracle_lib):
    """Clustered boxes of mixed sizes: the clustered tree costs less than the radix tree
    of the same Morton order (the quality PLOC is built for)."""
    rng = np.random.default_rng(7)
    centres = rng.uniform(-100, 100, (40, 3))
    pts = centres[rng.integers(0, 40, 3000)] + rng.normal(0, 4, (3000, 3))
    ext = np.exp(rng.normal(-0.5, 0.8, (3000, 3)))
    boxes = np.concatenate([pts - ext, pts + ext], 1).astype(np.float32)
    p, l = oracle_lib.ploc_f32(boxes), oracle_lib.lbvh_f32(boxes)
    assert sah_cost(p, boxes) < 0.9 * sah_cost(l, boxes)
