"""The traversal-stack bound: a scene whose TLAS and BLAS are both deep, traced
by one ray that enters every box, needs more than PR_STACK_DEPTH stack
entries. The kernel must finish, report PR_ERR_STACK_OVERFLOW in the scene's
error word, and write the pixel (pushes are bounds-checked, so nothing is
written outside the stack).

Construction: box centroids whose Morton codes are 0, 2^0, 2^1, ..., 2^29 and
2^30 - 1, each repeated 16 times. The radix tree over those keys has a left
spine of 30 single-bit splits above a 16-leaf cluster (34 levels). Every box
has its lower corner at the origin, so a ray along +x from x = -1 enters all of
them at t = 1: with equal entry distances the left child is visited first and
every right sibling waits on the stack. The TLAS holds 512 instances of one
BLAS of 512 such AABBs; each primitive is a small sphere the ray misses, so no
hit ever shortens the ray and every node is visited.
"""
import numpy as np
import pytest

import scenes

CHAIN_BITS = 30
CLUSTER = 16
STACK_DEPTH = 64


def _chain_centroids() -> np.ndarray:
    """Centroids in [1, 2]^3 whose 10-bit-per-axis Morton codes (x highest) are
    0, 2^b for b = 0..29 and 2^30 - 1, each CLUSTER times."""
    pts = [np.ones(3)]
    for b in range(CHAIN_BITS):
        level, axis = b // 3, 2 - b % 3
        c = np.ones(3)
        c[axis] = 1.0 + (2 ** level + 0.5) / 1024.0
        pts.append(c)
    pts.append(np.full(3, 2.0))
    return np.repeat(np.array(pts), CLUSTER, axis=0)


def deep_stack_workload(width=1, height=1) -> scenes.Workload:
    cen = _chain_centroids()
    b = scenes.SceneBuilder()
    scenes._standard_rays(b)
    hr, hs = b.add_hit_group(scenes.IS_SPHERE, scenes.CHS_LAMBERT), b.add_hit_group(scenes.IS_SPHERE)
    mat = b.add_material((0.8, 0.8, 0.8))
    aabbs = np.concatenate([np.zeros_like(cen), 2.0 * cen], 1)                 # [0, 2c]: centroid c
    prm = [scenes.params_row(1.9, 1.9, 1.9, 0.05) for _ in range(len(cen))]    # inside every box, off the ray
    blas = b.add_blas([b.add_geometry(aabbs, prm)])
    b.add_record(hr, mat, scenes.IS_SPHERE, 0)
    b.add_record(hs, mat, scenes.IS_SPHERE, 0)
    # BLAS root box [0, 4]^3; instance k scales it by c_k / 2, so its world box is [0, 2 c_k]
    for c in cen:
        xf = np.zeros((3, 4), np.float32)
        xf[0, 0], xf[1, 1], xf[2, 2] = c / 2.0
        b.add_instance(blas, xf.reshape(-1), 0)
    cam = scenes.Camera(np.float32([-1.0, 0.5, 0.5]), np.float32([0.0, 0.5, 0.5]), np.float32([0, 1, 0]), 1.0)
    return scenes.Workload(b.build("deep-stack"), cam, scenes.TraceParams(width, height))


def _left_first_stack_need(lv) -> list:
    """Stack entries held at each leaf (by sorted position) in a depth-first
    walk that visits the left child first and pushes the right one: the count
    of left turns on the leaf's path."""
    child = lv["child"]
    need = [0] * len(lv["perm"])
    todo = [(0, 0)]
    while todo:
        node, held = todo.pop()
        for side, ref in enumerate(child[node]):
            h = held + (1 if side == 0 else 0)     # going left keeps the right sibling pushed
            if ref >= 0:
                todo.append((int(ref), h))
            else:
                need[int(ref) & 0x7FFFFFFF] = h
    return need


def test_deep_scene_needs_more_than_the_stack(oracle_lib):
    """On the reference LBVH of this scene the leftmost TLAS leaf is reached with
    34 pushes and the BLAS below it needs 34 more: past the 64-entry bound."""
    w = deep_stack_workload()
    tlas = oracle_lib.lbvh_f32(oracle_lib.instance_boxes_f32(w.scene))
    blas = oracle_lib.lbvh_f32(oracle_lib.blas_leaf_boxes(w.scene, 0))
    t_need, b_need = _left_first_stack_need(tlas), _left_first_stack_need(blas)
    assert t_need[0] == CHAIN_BITS + 4 and b_need[0] == CHAIN_BITS + 4
    assert t_need[0] + max(b_need) > STACK_DEPTH
    # the oracle (no stack) sees a plain miss
    px = oracle_lib.render(w)
    assert px["flags"][0] & 1 == 0


@pytest.mark.gpu
@pytest.mark.parametrize("binary_tlas", [False, True])
def test_stack_overflow_sets_the_error_bit(binary_tlas):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2012_10357_b300 as pr
    w = deep_stack_workload()
    scene = pr.Scene(w.scene)
    assert scene.error_word() == 0
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = scene.trace(w.camera, w.params, ray_counter=counter, binary_tlas=binary_tlas)
    torch.cuda.synchronize()
    err = scene.error_word()
    assert err & (1 << pr.PR_ERR_STACK_OVERFLOW), err
    assert int(counter.item()) == 1
    assert torch.isfinite(out).all()
    # the word is cleared by the read; a shallow scene traced afterwards reports nothing
    assert scene.error_word() == 0
    scene.close()
    ok = pr.Scene(scenes.small_analytic().scene)
    ok.trace(scenes.small_analytic().camera, scenes.small_analytic().params)
    torch.cuda.synchronize()
    assert ok.error_word() == 0
    ok.close()
