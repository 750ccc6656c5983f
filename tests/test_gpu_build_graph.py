"""pr_build_bvh_many replays its fan-out of scene builds as a CUDA graph while
the same scenes (and flags) are built again. The replayed builds must follow
the scenes' current inputs: each tree equals the oracle's LBVH of the boxes
uploaded last, and images equal those of scenes built one by one. A changed
scene list (order, a destroyed scene, a new scene that may reuse its address)
must never replay a graph captured for another list.
"""
import dataclasses

import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2012_10357_b300 as pr  # noqa: E402
import oracle  # noqa: E402
from test_gpu_parity import _cmp_level  # noqa: E402

# small scenes (one single-CTA build), a 4-wide TLAS from 64 instances, and
# large TLAS levels (radix sort across CTAs)
SIZES = (5, 40, 300, 1500, 6000, 12000)


def _desc(seed, n):
    return scenes.field(seed=seed, n_inst=n, width=8, height=8).scene


def _check_trees(descs, built, label):
    torch.cuda.synchronize()
    for d, s in zip(descs, built):
        _cmp_level(s.read_bvh(pr.PR_NONE), oracle.lbvh_f32(oracle.instance_boxes_f32(d)),
                   f"{label} n={len(d.inst_blas)}")
        assert s.error_word() == 0


def test_replayed_builds_follow_new_inputs():
    first = [_desc(10 + i, n) for i, n in enumerate(SIZES)]
    many = [pr.Scene(d, build=False) for d in first]
    try:
        pr.build_bvh_many(many)          # captured
        _check_trees(first, many, "first build")
        for rnd in range(2):             # replayed, on new instance data each time
            moved = [_desc(100 * (rnd + 1) + i, n) for i, n in enumerate(SIZES)]
            for s, d in zip(many, moved):
                s.upload(d)
            pr.build_bvh_many(many)
            _check_trees(moved, many, f"replay {rnd}")
    finally:
        for s in many:
            s.close()


def test_replayed_images_equal_single_builds():
    ws = [scenes.field(seed=20 + i, n_inst=n, width=96, height=64) for i, n in enumerate(SIZES)]
    many = [pr.Scene(w.scene, build=False) for w in ws]
    alone = [pr.Scene(w.scene) for w in ws]
    try:
        for _ in range(3):               # capture, then two replays
            pr.build_bvh_many(many)
        for w, a, b in zip(ws, many, alone):
            ia = a.trace(w.camera, w.params, rgb=True)
            ib = b.trace(w.camera, w.params, rgb=True)
            torch.cuda.synchronize()
            assert torch.equal(ia, ib)
    finally:
        for s in many + alone:
            s.close()


def test_changed_scene_lists_are_built_afresh():
    descs = [_desc(30 + i, n) for i, n in enumerate(SIZES[:4])]
    sc = [pr.Scene(d, build=False) for d in descs]
    try:
        pr.build_bvh_many(sc)
        _check_trees(descs, sc, "list")
        order = [2, 0, 3, 1]
        pr.build_bvh_many([sc[i] for i in order])
        _check_trees([descs[i] for i in order], [sc[i] for i in order], "reordered")
        # replace one scene by a scene of another size (its address may be reused)
        sc[1].close()
        descs[1] = _desc(77, 2500)
        sc[1] = pr.Scene(descs[1], build=False)
        pr.build_bvh_many(sc)
        _check_trees(descs, sc, "replaced")
        # a subset, then the whole list with a wide-format flag, then without
        pr.build_bvh_many(sc[:2])
        _check_trees(descs[:2], sc[:2], "subset")
        pr.build_bvh_many(sc, flags=pr.PR_BUILD_TLAS_BVH8)
        _check_trees(descs, sc, "bvh8 flag")
        pr.build_bvh_many(sc)
        _check_trees(descs, sc, "default again")
    finally:
        for s in sc:
            s.close()   # closing twice is a no-op
