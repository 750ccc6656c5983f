"""PLOC TLAS builds (PR_BUILD_TLAS_PLOC) on a B300, through the C ABI.

The device tree must equal the reference PLOC builder (oracle.ploc_f32) bit for
bit on the instance boxes of the reference (same Morton order, same merges,
same node numbers and child boxes); images must equal those of the LBVH build
bit for bit (the closest hit does not depend on the tree's shape); builds are
deterministic, and pr_build_bvh_many_ex gives the trees of single builds.
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

PLOC = pr.PR_BUILD_TLAS_PLOC


def _identical_instances(n):
    w = scenes.field(n_inst=n, width=8, height=8)
    rep = {k: np.ascontiguousarray(np.repeat(getattr(w.scene, k)[:1], n, axis=0))
           for k in ("inst_xform", "inst_blas", "inst_sbt_offset")}
    return dataclasses.replace(w.scene, **rep)


@pytest.mark.parametrize("n", [1025, 1500, 5000, 30000, 100000])
def test_ploc_tlas_matches_reference_bit_for_bit(n):
    sc = scenes.field(n_inst=n, width=8, height=8).scene
    scene = pr.Scene(sc, build_flags=PLOC)
    torch.cuda.synchronize()
    _cmp_level(scene.read_bvh(pr.PR_NONE), oracle.ploc_f32(oracle.instance_boxes_f32(sc)), f"PLOC TLAS n={n}")
    # the BLAS levels stay LBVHs
    for b in range(len(sc.blas_geom_begin)):
        _cmp_level(scene.read_bvh(b), oracle.lbvh_f32(oracle.blas_leaf_boxes(sc, b)), f"BLAS {b}")
    assert scene.error_word() == 0
    scene.close()


def test_ploc_identical_instances():
    """All instance boxes equal: every area ties, the tie rule pairs neighbours and the
    tree halves the list each round (the reference tree, bit for bit)."""
    sc = _identical_instances(4096)
    scene = pr.Scene(sc, build_flags=PLOC)
    torch.cuda.synchronize()
    ref = oracle.ploc_f32(oracle.instance_boxes_f32(sc))
    _cmp_level(scene.read_bvh(pr.PR_NONE), ref, "identical instances")
    assert scene.error_word() == 0
    scene.close()


def test_small_tlas_ignores_the_flag():
    sc = scenes.field(n_inst=900, width=8, height=8).scene
    scene = pr.Scene(sc, build_flags=PLOC)
    torch.cuda.synchronize()
    _cmp_level(scene.read_bvh(pr.PR_NONE), oracle.lbvh_f32(oracle.instance_boxes_f32(sc)), "900-instance TLAS")
    scene.close()


@pytest.mark.parametrize("n,binary", [(30000, False), (30000, True), (100000, False)])
def test_ploc_images_equal_lbvh_images(n, binary):
    w = scenes.field(n_inst=n, width=640, height=360)
    imgs, errs, visits = [], [], []
    for flags in (0, PLOC):
        scene = pr.Scene(w.scene, build_flags=flags)
        out, aov = scene.trace(w.camera, w.params, want_aov=True, binary_tlas=binary)
        work = scene.trace_work(w.camera, w.params, binary_tlas=binary)
        torch.cuda.synchronize()
        imgs.append((out.cpu().numpy(), pr.aov_to_numpy(aov)))
        errs.append(scene.error_word())
        visits.append(work["tlas_nodes" if binary else "tlas_nodes4"])
        scene.close()
    assert errs == [0, 0]
    assert np.array_equal(imgs[0][0], imgs[1][0])
    for k in imgs[0][1].dtype.names or ():
        assert np.array_equal(imgs[0][1][k], imgs[1][1][k]), k
    assert visits[1] < visits[0]          # the clustered tree is visited less


def test_ploc_rebuild_is_deterministic():
    sc = scenes.field(n_inst=20000, width=8, height=8).scene
    scene = pr.Scene(sc, build_flags=PLOC)
    first = scene.read_bvh(pr.PR_NONE)
    for _ in range(3):
        scene.build_bvh(flags=PLOC)
        again = scene.read_bvh(pr.PR_NONE)
        for k in first:
            assert np.array_equal(first[k], again[k]), k
    scene.close()


def test_build_many_ex_equals_single_builds():
    descs = [scenes.field(seed=s, n_inst=n, width=8, height=8).scene
             for s, n in ((1, 3000), (2, 800), (3, 12000), (4, 2000), (5, 5000))]
    many = [pr.Scene(d, build=False) for d in descs]
    pr.build_bvh_many(many, flags=PLOC)
    torch.cuda.synchronize()
    for d, s in zip(descs, many):
        n = len(d.inst_blas)
        ref = oracle.ploc_f32 if n > 1024 else oracle.lbvh_f32
        _cmp_level(s.read_bvh(pr.PR_NONE), ref(oracle.instance_boxes_f32(d)), f"many_ex n={n}")
        assert s.error_word() == 0
        s.close()


def test_unknown_build_flag_is_rejected():
    sc = scenes.field(n_inst=2000, width=8, height=8).scene
    scene = pr.Scene(sc, build=False)
    with pytest.raises(pr.PrError) as e:
        scene.build_bvh(flags=0x10)
    assert e.value.status == pr.PR_ERR_INVALID_ARG
    scene.close()
