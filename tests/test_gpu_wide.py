"""Wide TLAS formats on a B300: depth-parity 4-wide, 8-wide float and 8-wide quantised
nodes, against the default (greedy 4-wide) build.

Each format must give the images (RGB and every AOV field) of the default build
bit for bit: the closest hit does not depend on the tree's shape, and the
quantised boxes are conservative by construction (they contain the float boxes
by a margin larger than the slab tests' rounding). The work counters show which
traversal ran; the error word stays clear; batched launches of such scenes
fall back to the binary TLAS and still match.
"""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2012_10357_b300 as pr  # noqa: E402

FORMATS = {"parity4": pr.PR_BUILD_TLAS_PARITY4, "bvh8": pr.PR_BUILD_TLAS_BVH8, "bvh8_f32": pr.PR_BUILD_TLAS_BVH8_F32}
COUNTER = {"parity4": "tlas_nodes4", "bvh8": "tlas_nodes8q", "bvh8_f32": "tlas_nodes8"}


def _render(w, flags):
    scene = pr.Scene(w.scene, build_flags=flags)
    out, aov = scene.trace(w.camera, w.params, want_aov=True)
    work = scene.trace_work(w.camera, w.params)
    torch.cuda.synchronize()
    res = out.cpu().numpy(), pr.aov_to_numpy(aov), work, scene.error_word()
    scene.close()
    return res


def _same(a, b):
    assert np.array_equal(a[0], b[0])
    for k in a[1].dtype.names or ():
        assert np.array_equal(a[1][k], b[1][k]), k


_REF = {}


def _reference(n):
    if n not in _REF:
        _REF[n] = _render(scenes.field(n_inst=n, width=640, height=360), 0)
    return _REF[n]


@pytest.mark.parametrize("fmt", list(FORMATS))
@pytest.mark.parametrize("n", [200, 30000, 100000])
@pytest.mark.parametrize("ploc", [False, True])
def test_wide_formats_give_the_default_images(fmt, n, ploc):
    w = scenes.field(n_inst=n, width=640, height=360)
    flags = FORMATS[fmt] | (pr.PR_BUILD_TLAS_PLOC if ploc else 0)
    got = _render(w, flags)
    ref = _reference(n)
    _same(got, ref)
    assert got[3] == 0
    assert got[2]["rays"] == ref[2]["rays"]
    assert got[2][COUNTER[fmt]] > 0
    others = {"tlas_nodes4", "tlas_nodes8", "tlas_nodes8q"} - {COUNTER[fmt]}
    assert all(got[2][k] == 0 for k in others)


def test_eight_wide_visits_fewer_nodes():
    ref = _reference(100000)      # greedy 4-wide
    q = _render(scenes.field(n_inst=100000, width=640, height=360), pr.PR_BUILD_TLAS_BVH8)
    assert q[2]["tlas_nodes8q"] < 0.8 * ref[2]["tlas_nodes4"]


def test_few_instances_keep_the_binary_tlas():
    w = scenes.teaser(width=160, height=90)
    a = _render(w, 0)
    b = _render(w, pr.PR_BUILD_TLAS_BVH8)
    _same(a, b)
    assert b[2]["tlas_nodes8q"] == 0 and b[2]["tlas_nodes"] > 0


def test_batched_launch_of_an_eight_wide_scene():
    ws = [scenes.field(seed=s, n_inst=n, width=320, height=180) for s, n in ((1, 5000), (2, 300))]
    objs = [pr.Scene(w.scene, build_flags=pr.PR_BUILD_TLAS_BVH8) for w in ws]
    plain = [pr.Scene(w.scene) for w in ws]
    outs = [torch.empty((w.params.height, w.params.width, 4), dtype=torch.float32, device="cuda") for w in ws]
    batch = pr.Batch(len(ws), sum(w.params.width * w.params.height for w in ws))
    batch.trace([(o, w.camera, w.params, out) for o, w, out in zip(objs, ws, outs)], graph=True)
    torch.cuda.synchronize()
    for p, w, out in zip(plain, ws, outs):
        ref = p.trace(w.camera, w.params)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    for o in objs + plain:
        assert o.error_word() == 0
        o.close()
    batch.close()


def test_conflicting_wide_formats_are_rejected():
    sc = scenes.field(n_inst=2000, width=8, height=8).scene
    scene = pr.Scene(sc, build=False)
    for flags in (pr.PR_BUILD_TLAS_BVH8 | pr.PR_BUILD_TLAS_BVH8_F32,
                  pr.PR_BUILD_TLAS_PARITY4 | pr.PR_BUILD_TLAS_BVH8):
        with pytest.raises(pr.PrError) as e:
            scene.build_bvh(flags=flags)
        assert e.value.status == pr.PR_ERR_INVALID_ARG
    scene.close()


def test_rebuild_switches_formats():
    w = scenes.field(n_inst=20000, width=320, height=180)
    scene = pr.Scene(w.scene, build_flags=pr.PR_BUILD_TLAS_BVH8_F32)
    first = scene.trace(w.camera, w.params).clone()
    for flags in (0, pr.PR_BUILD_TLAS_BVH8, pr.PR_BUILD_TLAS_PARITY4, pr.PR_BUILD_TLAS_BVH8_F32):
        scene.build_bvh(flags=flags)
        img = scene.trace(w.camera, w.params)
        torch.cuda.synchronize()
        assert torch.equal(img, first)
    assert scene.error_word() == 0
    scene.close()
