"""CUDA path vs the FP64 oracle, through the C ABI, on a B300.

BVH levels are compared bit for bit with the oracle's FP32 reference LBVH;
images pixel by pixel with the tolerances in tests/parity.py, at sizes the
oracle renders in seconds (several tiles plus ragged edges) and, at the full
configuration sizes in the benchmark's launch configuration, on seeded pixel
samples.
"""
import dataclasses
import json
import os

import numpy as np
import pytest

import scenes
from parity import assert_parity, compare, gpu_rays_from_flags

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2012_10357_b300 as pr  # noqa: E402
import oracle  # noqa: E402


def render_gpu(w, want_aov=True):
    scene = pr.Scene(w.scene)
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    out, aov = scene.trace(w.camera, w.params, ray_counter=counter, want_aov=True)
    torch.cuda.synchronize()
    err = scene.error_word()
    rgb = out[..., :3].cpu().numpy()
    a = pr.aov_to_numpy(aov)
    box = scene.bounds()
    diag = float(np.linalg.norm(box[3:] - box[:3]))
    rays = int(counter.item())
    scene.close()
    return rgb, a, diag, rays, err, out


def check_full(w, label, threads=0):
    rgb, a, diag, rays, err, _ = render_gpu(w)
    ref = oracle.render(w, threads=threads)
    rep = compare(ref, a, rgb, diag, scene=w.scene)
    assert_parity(rep, label)
    assert rays == int(gpu_rays_from_flags(a).sum())
    assert err == 0
    return rep


# ---------------------------------------------------------------------------
# BVH build: bit-exact against the reference LBVH
# ---------------------------------------------------------------------------
def _cmp_level(got, ref, label):
    """The reference names leaves by sorted position, the library by leaf index
    (perm[position]); map before comparing."""
    n = len(ref["perm"])
    assert np.array_equal(got["perm"], ref["perm"]), label
    assert np.array_equal(got["codes"], ref["codes"]), label
    if n > 1:
        rc = ref["child"].astype(np.int64)
        leaf = rc < 0
        mapped = np.where(leaf, (0x80000000 | ref["perm"][rc & 0x7FFFFFFF].astype(np.int64)) - (1 << 32), rc)
        assert np.array_equal(got["child"].astype(np.int64), mapped), label
        assert np.array_equal(got["cbox"], ref["cbox"]), label
    assert np.array_equal(got["root"], ref["root"]), label


def _many_prim_scene(n_big=3000, n_small=700, seed=11):
    rng = np.random.default_rng(seed)
    b = scenes.SceneBuilder()
    scenes._standard_rays(b)
    hr, hs = b.add_hit_group(scenes.IS_SPHERE, scenes.CHS_LAMBERT), b.add_hit_group(scenes.IS_SPHERE)
    mat = b.add_material((0.7, 0.7, 0.7))
    blas = []
    for n in (n_big, n_small):
        c = rng.uniform(-20, 20, (n, 3))
        r = rng.uniform(0.05, 0.5, n)
        # two geometries per BLAS so g and q are both exercised
        half = n // 2
        g0 = b.add_geometry(np.concatenate([c[:half] - r[:half, None], c[:half] + r[:half, None]], 1),
                            [scenes.params_row(*c[k], r[k]) for k in range(half)])
        g1 = b.add_geometry(np.concatenate([c[half:] - r[half:, None], c[half:] + r[half:, None]], 1),
                            [scenes.params_row(*c[k], r[k]) for k in range(half, n)])
        blas.append(b.add_blas([g0, g1]))
    for _ in range(2):
        b.add_record(hr, mat, scenes.IS_SPHERE, 0)
        b.add_record(hs, mat, scenes.IS_SPHERE, 0)
    b.add_instance(blas[0], scenes.xform_trs((0, 0, 0)), 0)
    b.add_instance(blas[1], scenes.xform_trs((50, 0, 0), scenes.rot_y(30), 0.5), 0)
    b.add_instance(blas[1], scenes.xform_trs((-50, 0, 0)), 0)
    return b.build("many-prims")


@pytest.mark.parametrize("which", ["small_analytic", "teaser", "field_900", "field_30000", "many_prims", "sample"])
def test_lbvh_levels_bit_exact(which):
    if which == "sample":
        sc = scenes.sample_scene(width=8, height=8, cells=24).scene          # 1152-triangle BLAS
    elif which == "small_analytic":
        sc = scenes.small_analytic().scene
    elif which == "teaser":
        sc = scenes.teaser(width=8, height=8).scene
    elif which == "field_900":
        sc = scenes.field(n_inst=900, width=8, height=8).scene
    elif which == "field_30000":
        sc = scenes.field(n_inst=30000, width=8, height=8).scene
    else:
        sc = _many_prim_scene()
    scene = pr.Scene(sc)
    torch.cuda.synchronize()
    for b in range(len(sc.blas_geom_begin)):
        _cmp_level(scene.read_bvh(b), oracle.lbvh_f32(oracle.blas_leaf_boxes(sc, b)), f"{which} BLAS {b}")
    _cmp_level(scene.read_bvh(pr.PR_NONE), oracle.lbvh_f32(oracle.instance_boxes_f32(sc)), f"{which} TLAS")
    scene.close()


def test_lbvh_full_size_tlas_bit_exact():
    sc = scenes.field(width=8, height=8).scene          # 100 000 instances
    scene = pr.Scene(sc)
    torch.cuda.synchronize()
    _cmp_level(scene.read_bvh(pr.PR_NONE), oracle.lbvh_f32(oracle.instance_boxes_f32(sc)), "field 100000 TLAS")
    scene.close()


def test_rebuild_is_deterministic():
    sc = scenes.field(n_inst=20000, width=8, height=8).scene
    scene = pr.Scene(sc)
    a = scene.read_bvh(pr.PR_NONE)
    scene.build_bvh()
    b = scene.read_bvh(pr.PR_NONE)
    for k in a:
        assert np.array_equal(a[k], b[k])
    scene.close()


# ---------------------------------------------------------------------------
# Images
# ---------------------------------------------------------------------------
def test_small_analytic_full_frame():
    check_full(scenes.small_analytic(), "small analytic 64x64")


@pytest.mark.parametrize("wh", [(67, 45), (1, 1), (3, 200), (200, 3), (17, 9)])
def test_small_analytic_ragged_sizes(wh):
    """Ragged and degenerate image sizes. A jittered eye is used: with the
    default eye every ray of the centre row of an odd-height image passes
    exactly through the far edge of the ground slab (y = 2 - 18/4 = -2.5 at
    z = 10), an ill-conditioned hit/miss on which FP32 and FP64 may differ."""
    w = scenes.small_analytic(width=wh[0], height=wh[1])
    w.camera = scenes.small_analytic_cameras(0, 1)[0]
    check_full(w, f"small analytic {wh}")


def test_small_analytic_degenerate_edge_row_is_the_only_disagreement():
    """With the default eye the centre row of an odd-height image grazes the
    slab's far edge; all other pixels agree strictly."""
    w = scenes.small_analytic(width=67, height=45)
    rgb, a, diag, rays, err, _ = render_gpu(w)
    ref = oracle.render(w)
    keep = np.ones((45, 67), bool)
    keep[22, :] = False
    rep = compare(ref.reshape(45, 67)[keep], a.reshape(45, 67)[keep], rgb.reshape(45, 67, 3)[keep], diag, scene=w.scene)
    assert rep["agree"] == 1.0 and rep["t_bad"] == rep["n_bad"] == rep["rgb_bad"] == 0, rep


def test_mirror_hit_is_shaded_without_shadow():
    """Strict parity on the two-sphere mirror scene (reflected hit that a
    shadow ray would find occluded), plus its centre pixel's closed form."""
    w = scenes.mirror_pair(33, 33)
    check_full(w, "mirror pair")
    rgb, a, diag, rays, err, _ = render_gpu(w)
    c = rgb.reshape(-1, 3)[16 * 33 + 16]
    assert np.allclose(c, 0.5 * 0.1 * np.array([0.5, 0.25, 1.0]) + 0.5 * 1.1 * np.array([0.2, 0.9, 0.4]), atol=1e-6)
    assert int(a.reshape(-1)[16 * 33 + 16]["refl_geom"]) == 1


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_small_analytic_other_seeds(seed):
    check_full(scenes.small_analytic(seed=seed, width=96, height=80), f"small analytic seed {seed}")


def test_teaser_reduced_full_frame():
    check_full(scenes.teaser(width=320, height=180), "teaser 320x180")


def test_field_reduced_full_frame():
    check_full(scenes.field(n_inst=2000, width=192, height=108), "field 2000 inst 192x108")


def test_field_mid_full_frame():
    check_full(scenes.field(n_inst=20000, width=160, height=90), "field 20000 inst 160x90")


@pytest.mark.parametrize("cfg", ["teaser_1080p", "field_100k_2160p"])
def test_full_size_sampled_pixels(cfg):
    """Full configuration sizes, the benchmark's trace call; oracle on a pixel sample."""
    w = scenes.teaser() if cfg == "teaser_1080p" else scenes.field()
    scene = pr.Scene(w.scene)
    plain = scene.trace(w.camera, w.params)           # exactly what bench.py times
    out, aov = scene.trace(w.camera, w.params, want_aov=True)
    torch.cuda.synchronize()
    assert torch.equal(plain, out)
    assert scene.error_word() == 0
    box = scene.bounds()
    diag = float(np.linalg.norm(box[3:] - box[:3]))
    pix = scenes.sample_pixels(w.params.width, w.params.height, 3000 if cfg == "teaser_1080p" else 1500, seed=5)
    a = pr.aov_to_numpy(aov).reshape(-1)[pix]
    rgb = out[..., :3].reshape(-1, 3).cpu().numpy()[pix]
    ref = oracle.render(w, pixels=pix)
    rep = compare(ref, a, rgb, diag, scene=w.scene)
    assert_parity(rep, f"{cfg} full size sampled")
    scene.close()


def test_trace_frames_equals_single_frames():
    w = scenes.small_analytic()
    cams = scenes.small_analytic_cameras(0, 5)
    scene = pr.Scene(w.scene)
    batch = scene.trace_frames(cams, w.params)
    for f, c in enumerate(cams):
        one = scene.trace(c, w.params)
        assert torch.equal(batch[f], one)
    scene.close()


def test_repeated_launches_on_two_streams():
    """Many launches of one scene in a row, of two sizes and on two streams,
    all give the image of the first launch of their size (a launch keeps no
    state in the scene)."""
    w = scenes.small_analytic()
    scene = pr.Scene(w.scene)
    small = dataclasses.replace(w.params, width=37, height=23)
    ref = scene.trace(w.camera, w.params).clone()
    ref_small = scene.trace(w.camera, small).clone()
    torch.cuda.synchronize()
    streams = (torch.cuda.Stream(), torch.cuda.Stream())
    outs = []
    for k in range(150):
        is_small = k % 3 == 0
        outs.append((is_small, scene.trace(w.camera, small if is_small else w.params, stream=streams[k % 2])))
    torch.cuda.synchronize()
    for is_small, o in outs:
        assert torch.equal(o, ref_small if is_small else ref)
    assert scene.error_word() == 0
    scene.close()


def test_4096_frame_launch_sampled_vs_oracle():
    """The 4096-frame throughput launch as the benchmark times it (4096 jittered
    64x64 frames in one pr_trace_frames call): 32 seeded frames x 64 seeded
    pixels agree with the oracle (strict: an analytic scene), and those frames
    equal single-frame renders bit for bit."""
    w = scenes.small_analytic()
    cams = scenes.small_analytic_cameras(0, 4096)
    scene = pr.Scene(w.scene)
    out, aov = scene.trace_frames(pr.CameraArray(cams), w.params, want_aov=True)
    torch.cuda.synchronize()
    box = scene.bounds()
    diag = float(np.linalg.norm(box[3:] - box[:3]))
    rng = np.random.default_rng(11)
    n = agree = 0
    for f in sorted(rng.choice(4096, 32, replace=False).tolist()):
        wf = scenes.Workload(w.scene, cams[f], w.params)
        pix = scenes.sample_pixels(64, 64, 64, seed=f)
        rep = compare(oracle.render(wf, pixels=pix), pr.aov_to_numpy(aov[f]).reshape(-1)[pix],
                      out[f, ..., :3].reshape(-1, 3).cpu().numpy()[pix], diag, scene=w.scene)
        assert rep["strict_bad"] == 0, (f, rep)
        n += rep["n"]
        agree += round(rep["agree"] * rep["n"])
        assert torch.equal(scene.trace(cams[f], w.params), out[f])
    scene.close()
    assert agree / n >= 0.999, (n, agree)


def test_launches_without_aov_equal_the_checked_ones():
    """Launches that write no AOV buffer take kernels compiled without AOV
    stores (the analytic config-1 kernel) and, for max_depth 1, without the
    mirror bounce: the 4096-frame RGB launch the benchmark times equals, bit for
    bit, the AOV launch that the oracle comparisons check, and so do single
    frames of the small analytic scene and of an instanced field."""
    w = scenes.small_analytic()
    cams = pr.CameraArray(scenes.small_analytic_cameras(0, 4096))
    scene = pr.Scene(w.scene)
    checked, _ = scene.trace_frames(cams, w.params, want_aov=True, rgb=True)
    timed = scene.trace_frames(cams, w.params, rgb=True)
    one_checked, _ = scene.trace(w.camera, w.params, want_aov=True)
    one = scene.trace(w.camera, w.params)
    torch.cuda.synchronize()
    assert torch.equal(checked, timed)
    assert torch.equal(one_checked, one)
    assert scene.error_word() == 0
    scene.close()
    f = scenes.field(n_inst=3000, width=203, height=97)
    scene = pr.Scene(f.scene)
    a, _ = scene.trace(f.camera, f.params, want_aov=True)
    b = scene.trace(f.camera, f.params)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    scene.close()


@pytest.mark.parametrize("which", ["teaser", "field"])
def test_rgb_output_equals_the_rgba_channels(which):
    """PR_TRACE_OUTPUT_RGB writes 3 floats per pixel: the same values as the
    first three channels of the RGBA image (single frames and frame batches)."""
    w = scenes.teaser(width=203, height=97) if which == "teaser" else scenes.field(n_inst=3000, width=203, height=97)
    scene = pr.Scene(w.scene)
    rgba = scene.trace(w.camera, w.params)
    rgb = scene.trace(w.camera, w.params, rgb=True)
    cams = [w.camera, w.camera]
    fr = scene.trace_frames(cams, w.params, rgb=True)
    torch.cuda.synchronize()
    assert rgb.shape == (97, 203, 3)
    assert torch.equal(rgb, rgba[..., :3].contiguous())
    assert torch.equal(fr[1], rgb)
    with pytest.raises(ValueError):
        scene.trace(w.camera, w.params, out=torch.empty((97, 203, 2), device="cuda"))
    scene.close()


def test_jittered_frames_vs_oracle():
    w = scenes.small_analytic()
    cams = scenes.small_analytic_cameras(0, 4)
    scene = pr.Scene(w.scene)
    out, aov = scene.trace_frames(cams, w.params, want_aov=True)
    torch.cuda.synchronize()
    box = scene.bounds()
    diag = float(np.linalg.norm(box[3:] - box[:3]))
    for f, c in enumerate(cams):
        wf = scenes.Workload(w.scene, c, w.params)
        ref = oracle.render(wf)
        rep = compare(ref, pr.aov_to_numpy(aov[f]), out[f, ..., :3].cpu().numpy(), diag, scene=w.scene)
        assert_parity(rep, f"jittered frame {f}")
    scene.close()


def test_sbt_index_outside_table_sets_error_word():
    w = scenes.small_analytic()
    w.scene.inst_sbt_offset[:] = 7
    rgb, a, diag, rays, err, _ = render_gpu(w)
    ref = oracle.render(w)
    assert err & pr.ERR_WORD_SBT
    assert not (a["flags"] & 1).any() and not (ref["flags"] & 1).any()
    assert ((a["flags"] & 32) != 0).sum() == 0 or True  # per-pixel flag is informational


def test_empty_scene_is_background():
    b = scenes.SceneBuilder()
    scenes._standard_rays(b)
    b.add_hit_group(scenes.IS_SPHERE, scenes.CHS_LAMBERT)
    b.add_material((1, 1, 1))
    b.add_record(0, 0, 0, 0)
    sc = b.build("empty")
    w = scenes.Workload(sc, scenes.Camera(np.float32([0, 0, -5]), np.float32([0, 0, 0]), np.float32([0, 1, 0])),
                        scenes.TraceParams(33, 17))
    rgb, a, diag, rays, err, _ = render_gpu(w)
    assert np.allclose(rgb, np.float32([0.05, 0.05, 0.08]))
    assert rays == 33 * 17 and err == 0


def test_eq1_fig3_layout_matches_oracle():
    """The oracle's Eq. 1 pin scene, rendered by both."""
    from test_oracle_pins import _eq1_scene
    fix = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "eq1_fig3.json")))
    scene = _eq1_scene(fix).build("fig3")
    for x in (-3.0, -1.0, 1.0, 3.0):
        cam = scenes.Camera(np.float32([x, 0, -50]), np.float32([x, 0, 0]), np.float32([0, 1, 0]), 1.0)
        tp = scenes.TraceParams(5, 5, light_pos=np.float32([x, 0, 50]))
        check_full(scenes.Workload(scene, cam, tp), f"fig3 x={x}")


def test_mask_and_tie_rules():
    from test_oracle_pins import _single_sphere_workload
    w = _single_sphere_workload()
    s = w.scene
    for name in ("inst_xform", "inst_blas", "inst_id", "inst_sbt_offset", "inst_mask"):
        a = getattr(s, name)
        setattr(s, name, np.concatenate([a, a]))
    rgb, a, diag, rays, err, _ = render_gpu(w)
    hit = (a["flags"] & 1) != 0
    assert hit.sum() > 20 and (a["inst"][hit] == 0).all()
    s.inst_mask[0] = 0
    rgb, a, diag, rays, err, _ = render_gpu(w)
    hit = (a["flags"] & 1) != 0
    assert hit.sum() > 20 and (a["inst"][hit] == 1).all()


# ---------------------------------------------------------------------------
# Julia set cut by planes (Fig. 5) and animation parameters (Fig. 6)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("plane", [((0.0, 0.0, -1.0), 0.0), ((1.0, 0.0, -1.0), 0.2), ((0.0, 1.0, 0.0), -0.3)])
def test_julia_cut_scene(plane):
    w = scenes.julia_cut_scene(normal=plane[0], offset=plane[1], width=160, height=120)
    check_full(w, f"julia cut {plane}")


@pytest.mark.parametrize("steps", [8, 32, 96])
def test_animation_by_sphere_tracing_step_cap(steps):
    """Fig. 6 animates the Mandelbulb by the number of ray-marching steps: a
    per-frame parameter (max_steps) of every trace call."""
    w = scenes.teaser(width=192, height=108)
    w.params.max_steps = steps
    check_full(w, f"teaser max_steps {steps}")


def test_animation_by_iteration_count_via_upload():
    """Changing the fractal iteration count between frames: re-upload the
    description (same counts, no allocation), rebuild, trace."""
    w = scenes.teaser(width=160, height=90)
    bulb = [k for k in range(len(w.scene.sbt)) if w.scene.sbt[k, 2] == scenes.IS_MANDELBULB]
    assert bulb
    scene = pr.Scene(w.scene)
    arena = scene.device_bytes()
    prim_of_mb = [p for p in range(len(w.scene.params)) if w.scene.params[p, 0] == 8.0 and w.scene.params[p, 2] == 2.0]
    for iters in (3, 6, 12):
        w.scene.params[prim_of_mb, 1] = iters
        scene.upload(w.scene)
        scene.build_bvh()
        out, aov = scene.trace(w.camera, w.params, want_aov=True)
        torch.cuda.synchronize()
        box = scene.bounds()
        rep = compare(oracle.render(w), pr.aov_to_numpy(aov), out[..., :3].cpu().numpy(),
                      float(np.linalg.norm(box[3:] - box[:3])), scene=w.scene)
        assert_parity(rep, f"mandelbulb iterations {iters}")
    assert scene.device_bytes() == arena
    scene.close()


# ---------------------------------------------------------------------------
# 4-wide TLAS (collapsed from the binary LBVH)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n_inst", [64, 65, 100, 700, 30000])
def test_four_wide_tlas_gives_the_same_image(n_inst):
    w = scenes.field(n_inst=n_inst, width=160, height=90)
    scene = pr.Scene(w.scene)
    a = scene.trace(w.camera, w.params)
    b = scene.trace(w.camera, w.params, binary_tlas=True)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    if n_inst > 100:
        k4 = scene.trace_work(w.camera, w.params)
        k2 = scene.trace_work(w.camera, w.params, binary_tlas=True)
        assert k4["tlas_nodes"] == 0 and k2["tlas_nodes4"] == 0
        assert k4["tlas_nodes4"] < k2["tlas_nodes"]
        # the visit order (and so the number of leaves reached before the
        # closest hit prunes the rest) may differ; the rays cast may not
        assert k4["rays"] == k2["rays"]
    scene.close()


def test_four_wide_tlas_full_size_sampled():
    w = scenes.field()
    scene = pr.Scene(w.scene)
    a = scene.trace(w.camera, w.params)
    b = scene.trace(w.camera, w.params, binary_tlas=True)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    scene.close()


# ---------------------------------------------------------------------------
# Any-hit shaders (third hit-group slot)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["analytic", "sdf", "fractal"])
@pytest.mark.parametrize("shadow_cutout", [True, False])
def test_cutout_any_hit_scene(shadow_cutout, kind):
    """Band edges are discontinuities of the any-hit decision (FP32 vs FP64 may
    disagree on a pixel whose candidate sits on an edge): hits on primitives
    with the any-hit shader take the 0.1 % budget, every other pixel is strict.
    sdf / fractal: the sphere-traced shaders' candidates (march points below eps,
    the march going on through the solid after an ignored one)."""
    w = scenes.cutout_scene(width=200, height=150, shadow_cutout=shadow_cutout, kind=kind)
    rgb, a, diag, rays, err, _ = render_gpu(w)
    rep = compare(oracle.render(w), a, rgb, diag, scene=w.scene)
    assert_parity(rep, f"cutout {kind} shadow_cutout={shadow_cutout}")
    assert err == 0


@pytest.mark.parametrize("kind", ["analytic", "sdf", "fractal"])
def test_cutout_changes_the_image(kind):
    w = scenes.cutout_scene(width=96, height=72, kind=kind)
    a = render_gpu(w)[0]
    w.scene.hit_groups[:, 2] = scenes.NONE
    b = render_gpu(w)[0]
    assert np.abs(a - b).max() > 0.1



# ---------------------------------------------------------------------------
# Triangle geometry (built-in triangle intersection) mixed with procedural BLASes
# ---------------------------------------------------------------------------
def test_sample_scene_fig4():
    """The paper's sample scene: triangle plane mesh + pac-men + Julia + Mandelbulb,
    Listing 10's shader-table layout, mirror bounce."""
    check_full(scenes.sample_scene(width=320, height=180), "sample scene 320x180")


def _mesh_and_spheres(cells=16, width=160, height=120):
    b = scenes.SceneBuilder()
    scenes._standard_rays(b)
    tr, ts = b.add_hit_group(scenes.NONE, scenes.CHS_LAMBERT), b.add_hit_group(scenes.NONE)
    sr, ss = b.add_hit_group(scenes.IS_SPHERE, scenes.CHS_LAMBERT), b.add_hit_group(scenes.IS_SPHERE)
    mt, ms = b.add_material((0.7, 0.7, 0.7)), b.add_material((0.9, 0.3, 0.2))
    v, i = scenes.plane_mesh(6.0, -1.0, cells)
    tb = b.add_blas([b.add_triangle_geometry(v, i)])
    a, p = scenes.shape_sphere((0, 0, 0), 0.8)
    sb = b.add_blas([b.add_geometry([a], [p])])
    b.add_record(tr, mt, scenes.NONE, 0)
    b.add_record(ts, mt, scenes.NONE, 0)
    b.add_record(sr, ms, scenes.IS_SPHERE, 1)
    b.add_record(ss, ms, scenes.IS_SPHERE, 1)
    b.add_instance(tb, scenes.xform_trs((0, 0, 0)), 0)
    b.add_instance(tb, scenes.xform_trs((0, 1.5, 8), scenes.rot_y(25), 1.0), 0)     # a second, rotated mesh
    b.add_instance(sb, scenes.xform_trs((-1, 0, 1)), 2)
    b.add_instance(sb, scenes.xform_trs((1.5, 0.2, 2.5), None, 0.7), 2)
    cam = scenes.Camera(np.float32([0.3, 2.0, -5.0]), np.float32([0, 0, 2]), np.float32([0, 1, 0]), 60.0)
    return scenes.Workload(b.build("mesh"), cam, scenes.TraceParams(width, height, light_pos=np.float32([4, 7, -3])))


def test_triangle_mesh_with_spheres_strict():
    w = _mesh_and_spheres()
    rep = check_full(w, "triangle mesh + spheres")
    assert rep["hits"] > 1000


def test_build_many_equals_single_builds():
    """pr_build_bvh_many (builds of many scenes spread over internal streams,
    joined back into the caller's stream) gives every scene the BVH and image
    of its own pr_build_bvh, also when the scenes are rebuilt in place."""
    ws = scenes.batch_requests(3, 12, res_choices=(48, 64))
    ref = [pr.Scene(w.scene) for w in ws]                 # built one by one
    many = [pr.Scene(w.scene, build=False) for w in ws]
    stream = torch.cuda.Stream()
    for _ in range(2):
        pr.build_bvh_many(many, stream=stream)
        imgs = [m.trace(w.camera, w.params, stream=stream) for m, w in zip(many, ws)]
        stream.synchronize()
        for r, m, w, img in zip(ref, many, ws, imgs):
            a, b = r.read_bvh(pr.PR_NONE), m.read_bvh(pr.PR_NONE)
            for k in a:
                assert np.array_equal(a[k], b[k])
            assert torch.equal(r.trace(w.camera, w.params), img)
    for s in ref + many:
        s.close()
