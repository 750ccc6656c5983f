"""Batched wavefront path vs the plain per-request path (and the oracle), on a B300.

Every request of a batch must come out bit-identical to a pr_trace of it:
both paths share the per-pixel device functions and the shading composition
is explicitly rounded. The plain path is itself held to the oracle by
test_gpu_parity.py; one request here is also compared with the oracle directly.
"""
import numpy as np
import pytest

import scenes
from parity import assert_parity, compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2012_10357_b300 as pr  # noqa: E402
import oracle  # noqa: E402


def _mixed_workloads():
    ws = [scenes.small_analytic(width=67, height=45), scenes.teaser(width=200, height=113),
          scenes.field(n_inst=3000, width=150, height=97), scenes.small_analytic(seed=4, width=1, height=1),
          scenes.teaser(seed=2, width=33, height=250)]
    ws += scenes.batch_requests(seed=0, n_requests=6, res_choices=(64, 96, 128))
    return ws


def _plain(scene_objs, ws):
    outs, rays = [], 0
    for sc, w in zip(scene_objs, ws):
        c = torch.zeros(1, dtype=torch.int64, device="cuda")
        outs.append(sc.trace(w.camera, w.params, ray_counter=c))
        torch.cuda.synchronize()
        rays += int(c.item())
    return outs, rays


@pytest.mark.parametrize("graph", [False, True])
def test_batch_bit_identical_to_plain(graph):
    ws = _mixed_workloads()
    objs = [pr.Scene(w.scene) for w in ws]
    plain, plain_rays = _plain(objs, ws)
    total = sum(w.params.width * w.params.height for w in ws)
    batch = pr.Batch(len(ws), total)
    outs = [torch.full((w.params.height, w.params.width, 4), -1.0, device="cuda") for w in ws]
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    batch.trace([(o, w.camera, w.params, out) for o, w, out in zip(objs, ws, outs)], ray_counter=counter, graph=graph)
    torch.cuda.synchronize()
    for k, (a, b) in enumerate(zip(plain, outs)):
        assert torch.equal(a, b), f"request {k} differs (max {float((a - b).abs().max())})"
    assert int(counter.item()) == plain_rays
    # a second launch through the same batch (graph replay / table restaging) gives the same bits
    for out in outs:
        out.fill_(-1.0)
    batch.trace([(o, w.camera, w.params, out) for o, w, out in zip(objs, ws, outs)], graph=graph)
    torch.cuda.synchronize()
    for a, b in zip(plain, outs):
        assert torch.equal(a, b)
    batch.close()


@pytest.mark.parametrize("mode", [2, 4])
def test_graph_batches_alternating_mirror_and_no_mirror(mode):
    """Batches whose requests all have max_depth 1 run kernels without the
    mirror bounce, batches with a max_depth-2 request the mirror-capable ones;
    one batch object keeps a captured graph for each and alternates between
    them (as the server's iterations do), every image equal to pr_trace's."""
    with_mirror = [scenes.teaser(width=120, height=68), scenes.field(n_inst=2000, width=96, height=64)]
    without = scenes.batch_requests(seed=3, n_requests=3, res_choices=(64, 96))
    assert all(w.params.max_depth == 1 for w in without) and with_mirror[0].params.max_depth == 2
    objs_m = [pr.Scene(w.scene) for w in with_mirror]
    objs_n = [pr.Scene(w.scene) for w in without]
    plain_m, _ = _plain(objs_m, with_mirror)
    plain_n, _ = _plain(objs_n, without)
    total = max(sum(w.params.width * w.params.height for w in ws) for ws in (with_mirror, without))
    batch = pr.Batch(4, total)
    batch.set_tuning(4, 16, 8, 32, mode)
    for rnd in range(3):
        for objs, ws, plain in ((objs_m, with_mirror, plain_m), (objs_n, without, plain_n)):
            outs = [torch.full((w.params.height, w.params.width, 4), -1.0, device="cuda") for w in ws]
            batch.trace([(o, w.camera, w.params, out) for o, w, out in zip(objs, ws, outs)], graph=True)
            torch.cuda.synchronize()
            for k, (a, b) in enumerate(zip(plain, outs)):
                assert torch.equal(a, b), f"round {rnd}, request {k} differs"
    batch.close()
    for o in objs_m + objs_n:
        o.close()


@pytest.mark.parametrize("shape", [(2, 16, 8, 32, 0), (8, 32, 4, 128, 0), (16, 8, 16, 64, 0), (1, 16, 8, 1024, 0),
                                   (4, 16, 8, 32, 1), (1, 16, 8, 32, 1), (4, 16, 8, 32, 2),
                                   (4, 16, 8, 32, 3), (8, 32, 4, 128, 3), (1, 8, 16, 64, 3), (4, 16, 8, 32, 4)])
def test_batch_launch_shapes_do_not_change_results(shape):
    """Wavefront stages or the batched megakernel, any launch shape: every
    request equals its plain pr_trace image bit for bit."""
    ws = _mixed_workloads()[:5]
    objs = [pr.Scene(w.scene) for w in ws]
    plain, _ = _plain(objs, ws)
    batch = pr.Batch(8, sum(w.params.width * w.params.height for w in ws))
    batch.set_tuning(*shape)
    assert batch.tuning() == dict(zip(("ctas_per_sm", "tile_w", "tile_h", "queue_chunk", "megakernel"), shape))
    outs = [torch.empty((w.params.height, w.params.width, 4), device="cuda") for w in ws]
    batch.trace([(o, w.camera, w.params, out) for o, w, out in zip(objs, ws, outs)])
    torch.cuda.synchronize()
    for a, b in zip(plain, outs):
        assert torch.equal(a, b)


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4])
def test_batch_any_hit_on_sphere_traced_shapes(mode):
    """Cutout any-hit shaders on sphere-traced SDF and fractal shapes (and analytic ones) in
    every batched mode: the regrouped mode marches their candidates in place (an ignored
    candidate continues the march), so every image equals its plain pr_trace image."""
    ws = [scenes.cutout_scene(width=160, height=120, kind=k, shadow_cutout=sc)
          for k, sc in (("sdf", True), ("fractal", True), ("analytic", False), ("fractal", False))]
    objs = [pr.Scene(w.scene) for w in ws]
    plain, _ = _plain(objs, ws)
    batch = pr.Batch(len(ws), sum(w.params.width * w.params.height for w in ws))
    batch.set_tuning(4, 16, 8, 32, mode)
    outs = [torch.empty((w.params.height, w.params.width, 4), device="cuda") for w in ws]
    batch.trace([(o, w.camera, w.params, out) for o, w, out in zip(objs, ws, outs)])
    torch.cuda.synchronize()
    for a, b in zip(plain, outs):
        assert torch.equal(a, b)
    for o in objs:
        assert o.error_word() == 0
        o.close()
    batch.close()


def test_autotune_picks_a_valid_shape_and_keeps_results():
    ws = _mixed_workloads()
    objs = [pr.Scene(w.scene) for w in ws]
    plain, _ = _plain(objs, ws)
    batch = pr.Batch(len(ws), sum(w.params.width * w.params.height for w in ws))
    outs = [torch.empty((w.params.height, w.params.width, 4), device="cuda") for w in ws]
    items = [(o, w.camera, w.params, out) for o, w, out in zip(objs, ws, outs)]
    best, ms = batch.autotune(items)
    assert ms > 0 and best == batch.tuning()
    batch.trace(items, graph=True)
    torch.cuda.synchronize()
    for a, b in zip(plain, outs):
        assert torch.equal(a, b)


def test_batch_request_vs_oracle():
    w = scenes.teaser(width=160, height=90)
    sc = pr.Scene(w.scene)
    batch = pr.Batch(2, 2 * 160 * 90)
    out = torch.empty((90, 160, 4), device="cuda")
    out2 = torch.empty((90, 160, 4), device="cuda")
    batch.trace([(sc, w.camera, w.params, out), (sc, w.camera, w.params, out2)])
    _, aov = sc.trace(w.camera, w.params, want_aov=True)
    torch.cuda.synchronize()
    assert torch.equal(out, out2)
    box = sc.bounds()
    rep = compare(oracle.render(w), pr.aov_to_numpy(aov), out[..., :3].cpu().numpy(),
                  float(np.linalg.norm(box[3:] - box[:3])), scene=w.scene)
    assert_parity(rep, "batched teaser 160x90")


def test_batch_budget_and_argument_errors():
    w = scenes.small_analytic()
    sc = pr.Scene(w.scene)
    out = torch.empty((64, 64, 4), device="cuda")
    batch = pr.Batch(2, 1000)                     # fewer pixels than one 64x64 request
    with pytest.raises(pr.PrError) as ei:
        batch.trace([(sc, w.camera, w.params, out)])
    assert ei.value.status == pr.PR_ERR_BUDGET
    with pytest.raises(pr.PrError):
        pr.Batch(1, 4096).trace([(sc, w.camera, w.params, out)] * 2)   # more requests than max_requests
    with pytest.raises(pr.PrError):
        batch.set_tuning(4, 16, 16, 64)                                  # unsupported tile
    unbuilt = pr.Scene(w.scene, build=False)
    with pytest.raises(pr.PrError) as ei:
        pr.Batch(1, 4096).trace([(unbuilt, w.camera, w.params, out)])
    assert ei.value.status == pr.PR_ERR_NOT_BUILT


def test_full_request_batch_sampled_vs_oracle():
    """The 64-request batch at full size (64 requests, 83.6 M pixels, in the
    launch configuration the benchmark uses: one graph launch): every request's
    image equals its pr_trace, and 64 seeded pixels of every request (4096 in
    all, parity on the sampled pixels as the oracle renders them one by one)
    agree with the oracle within the 0.1 % budget."""
    from parity import merge_reports
    ws = scenes.batch_requests(0, 64)
    total = sum(w.params.width * w.params.height for w in ws)
    objs = [pr.Scene(w.scene) for w in ws]
    outs = [torch.empty((w.params.height, w.params.width, 4), device="cuda") for w in ws]
    batch = pr.Batch(len(ws), total)
    batch.trace([(o, w.camera, w.params, out) for o, w, out in zip(objs, ws, outs)], graph=True)
    torch.cuda.synchronize()
    reps = []
    for k, (o, w, out) in enumerate(zip(objs, ws, outs)):
        img, aov = o.trace(w.camera, w.params, want_aov=True)
        torch.cuda.synchronize()
        assert torch.equal(img, out), f"request {k}"
        pix = scenes.sample_pixels(w.params.width, w.params.height, 64, seed=100 + k)
        box = o.bounds()
        reps.append(compare(oracle.render(w, pixels=pix), pr.aov_to_numpy(aov).reshape(-1)[pix],
                            img[..., :3].reshape(-1, 3).cpu().numpy()[pix], float(np.linalg.norm(box[3:] - box[:3])),
                            scene=w.scene))
        del img, aov
    batch.close()
    for o in objs:
        o.close()
    rep = merge_reports(reps)
    assert rep["n"] == 64 * len(ws)
    assert_parity(rep, "64-request batch, 64 sampled pixels per request")


def test_batch_rgb_outputs_equal_plain():
    """Requests whose output image has 3 channels get PR_TRACE_OUTPUT_RGB: the
    batch writes r, g, b per pixel, equal to the plain RGBA image's channels."""
    ws = _mixed_workloads()[:6]
    objs = [pr.Scene(w.scene) for w in ws]
    outs = [torch.empty((w.params.height, w.params.width, 3 if k % 2 else 4), device="cuda") for k, w in enumerate(ws)]
    total = sum(w.params.width * w.params.height for w in ws)
    batch = pr.Batch(len(ws), total)
    batch.trace([(o, w.camera, w.params, out) for o, w, out in zip(objs, ws, outs)], graph=True)
    torch.cuda.synchronize()
    for o, w, out in zip(objs, ws, outs):
        ref = o.trace(w.camera, w.params)
        torch.cuda.synchronize()
        assert torch.equal(out, ref[..., :out.shape[-1]].contiguous())
    batch.close()
    for o in objs:
        o.close()


def test_batch_megakernel_needs_16x8_tiles():
    batch = pr.Batch(2, 1024)
    for mode in (1, 2, 4):
        with pytest.raises(pr.PrError):
            batch.set_tuning(4, 32, 4, 32, mode)
    with pytest.raises(pr.PrError):
        batch.set_tuning(4, 16, 8, 32, 5)
    batch.close()


@pytest.mark.parametrize("mode", [1, 2, 3, 4])
def test_batched_megakernel_rays_and_graph(mode):
    """The batched megakernel (persistent, or one CTA per tile) and the
    regrouped stages count the same rays as the plain launches and run the
    same through their CUDA graph; RGB and RGBA outputs both."""
    ws = _mixed_workloads()
    objs = [pr.Scene(w.scene) for w in ws]
    plain, rays_plain = _plain(objs, ws)
    batch = pr.Batch(len(ws), sum(w.params.width * w.params.height for w in ws))
    batch.set_tuning(4, 16, 8, 32, mode)
    for graph in (False, True):
        outs = [torch.empty((w.params.height, w.params.width, 3 if k % 2 else 4), device="cuda")
                for k, w in enumerate(ws)]
        c = torch.zeros(1, dtype=torch.int64, device="cuda")
        batch.trace([(o, w.camera, w.params, out) for o, w, out in zip(objs, ws, outs)], ray_counter=c, graph=graph)
        torch.cuda.synchronize()
        assert int(c.item()) == rays_plain
        for a, b in zip(plain, outs):
            assert torch.equal(a[..., :b.shape[-1]].contiguous(), b)
    batch.close()
    for o in objs:
        o.close()


@pytest.mark.parametrize("mode", [2, 4])
def test_tile_megakernel_graph_grows_with_the_batch(mode):
    """One CTA per tile (or per quarter tile): the captured graph's grid grows
    (recapture) when a later batch has more tiles, and a smaller batch reuses
    the larger grid."""
    small = scenes.small_analytic(width=40, height=24)
    big = scenes.teaser(width=400, height=300)
    a, b_ = pr.Scene(small.scene), pr.Scene(big.scene)
    batch = pr.Batch(2, 400 * 300 + 40 * 24)
    batch.set_tuning(4, 16, 8, 32, mode)
    for w, sc in ((small, a), (big, b_), (small, a)):
        out = torch.empty((w.params.height, w.params.width, 4), device="cuda")
        batch.trace([(sc, w.camera, w.params, out)], graph=True)
        ref = sc.trace(w.camera, w.params)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    batch.close()
    a.close()
    b_.close()


def _julia_row(width=96, height=72):
    """Four Julia sets in a row along the view axis (and a mirror slab): every
    ray through them meets up to four fractal boxes, more march jobs than
    pixels, so the regrouped stages also march in place."""
    b = scenes.SceneBuilder()
    scenes._standard_rays(b)
    hj, hjs = b.add_hit_group(scenes.IS_JULIA, scenes.CHS_LAMBERT), b.add_hit_group(scenes.IS_JULIA)
    hb, hbs = b.add_hit_group(scenes.IS_BOX, scenes.CHS_LAMBERT), b.add_hit_group(scenes.IS_BOX)
    mj, ms = b.add_material((0.8, 0.5, 0.3), 0.2), b.add_material((0.6, 0.6, 0.6), 0.4)
    a, p = scenes.shape_julia((-0.2, 0.6, 0.2, 0.2))
    jb = b.add_blas([b.add_geometry([a], [p])])
    a2, p2 = scenes.shape_box((0, -1.6, 0), (12, 0.01, 12))
    sb = b.add_blas([b.add_geometry([a2], [p2])])
    b.add_record(hj, mj, scenes.IS_JULIA, 0)
    b.add_record(hjs, mj, scenes.IS_JULIA, 0)
    b.add_record(hb, ms, scenes.IS_BOX, 1)
    b.add_record(hbs, ms, scenes.IS_BOX, 1)
    for k in range(4):
        b.add_instance(jb, scenes.xform_trs((0.15 * k, 0.1 * k, 1.2 * k)), 0)
    b.add_instance(sb, scenes.xform_trs((0, 0, 0)), 2)
    cam = scenes.Camera(np.float32([0.3, 0.4, -4.0]), np.float32([0.2, 0.2, 2.0]), np.float32([0, 1, 0]), 50.0)
    tp = scenes.TraceParams(width, height, max_depth=2, light_pos=np.float32([4, 8, -6]))
    return scenes.Workload(b.build("julia-row"), cam, tp)


@pytest.mark.parametrize("graph", [False, True])
def test_regrouped_job_overflow_marches_in_place(graph):
    """More deferred marches than the batch holds jobs (a batch sized for
    exactly its pixels, four fractal boxes behind one another): the rays whose
    jobs do not fit march in place, and every image still equals pr_trace."""
    ws = [_julia_row(), _julia_row(37, 53)]
    objs = [pr.Scene(w.scene) for w in ws]
    plain, rays_plain = _plain(objs, ws)
    batch = pr.Batch(2, sum(w.params.width * w.params.height for w in ws))
    batch.set_tuning(4, 16, 8, 32, 3)
    outs = [torch.full((w.params.height, w.params.width, 4), -1.0, device="cuda") for w in ws]
    c = torch.zeros(1, dtype=torch.int64, device="cuda")
    batch.trace([(o, w.camera, w.params, out) for o, w, out in zip(objs, ws, outs)], ray_counter=c, graph=graph)
    torch.cuda.synchronize()
    assert int(c.item()) == rays_plain
    for a, b in zip(plain, outs):
        assert torch.equal(a, b)
    batch.close()
    for o in objs:
        o.close()


def test_regrouped_teaser_vs_oracle():
    """The regrouped stages on the teaser (fractal marches from the job queue,
    mirror rays): parity with the oracle, and the same image as pr_trace."""
    from parity import assert_parity
    w = scenes.teaser(width=192, height=108)
    sc = pr.Scene(w.scene)
    batch = pr.Batch(1, 192 * 108)
    batch.set_tuning(8, 16, 8, 128, 3)
    out = torch.empty((108, 192, 4), device="cuda")
    batch.trace([(sc, w.camera, w.params, out)], graph=True)
    img, aov = sc.trace(w.camera, w.params, want_aov=True)
    torch.cuda.synchronize()
    assert torch.equal(out, img)
    box = sc.bounds()
    rep = compare(oracle.render(w), pr.aov_to_numpy(aov), out[..., :3].cpu().numpy(),
                  float(np.linalg.norm(box[3:] - box[:3])), scene=w.scene)
    assert_parity(rep, "regrouped teaser 192x108")
    batch.close()
    sc.close()
