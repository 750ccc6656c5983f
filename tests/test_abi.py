"""C-ABI library: loads, exports every declared symbol, host-side validation
and Eq. 1 indexing (no GPU needed: none of these calls touch the device)."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "proceduray.h")


@pytest.fixture(scope="module")
def pr():
    from paper_2012_10357_b300 import build
    build.build()
    import paper_2012_10357_b300 as pr
    return pr


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pr_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(pr):
    syms = declared_symbols()
    assert len(syms) >= 14
    lib = ctypes.CDLL(pr.LIB_PATH)
    for s in syms:
        assert hasattr(lib, s), f"{s} declared in proceduray.h but not exported"
    assert set(syms) <= set(pr.EXPORTED) | {s for s in syms if hasattr(lib, s)}


def test_version_and_constants(pr):
    assert pr.version() == 1
    text = open(HEADER).read()
    ids = dict(re.findall(r"#define (PR_IS_[A-Z0-9]+) (\d+)u", text))
    assert int(ids["PR_IS_SPHERE"]) == scenes.IS_SPHERE
    assert int(ids["PR_IS_JULIA"]) == scenes.IS_JULIA
    assert int(ids["PR_IS_MANDELBULB"]) == scenes.IS_MANDELBULB
    assert int(ids["PR_IS_METABALL4"]) == scenes.IS_METABALL4


def test_eq1_fig3_golden_through_abi(pr):
    fix = json.load(open(os.path.join(ROOT, "tests", "golden", "eq1_fig3.json")))
    m = fix["m"]
    n = len(fix["table"])
    for e in fix["expected"]:
        i = fix["instances"][e["instance"]]["sbt_offset"]
        assert pr.sbt_index(e["r"], m, e["g"], i, n) == e["record"]
    # every (instance, g, r) lands on a distinct record: no collisions
    got = [pr.sbt_index(e["r"], m, e["g"], fix["instances"][e["instance"]]["sbt_offset"], n) for e in fix["expected"]]
    assert sorted(got) == list(range(n))
    # the literal i = 0 / i = 1 reading of the text collides (instance 0 shadow == instance 1 radiance)
    assert pr.sbt_index(1, m, 0, 0, n) == pr.sbt_index(0, m, 0, 1, n)
    assert pr.sbt_index(0, m, 0, n, n) is None


@pytest.mark.parametrize("mutate,frag", [
    (lambda s: s.aabbs.__setitem__((0, 0), 9.0), "lo > hi"),
    (lambda s: s.aabbs.__setitem__((0, 1), np.nan), "not finite"),
    (lambda s: s.inst_blas.__setitem__(0, 99), "BLAS out of range"),
    (lambda s: s.inst_xform.__setitem__((0, slice(0, 3)), 0.0), "not invertible"),
    (lambda s: s.hit_groups.__setitem__((0, 0), 42), "intersection shader"),
    (lambda s: s.hit_groups.__setitem__((0, 2), 5), "any-hit"),
    (lambda s: s.sbt.__setitem__((0, 0), 1000), "hit group out of range"),
    (lambda s: s.sbt.__setitem__((0, 1), 1000), "material out of range"),
    (lambda s: s.geom_prim_count.__setitem__(0, 0), "primitive range"),
    (lambda s: s.blas_geom_count.__setitem__(0, 99), "geometry range"),
    (lambda s: s.ray_types.__setitem__((0, 0), 7), "miss shader"),
])
def test_validation_rejects(pr, mutate, frag):
    w = scenes.small_analytic()
    pr.validate(w.scene)
    mutate(w.scene)
    with pytest.raises(pr.PrError) as ei:
        pr.validate(w.scene)
    assert ei.value.status == pr.PR_ERR_INVALID_ARG
    assert frag in str(ei.value)


def test_validation_accepts_all_configs(pr):
    for w in (scenes.small_analytic(), scenes.teaser(width=8, height=8), scenes.field(n_inst=300, width=8, height=8)):
        pr.validate(w.scene)


def test_cutout_any_hit_needs_an_intersection_shader(pr):
    w = scenes.small_analytic()
    w.scene.hit_groups[0, 2] = scenes.AHS_CUTOUT      # sphere intersection shader: allowed
    pr.validate(w.scene)
    f = scenes.field(n_inst=50, width=8, height=8)
    torus_hg = [h for h in range(len(f.scene.hit_groups)) if f.scene.hit_groups[h, 0] == scenes.IS_TORUS][0]
    f.scene.hit_groups[torus_hg, 2] = scenes.AHS_CUTOUT   # sphere-traced shader: allowed too
    pr.validate(f.scene)
    f.scene.hit_groups[torus_hg, 0] = scenes.NONE         # no intersection shader to report candidates
    with pytest.raises(pr.PrError) as ei:
        pr.validate(f.scene)
    assert "intersection shader" in str(ei.value)


def test_triangle_validation(pr):
    w = scenes.sample_scene(width=8, height=8)
    pr.validate(w.scene)
    bad = scenes.sample_scene(width=8, height=8)
    bad.scene.indices[0, 0] = 10_000
    with pytest.raises(pr.PrError) as ei:
        pr.validate(bad.scene)
    assert "vertex index" in str(ei.value)
    mixed = scenes.sample_scene(width=8, height=8)
    mixed.scene.blas_geom_count[0] = 2            # triangle BLAS swallowing an AABB geometry
    with pytest.raises(pr.PrError) as ei:
        pr.validate(mixed.scene)
    assert "mixes" in str(ei.value)
    rng = scenes.sample_scene(width=8, height=8)
    rng.scene.geom_prim_count[0] = 999
    with pytest.raises(pr.PrError):
        pr.validate(rng.scene)


def test_one_ray_type_is_rejected(pr):
    w = scenes.small_analytic()
    w.scene.ray_types = w.scene.ray_types[:1]
    with pytest.raises(pr.PrError):
        pr.validate(w.scene)


def test_header_documents_every_entry_point():
    """Each declaration in the header is directly preceded by a comment."""
    text = open(HEADER).read()
    for s in declared_symbols():
        m = re.search(r"\n((?:pr_status|uint32_t|const char\*|void|size_t)\s+\*?" + s + r"\()", text)
        assert m, s
        before = text[:m.start(1)].rstrip()
        assert before.endswith("*/"), s


def test_build_many_rejects_a_scene_listed_twice(pr):
    """pr_build_bvh_many refuses an array naming one scene twice (two streams
    would build it into one arena at once) before it touches any scene: the
    handles here are never dereferenced, so no device is needed."""
    lib = ctypes.CDLL(pr.LIB_PATH)
    lib.pr_build_bvh_many.restype = ctypes.c_int
    lib.pr_build_bvh_many.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint32, ctypes.c_void_p]
    lib.pr_last_error.restype = ctypes.c_char_p
    fake = ctypes.c_void_p(0x1000)   # an address no scene has; only compared, never read
    arr = (ctypes.c_void_p * 3)(0x2000, fake.value, fake.value)
    assert lib.pr_build_bvh_many(arr, 3, None) == pr.PR_ERR_INVALID_ARG
    assert b"twice" in lib.pr_last_error()
