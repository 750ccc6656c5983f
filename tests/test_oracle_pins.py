"""Pins of the CPU FP64 oracle against facts independent of it.

Each test checks the oracle against closed forms, brute force, invariants or
the paper's worked examples (Eq. 1 / Fig. 3, Listing 10), so that a dropped
term, a wrong sign or index, or a transposed operand in the oracle fails here.
No GPU is needed.
"""
import json
import math
import os

import numpy as np
import pytest

import scenes
from scenes import (IS_BOX, IS_CAPSULE, IS_JULIA, IS_MANDELBULB, IS_METABALL4, IS_PACMAN,
                    IS_ROUNDBOX, IS_SPHERE, IS_TORUS)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


# --------------------------------------------------------------------------
# Analytic intersection shaders
# --------------------------------------------------------------------------
def test_sphere_closed_form(O):
    prm = [0, 0, 0, 1]
    t, n, _ = O.intersect(IS_SPHERE, prm, [0, 0, -5], [0, 0, 1], 0.0)
    assert t == pytest.approx(4.0, abs=1e-12) and np.allclose(n, [0, 0, -1])
    # origin inside: the far root
    t, n, _ = O.intersect(IS_SPHERE, prm, [0, 0, 0.5], [0, 0, 1], 0.0)
    assert t == pytest.approx(0.5, abs=1e-12) and np.allclose(n, [0, 0, 1])
    # non-unit direction: t is measured in units of |d|
    t, _, _ = O.intersect(IS_SPHERE, [1, 2, 3, 0.5], [1, 2, -7], [0, 0, 4], 0.0)
    assert t == pytest.approx((10 - 0.5) / 4, abs=1e-12)
    # a line passing just outside the radius misses; just inside hits
    assert O.intersect(IS_SPHERE, prm, [1 + 1e-9, 0, -5], [0, 0, 1], 0.0) is None
    assert O.intersect(IS_SPHERE, prm, [1 - 1e-9, 0, -5], [0, 0, 1], 0.0) is not None
    # tmin past both roots
    assert O.intersect(IS_SPHERE, prm, [0, 0, -5], [0, 0, 1], 6.5) is None


def _first_inside(inside_fn, o, d, t_max, n=20000):
    ts = np.linspace(0.0, t_max, n)
    ins = inside_fn(o[None] + ts[:, None] * d[None])
    idx = np.argmax(ins)
    return ts[idx] if ins[idx] else None


def test_sphere_random_rays_geometric(O):
    """Hit iff the line passes within R of the centre (cross-product distance);
    the hit lies on the sphere and no earlier sample point is inside."""
    rng = np.random.default_rng(1)
    c, R = np.array([0.25, -0.125, 0.125]), 0.75
    for _ in range(300):
        o = rng.uniform(-4, 4, 3)
        if np.linalg.norm(o - c) < R + 0.05:
            continue
        d = _unit(c + rng.normal(scale=0.6, size=3) - o) * rng.uniform(0.5, 2.0)
        line_dist = np.linalg.norm(np.cross(c - o, d)) / np.linalg.norm(d)
        ahead = np.dot(c - o, d) > 0
        res = O.intersect(IS_SPHERE, [*c, R], o, d, 0.0)
        if abs(line_dist - R) < 1e-6:
            continue
        assert (res is not None) == (line_dist < R and ahead)
        if res:
            t, n, _ = res
            p = o + t * d
            assert np.linalg.norm(p - c) == pytest.approx(R, abs=1e-9)
            assert np.allclose(n, (p - c) / R, atol=1e-9)
            t_ref = _first_inside(lambda P: np.linalg.norm(P - c, axis=1) <= R, o, d, 2 * t + 1)
            assert t_ref is not None and abs(t_ref - t) <= (2 * t + 1) / 20000 + 1e-9


def test_box_closed_form_and_random(O):
    prm = [0, 0, 0, 1, 1, 1]
    t, n, _ = O.intersect(IS_BOX, prm, [-5, 0.2, 0.3], [1, 0, 0], 0.0)
    assert t == pytest.approx(4.0) and np.allclose(n, [-1, 0, 0])
    t, n, _ = O.intersect(IS_BOX, prm, [0.2, 7, 0.3], [0, -2, 0], 0.0)
    assert t == pytest.approx(3.0) and np.allclose(n, [0, 1, 0])
    t, n, _ = O.intersect(IS_BOX, prm, [0.0, 0.0, 0.0], [0, 0, 1], 0.0)   # inside: exit face
    assert t == pytest.approx(1.0) and np.allclose(n, [0, 0, 1])
    assert O.intersect(IS_BOX, prm, [-5, 1.5, 0], [1, 0, 0], 0.0) is None
    # entering exactly through an edge: the tie goes to the lowest axis (x before y)
    t, n, _ = O.intersect(IS_BOX, prm, [-5, -5, 0.5], [1, 1, 0], 0.0)
    assert t == pytest.approx(4.0) and np.allclose(n, [-1, 0, 0])
    rng = np.random.default_rng(2)
    c, e = np.array([0.5, -0.25, 0.125]), np.array([0.75, 0.375, 1.125])
    inside = lambda P: np.all(np.abs(P - c) <= e, axis=1)
    hits = 0
    for _ in range(300):
        o = rng.uniform(-4, 4, 3)
        if inside(o[None])[0]:
            continue
        d = _unit(c + rng.normal(scale=0.8, size=3) - o)
        res = O.intersect(IS_BOX, [*c, *e], o, d, 0.0)
        t_ref = _first_inside(inside, o, d, 12.0)
        if res is None:
            assert t_ref is None
            continue
        hits += 1
        t, n, _ = res
        p = o + t * d
        assert np.max(np.abs(p - c) / e) == pytest.approx(1.0, abs=1e-9)
        k = int(np.argmax(np.abs(n)))
        assert abs(abs(p[k] - c[k]) - e[k]) < 1e-9 and np.sign(n[k]) == np.sign(p[k] - c[k])
        assert np.dot(n, d) < 0
        assert t_ref is not None and abs(t_ref - t) <= 12.0 / 20000 + 1e-9
    assert hits > 50


def _pacman_inside(P, c, R, a):
    q = P - c
    n1 = np.array([-math.sin(a), math.cos(a), 0.0])
    n2 = np.array([-math.sin(a), -math.cos(a), 0.0])
    in_ball = np.linalg.norm(q, axis=1) <= R
    in_wedge = (q @ n1 < 0) & (q @ n2 < 0)
    return in_ball & ~in_wedge


def test_pacman_reductions(O):
    a = float(np.float32(math.radians(30)))   # parameters are stored as float32
    prm = [0, 0, 0, 1, a]
    # a ray meeting the back of the ball (outside the mouth) reduces to the sphere
    t, n, _ = O.intersect(IS_PACMAN, prm, [-5, 0.1, 0.2], [1, 0, 0], 0.0)
    ts, ns, _ = O.intersect(IS_SPHERE, [0, 0, 0, 1], [-5, 0.1, 0.2], [1, 0, 0], 0.0)
    assert t == pytest.approx(ts, abs=1e-12) and np.allclose(n, ns)
    # a ray entering the mouth hits wedge plane 1 where x = y / tan(a)
    y0 = 0.1
    t, n, _ = O.intersect(IS_PACMAN, prm, [5, y0, 0], [-1, 0, 0], 0.0)
    assert t == pytest.approx(5 - y0 / math.tan(a), abs=1e-12)
    assert np.allclose(n, [math.sin(a), -math.cos(a), 0])     # -n1
    # and by symmetry wedge plane 2 below the axis
    t, n, _ = O.intersect(IS_PACMAN, prm, [5, -y0, 0], [-1, 0, 0], 0.0)
    assert t == pytest.approx(5 - y0 / math.tan(a), abs=1e-12)
    assert np.allclose(n, [math.sin(a), math.cos(a), 0])      # -n2
    # a ray along z inside the mouth, away from the ball's rim, never meets the solid
    assert O.intersect(IS_PACMAN, prm, [0.6, 0.0, -5], [0, 0, 1], 0.0) is None
    # the same ray outside the mouth meets the sphere
    assert O.intersect(IS_PACMAN, prm, [-0.6, 0.0, -5], [0, 0, 1], 0.0) is not None


def _band(y):
    return 4 * y - math.floor(4 * y)


def _sphere_roots(o, d, r):
    b, c = np.dot(o, d), np.dot(o, o) - r * r
    disc = b * b - c
    return None if disc < 0 else (-b - math.sqrt(disc), -b + math.sqrt(disc))


def test_sphere_traced_cutout_on_level_rays(O):
    """A capsule of zero half-height is a ball. On a ray with d.y = 0 every candidate has
    the same y: a kept band gives the ball's entry root (to the march tolerance), a
    removed band ignores every candidate and the march goes through the ball: a miss."""
    r = 0.45
    prm = [0.0, r]
    kept = removed = 0
    for y0 in np.linspace(-0.4, 0.4, 33):
        for x0 in (-0.2, 0.0, 0.15):
            o, d = np.array([x0, y0, -3.0]), np.array([0.0, 0.0, 1.0])
            roots = _sphere_roots(o, d, r)
            if roots is None or abs(_band(y0) - 0.5) < 1e-6 or _band(y0) < 1e-6:
                continue
            res = O.intersect(IS_CAPSULE, prm, o, d, 0.0, 10.0, eps=1e-6, max_steps=512,
                              ahs_id=scenes.AHS_CUTOUT)
            if _band(y0) >= 0.5:
                kept += 1
                assert res is not None and res[0] == pytest.approx(roots[0], abs=1e-5)
            else:
                removed += 1
                assert res is None
    assert kept > 10 and removed > 10


def test_sphere_traced_cutout_marches_through_the_solid(O):
    """Rays that enter a ball (capsule of zero half-height) in a removed band and climb
    into a kept band before leaving it: the march goes on through the solid and reports
    the first kept point it visits, inside the ball or on its surface; rays that stay in
    removed bands miss; without the shader the entry root."""
    r = 0.45
    prm = [0.0, r]
    eps = 1e-6
    hits = misses = 0
    for slope, y0 in [(sl, y) for sl in (0.05, 0.3) for y in np.linspace(-1.4, 0.2, 161)]:
        o, d = np.array([-3.0, y0, 0.05]), _unit([1.0, slope, 0.0])
        roots = _sphere_roots(o, d, r)
        if roots is None:
            continue
        ys = [(o + t * d)[1] for t in np.linspace(roots[0], roots[1], 4001)]
        if min(min(abs(_band(y) - 0.5), _band(y), 1 - _band(y)) for y in (ys[0], ys[-1])) < 1e-4:
            continue                                   # the chord starts or ends on a band edge: skip
        n_entry = (o + roots[0] * d) / r
        if abs(np.dot(n_entry, d)) < 0.2:
            continue                                   # grazing entry: the march tolerance stretches along the ray
        plain = O.intersect(IS_CAPSULE, prm, o, d, 0.0, 10.0, eps=eps, max_steps=2048)
        assert plain is not None and plain[0] == pytest.approx(roots[0], abs=1e-4)
        res = O.intersect(IS_CAPSULE, prm, o, d, 0.0, 10.0, eps=eps, max_steps=2048, ahs_id=scenes.AHS_CUTOUT)
        first_kept = next((t for t, y in zip(np.linspace(roots[0], roots[1], 4001), ys) if _band(y) >= 0.5), None)
        if first_kept is None:
            misses += 1
            assert res is None
            continue
        hits += 1
        assert res is not None
        p = o + res[0] * d
        assert _band(p[1]) >= 0.5                       # the any-hit shader kept it
        assert np.linalg.norm(p) <= r + 1e-5            # in or on the ball
        assert roots[0] - 1e-5 <= res[0] <= roots[1] + 1e-5
        if _band((o + roots[0] * d)[1]) >= 0.5:
            assert res[0] == pytest.approx(roots[0], abs=1e-4)
        else:
            assert res[0] >= first_kept - 1e-3          # no kept point is reported before the chord reaches one
    assert hits > 5 and misses > 5


def test_cutout_any_hit_skips_banded_candidates(O):
    """Unit sphere, ray in the y-z plane: the front point lies in a removed band
    (frac(4y) < 1/2), the back point in a kept band, so the far root is reported;
    with the back point removed too the ray misses; without the shader the near root."""
    d = _unit([0.0, 0.35, 1.0])
    band = lambda y: 4 * y - math.floor(4 * y)

    def roots_of(o):
        b, c = np.dot(o, d), np.dot(o, o) - 1.0
        disc = b * b - c
        return None if disc < 0 else (-b - math.sqrt(disc), -b + math.sqrt(disc))

    o = None
    for dy in np.linspace(-1.6, -0.2, 141):            # pick a ray with this geometry
        cand = np.array([0.0, dy, -3.0])
        r = roots_of(cand)
        if r and band((cand + r[0] * d)[1]) < 0.45 and band((cand + r[1] * d)[1]) > 0.55:
            o = cand
            break
    assert o is not None
    t0, t1 = roots_of(o)
    t, n, _ = O.intersect(IS_SPHERE, [0, 0, 0, 1], o, d, 0.0, ahs_id=scenes.AHS_CUTOUT)
    assert t == pytest.approx(t1, abs=1e-12)
    t, n, _ = O.intersect(IS_SPHERE, [0, 0, 0, 1], o, d, 0.0)
    assert t == pytest.approx(t0, abs=1e-12)
    # shift the ray so that both candidates fall in removed bands: no hit
    for dy in np.linspace(-0.2, 0.2, 81):
        o2 = o + np.array([0.0, dy, 0.0])
        r = roots_of(o2)
        if r is None:
            continue
        ya, yb = [(o2 + t * d)[1] for t in r]
        if min(abs(band(ya) - 0.5), abs(band(yb) - 0.5), band(ya), band(yb)) < 1e-9:
            continue                                    # on a band edge: ill-conditioned
        res = O.intersect(IS_SPHERE, [0, 0, 0, 1], o2, d, 0.0, ahs_id=scenes.AHS_CUTOUT)
        expect = None if (band(ya) < 0.5 and band(yb) < 0.5) else (r[0] if band(ya) >= 0.5 else r[1])
        if expect is None:
            assert res is None
        else:
            assert res is not None and res[0] == pytest.approx(expect, abs=1e-9)
    # box: entry face removed, exit face kept
    t, n, _ = O.intersect(IS_BOX, [0, 0, 0, 1, 1, 1], [-5, 0.1, 0.0], [1, 0.06, 0], 0.0, ahs_id=scenes.AHS_CUTOUT)
    ye = 0.1 + 0.06 * 4.0
    assert band(ye) < 0.5 and t == pytest.approx(6.0) and np.allclose(n, [1, 0, 0])


def _one_triangle_workload(v, eye, look):
    b = scenes.SceneBuilder()
    scenes._standard_rays(b)
    hr, hs = b.add_hit_group(scenes.NONE, scenes.CHS_LAMBERT), b.add_hit_group(scenes.NONE)
    m = b.add_material((0.5, 0.5, 0.5))
    blas = b.add_blas([b.add_triangle_geometry(np.asarray(v, np.float32), [[0, 1, 2]])])
    b.add_record(hr, m, scenes.NONE, 0)
    b.add_record(hs, m, scenes.NONE, 0)
    b.add_instance(blas, scenes.xform_trs((0, 0, 0)), 0)
    cam = scenes.Camera(np.float32(eye), np.float32(look), np.float32([0, 1, 0]), 1.0)
    return scenes.Workload(b.build("tri"), cam, scenes.TraceParams(1, 1, light_pos=np.float32([0, 0, -50])))


def test_triangle_hits_by_half_spaces(O):
    """Built-in triangle test: a ray along +z through (x, y) meets the triangle
    (0,0,0), (2,0,0), (0,2,0) iff x >= 0, y >= 0, x + y <= 2 (half-space test,
    independent of the barycentric solve), at t = 10 with normal +-z."""
    tri = [[0, 0, 0], [2, 0, 0], [0, 2, 0]]
    for x in np.linspace(-0.5, 2.5, 13):
        for y in np.linspace(-0.5, 2.5, 13):
            inside = x >= 0 and y >= 0 and x + y <= 2
            if min(abs(x), abs(y), abs(x + y - 2)) < 1e-9:
                continue
            px = O.render(_one_triangle_workload(tri, [x, y, -10], [x, y, 0]))[0]
            assert bool(px["flags"] & 1) == inside, (x, y)
            if inside:
                assert px["t"] == pytest.approx(10.0, abs=1e-9)
                assert np.allclose(np.abs(px["n"]), [0, 0, 1])


def test_triangle_slanted_plane_point(O):
    """A slanted triangle: the hit point must satisfy the plane equation."""
    tri = np.array([[-3, -2, 1], [4, -1, 3], [0, 3, 6]], np.float64)
    n = np.cross(tri[1] - tri[0], tri[2] - tri[0])
    for x, y in [(0.0, 0.0), (0.5, 0.7), (-0.4, 1.2)]:
        px = O.render(_one_triangle_workload(tri, [x, y, -10], [x, y, 0]))[0]
        assert px["flags"] & 1
        p = np.float32([x, y, -10.0]).astype(np.float64) + px["t"] * np.array([0, 0, 1.0])   # the eye is float32
        assert abs(np.dot(n, p - tri[0])) < 1e-9 * np.linalg.norm(n)


def test_pacman_random_dense_membership(O):
    rng = np.random.default_rng(3)
    a = float(np.float32(math.radians(30)))
    c, R = np.zeros(3), 1.0
    inside = lambda P: _pacman_inside(P, c, R, a)
    hits = 0
    for _ in range(400):
        o = rng.uniform(-3, 3, 3)
        if np.linalg.norm(o) < 1.2:
            continue
        d = _unit(rng.normal(scale=0.5, size=3) + np.array([0.5, 0, 0]) - o)
        res = O.intersect(IS_PACMAN, [*c, R, a], o, d, 0.0)
        t_ref = _first_inside(inside, o, d, 8.0, n=40000)
        step = 8.0 / 40000
        if res is None:
            assert t_ref is None
            continue
        hits += 1
        assert t_ref is not None and abs(t_ref - res[0]) <= step + 1e-9
    assert hits > 100


# --------------------------------------------------------------------------
# Signed distance functions and sphere tracing
# --------------------------------------------------------------------------
def test_sdf_closed_forms(O):
    assert O.de(IS_TORUS, [1, 0.25], [1, 0, 0]) == pytest.approx(-0.25)
    assert O.de(IS_TORUS, [1, 0.25], [2.25, 0, 0]) == pytest.approx(1.0)
    assert O.de(IS_TORUS, [1, 0.25], [0, 0, 0]) == pytest.approx(0.75)
    assert O.de(IS_TORUS, [1, 0.25], [0, 2, 1]) == pytest.approx(1.75)
    assert O.de(IS_CAPSULE, [0.6, 0.3], [0, 1.4, 0]) == pytest.approx(0.5)
    assert O.de(IS_CAPSULE, [0.6, 0.3], [1, 0.2, 0]) == pytest.approx(0.7)
    assert O.de(IS_CAPSULE, [0.6, 0.3], [0, 0, 0]) == pytest.approx(-0.3)
    rb = [0.6, 0.6, 0.6, 0.15]
    assert O.de(IS_ROUNDBOX, rb, [1, 0, 0]) == pytest.approx(0.4)
    assert O.de(IS_ROUNDBOX, rb, [0, 0, 0]) == pytest.approx(-0.6)
    # corner: distance to the rounding sphere centred at (0.45,0.45,0.45)
    p = np.array([1.0, 1.0, 1.0])
    assert O.de(IS_ROUNDBOX, rb, p) == pytest.approx(np.linalg.norm(p - 0.45) - 0.15)
    # metaballs far apart: smooth-min equals plain min of ball distances
    mb = [-3, 0, 0, 3, 0, 0, 0, -3, 0, 0, 3, 0, 0.3, 0.3, 0.3, 0.3]
    assert O.de(IS_METABALL4, mb, [-3, 1, 0]) == pytest.approx(0.7)
    # two touching balls: the smooth union bulges out by k/4 where distances tie
    mb2 = [-0.5, 0, 0, 0.5, 0, 0, 0, 9, 0, 0, -9, 0, 0.4, 0.4, 0.1, 0.1]
    d_plain = math.hypot(0.5, 0.3) - 0.4
    assert O.de(IS_METABALL4, mb2, [0, 0.3, 0]) == pytest.approx(d_plain - 0.2 / 4)


def _bisect_root(f, t0, t1, it=80):
    for _ in range(it):
        tm = 0.5 * (t0 + t1)
        if f(tm) < 0:
            t1 = tm
        else:
            t0 = tm
    return t1


@pytest.mark.parametrize("is_id,prm", [
    (IS_TORUS, [1, 0.25]), (IS_ROUNDBOX, [0.6, 0.6, 0.6, 0.15]), (IS_CAPSULE, [0.6, 0.3]),
    (IS_METABALL4, list(scenes.shape_metaball4(np.random.default_rng(5))[1]))])
def test_sdf_sphere_tracing_vs_bisection(O, is_id, prm):
    """The first sign change of the SDF along the ray (dense sampling then
    bisection to ~1e-15) bounds the sphere-traced t from above, within eps."""
    rng = np.random.default_rng(4)
    eps = 1e-4
    hits = 0
    for _ in range(70):
        o = _unit(rng.normal(size=3)) * 3.0
        d = _unit(rng.normal(scale=0.35, size=3) - o)
        f = lambda t: O.de(is_id, prm, o + t * d)
        ts = np.linspace(0, 6, 1501)
        vals = np.array([f(t) for t in ts])
        neg = np.nonzero(vals < 0)[0]
        res = O.intersect(is_id, prm, o, d, 0.0, 6.0, eps, 256)
        if len(neg) == 0:
            if res is not None:   # grazing: must still be within eps of the surface
                assert abs(f(res[0])) < eps
            continue
        k = neg[0]
        t_star = _bisect_root(f, ts[k - 1], ts[k])
        assert res is not None
        hits += 1
        t, n, steps = res
        assert t <= t_star + 1e-12
        assert f(t) < eps and t_star - t < 50 * eps
        assert 1 <= steps <= 256
        assert abs(np.linalg.norm(n) - 1) < 1e-12
    assert hits > 20


# --------------------------------------------------------------------------
# Normals of sphere-traced hits against closed-form gradients
# --------------------------------------------------------------------------
# The oracle's sphere-traced normal is the normalised central difference of the
# estimate (step eps |d|). For the exact SDFs the gradient has a closed form
# written from the geometry (the direction from the closest point of the core
# set: ring circle, segment, inner box); for the smooth-min metaballs it is the
# chain rule of the polynomial smooth minimum. A swapped or wrong-axis stencil,
# or a sign error inside an SDF, moves these normals by far more than 1e-3 rad.
def _grad_torus(p, R, r):
    rho = math.hypot(p[0], p[2])
    core = np.array([R * p[0] / rho, 0.0, R * p[2] / rho])
    return _unit(p - core)


def _grad_capsule(p, h, r):
    return _unit(p - np.array([0.0, min(max(p[1], -h), h), 0.0]))


def _grad_roundbox(p, b, rr):
    e = np.asarray(b, np.float64) - rr
    v = p - np.clip(p, -e, e)          # face, edge or corner region of the inner box
    assert np.linalg.norm(v) > 0.5 * rr
    return _unit(v)


def _grad_metaball4(p, prm, k=0.2):
    """Chain rule through smin(smin(smin(d0, d1), d2), d3): with
    h = max(k - |a - b|, 0) / k, d smin / d min(a, b) = 1 - h/2 and
    d smin / d max(a, b) = h/2."""
    prm = np.asarray(prm, np.float64)
    cs, rs = prm[:12].reshape(4, 3), prm[12:16]
    dist = [np.linalg.norm(p - cs[i]) - rs[i] for i in range(4)]
    grad = [_unit(p - cs[i]) for i in range(4)]

    def smin_with_grad(a, ga, b, gb):
        h = max(k - abs(a - b), 0.0) / k
        wa, wb = (1 - h / 2, h / 2) if a <= b else (h / 2, 1 - h / 2)
        return min(a, b) - h * h * k * 0.25, wa * ga + wb * gb

    m, g = smin_with_grad(dist[0], grad[0], dist[1], grad[1])
    m, g = smin_with_grad(m, g, dist[2], grad[2])
    m, g = smin_with_grad(m, g, dist[3], grad[3])
    return _unit(g)


_FAR_METABALLS = [-1.5, 0, 0, 1.5, 0, 0, 0, 1.5, 0, 0, -1.5, 0, 0.4, 0.3, 0.35, 0.25]


@pytest.mark.parametrize("is_id,prm,grad", [
    (IS_TORUS, [1, 0.25], lambda p: _grad_torus(p, 1.0, 0.25)),
    (IS_TORUS, [0.7, 0.3], lambda p: _grad_torus(p, 0.7, 0.3)),
    (IS_CAPSULE, [0.6, 0.3], lambda p: _grad_capsule(p, 0.6, 0.3)),
    (IS_ROUNDBOX, [0.6, 0.6, 0.6, 0.15], lambda p: _grad_roundbox(p, [0.6, 0.6, 0.6], 0.15)),
    (IS_ROUNDBOX, [0.9, 0.4, 0.6, 0.1], lambda p: _grad_roundbox(p, [0.9, 0.4, 0.6], 0.1)),
    # far-apart balls: the smooth minimum is the plain one, each ball's normal radial
    (IS_METABALL4, _FAR_METABALLS, lambda p: _grad_metaball4(p, _FAR_METABALLS)),
    (IS_METABALL4, list(scenes.shape_metaball4(np.random.default_rng(5))[1]),
     lambda p: _grad_metaball4(p, scenes.shape_metaball4(np.random.default_rng(5))[1])),
], ids=["torus", "torus_thick", "capsule", "roundbox", "roundbox_aniso", "metaballs_apart", "metaballs_blend"])
def test_sphere_traced_normal_is_the_sdf_gradient(O, is_id, prm, grad):
    """At sphere-traced hits of random rays (eps 1e-4, |d| = 1 and |d| != 1),
    the oracle's normal is within 1e-3 rad of the closed-form gradient."""
    rng = np.random.default_rng(17)
    eps = 1e-4
    hits, worst = 0, 0.0
    for k in range(160):
        o = _unit(rng.normal(size=3)) * 3.0
        aim = rng.uniform(-0.5, 0.5, 3)
        if prm is _FAR_METABALLS:      # aim at one of the separated balls
            aim = 0.6 * aim + np.reshape(prm[:12], (4, 3))[k % 4]
        d = _unit(aim - o)
        if k % 2:
            d = d * 0.6        # an object-space direction of a scaled instance: t shared with world
        res = O.intersect(is_id, prm, o, d, 0.0, 10.0, eps, 256)
        if res is None:
            continue
        t, n, _ = res
        p = o + t * d
        ang = math.acos(min(1.0, abs(float(np.dot(n, grad(p))))))
        assert float(np.dot(n, grad(p))) > 0, (k, p, n)          # outward, not flipped
        worst = max(worst, ang)
        hits += 1
    assert hits >= 60, hits
    assert worst <= 1e-3, worst


def test_julia_c0_normal_is_radial(O):
    """c = 0: the estimate 0.5 r ln r is radial, so sphere-traced hits near the
    unit ball carry the radial normal p / |p| (pins the stencil on a fractal
    estimator). eps = 1e-2 keeps the stencil outside the 12-iteration filled
    set (radius 4^(1/4096) = 1.00034), where the estimate jumps to 0."""
    rng = np.random.default_rng(23)
    prm = [0, 0, 0, 0, 12, 4]
    hits = 0
    for _ in range(60):
        o = _unit(rng.normal(size=3)) * 3.0
        d = _unit(rng.uniform(-0.6, 0.6, 3) - o)
        res = O.intersect(IS_JULIA, prm, o, d, 0.0, 10.0, 1e-2, 256)
        if res is None:
            continue
        t, n, _ = res
        p = o + t * d
        assert math.acos(min(1.0, float(np.dot(n, _unit(p))))) <= 1e-3
        hits += 1
    assert hits >= 30


def test_julia_c0_closed_form(O):
    """c = 0: q_n = q^(2^n), so the estimate collapses to 0.5 |q| ln|q| outside
    the unit ball and the 12-iteration filled set is the unit ball itself."""
    prm = [0, 0, 0, 0, 12, 4]
    for r in (1.3, 2.0, 3.5, 10.0):
        p = _unit([0.3, -0.5, 0.8]) * r
        assert O.de(IS_JULIA, prm, p) == pytest.approx(0.5 * r * math.log(r), rel=1e-12)
    assert O.de(IS_JULIA, prm, [0.2, 0.3, -0.4]) == 0.0
    # points just outside the unit ball whose orbit has not escaped after 12 steps
    assert O.de(IS_JULIA, prm, [1.0001, 0, 0]) == 0.0


def test_julia_cut_closed_form(O):
    """c = 0 cut by n = (0,0,-1), d = 0: the half ball z >= 0. The estimate is
    max(Julia estimate, plane distance); a ray along +z through the ball's
    centre meets the cut face at z = 0 with normal -z."""
    prm = [0, 0, 0, 0, 12, 4, 0, 0, -1, 0]
    assert O.de(scenes.IS_JULIA_CUT, prm, [0, 0, -0.5]) == pytest.approx(0.5)      # removed half of the ball
    assert O.de(scenes.IS_JULIA_CUT, prm, [0.1, 0.2, 0.5]) == 0.0                   # kept half: inside
    p = _unit([0.3, -0.5, 0.8]) * 2.0                                               # outside both: the larger bound
    assert O.de(scenes.IS_JULIA_CUT, prm, p) == pytest.approx(max(0.5 * 2 * math.log(2), -p[2]))
    t, n, _ = O.intersect(scenes.IS_JULIA_CUT, prm, [0.05, 0.02, -3], [0, 0, 1], 0.0, 10.0, 1e-5, 256)
    assert t == pytest.approx(3.0, abs=2e-5) and np.allclose(n, [0, 0, -1], atol=1e-3)
    # the same ray with the half-space flipped keeps the front half: the ball's sphere at z ~ -1
    prm2 = [0, 0, 0, 0, 12, 4, 0, 0, 1, 0]
    t2, _, _ = O.intersect(scenes.IS_JULIA_CUT, prm2, [0.05, 0.02, -3], [0, 0, 1], 0.0, 10.0, 1e-5, 256)
    assert t2 == pytest.approx(3.0 - math.sqrt(1 - 0.05 ** 2 - 0.02 ** 2), abs=1e-3)


def test_mandelbulb_axis_reduces_to_real_iteration(O):
    """On the +z axis (theta = 0) the power map is z -> z^8 on the real line."""
    for a in (1.05, 1.2, 0.9, 0.5):
        z, dr, val = a, 1.0, 0.0
        for _ in range(12):
            dr = 8 * abs(z) ** 7 * dr + 1
            z = z ** 8 + a
            if abs(z) > 2:
                val = 0.5 * math.log(abs(z)) * abs(z) / dr
                break
        assert O.de(IS_MANDELBULB, [8, 12, 2], [0, 0, a]) == pytest.approx(val, rel=1e-12, abs=1e-300)


def test_triplex_pow_matches_complex_form(O):
    """z^8 in spherical form equals the trig-free form Im((z+i rho)^8) * e^(8i phi),
    Re((z + i rho)^8) built from complex powers (away from r = 0)."""
    rng = np.random.default_rng(6)
    for _ in range(500):
        z = rng.uniform(-1.5, 1.5, 3)
        x, y, zz = z
        rho = math.hypot(x, y)
        w = complex(zz, rho) ** 8
        u = (complex(x, y) / rho) ** 8
        ref = np.array([w.imag * u.real, w.imag * u.imag, w.real])
        got = O.triplex_pow(z, 8.0)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * np.linalg.norm(z) ** 8)


def _julia_filled(c, P, iters):
    q = np.concatenate([P, np.zeros((len(P), 1))], 1)
    alive = np.ones(len(P), bool)
    for _ in range(iters):
        a, b, cc, d = q.T
        q = np.stack([a * a - b * b - cc * cc - d * d, 2 * a * b, 2 * a * cc, 2 * a * d], 1) + c
        alive &= (q * q).sum(1) <= 16.0
        q[~alive] = 0
    return alive


def _bulb_filled(P, iters):
    z = P.copy()
    alive = np.ones(len(P), bool)
    for _ in range(iters):
        x, y, zz = z.T
        rho = np.sqrt(x * x + y * y)
        w = (zz + 1j * rho) ** 8
        u = np.where(rho > 0, (x + 1j * y) / np.where(rho > 0, rho, 1), 1) ** 8
        z = np.stack([w.imag * u.real, w.imag * u.imag, w.real], 1) + P
        alive &= np.sqrt((z * z).sum(1)) <= 2.0
        z[~alive] = 0
    return alive


@pytest.mark.parametrize("kind", ["julia", "mandelbulb"])
def test_fractal_estimate_never_overshoots(O, kind):
    """Invariant: from a point p outside the set with estimate d above the
    hit threshold, the ball of radius d around p holds no point of the filled
    set (64 random samples per point; membership by independent iteration:
    quaternion squaring in numpy, resp. the complex-power Mandelbulb map). The
    reference sets use deeper iteration (20 resp. 40), i.e. points of the
    actual fractal; the 12-iteration set is fatter than what the estimate
    measures (its thin filaments are not seen by it). Points are those the
    marcher steps from: estimate above 4e-3 object units, below the teaser
    scene's hit threshold (1e-4 x diagonal / instance scale ~ 4.8e-3)."""
    rng = np.random.default_rng(7)
    if kind == "julia":
        c = scenes.julia_c(np.random.default_rng(0))
        is_id, prm, ext = IS_JULIA, [*c, 12, 4], 1.6
        inside = lambda P: _julia_filled(c, P, 20)
    else:
        is_id, prm, ext = IS_MANDELBULB, [8, 12, 2], 1.25
        inside = lambda P: _bulb_filled(P, 40)
    tested = 0
    for _ in range(900):
        p = rng.uniform(-ext, ext, 3)
        d = O.de(is_id, prm, p)
        if d <= 4e-3:
            continue
        tested += 1
        dirs = rng.normal(size=(64, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        P = p + dirs * rng.uniform(0, 1, (64, 1)) * d
        assert not inside(P).any(), f"estimate {d} overshoots at {p}"
    assert tested > 500


# --------------------------------------------------------------------------
# Camera, shading, traversal semantics
# --------------------------------------------------------------------------
def _single_sphere_workload(width=33, height=33, light=(0, 0, -10), albedo=(0.5, 0.25, 1.0), kr=0.0,
                            max_depth=1):
    b = scenes.SceneBuilder()
    scenes._standard_rays(b)
    hr, hs = b.add_hit_group(IS_SPHERE, scenes.CHS_LAMBERT), b.add_hit_group(IS_SPHERE)
    mat = b.add_material(albedo, kr)
    aabb, prm = scenes.shape_sphere((0, 0, 0), 1.0)
    blas = b.add_blas([b.add_geometry([aabb], [prm])])
    b.add_record(hr, mat, IS_SPHERE, 0)
    b.add_record(hs, mat, IS_SPHERE, 0)
    b.add_instance(blas, scenes.xform_trs((0, 0, 0)), 0)
    cam = scenes.Camera(np.float32([0, 0, -10]), np.float32([0, 0, 0]), np.float32([0, 1, 0]), 60.0)
    tp = scenes.TraceParams(width, height, max_depth=max_depth, light_pos=np.float32(light))
    return scenes.Workload(b.build("one-sphere"), cam, tp)


def test_head_on_lambert_closed_form(O):
    """Odd image: the centre pixel looks along the axis, meets the pole at t = 9
    with n = l, so the radiance is albedo * (k_a + I)."""
    w = _single_sphere_workload()
    px = O.render(w, pixels=[16 * 33 + 16])[0]
    assert px["flags"] & 1 and px["t"] == pytest.approx(9.0, abs=1e-12)
    assert np.allclose(px["n"], [0, 0, -1])
    assert np.allclose(px["rgb"], np.array([0.5, 0.25, 1.0]) * 1.1, atol=1e-12)
    assert px["rays"] == 2 and px["flags"] & 4


def test_camera_rows_and_background(O):
    """Top-row pixel centre elevation is atan(tan(30 deg) * (1 - 1/H)); misses
    return the background and cast exactly one ray."""
    w = _single_sphere_workload(width=33, height=33)
    # move the sphere out of view: all pixels miss
    w.scene.inst_xform[0, 3] = 100.0
    img = O.render(w)
    assert not (img["flags"] & 1).any()
    assert np.allclose(img["rgb"], [0.05, 0.05, 0.08], atol=1e-7)
    assert (img["rays"] == 1).all()
    # put a huge sphere so the top-centre pixel's ray meets it: compare hit point elevation
    w.scene.inst_xform[0, 3] = 0.0
    w.scene.inst_xform[0, [0, 5, 10]] = 9.5
    w.scene.aabbs[0] = [-1, -1, -1, 1, 1, 1]
    px = O.render(w, pixels=[16])[0]
    p = np.array([0, 0, -10.0]) + px["t"] * _unit([0, math.tan(math.radians(30)) * (1 - 1 / 33), 1])
    assert np.linalg.norm(p) == pytest.approx(9.5, abs=1e-9)


def test_shadow_any_hit_and_mirror_miss(O):
    """Light behind an occluder: the lit side pixel is shadowed iff the occluder
    lies between; a mirror bounce that escapes adds k_r * background."""
    w = _single_sphere_workload(light=(0, 0, -10), kr=0.3, max_depth=2)
    px = O.render(w, pixels=[16 * 33 + 16])[0]
    # mirror ray goes straight back to the camera side and escapes
    bg = np.array([0.05, 0.05, 0.08])
    direct = np.array([0.5, 0.25, 1.0]) * 1.1
    assert np.allclose(px["rgb"], 0.7 * direct + 0.3 * bg, atol=1e-7)
    assert px["rays"] == 3 and px["flags"] & 8 and not px["flags"] & 16
    # add an occluding sphere between pole and light: the pixel is occluded
    b = scenes.SceneBuilder()
    scenes._standard_rays(b)
    hr, hs = b.add_hit_group(IS_SPHERE, scenes.CHS_LAMBERT), b.add_hit_group(IS_SPHERE)
    mat = b.add_material((0.5, 0.25, 1.0), 0.0)
    a0, p0 = scenes.shape_sphere((0, 0, 0), 1.0)
    a1, p1 = scenes.shape_sphere((0, 3, -3), 0.5)
    blas = b.add_blas([b.add_geometry([a0], [p0]), b.add_geometry([a1], [p1])])
    for _ in range(2):
        b.add_record(hr, mat, IS_SPHERE, 0)
        b.add_record(hs, mat, IS_SPHERE, 0)
    b.add_instance(blas, scenes.xform_trs((0, 0, 0)), 0)
    cam = scenes.Camera(np.float32([0, 0, -10]), np.float32([0, 0, 0]), np.float32([0, 1, 0]), 60.0)
    tp = scenes.TraceParams(33, 33, light_pos=np.float32([0, 6, -6]))
    px = O.render(scenes.Workload(b.build(), cam, tp), pixels=[16 * 33 + 16])[0]
    assert px["flags"] & 2 and not px["flags"] & 4
    assert np.allclose(px["rgb"], np.array([0.5, 0.25, 1.0]) * 0.1, atol=1e-12)


def test_mirror_hit_is_shaded_without_shadow(O):
    """Sphere A (k_r = 0.5) seen head-on with the light behind it: its front
    pole gets ambient only (n.l = -1, no shadow ray). The mirror ray returns
    along the axis, past the camera, to sphere B behind it; B's pole faces the
    light (n.l = 1) but A lies between them. The reflected hit is shaded
    without a shadow ray, so it is lit: rgb = 0.5 * 0.1 a_A + 0.5 * 1.1 a_B.
    A shadowed reflection would give 0.5 * 0.1 a_B instead."""
    a_A, a_B = np.array([0.5, 0.25, 1.0]), np.array([0.2, 0.9, 0.4])
    px = O.render(scenes.mirror_pair(), pixels=[16 * 33 + 16])[0]
    assert px["flags"] & 1 and not px["flags"] & 2       # hit, no shadow ray (n.l < 0)
    assert px["flags"] & 8 and px["flags"] & 16           # mirror ray cast and hit
    assert (px["refl_inst"], px["refl_geom"], px["refl_prim"]) == (0, 1, 0)
    assert px["refl_t"] == pytest.approx(18.0, abs=0.01)  # from the offset origin near z = -1 to z = -19
    assert px["rays"] == 2
    assert np.allclose(px["rgb"], 0.5 * 0.1 * a_A + 0.5 * 1.1 * a_B, atol=1e-12)


def test_tie_keeps_lower_instance(O):
    """Two instances of the same sphere at the same place: exact tie in t, the
    lower (instance, geometry, primitive) key wins."""
    w = _single_sphere_workload()
    s = w.scene
    for name in ("inst_xform", "inst_blas", "inst_id", "inst_sbt_offset", "inst_mask"):
        a = getattr(s, name)
        setattr(s, name, np.concatenate([a, a]))
    img = O.render(w)
    hit = (img["flags"] & 1) != 0
    assert hit.sum() > 20 and (img["inst"][hit] == 0).all()


def test_instance_mask_zero_skips(O):
    w = _single_sphere_workload()
    w.scene.inst_mask[:] = 0
    img = O.render(w)
    assert not (img["flags"] & 1).any()


# --------------------------------------------------------------------------
# Eq. 1 shader-table indexing: worked example and Listing 10 layout
# --------------------------------------------------------------------------
def _eq1_scene(fix):
    """Procedural stand-in of the Fig. 3 example. Each record gets its own
    material (albedo encodes the record number); shadow records' hit groups
    have no intersection shader unless they are 'probe' records."""
    b = scenes.SceneBuilder(sbt_stride_m=fix["m"])
    scenes._standard_rays(b)
    hr = b.add_hit_group(IS_BOX, scenes.CHS_LAMBERT)
    hs = b.add_hit_group(IS_BOX)
    nrec = len(fix["table"])
    for k in range(nrec):
        mat = b.add_material((0.01 * (k + 1), 0.5, 0.5), 0.0)
        b.add_record(hr if k % 2 == 0 else hs, mat, IS_BOX, k)
    # "triangle" BLAS: two slab-like boxes (g = 0 left, g = 1 right); procedural BLAS: one box
    aL, pL = scenes.shape_box((-3, 0, 0), (0.8, 0.8, 0.8))
    aR, pR = scenes.shape_box((-1, 0, 0), (0.8, 0.8, 0.8))
    aP, pP = scenes.shape_box((0, 0, 0), (0.8, 0.8, 0.8))
    tri = b.add_blas([b.add_geometry([aL], [pL]), b.add_geometry([aR], [pR])])
    proc = b.add_blas([b.add_geometry([aP], [pP])])
    xs = {"T": 0.0, "P0": 1.0, "P1": 3.0}
    for inst in fix["instances"]:
        blas = tri if inst["blas"] == "triangle" else proc
        b.add_instance(blas, scenes.xform_trs((xs[inst["label"]], 0, 0)), inst["sbt_offset"])
    return b


def test_eq1_worked_example_fig3(O):
    fix = json.load(open(os.path.join(GOLDEN, "eq1_fig3.json")))
    b = _eq1_scene(fix)
    scene = b.build("fig3")
    # orthographic-like probing: one camera looking down -z from far away at each geometry centre
    centres = {(0, 0): -3.0, (0, 1): -1.0, (1, 0): 1.0, (2, 0): 3.0}
    for e in fix["expected"]:
        if e["r"] != 0:
            continue
        x = centres[(e["instance"], e["g"])]
        cam = scenes.Camera(np.float32([x, 0, -50]), np.float32([x, 0, 0]), np.float32([0, 1, 0]), 1.0)
        tp = scenes.TraceParams(3, 3, light_pos=np.float32([x, 0, 50]))   # light behind: ambient only
        px = O.render(scenes.Workload(scene, cam, tp), pixels=[4])[0]
        assert px["flags"] & 1 and px["inst"] == e["instance"] and px["geom"] == e["g"]
        rec = int(round(px["rgb"][0] / 0.1 / 0.01)) - 1
        assert rec == e["record"], (e, rec)
    # shadow records (r = 1): give exactly one shadow record a working intersection shader
    for e in fix["expected"]:
        if e["r"] != 1:
            continue
        b2 = _eq1_scene(fix)
        probe = b2.add_hit_group(IS_BOX)
        none = b2.add_hit_group(scenes.NONE)
        for k in range(len(b2.sbt)):
            if k % 2 == 1:
                h, m, pt, ii = b2.sbt[k]
                b2.sbt[k] = (probe if k == e["record"] else none, m, pt, ii)
        # receiver: a big floor box instance using its own records, lit from above through the probe geometry
        b2.hit_groups.append((IS_BOX, scenes.CHS_LAMBERT, scenes.NONE))
        floor_hg = len(b2.hit_groups) - 1
        fmat = b2.add_material((0.5, 0.5, 0.5), 0.0)
        off = len(b2.sbt)
        b2.add_record(floor_hg, fmat, IS_BOX, 99)
        b2.add_record(none, fmat, IS_BOX, 99)
        fa, fp = scenes.shape_box((0, 0, 0), (10, 0.01, 10))
        fb = b2.add_blas([b2.add_geometry([fa], [fp])])
        b2.add_instance(fb, scenes.xform_trs((0, -5, 0)), off)
        scene2 = b2.build()
        x = centres[(e["instance"], e["g"])]
        for xx, expect_lit in [(x, False)] + [(xo, True) for xo in centres.values() if xo != x]:
            cam = scenes.Camera(np.float32([xx, -4.0, -20]), np.float32([xx, -4.99, 0]), np.float32([0, 1, 0]), 1.0)
            tp = scenes.TraceParams(3, 3, light_pos=np.float32([xx, 40, 0]))
            px = O.render(scenes.Workload(scene2, cam, tp), pixels=[4])[0]
            assert px["inst"] == 3 and px["flags"] & 2
            assert bool(px["flags"] & 4) == expect_lit, (e, xx)


def test_listing10_layout(O):
    """Build the sample's table with the procedural part of Listing 10 (geometry
    order Julia, Pacman, Mandelbulb; two pac-men); each instance must reach the
    record carrying its running instanceIndex and its geometry's material."""
    fix = json.load(open(os.path.join(GOLDEN, "listing10_layout.json")))
    b = scenes.SceneBuilder(sbt_stride_m=2)
    scenes._standard_rays(b)
    # record 0/1: the plane ("Triangle") stand-in
    plane_r = b.add_hit_group(IS_BOX, scenes.CHS_LAMBERT)
    plane_s = b.add_hit_group(IS_BOX)
    pm = b.add_material((0.9, 0.9, 0.9), 0.0)
    b.add_record(plane_r, pm, IS_BOX, 0)
    b.add_record(plane_s, pm, IS_BOX, 0)
    # all three procedural types drawn as unit spheres so the probe camera sees them alike
    kinds = {"Julia": 0, "Pacman": 1, "Mandelbulb": 2}
    hg = {k: (b.add_hit_group(IS_SPHERE, scenes.CHS_LAMBERT), b.add_hit_group(IS_SPHERE)) for k in kinds}
    mats = {k: b.add_material((0.02 * (v + 1), 0.3, 0.3), 0.0) for k, v in kinds.items()}
    instance_index = 0
    x = 0.0
    placed = []
    for geo in fix["geometries"]:
        a, p = scenes.shape_sphere((0, 0, 0), 0.5)
        blas = b.add_blas([b.add_geometry([a], [p])])
        for j in range(geo["instances"]):
            off = len(b.sbt)
            assert off == fix["instance_sbt_offset"][f"{geo['name']}#{j}"]
            rr, rs = hg[geo["name"]]
            b.add_record(rr, mats[geo["name"]], IS_SPHERE, instance_index)
            b.add_record(rs, mats[geo["name"]], IS_SPHERE, instance_index)
            b.add_instance(blas, scenes.xform_trs((x, 0, 0)), off)
            placed.append((geo["name"], instance_index, x))
            instance_index += 1
            x += 2.0
    scene = b.build("listing10")
    assert len(scene.sbt) == len(fix["records"])
    for k, rec in enumerate(fix["records"]):
        if rec["instance_index"] is not None:
            assert scene.sbt[k, 3] == rec["instance_index"]
            assert scene.sbt[k, 1] == mats[fix["geometries"][[g["name"] for g in fix["geometries"]].index(
                rec["hit_group"].replace("_Shadow", ""))]["name"]]
    for name, ii, xpos in placed:
        cam = scenes.Camera(np.float32([xpos, 0, -50]), np.float32([xpos, 0, 0]), np.float32([0, 1, 0]), 1.0)
        tp = scenes.TraceParams(3, 3, light_pos=np.float32([xpos, 0, 50]))
        px = O.render(scenes.Workload(scene, cam, tp), pixels=[4])[0]
        assert px["inst"] == ii
        assert int(round(px["rgb"][0] / 0.1 / 0.02)) - 1 == kinds[name]


def test_sbt_index_out_of_range_flags_and_misses(O):
    w = _single_sphere_workload()
    w.scene.inst_sbt_offset[:] = 7     # past the 2-record table
    img = O.render(w)
    assert (img["flags"] & 32).any() and not (img["flags"] & 1).any()


# --------------------------------------------------------------------------
# FP32 reference LBVH
# --------------------------------------------------------------------------
def test_morton_spread_known_values(O):
    # single boxes at the corners of the centroid bounds quantise to 0 / 1023 per axis
    boxes = np.array([[0, 0, 0, 0, 0, 0], [1, 0, 0, 1, 0, 0], [0, 1, 0, 0, 1, 0], [0, 0, 1, 0, 0, 1],
                      [1, 1, 1, 1, 1, 1]], np.float32)
    r = O.lbvh_f32(boxes)
    code_of = dict(zip(r["perm"].tolist(), r["codes"].tolist()))
    assert code_of[0] == 0
    assert code_of[1] == 0x24924924          # x bits at positions 3b+2
    assert code_of[2] == 0x12492492          # y at 3b+1
    assert code_of[3] == 0x09249249          # z at 3b
    assert code_of[4] == 0x3FFFFFFF


def _check_tree(r, boxes, keys):
    n = len(boxes)
    perm, child, cbox = r["perm"], r["child"], r["cbox"]
    assert sorted(perm.tolist()) == list(range(n))
    assert np.all(np.diff(keys[perm]) > 0)
    seen = np.zeros(n, int)

    def visit(node):
        """returns (first, last, box) of the subtree"""
        rng_, bx = [], []
        for side in (0, 1):
            ref = int(child[node, side])
            if ref < 0:
                leaf = ref & 0x7FFFFFFF
                seen[leaf] += 1
                rng_.append((leaf, leaf))
                b = boxes[perm[leaf]]
            else:
                f, l, b = visit(ref)
                rng_.append((f, l))
            assert np.array_equal(cbox[node, 6 * side:6 * side + 6], b)
            bx.append(b)
        (f0, l0), (f1, l1) = rng_
        assert l0 + 1 == f1
        assert node in (f0, l1)                  # internal node index is one end of its range
        # split at the highest differing bit: prefix of left range shared strictly more
        kf, kl, ks = keys[perm[f0]], keys[perm[l1]], keys[perm[l0]]
        common = 64 - int(kf ^ kl).bit_length()
        assert 64 - int(kf ^ ks).bit_length() > common
        assert 64 - int(kf ^ keys[perm[f1]]).bit_length() == common
        return f0, l1, np.concatenate([np.minimum(bx[0][:3], bx[1][:3]), np.maximum(bx[0][3:], bx[1][3:])])

    f, l, root = visit(0)
    assert (f, l) == (0, n - 1) and np.array_equal(root, r["root"])
    assert (seen == 1).all()


@pytest.mark.parametrize("n", [2, 3, 7, 64, 1000])
def test_lbvh_tree_is_the_radix_tree(O, n):
    rng = np.random.default_rng(n)
    lo = rng.uniform(-10, 10, (n, 3)).astype(np.float32)
    boxes = np.concatenate([lo, lo + rng.uniform(0, 2, (n, 3)).astype(np.float32)], 1)
    if n == 64:                                  # duplicate Morton codes
        boxes[32:] = boxes[:32]
    r = O.lbvh_f32(boxes)
    keys = (r["codes"].astype(np.uint64)[np.argsort(r["perm"])] << np.uint64(32)) | np.arange(n, dtype=np.uint64)
    _check_tree(r, boxes, keys)


def test_lbvh_single_leaf(O):
    box = np.array([[1, 2, 3, 4, 5, 6]], np.float32)
    r = O.lbvh_f32(box)
    assert r["perm"].tolist() == [0] and np.array_equal(r["root"], box[0])


def test_instance_boxes_f32_close_to_fp64_corners(O):
    w = scenes.field(seed=3, n_inst=500, width=8, height=8)
    b32 = O.instance_boxes_f32(w.scene).astype(np.float64)
    s = w.scene
    for k in range(len(s.inst_blas)):
        m = s.inst_xform[k].reshape(3, 4).astype(np.float64)
        a = s.aabbs[s.inst_blas[k]].astype(np.float64)
        corners = np.array([[a[0 + 3 * ((c >> j) & 1) + j] for j in range(3)] for c in range(8)])
        w_ = corners @ m[:, :3].T + m[:, 3]
        ref = np.concatenate([w_.min(0), w_.max(0)])
        assert np.allclose(b32[k], ref, rtol=0, atol=1e-5 * (1 + np.abs(ref).max()))
