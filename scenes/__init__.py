"""Seeded synthetic scene generators (shared input for the renderer and the oracle).

This module only draws and lays out input arrays: AABBs, primitive parameters,
instance transforms, hit groups, materials, shader-table records, cameras and
trace parameters. It holds none of the rendering arithmetic (no intersection,
traversal, shading or BVH code), so both the CUDA path and the CPU oracle can
consume the same scenes without sharing any of the method's code.

Scene vocabulary follows the paper's entity model (Section 3.1.1, 3.1.5,
Listings 2-10): procedural geometries made of AABBs, one BLAS per geometry set,
instances of BLASes in one TLAS, hit groups {intersection, closest-hit,
any-hit}, and shader-table records reached with the indexing rule of Eq. 1,
``record = r + m*g + i``.

The paper's own scenes are not released (the shaders and scene files live in a
separate chapter and repository), so the configurations below are synthetic
stand-ins shaped like the paper's teaser and sample scene (two pac-men, a
quaternion Julia set, a Mandelbulb, a ground plane) and an instanced field of
the same primitive types.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# --------------------------------------------------------------------------
# Shader ids. These numbers are part of the scene input format: hit groups
# name built-in device shaders by id, like DXR hit groups name exports.
# --------------------------------------------------------------------------
IS_SPHERE = 0
IS_BOX = 1
IS_PACMAN = 2
IS_TORUS = 3
IS_ROUNDBOX = 4
IS_CAPSULE = 5
IS_METABALL4 = 6
IS_JULIA = 7
IS_MANDELBULB = 8
IS_JULIA_CUT = 9
N_IS = 10
SPHERE_TRACED = (IS_TORUS, IS_ROUNDBOX, IS_CAPSULE, IS_METABALL4, IS_JULIA, IS_MANDELBULB, IS_JULIA_CUT)

CHS_LAMBERT = 0
AHS_CUTOUT = 0
GEOM_AABBS = 0
GEOM_TRIANGLES = 1
MISS_BACKGROUND = 0
MISS_SHADOW = 1
NONE = 0xFFFFFFFF

RAY_TERMINATE_ON_FIRST_HIT = 1
RAY_SKIP_CLOSEST_HIT = 2

RAY_RADIANCE = 0
RAY_SHADOW = 1

N_PARAMS = 16  # floats of shape parameters per AABB primitive

IS_NAMES = ["sphere", "box", "pacman", "torus", "roundbox", "capsule",
            "metaball4", "julia", "mandelbulb", "julia_cut"]


@dataclasses.dataclass
class SceneDesc:
    """Flat arrays describing one scene (all host, little-endian).

    aabbs            float32 [P,6]   object-space lo.xyz, hi.xyz of every AABB primitive
    params           float32 [P,16]  shape parameters of every primitive
    geom_prim_begin  uint32  [G]     first primitive of each geometry
    geom_prim_count  uint32  [G]
    blas_geom_begin  uint32  [B]     first geometry of each BLAS (g = index inside the BLAS)
    blas_geom_count  uint32  [B]
    inst_xform       float32 [I,12]  object->world, row-major 3x4
    inst_blas        uint32  [I]
    inst_id          uint32  [I]     user instance id (DXR InstanceID)
    inst_sbt_offset  uint32  [I]     Eq. 1 instance contribution i, in records
    inst_mask        uint32  [I]     8-bit instance mask
    hit_groups       uint32  [H,3]   is_id, chs_id, ahs_id (NONE = absent)
    materials        float32 [M,4]   albedo rgb, mirror reflectance
    sbt              uint32  [R,4]   hit_group, material, prim_type, instance_index
    ray_types        uint32  [T,2]   miss_id, flags
    sbt_stride_m     int             Eq. 1 geometry multiplier m
    geom_type        uint32  [G]     GEOM_AABBS or GEOM_TRIANGLES (None: all AABBs); a triangle
                                     geometry's prim range indexes `indices`
    vertices         float32 [V,3]   triangle vertices (object space)
    indices          uint32  [T,3]   triangle vertex indices
    """
    aabbs: np.ndarray
    params: np.ndarray
    geom_prim_begin: np.ndarray
    geom_prim_count: np.ndarray
    blas_geom_begin: np.ndarray
    blas_geom_count: np.ndarray
    inst_xform: np.ndarray
    inst_blas: np.ndarray
    inst_id: np.ndarray
    inst_sbt_offset: np.ndarray
    inst_mask: np.ndarray
    hit_groups: np.ndarray
    materials: np.ndarray
    sbt: np.ndarray
    ray_types: np.ndarray
    sbt_stride_m: int = 2
    name: str = ""
    geom_type: Optional[np.ndarray] = None       # uint32 [G]: 0 AABBs, 1 triangles (None: all AABBs)
    vertices: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 3), np.float32))
    indices: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 3), np.uint32))

    def counts(self):
        return dict(prims=len(self.aabbs), geoms=len(self.geom_prim_begin),
                    blas=len(self.blas_geom_begin), inst=len(self.inst_blas),
                    hit_groups=len(self.hit_groups), materials=len(self.materials),
                    records=len(self.sbt), ray_types=len(self.ray_types))

    def nbytes(self) -> int:
        return int(sum(getattr(self, f.name).nbytes for f in dataclasses.fields(self)
                       if isinstance(getattr(self, f.name), np.ndarray)))


@dataclasses.dataclass
class Camera:
    """Pinhole camera: eye, look-at point, up vector, vertical field of view (degrees)."""
    eye: np.ndarray
    look_at: np.ndarray
    up: np.ndarray
    vfov_deg: float = 60.0


@dataclasses.dataclass
class TraceParams:
    """Frame parameters. eps_rel scales the scene diagonal into the world epsilon."""
    width: int
    height: int
    max_depth: int = 1          # 1: primary (+shadow); 2: plus one mirror bounce
    max_steps: int = 256        # sphere-tracing step cap
    light_pos: np.ndarray = dataclasses.field(default_factory=lambda: np.array([5, 8, -5], np.float32))
    light_intensity: float = 1.0
    eps_rel: float = 1e-4
    ambient: float = 0.1
    background: np.ndarray = dataclasses.field(default_factory=lambda: np.array([0.05, 0.05, 0.08], np.float32))


@dataclasses.dataclass
class Workload:
    scene: SceneDesc
    camera: Camera
    params: TraceParams
    name: str = ""


def _f32(x):
    return np.asarray(x, dtype=np.float32)


def _u32(x):
    return np.asarray(x, dtype=np.uint32)


def params_row(*vals) -> np.ndarray:
    row = np.zeros(N_PARAMS, np.float32)
    row[: len(vals)] = vals
    return row


def xform_trs(translation, rot3x3=None, scale=1.0) -> np.ndarray:
    """object->world 3x4 = [scale*R | t], row-major, float32."""
    r = np.eye(3) if rot3x3 is None else np.asarray(rot3x3, np.float64)
    m = np.zeros((3, 4), np.float64)
    m[:, :3] = r * scale
    m[:, 3] = translation
    return m.astype(np.float32).reshape(12)


def rot_y(deg: float) -> np.ndarray:
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], np.float64)


def quat_to_mat(q) -> np.ndarray:
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]], np.float64)


def random_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random unit quaternions (Shoemake 1992, 'Uniform random rotations')."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    return np.stack([b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2),
                     a * np.cos(2 * np.pi * u2), b * np.sin(2 * np.pi * u3)], axis=1)


class SceneBuilder:
    """Incremental scene assembly in the paper's build order (Listing 1):
    ray types -> hit groups -> geometry -> instances -> shader-table entries."""

    def __init__(self, sbt_stride_m: int = 2):
        self.aabbs: List[np.ndarray] = []
        self.params: List[np.ndarray] = []
        self.geoms: List[tuple] = []
        self.blas: List[tuple] = []
        self.inst: List[tuple] = []
        self.hit_groups: List[tuple] = []
        self.materials: List[tuple] = []
        self.sbt: List[tuple] = []
        self.ray_types: List[tuple] = []
        self.m = sbt_stride_m

    def add_ray_type(self, miss_id, flags=0) -> int:
        self.ray_types.append((miss_id, flags))
        return len(self.ray_types) - 1

    def add_hit_group(self, is_id, chs_id=NONE, ahs_id=NONE) -> int:
        self.hit_groups.append((is_id, chs_id, ahs_id))
        return len(self.hit_groups) - 1

    def add_material(self, albedo, reflectance=0.0) -> int:
        self.materials.append((*albedo, reflectance))
        return len(self.materials) - 1

    def add_geometry(self, aabbs, params) -> int:
        """A procedural geometry: a list of AABBs with one parameter row each."""
        begin = sum(len(a) for a in self.aabbs)
        aabbs = np.asarray(aabbs, np.float32).reshape(-1, 6)
        params = np.asarray(params, np.float32).reshape(-1, N_PARAMS)
        assert len(aabbs) == len(params)
        self.aabbs.append(aabbs)
        self.params.append(params)
        self.geoms.append((begin, len(aabbs), GEOM_AABBS))
        return len(self.geoms) - 1

    def add_triangle_geometry(self, vertices, indices) -> int:
        """A triangle geometry (built-in triangle intersection): vertices [V,3], indices [T,3]."""
        if not hasattr(self, "tris"):
            self.verts, self.tris = [], []
        vbase = sum(len(v) for v in self.verts)
        tbegin = sum(len(t) for t in self.tris)
        self.verts.append(np.asarray(vertices, np.float32).reshape(-1, 3))
        self.tris.append(np.asarray(indices, np.uint32).reshape(-1, 3) + np.uint32(vbase))
        self.geoms.append((tbegin, len(self.tris[-1]), GEOM_TRIANGLES))
        return len(self.geoms) - 1

    def add_blas(self, geom_ids) -> int:
        """A BLAS over consecutive geometries; g is the position inside the BLAS."""
        geom_ids = list(geom_ids)
        assert geom_ids == list(range(geom_ids[0], geom_ids[0] + len(geom_ids)))
        self.blas.append((geom_ids[0], len(geom_ids)))
        return len(self.blas) - 1

    def add_instance(self, blas, xform12, sbt_offset, inst_id=None, mask=0xFF) -> int:
        if inst_id is None:
            inst_id = len(self.inst)
        self.inst.append((np.asarray(xform12, np.float32), blas, inst_id, sbt_offset, mask))
        return len(self.inst) - 1

    def add_record(self, hit_group, material, prim_type, instance_index) -> int:
        self.sbt.append((hit_group, material, prim_type, instance_index))
        return len(self.sbt) - 1

    def build(self, name="") -> SceneDesc:
        G = len(self.geoms)
        return SceneDesc(
            aabbs=np.concatenate(self.aabbs).astype(np.float32) if self.aabbs else np.zeros((0, 6), np.float32),
            params=np.concatenate(self.params).astype(np.float32) if self.params else np.zeros((0, N_PARAMS), np.float32),
            geom_prim_begin=_u32([g[0] for g in self.geoms]).reshape(G),
            geom_prim_count=_u32([g[1] for g in self.geoms]).reshape(G),
            blas_geom_begin=_u32([b[0] for b in self.blas]).reshape(-1),
            blas_geom_count=_u32([b[1] for b in self.blas]).reshape(-1),
            inst_xform=np.stack([i[0] for i in self.inst]).astype(np.float32) if self.inst else np.zeros((0, 12), np.float32),
            inst_blas=_u32([i[1] for i in self.inst]).reshape(-1),
            inst_id=_u32([i[2] for i in self.inst]).reshape(-1),
            inst_sbt_offset=_u32([i[3] for i in self.inst]).reshape(-1),
            inst_mask=_u32([i[4] for i in self.inst]).reshape(-1),
            hit_groups=_u32(self.hit_groups).reshape(-1, 3),
            materials=_f32(self.materials).reshape(-1, 4),
            sbt=_u32(self.sbt).reshape(-1, 4),
            ray_types=_u32(self.ray_types).reshape(-1, 2),
            sbt_stride_m=self.m, name=name,
            geom_type=(_u32([g[2] for g in self.geoms]).reshape(G)
                       if any(g[2] != GEOM_AABBS for g in self.geoms) else None),
            vertices=(np.concatenate(self.verts).astype(np.float32) if getattr(self, "verts", None)
                      else np.zeros((0, 3), np.float32)),
            indices=(np.concatenate(self.tris).astype(np.uint32) if getattr(self, "tris", None)
                     else np.zeros((0, 3), np.uint32)))


# --------------------------------------------------------------------------
# Object-space shapes of the procedural primitive types (unit-sized).
# --------------------------------------------------------------------------
PACMAN_HALF_ANGLE = math.radians(30.0)   # 60 degree mouth
METABALL_K = 0.2                          # polynomial smooth-min width


def shape_sphere(c=(0, 0, 0), r=1.0):
    c = np.asarray(c, np.float64)
    return np.concatenate([c - r, c + r]), params_row(*c, r)


def shape_box(c, h):
    c, h = np.asarray(c, np.float64), np.asarray(h, np.float64)
    return np.concatenate([c - h, c + h]), params_row(*c, *h)


def shape_pacman(r=1.0):
    return np.array([-r, -r, -r, r, r, r]), params_row(0, 0, 0, r, PACMAN_HALF_ANGLE)


def shape_torus(R=1.0, r=0.25):
    return np.array([-(R + r), -r, -(R + r), R + r, r, R + r]), params_row(R, r)


def shape_roundbox(b=0.6, rr=0.15):
    return np.array([-b, -b, -b, b, b, b]), params_row(b, b, b, rr)


def shape_capsule(h=0.6, r=0.3):
    return np.array([-r, -(h + r), -r, r, h + r, r]), params_row(h, r)


def shape_metaball4(rng: np.random.Generator):
    # four ball centres with |c| <= 0.5 and radii in [0.25, 0.4]; smooth-min bulges by <= k/4
    cs = []
    while len(cs) < 4:
        c = rng.uniform(-0.5, 0.5, 3)
        if np.linalg.norm(c) <= 0.5:
            cs.append(c)
    rs = rng.uniform(0.25, 0.4, 4)
    return np.array([-1.0, -1.0, -1.0, 1.0, 1.0, 1.0]), params_row(*np.concatenate(cs), *rs)


def julia_c(rng: np.random.Generator, radius=0.8) -> np.ndarray:
    """Julia constant drawn uniformly from the 4-ball |c| <= radius."""
    while True:
        c = rng.uniform(-radius, radius, 4)
        if np.linalg.norm(c) <= radius:
            return c


def shape_julia(c, iters=12, escape=4.0):
    return np.array([-1.6] * 3 + [1.6] * 3), params_row(*c, iters, escape)


def shape_julia_cut(c, normal, offset, iters=12, escape=4.0):
    """Julia set cut by the half-space normal.p <= offset (the paper's Fig. 5)."""
    n = np.asarray(normal, np.float64)
    n = n / np.linalg.norm(n)
    return np.array([-1.6] * 3 + [1.6] * 3), params_row(*c, iters, escape, *n, offset)


JULIA_CUT_C = (-0.2, 0.6, 0.2, 0.2)   # a connected set (|c| = 0.69), so the cut face is solid


def julia_cut_scene(seed: int = 0, normal=(0.0, 0.0, -1.0), offset=0.0, width=320, height=240,
                    max_steps=256, c=JULIA_CUT_C) -> Workload:
    """A quaternion Julia set cut by one plane (Fig. 5), on a ground slab, the
    camera facing the cut. c = None draws c from the seed like the teaser scene."""
    rng = np.random.default_rng(seed)
    b = SceneBuilder(sbt_stride_m=2)
    _standard_rays(b)
    c = julia_c(rng) if c is None else np.asarray(c, np.float64)
    hr, hs = b.add_hit_group(IS_JULIA_CUT, CHS_LAMBERT), b.add_hit_group(IS_JULIA_CUT)
    gr, gs = b.add_hit_group(IS_BOX, CHS_LAMBERT), b.add_hit_group(IS_BOX)
    mj = b.add_material((0.75, 0.35, 0.85), 0.0)
    mg = b.add_material((0.6, 0.6, 0.6), 0.0)
    aabb, prm = shape_julia_cut(c, normal, offset)
    bj = b.add_blas([b.add_geometry([aabb], [prm])])
    ag, pg = shape_box((0, -2.205, 0), (8, 0.005, 8))
    bg = b.add_blas([b.add_geometry([ag], [pg])])
    b.add_record(hr, mj, IS_JULIA_CUT, 0)
    b.add_record(hs, mj, IS_JULIA_CUT, 0)
    b.add_record(gr, mg, IS_BOX, 1)
    b.add_record(gs, mg, IS_BOX, 1)
    b.add_instance(bj, xform_trs((0, 0, 0), None, 1.3), 0)
    b.add_instance(bg, xform_trs((0, 0, 0)), 2)
    cam = Camera(_f32([0.5, 1.5, -5]), _f32([0, 0, 0]), _f32([0, 1, 0]), 60.0)
    tp = TraceParams(width, height, max_depth=1, max_steps=max_steps, light_pos=_f32([3, 6, -6]))
    return Workload(b.build("julia-cut"), cam, tp, "julia-cut")


def mirror_pair(width: int = 33, height: int = 33) -> Workload:
    """Two unit spheres on the view axis: A at the origin (albedo (0.5, 0.25, 1),
    k_r = 0.5) in front of the camera, B at z = -20 behind the camera (albedo
    (0.2, 0.9, 0.4)); the light at z = 5 behind A. The mirror ray of A's front
    pole returns along the axis to B's pole, which faces the light with A in
    between (a reflected hit that a shadow ray would find occluded)."""
    b = SceneBuilder()
    _standard_rays(b)
    hr, hs = b.add_hit_group(IS_SPHERE, CHS_LAMBERT), b.add_hit_group(IS_SPHERE)
    m_a, m_b = b.add_material((0.5, 0.25, 1.0), 0.5), b.add_material((0.2, 0.9, 0.4), 0.0)
    g0, p0 = shape_sphere((0, 0, 0), 1.0)
    g1, p1 = shape_sphere((0, 0, -20), 1.0)
    blas = b.add_blas([b.add_geometry([g0], [p0]), b.add_geometry([g1], [p1])])
    for mat in (m_a, m_b):
        b.add_record(hr, mat, IS_SPHERE, 0)
        b.add_record(hs, mat, IS_SPHERE, 0)
    b.add_instance(blas, xform_trs((0, 0, 0)), 0)
    cam = Camera(_f32([0, 0, -10]), _f32([0, 0, 0]), _f32([0, 1, 0]), 60.0)
    tp = TraceParams(width, height, max_depth=2, light_pos=_f32([0, 0, 5]))
    return Workload(b.build("mirror-pair"), cam, tp, "mirror_pair")


def cutout_scene(seed: int = 0, width=256, height=192, shadow_cutout: bool = True, kind: str = "analytic",
                 max_steps: int = 256) -> Workload:
    """Shapes whose hit groups carry the cutout any-hit shader (bands removed along
    object y), over a ground slab; with shadow_cutout the shadow hit groups carry it
    too, so shadows show the bands. kind: "analytic" (sphere, box, pac-man), "sdf"
    (torus, rounded box, capsule, metaballs: sphere-traced exact SDFs) or "fractal"
    (quaternion Julia, Mandelbulb)."""
    rng = np.random.default_rng(seed)
    b = SceneBuilder(sbt_stride_m=2)
    _standard_rays(b)
    gr, gs = b.add_hit_group(IS_BOX, CHS_LAMBERT), b.add_hit_group(IS_BOX)
    mg = b.add_material((0.6, 0.6, 0.6), 0.0)
    ag, pg = shape_box((0, -1.505, 0), (8, 0.005, 8))
    bg = b.add_blas([b.add_geometry([ag], [pg])])
    b.add_record(gr, mg, IS_BOX, 0)
    b.add_record(gs, mg, IS_BOX, 0)
    b.add_instance(bg, xform_trs((0, 0, 0)), 0)
    if kind == "analytic":
        shapes = [(IS_SPHERE, shape_sphere((0, 0, 0), 1.0), (0.9, 0.3, 0.2), (-2.2, 0.0, 0.5)),
                  (IS_BOX, shape_box((0, 0, 0), (0.8, 0.9, 0.7)), (0.3, 0.4, 0.9), (0.0, -0.2, 1.5)),
                  (IS_PACMAN, shape_pacman(1.0), (0.95, 0.85, 0.1), (2.2, 0.0, 0.5))]
    elif kind == "sdf":
        shapes = [(IS_TORUS, shape_torus(0.9, 0.35), (0.9, 0.3, 0.2), (-3.0, -0.3, 0.5)),
                  (IS_ROUNDBOX, shape_roundbox(0.7, 0.15), (0.3, 0.4, 0.9), (-1.0, -0.4, 1.5)),
                  (IS_CAPSULE, shape_capsule(0.6, 0.45), (0.95, 0.85, 0.1), (1.0, -0.3, 0.5)),
                  (IS_METABALL4, shape_metaball4(rng), (0.3, 0.85, 0.4), (3.0, -0.3, 1.0))]
    else:
        shapes = [(IS_JULIA, shape_julia(JULIA_CUT_C), (0.75, 0.35, 0.85), (-1.6, 0.0, 0.8)),
                  (IS_MANDELBULB, shape_mandelbulb(), (0.35, 0.65, 0.95), (1.6, -0.2, 0.8))]
    for is_id, (aabb, prm), alb, pos in shapes:
        hr = b.add_hit_group(is_id, CHS_LAMBERT, AHS_CUTOUT)
        hs = b.add_hit_group(is_id, NONE, AHS_CUTOUT if shadow_cutout else NONE)
        m = b.add_material(alb, 0.0)
        blas = b.add_blas([b.add_geometry([aabb], [prm])])
        off = len(b.sbt)
        b.add_record(hr, m, is_id, len(b.inst))
        b.add_record(hs, m, is_id, len(b.inst))
        b.add_instance(blas, xform_trs(pos, rot_y(rng.uniform(-40, 40))), off)
    eye = [0, 2.5, -6.5] if kind == "analytic" else [0, 2.5, -7.5]
    cam = Camera(_f32(eye), _f32([0, -0.2, 0.6]), _f32([0, 1, 0]), 60.0)
    tp = TraceParams(width, height, max_depth=1, light_pos=_f32([-3, 7, -4]), max_steps=max_steps)
    return Workload(b.build("cutout" if kind == "analytic" else f"cutout-{kind}"), cam, tp, "cutout")


def shape_mandelbulb(power=8, iters=12, bailout=2.0):
    return np.array([-1.25] * 3 + [1.25] * 3), params_row(power, iters, bailout)


def _standard_rays(b: SceneBuilder):
    rr = b.add_ray_type(MISS_BACKGROUND, 0)
    rs = b.add_ray_type(MISS_SHADOW, RAY_TERMINATE_ON_FIRST_HIT | RAY_SKIP_CLOSEST_HIT)
    assert (rr, rs) == (RAY_RADIANCE, RAY_SHADOW)


# --------------------------------------------------------------------------
# Tiny analytic scene (64x64): one BLAS with four geometries.
# --------------------------------------------------------------------------
def small_analytic(seed: int = 0, width: int = 64, height: int = 64) -> Workload:
    rng = np.random.default_rng(seed)
    b = SceneBuilder(sbt_stride_m=2)
    _standard_rays(b)
    hg_sph = b.add_hit_group(IS_SPHERE, CHS_LAMBERT)
    hg_sph_s = b.add_hit_group(IS_SPHERE)
    hg_box = b.add_hit_group(IS_BOX, CHS_LAMBERT)
    hg_box_s = b.add_hit_group(IS_BOX)
    c0, c1 = rng.uniform(-2, 2, 3), rng.uniform(-2, 2, 3)
    r0, r1 = rng.uniform(0.3, 1.0, 2)
    he = rng.uniform(0.3, 0.8, 3)
    shapes = [shape_sphere(c0, r0), shape_sphere(c1, r1),
              shape_box((0, -1, 0), he), shape_box((0, -2.505, 0), (10, 0.005, 10))]
    groups = [(hg_sph, hg_sph_s, IS_SPHERE), (hg_sph, hg_sph_s, IS_SPHERE),
              (hg_box, hg_box_s, IS_BOX), (hg_box, hg_box_s, IS_BOX)]
    albedos = [(0.9, 0.3, 0.2), (0.2, 0.8, 0.3), (0.3, 0.4, 0.9), (0.7, 0.7, 0.7)]
    gids = [b.add_geometry([a], [p]) for a, p in shapes]
    blas = b.add_blas(gids)
    b.add_instance(blas, xform_trs((0, 0, 0)), sbt_offset=0)
    for g, ((hr, hs, pt), alb) in enumerate(zip(groups, albedos)):
        mat = b.add_material(alb, 0.0)
        b.add_record(hr, mat, pt, 0)   # record r + 2g, r = 0
        b.add_record(hs, mat, pt, 0)   # r = 1
    scene = b.build("small_analytic")
    cam = Camera(_f32([0, 2, -8]), _f32([0, 0, 0]), _f32([0, 1, 0]), 60.0)
    tp = TraceParams(width, height, max_depth=1, light_pos=_f32([5, 8, -5]))
    return Workload(scene, cam, tp, "small_analytic")


def small_analytic_cameras(seed: int, n_frames: int, base: Optional[Camera] = None) -> List[Camera]:
    """Per-frame cameras of the 4096-frame throughput run: eye jittered by U[-0.5,0.5]^3."""
    rng = np.random.default_rng(seed + 7919)
    base = base or Camera(_f32([0, 2, -8]), _f32([0, 0, 0]), _f32([0, 1, 0]), 60.0)
    jit = rng.uniform(-0.5, 0.5, (n_frames, 3))
    return [Camera(_f32(base.eye + j), base.look_at, base.up, base.vfov_deg) for j in jit]


# --------------------------------------------------------------------------
# Teaser-like scene (1920x1080): each primitive its own BLAS + hit groups.
# Shader-table layout follows Listing 10: per geometry (insertion order), per
# instance: a radiance record then a shadow record; instance_index runs across
# procedural geometries.
# --------------------------------------------------------------------------
def teaser(seed: int = 0, width: int = 1920, height: int = 1080) -> Workload:
    rng = np.random.default_rng(seed)
    b = SceneBuilder(sbt_stride_m=2)
    _standard_rays(b)
    c = julia_c(rng)
    kinds = [
        # (shape, is_id, albedo, reflectance, instance transforms)
        (shape_pacman(1.0), IS_PACMAN, (0.95, 0.85, 0.1), 0.2,
         [xform_trs((-3, 0, 0), rot_y(0.0)), xform_trs((3, 0, 0), rot_y(180.0))]),
        (shape_julia(c), IS_JULIA, (0.75, 0.35, 0.85), 0.2, [xform_trs((0, 1.2, 3), None, 1.5)]),
        (shape_mandelbulb(), IS_MANDELBULB, (0.35, 0.65, 0.95), 0.2, [xform_trs((0, 0.5, -1), None, 1.2)]),
        (shape_box((0, -1.205, 0), (20, 0.005, 20)), IS_BOX, (0.6, 0.6, 0.6), 0.4, [xform_trs((0, 0, 0))]),
    ]
    instance_index = 0
    for (aabb, prm), is_id, alb, kr, xforms in kinds:
        hr = b.add_hit_group(is_id, CHS_LAMBERT)
        hs = b.add_hit_group(is_id)
        mat = b.add_material(alb, kr)
        blas = b.add_blas([b.add_geometry([aabb], [prm])])
        for xf in xforms:
            off = len(b.sbt)
            b.add_record(hr, mat, is_id, instance_index)
            b.add_record(hs, mat, is_id, instance_index)
            b.add_instance(blas, xf, sbt_offset=off)
            instance_index += 1
    scene = b.build("teaser")
    cam = Camera(_f32([0, 3, -10]), _f32([0, 0, 0]), _f32([0, 1, 0]), 60.0)
    tp = TraceParams(width, height, max_depth=2, light_pos=_f32([6, 10, -6]))
    return Workload(scene, cam, tp, "teaser")


def plane_mesh(half: float, y: float, cells: int):
    """A square grid of 2*cells^2 triangles at height y spanning [-half, half]^2 in x, z."""
    xs = np.linspace(-half, half, cells + 1)
    verts = np.array([[x, y, z] for z in xs for x in xs], np.float32)
    idx = []
    for j in range(cells):
        for i in range(cells):
            a, b = j * (cells + 1) + i, j * (cells + 1) + i + 1
            c, d = a + cells + 1, b + cells + 1
            idx += [(a, c, b), (b, c, d)]
    return verts, np.array(idx, np.uint32)


def sample_scene(seed: int = 0, width: int = 640, height: int = 360, cells: int = 8) -> Workload:
    """The paper's sample scene (Fig. 4): a triangle plane mesh and procedural
    objects (two pac-men, a Julia set, a Mandelbulb). Shader table as Listing 10:
    the triangle records first (radiance, shadow), then per procedural geometry in
    insertion order (Julia, Pacman, Mandelbulb; Listing 4) and per instance of it,
    a radiance and a shadow record, instance_index running over all procedural
    instances and the material indexed by the procedural geometry ordinal."""
    rng = np.random.default_rng(seed)
    b = SceneBuilder(sbt_stride_m=2)
    _standard_rays(b)
    tri_r = b.add_hit_group(NONE, CHS_LAMBERT)         # built-in triangle intersection
    tri_s = b.add_hit_group(NONE)
    plane_mat = b.add_material((0.6, 0.6, 0.6), 0.4)
    v, i = plane_mesh(20.0, -1.2, cells)
    plane_blas = b.add_blas([b.add_triangle_geometry(v, i)])
    b.add_record(tri_r, plane_mat, NONE, 0)
    b.add_record(tri_s, plane_mat, NONE, 0)
    b.add_instance(plane_blas, xform_trs((0, 0, 0)), 0)
    c = julia_c(rng)
    kinds = [("Julia", shape_julia(c), IS_JULIA, (0.75, 0.35, 0.85), [xform_trs((0, 1.2, 3), None, 1.5)]),
             ("Pacman", shape_pacman(1.0), IS_PACMAN, (0.95, 0.85, 0.1),
              [xform_trs((-3, 0, 0), rot_y(0.0)), xform_trs((3, 0, 0), rot_y(180.0))]),
             ("Mandelbulb", shape_mandelbulb(), IS_MANDELBULB, (0.35, 0.65, 0.95),
              [xform_trs((0, 0.5, -1), None, 1.2)])]
    instance_index = 0
    for name, (aabb, prm), is_id, alb, xforms in kinds:
        hr, hs = b.add_hit_group(is_id, CHS_LAMBERT), b.add_hit_group(is_id)
        mat = b.add_material(alb, 0.2)                  # materialCb[primitiveIndex]
        blas = b.add_blas([b.add_geometry([aabb], [prm])])
        for xf in xforms:
            off = len(b.sbt)
            b.add_record(hr, mat, is_id, instance_index)
            b.add_record(hs, mat, is_id, instance_index)
            b.add_instance(blas, xf, sbt_offset=off)
            instance_index += 1
    cam = Camera(_f32([0, 3, -10]), _f32([0, 0, 0]), _f32([0, 1, 0]), 60.0)
    tp = TraceParams(width, height, max_depth=2, light_pos=_f32([6, 10, -6]))
    return Workload(b.build("sample"), cam, tp, "sample")


# --------------------------------------------------------------------------
# Instanced field of 8 primitive types (100 000 instances at 3840x2160; the batch
# requests use the same mix at other sizes).
# --------------------------------------------------------------------------
FIELD_TYPES = [IS_SPHERE, IS_TORUS, IS_ROUNDBOX, IS_CAPSULE, IS_METABALL4, IS_PACMAN,
               IS_JULIA, IS_MANDELBULB]
FIELD_PROBS = [0.3, 0.2, 0.15, 0.1, 0.1, 0.1, 0.025, 0.025]
FIELD_ALBEDO = [(0.9, 0.3, 0.2), (0.2, 0.8, 0.3), (0.3, 0.4, 0.9), (0.9, 0.8, 0.2),
                (0.8, 0.4, 0.8), (0.95, 0.85, 0.1), (0.75, 0.35, 0.85), (0.35, 0.65, 0.95)]


def instanced_field(seed: int, n_inst: int, side: float, origin=(0.0, 0.0, 0.0), name="field") -> SceneDesc:
    """n_inst instances of the 8 BLAS types, positions uniform in a cube of the given
    side, uniform scale log-uniform in [0.1, 2], uniformly random rotations.
    sbt_offset = 2*type: one radiance and one shadow record per primitive type."""
    rng = np.random.default_rng(seed)
    b = SceneBuilder(sbt_stride_m=2)
    _standard_rays(b)
    shapes = {IS_SPHERE: shape_sphere(), IS_TORUS: shape_torus(), IS_ROUNDBOX: shape_roundbox(),
              IS_CAPSULE: shape_capsule(), IS_METABALL4: shape_metaball4(rng),
              IS_PACMAN: shape_pacman(), IS_JULIA: shape_julia(julia_c(rng)),
              IS_MANDELBULB: shape_mandelbulb()}
    blas_of = {}
    for t, is_id in enumerate(FIELD_TYPES):
        aabb, prm = shapes[is_id]
        blas_of[t] = b.add_blas([b.add_geometry([aabb], [prm])])
        hr = b.add_hit_group(is_id, CHS_LAMBERT)
        hs = b.add_hit_group(is_id)
        mat = b.add_material(FIELD_ALBEDO[t], 0.0)
        b.add_record(hr, mat, is_id, t)
        b.add_record(hs, mat, is_id, t)
    types = rng.choice(len(FIELD_TYPES), size=n_inst, p=FIELD_PROBS)
    pos = rng.uniform(0.0, side, (n_inst, 3)) + np.asarray(origin)
    scale = np.exp(rng.uniform(math.log(0.1), math.log(2.0), n_inst))
    quats = random_quats(rng, n_inst)
    w, x, y, z = quats.T
    rot = np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)
    xf = np.zeros((n_inst, 3, 4), np.float64)
    xf[:, :, :3] = rot * scale[:, None, None]
    xf[:, :, 3] = pos
    scene = b.build(name)
    scene.inst_xform = xf.reshape(n_inst, 12).astype(np.float32)
    scene.inst_blas = types.astype(np.uint32)
    scene.inst_id = np.arange(n_inst, dtype=np.uint32)
    scene.inst_sbt_offset = (2 * types).astype(np.uint32)
    scene.inst_mask = np.full(n_inst, 0xFF, np.uint32)
    return scene


def field(seed: int = 0, width: int = 3840, height: int = 2160, n_inst: int = 100_000) -> Workload:
    side = 100.0 * (n_inst / 100_000) ** (1.0 / 3.0)
    scene = instanced_field(seed, n_inst, side, name="field")
    s = side / 100.0
    cam = Camera(_f32([50 * s, 50 * s, -60 * s]), _f32([50 * s, 50 * s, 50 * s]), _f32([0, 1, 0]), 60.0)
    tp = TraceParams(width, height, max_depth=1, light_pos=_f32([50 * s, 200 * s, -100 * s]))
    return Workload(scene, cam, tp, "field")


def orbit_camera(rng: np.random.Generator, center, diag) -> Camera:
    """Orbit pose around the scene centre: radius 0.6*diag, azimuth U[0,2pi), elevation U[10,60] deg."""
    az = rng.uniform(0, 2 * math.pi)
    el = math.radians(rng.uniform(10, 60))
    r = 0.6 * diag
    center = np.asarray(center, np.float64)
    eye = center + r * np.array([math.cos(el) * math.cos(az), math.sin(el), math.cos(el) * math.sin(az)])
    return Camera(_f32(eye), _f32(center), _f32([0, 1, 0]), 60.0)


def batch_requests(seed: int = 0, n_requests: int = 64, res_choices=(256, 512, 1024, 2048)) -> List[Workload]:
    """64 render requests: resolution from {256^2..2048^2}, instanced-field scenes with
    n = floor(10^U[0,4]) instances in a cube of side 100*(n/1e5)^(1/3), orbit cameras."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n_requests):
        res = int(rng.choice(res_choices))
        n = int(math.floor(10 ** rng.uniform(0, 4)))
        side = 100.0 * (n / 100_000) ** (1.0 / 3.0)
        scene = instanced_field(seed * 1000 + q + 1, n, side, name=f"req{q}")
        center = np.full(3, side / 2)
        cam = orbit_camera(rng, center, math.sqrt(3) * side + 4.0)
        tp = TraceParams(res, res, max_depth=1,
                         light_pos=_f32(center + np.array([0.0, 2.0 * side + 4.0, -side - 2.0])))
        out.append(Workload(scene, cam, tp, f"req{q}"))
    return out


def serving_request(rng: np.random.Generator, scene_pool: int = 16, build=None):
    """One serving request: a teaser or an instanced-field scene (50/50), seed from a pool
    of 16 per kind (so scenes repeat and a BVH cache can hit), resolution
    t~U[0,1], W=round(512+1408t), H=round(512+568t), orbit camera around the
    scene. build(kind, seed) may return an already generated description."""
    kind = int(rng.integers(0, 2))
    sseed = int(rng.integers(0, scene_pool))
    t = rng.uniform()
    w, h = int(round(512 + 1408 * t)), int(round(512 + 568 * t))
    known = build(kind, sseed) if build else None
    if kind == 0:
        wl = teaser(sseed, w, h) if known is None else Workload(known, None, teaser(sseed, 8, 8).params)
        wl.params.width, wl.params.height = w, h
        wl.camera = orbit_camera(rng, (0.0, 0.5, 1.0), 12.0)
    else:
        if known is None:
            wl = field(sseed, w, h)
        else:
            wl = Workload(known, None, TraceParams(w, h, max_depth=1, light_pos=_f32([50, 200, -100])))
        wl.params.width, wl.params.height = w, h
        wl.camera = orbit_camera(rng, np.full(3, 50.0), math.sqrt(3) * 100.0)
    return kind, sseed, wl


def sample_pixels(width: int, height: int, n: int, seed: int = 1) -> np.ndarray:
    """Seeded sample of distinct linear pixel indices (y*width + x), sorted."""
    rng = np.random.default_rng(seed)
    n = min(n, width * height)
    return np.sort(rng.choice(width * height, size=n, replace=False)).astype(np.int64)
