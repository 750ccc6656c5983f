"""Pixel-wise comparison of the CUDA path with the FP64 oracle.

Tolerance (the stated contract): the discrete outcome of every ray a pixel
casts must agree on >= 99.9 % of pixels — primary hit or miss and its
(instance, geometry, primitive) id, whether the shadow ray found an occluder,
whether the mirror ray hit and what. On the pixels that agree, the primary hit
distance is within 1e-3 x scene diagonal, the shading normal within 1e-2 rad
and the radiance within 1e-3 (max norm).

Reading for fractals and any-hit shaders (the only exception): the surface
point and normal of a quaternion Julia set or a Mandelbulb are ill-conditioned
between FP32 and FP64 (a hit a few epsilons away has an unrelated normal, and a
mirror ray from it lands elsewhere on the fractal), and an any-hit shader's
band test is a discontinuous decision on the candidate point. A pixel whose
primary or mirror hit (on either side) is on such a primitive may therefore
exceed the continuous tolerances; it then counts as a disagreeing pixel, inside
the same 0.1 % budget. Every other agreeing pixel, including hits on the
sphere-traced exact SDFs (torus, rounded box, capsule, metaballs), must be
within tolerance.
"""
from __future__ import annotations

import numpy as np

F_HIT, F_SHADOW, F_LIT, F_REFL, F_REFL_HIT, F_SBT = 1, 2, 4, 8, 16, 32
NONE = 0xFFFFFFFF

T_REL = 1e-3
N_RAD = 1e-2
RGB_ABS = 1e-3
AGREE_MIN = 0.999

IS_JULIA, IS_MANDELBULB, IS_JULIA_CUT = 7, 8, 9
ILL_CONDITIONED_IS = (IS_JULIA, IS_MANDELBULB, IS_JULIA_CUT)

# (label, report) of every assert_parity call of this process, printed at the
# end of the test session
REPORTS = []


def ill_conditioned_hits(scene, inst: np.ndarray, geom: np.ndarray) -> np.ndarray:
    """True where (instance, geometry) is a radiance hit on a fractal primitive or
    on one whose hit group has an any-hit shader (Eq. 1 record with r = 0)."""
    inst = inst.astype(np.int64)
    geom = geom.astype(np.int64)
    hit = (inst >= 0) & (inst < len(scene.inst_sbt_offset)) & (geom >= 0)
    out = np.zeros(len(inst), bool)
    if not hit.any():
        return out
    rec = int(scene.sbt_stride_m) * geom[hit] + np.asarray(scene.inst_sbt_offset, np.int64)[inst[hit]]
    ok = rec < len(scene.sbt)
    hg = np.asarray(scene.sbt, np.int64)[np.where(ok, rec, 0), 0]
    groups = np.asarray(scene.hit_groups, np.int64)
    is_id, ahs = groups[hg, 0], groups[hg, 2]
    bad = ok & (np.isin(is_id, ILL_CONDITIONED_IS) | (ahs != NONE))
    out[np.nonzero(hit)[0]] = bad
    return out


def compare(ref: np.ndarray, aov: np.ndarray, rgb: np.ndarray, diag: float, scene=None) -> dict:
    """ref: oracle pixels; aov: AOV structured array; rgb: [N,3] float32 radiance.
    scene: the description, to find the pixels of the fractal / any-hit reading
    (without it every pixel is held to the strict form)."""
    ref = ref.reshape(-1)
    aov = aov.reshape(-1)
    rgb = rgb.reshape(-1, 3).astype(np.float64)
    n = len(ref)
    as_u = lambda a: np.where(a.astype(np.int64) < 0, NONE, a.astype(np.int64))
    g_flags = aov["flags"].astype(np.int64)
    r_flags = ref["flags"].astype(np.int64)
    mask = F_HIT | F_SHADOW | F_LIT | F_REFL | F_REFL_HIT
    flags_eq = (g_flags & mask) == (r_flags & mask)
    g = lambda k: aov[k].astype(np.int64)
    ids_eq = (g("inst") == as_u(ref["inst"])) & (g("geom") == as_u(ref["geom"])) & (g("prim") == as_u(ref["prim"]))
    rids_eq = ((g("refl_inst") == as_u(ref["refl_inst"])) & (g("refl_geom") == as_u(ref["refl_geom"])) &
               (g("refl_prim") == as_u(ref["refl_prim"])))
    primary_eq = ((g_flags & F_HIT) == (r_flags & F_HIT)) & ids_eq
    agree = flags_eq & ids_eq & rids_eq
    hit = agree & ((r_flags & F_HIT) != 0)
    dt = np.abs(aov["t"].astype(np.float64) - ref["t"])
    cosang = np.clip(np.sum(aov["n"].astype(np.float64) * ref["n"], axis=1), -1.0, 1.0)
    ang = np.arccos(cosang)
    drgb = np.max(np.abs(rgb - ref["rgb"]), axis=1)
    t_bad = hit & (dt > T_REL * diag)
    n_bad = hit & (ang > N_RAD)
    rgb_bad = agree & (drgb > RGB_ABS)
    out_of_tol = t_bad | n_bad | rgb_bad
    ill = np.zeros(n, bool)
    if scene is not None:
        signed = lambda a: np.where(a.astype(np.int64) == NONE, -1, a.astype(np.int64))
        ill = (ill_conditioned_hits(scene, ref["inst"], ref["geom"]) |
               ill_conditioned_hits(scene, signed(aov["inst"]), signed(aov["geom"])) |
               ill_conditioned_hits(scene, ref["refl_inst"], ref["refl_geom"]) |
               ill_conditioned_hits(scene, signed(aov["refl_inst"]), signed(aov["refl_geom"])))
    strict_bad = agree & ~ill & out_of_tol
    budget_bad = ~agree | (agree & ill & out_of_tol)
    ok = agree & ~out_of_tol
    strict_hit = hit & ~ill
    return dict(
        n=n,
        agree_within_tol=float(ok.mean()) if n else 1.0,
        primary_agree=float(primary_eq.mean()) if n else 1.0,
        agree=float(agree.mean()) if n else 1.0,
        n_disagree=int((~agree).sum()),
        t_bad=int(t_bad.sum()), n_bad=int(n_bad.sum()), rgb_bad=int(rgb_bad.sum()),
        n_ill=int(ill.sum()), strict_bad=int(strict_bad.sum()), budget_bad=int(budget_bad.sum()),
        max_dt=float(dt[hit].max()) if hit.any() else 0.0,
        max_ang=float(ang[hit].max()) if hit.any() else 0.0,
        max_drgb=float(drgb[agree].max()) if agree.any() else 0.0,
        strict_max_dt_rel=float(dt[strict_hit].max() / diag) if strict_hit.any() else 0.0,
        strict_max_ang=float(ang[strict_hit].max()) if strict_hit.any() else 0.0,
        strict_max_drgb=float(drgb[agree & ~ill].max()) if (agree & ~ill).any() else 0.0,
        hits=int(hit.sum()), sbt_err_ref=int(((r_flags & F_SBT) != 0).sum()),
        sbt_err_gpu=int(((g_flags & F_SBT) != 0).sum()),
        rays_ref=int(ref["rays"].sum()),
    )


def assert_parity(rep: dict, label: str = ""):
    """>= 99.9 % of pixels agree on every ray's discrete outcome; every agreeing
    pixel outside the fractal / any-hit reading is within tolerance; pixels that
    disagree plus out-of-tolerance pixels of that reading stay within 0.1 %."""
    REPORTS.append((label, rep))
    msg = f"{label}: {rep}"
    assert rep["primary_agree"] >= AGREE_MIN, msg
    assert rep["agree"] >= AGREE_MIN, msg
    assert rep["strict_bad"] == 0, msg
    assert rep["budget_bad"] <= (1.0 - AGREE_MIN) * rep["n"] + 1e-9, msg


def merge_reports(reps) -> dict:
    """One report over several comparisons (e.g. the sampled pixels of many requests)."""
    n = sum(r["n"] for r in reps)
    out = {"n": n}
    for k in ("n_disagree", "t_bad", "n_bad", "rgb_bad", "n_ill", "strict_bad", "budget_bad", "hits", "sbt_err_ref",
              "sbt_err_gpu", "rays_ref"):
        out[k] = sum(r[k] for r in reps)
    for k in ("agree_within_tol", "primary_agree", "agree"):
        out[k] = sum(r[k] * r["n"] for r in reps) / n if n else 1.0
    for k in ("max_dt", "max_ang", "max_drgb", "strict_max_dt_rel", "strict_max_ang", "strict_max_drgb"):
        out[k] = max((r[k] for r in reps), default=0.0)
    return out


def summary_line(label: str, rep: dict) -> str:
    return (f"{label}: n={rep['n']} disagree={rep['n_disagree']} fractal/any-hit px={rep['n_ill']} "
            f"t_bad={rep['t_bad']} n_bad={rep['n_bad']} rgb_bad={rep['rgb_bad']} strict_bad={rep['strict_bad']} "
            f"budget_used={rep['budget_bad']}/{rep['n']} strict max |dt|/diag={rep['strict_max_dt_rel']:.2e} "
            f"angle={rep['strict_max_ang']:.2e} rad |drgb|={rep['strict_max_drgb']:.2e}")


def gpu_rays_from_flags(aov: np.ndarray) -> np.ndarray:
    f = aov["flags"].astype(np.int64)
    return 1 + ((f & F_SHADOW) != 0) + ((f & F_REFL) != 0)
