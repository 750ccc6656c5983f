"""Planted mistakes: each pin of the oracle must catch the mistake it guards.

Every case copies oracle.cpp, makes one plausible error in it (a swapped
stencil axis, a dropped term, a flipped sign, a wrong tie rule), compiles the
copy into a temporary library and runs the pin that should fail on it. A pin
that still passes on the planted copy does not pin what it claims. CPU only.
"""
import contextlib
import hashlib
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import scenes
import test_oracle_pins as pins
import test_oracle_ploc as ploc_pins
from scenes import IS_CAPSULE, IS_METABALL4, IS_TORUS


def _build_variant(replacements) -> str:
    with open(oracle._SRC) as f:
        src = f.read()
    for old, new in replacements:
        assert src.count(old) == 1, f"planted edit does not match exactly once: {old!r}"
        src = src.replace(old, new)
    tag = hashlib.sha1(src.encode()).hexdigest()[:16]
    out_dir = os.path.join(tempfile.gettempdir(), "pr_oracle_variants")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, f"oracle_{tag}.so")
    if not os.path.exists(so):
        cpp = os.path.join(out_dir, f"oracle_{tag}.cpp")
        with open(cpp, "w") as f:
            f.write(src)
        subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                        "-pthread", "-I", os.path.dirname(oracle._SRC), "-o", so + ".tmp", cpp], check=True)
        os.replace(so + ".tmp", so)
    return so


@contextlib.contextmanager
def _oracle_from(path: str):
    saved = oracle.lib()
    oracle._lib = oracle.load(path)
    try:
        yield oracle
    finally:
        oracle._lib = saved


_STENCIL = ("V3 g{distance_estimate(id, prm, p + V3{hh, 0, 0}) - distance_estimate(id, prm, p - V3{hh, 0, 0}),\n"
            "           distance_estimate(id, prm, p + V3{0, hh, 0}) - distance_estimate(id, prm, p - V3{0, hh, 0}),")
_STENCIL_XY = ("V3 g{distance_estimate(id, prm, p + V3{0, hh, 0}) - distance_estimate(id, prm, p - V3{0, hh, 0}),\n"
               "           distance_estimate(id, prm, p + V3{hh, 0, 0}) - distance_estimate(id, prm, p - V3{hh, 0, 0}),")


def _normal_pin(is_id, prm, grad):
    return lambda O: pins.test_sphere_traced_normal_is_the_sdf_gradient(O, is_id, prm, grad)


_TORUS = _normal_pin(IS_TORUS, [1, 0.25], lambda p: pins._grad_torus(p, 1.0, 0.25))
_CAPSULE = _normal_pin(IS_CAPSULE, [0.6, 0.3], lambda p: pins._grad_capsule(p, 0.6, 0.3))
_MB = list(scenes.shape_metaball4(np.random.default_rng(5))[1])
_METABALLS = _normal_pin(IS_METABALL4, _MB, lambda p: pins._grad_metaball4(p, _MB))

# (name, edits to oracle.cpp, pin that must fail)
CASES = [
    ("normal stencil: x and y components swapped", [(_STENCIL, _STENCIL_XY)], _TORUS),
    ("normal stencil: y component taken along z",
     [("p + V3{0, hh, 0}) - distance_estimate(id, prm, p - V3{0, hh, 0})",
       "p + V3{0, 0, hh}) - distance_estimate(id, prm, p - V3{0, 0, hh})")], _CAPSULE),
    ("normal stencil: one-sided difference",
     [("p + V3{0, hh, 0}) - distance_estimate(id, prm, p - V3{0, hh, 0})",
       "p + V3{0, hh, 0}) - distance_estimate(id, prm, p)")], _CAPSULE),
    ("torus: ring radius added instead of subtracted",
     [("double qx = std::sqrt(p.x * p.x + p.z * p.z) - R;", "double qx = std::sqrt(p.x * p.x + p.z * p.z) + R;")],
     _TORUS),
    ("capsule: segment clamped on x", [("double y = std::min(std::max(p.y, -hh), hh);",
                                        "double y = std::min(std::max(p.x, -hh), hh);")], _CAPSULE),
    ("smooth minimum: blend weight linear instead of squared",
     [("return std::min(a, b) - hh * hh * k * 0.25;", "return std::min(a, b) - hh * k * 0.25;")], _METABALLS),
    ("Eq. 1: geometry term m*g dropped",
     [("(uint64_t)r + (uint64_t)s->sbt_stride_m * g + s->inst_sbt_offset[k]", "(uint64_t)r + s->inst_sbt_offset[k]")],
     pins.test_eq1_worked_example_fig3),
    ("Julia estimate: factor 1/2 dropped",
     [("return 0.5 * r * std::log(r) / md;", "return r * std::log(r) / md;")], pins.test_julia_c0_closed_form),
    ("Mandelbulb derivative: +1 dropped",
     [("dr = n * std::pow(r, n - 1.0) * dr + 1.0;", "dr = n * std::pow(r, n - 1.0) * dr;")],
     pins.test_mandelbulb_axis_reduces_to_real_iteration),
    ("pac-man: wedge-face normal sign flipped",
     [(": -nrm[ev[i].kind];", ": nrm[ev[i].kind];")], pins.test_pacman_reductions),
    ("box: edge tie resolved to the highest axis",
     [("if (tn > te) { te = tn; ea = k; }   // ties keep the lowest axis index",
       "if (tn >= te) { te = tn; ea = k; }")], pins.test_box_closed_form_and_random),
    ("instance boxes: min and max swapped",
     [("lo = lo + std::min(a, b);\n        hi = hi + std::max(a, b);",
       "lo = lo + std::max(a, b);\n        hi = hi + std::min(a, b);")], pins.test_instance_boxes_f32_close_to_fp64_corners),
    ("sphere-traced any-hit: an ignored candidate ends the march",
     [("      t += std::max(std::fabs(dist), eps);\n      continue;", "      return false;")],
     pins.test_sphere_traced_cutout_marches_through_the_solid),
    ("sphere-traced any-hit: the march goes on by the signed estimate",
     [("      t += std::max(std::fabs(dist), eps);\n      continue;", "      t += std::max(dist, eps);\n      continue;")],
     pins.test_sphere_traced_cutout_marches_through_the_solid),
    ("sphere-traced any-hit: the shader is not consulted",
     [("    if (dist < eps && !any_hit_accepts(ahs, p)) {", "    if (false) {")],
     pins.test_sphere_traced_cutout_on_level_rays),
    ("PLOC: area tie resolved to the odd lower index",
     [("(lo & 1) != (lob & 1) ? (lo & 1) == 0 : lo < lob", "(lo & 1) != (lob & 1) ? (lo & 1) == 1 : lo < lob")],
     ploc_pins.test_ploc_tie_goes_to_the_even_lower_pair),
    ("PLOC: distance tie rule dropped",
     [("take = d != db ? d < db : (lo & 1)", "take = (lo & 1)")],
     lambda O: ploc_pins.test_ploc_equal_boxes_give_a_balanced_tree(O, 16)),
    ("PLOC: volume of the union instead of its surface area",
     [("const float s = std::fma(dx, dy, std::fma(dy, dz, dz * dx));", "const float s = dx * dy * dz;")],
     ploc_pins.test_ploc_flat_boxes_merge_by_area),
    ("PLOC: children of a merge swapped",
     [("child_out[2 * node + 0] = C[i].ref;\n      child_out[2 * node + 1] = C[j].ref;",
       "child_out[2 * node + 0] = C[j].ref;\n      child_out[2 * node + 1] = C[i].ref;")],
     ploc_pins.test_ploc_boxes_on_a_line),
    ("PLOC: merged node takes the place of the upper cluster",
     [("      if (mutual && j < i) continue;   // merged into the node made at j\n      if (!mutual) {",
       "      if (mutual && j > i) continue;\n      if (!mutual) {")],
     ploc_pins.test_ploc_boxes_on_a_line),
]


@pytest.mark.parametrize("name,edits,pin", CASES, ids=[c[0] for c in CASES])
def test_pin_catches_planted_mistake(oracle_lib, name, edits, pin):
    pin(oracle_lib)                       # the pin passes on the oracle as it is
    with _oracle_from(_build_variant(edits)) as variant:
        with pytest.raises(AssertionError):
            pin(variant)
