"""Algorithmic FP32 work per unit, counted from the kernel source formulas.

Counting convention: an FMA is 2 FLOPs; add, multiply, min, max, compare and
each special-function instruction (sqrt, rsqrt, reciprocal, divide, log,
sincos) count 1. The instrumented trace kernel (pr_trace_work) reports how many
times each unit ran; multiplying gives the FLOPs one frame needs, which over
the timed kernel's duration gives the achieved FP32 rate for the roofline.
"""
from __future__ import annotations

# per unit, from trace.cu / shaders.cuh
FLOPS = {
    "tlas_nodes": 50,        # two slab tests (6 FMA + 10 min/max each), clip to [tmin,tmax], order
    "tlas_nodes4": 104,      # four slab tests with clip (24 FMA + 44 min/max), masks, 5-exchange sort
    "blas_nodes": 50,
    "instances": 64,         # world->object origin (9 FMA) and direction (6 FMA + 3 MUL), 1/d, root-box slab
    "leaves": 25,            # primitive AABB slab + clip
    "sbt_lookups": 2,        # Eq. 1: r + m*g + i and its bounds check (integer; counted as 2)
    "is_calls_0": 32,        # sphere: closest approach, squared half chord, sqrt, root selection
    "is_calls_1": 33,        # box: per-axis reciprocal, two plane distances, min/max, entry/exit choice
    "is_calls_2": 52,        # pac-man: sphere chord + two wedge planes + event ordering
    "de_evals_3": 10 + 8,    # torus SDF (+ 8 per estimate: ray point, scale, hit test, step)
    "de_evals_4": 23 + 8,    # rounded box SDF
    "de_evals_5": 10 + 8,    # capsule SDF
    "de_evals_6": 70 + 8,    # four balls + three polynomial smooth minima
    "de_evals_7": 10 + 8,    # Julia setup + escape tail (iterations counted below)
    "de_evals_8": 5 + 8,     # Mandelbulb escape tail (iterations counted below)
    "de_evals_9": 10 + 6 + 8,  # cut Julia: Julia setup/tail + plane distance (iterations counted below)
    "julia_iters": 27,       # q^2 + c, |q'|^2 update, |q|^2, escape test
    "mandelbulb_iters": 54,  # trig-free z^8 (two complex cubes of squarings), dr update, escape test
    "shaded": 150,           # surface reconstruction, world normal, two Lambert evaluations
    "rays": 60,              # ray generation / shadow or mirror ray setup, 1/d, TLAS entry
}


def frame_flops(counters: dict) -> float:
    return float(sum(FLOPS.get(k, 0) * v for k, v in counters.items()))


def fp32_peak_tflops(n_sm: int, sm_mhz: float) -> float:
    """SMs x 128 FP32 lanes x 2 FLOP (FMA) x clock."""
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
