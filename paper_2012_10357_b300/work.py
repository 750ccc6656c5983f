"""Algorithmic FP32 work per unit, counted from the kernel source formulas.

Three kinds of operation are counted separately, by the pipe that executes
them on the SM:
  FMA pipe  FFMA counts 2 FLOPs, FADD and FMUL 1 (the roofline's FLOPs; its
            peak is SMs x 128 lanes x 2 x clock);
  ALU pipe  min / max (a three-input min or max is one), compares and
            selects on FP32 values;
  special   reciprocal, square root, reciprocal square root, logarithm,
            sine / cosine, division (one each; their FMA fix-ups inside the
            IEEE division and square root are not counted).
Integer index arithmetic, loads and control flow are not counted. The
instrumented trace kernel (pr_trace_work) reports how many times each unit
ran; multiplied with these figures it gives the work of one launch, and over
the timed kernel's duration the achieved rates.

Per-unit counts (trace.cu / tracer.cuh / shaders.cuh):
  rays        ray set-up: 1/d (3 special + 3 FMUL), -o/d (3 FMUL), and the
              average generation of a primary / shadow / mirror ray
              (normalisations, light direction, offsets)
  BVH2 node   two slab tests: 12 FFMA; 20 min/max + 3 compares
  4-wide node four slab tests: 24 FFMA; 16 min/max (entry and exit planes
              picked by the sign of d, so only the three-plane max / min
              and the clip to [tmin, t]) + 12 compares/selects + 5-exchange
              sort (15)
  8-wide node float nodes: eight slab tests, 48 FFMA; 80 min/max + 24
              compares/selects + 19-exchange sort (57). Quantised nodes:
              per node 3 FMUL + 3 FFMA (step / d, (origin - o) / d) and 12
              word selects (entry / exit bounds by the sign of d); per child
              6 byte-to-float decodes (byte permute + FADD) and 6 FFMA, 4
              min/max + 3 compares/selects; the sort (57)
  instance    world->object origin (9 FFMA) and direction (6 FFMA + 3 FMUL),
              1/d, -o/d, BLAS root-box slab test (6 FFMA, 10 min/max)
  leaf        primitive AABB slab test: 6 FFMA, 11 min/max/compare
  sphere IS   closest approach, squared half chord, root choice
  box IS      per axis 1/d, two plane distances, entry / exit bookkeeping
  pac-man IS  sphere chord, two wedge planes, sincos, event ordering
  DE eval     estimate at one point plus the march step around it
              (point o + t d: 3 FFMA; scale, hit test, advance); fractal
              estimates count their set-up and escape tail here and their
              iterations below
  iteration   one Julia (q^2 + c, |q'|^2, |q|^2) or Mandelbulb (trig-free z^8,
              dr) iteration
  shaded      surface reconstruction: record, object-space point, analytic
              normal, world normal through the inverse transpose, light
              direction, Lambert
The normal stencil's six estimates per sphere-traced hit are counted as DE
evaluations, i.e. with a march step's 4 FFMA that a stencil point does not
need (an over-count of at most 8 FLOPs per stencil estimate).
"""
from __future__ import annotations

# (FMA-pipe FLOPs, ALU ops, special ops) per unit
UNITS = {
    "rays": (34, 6, 4),
    "tlas_nodes": (24, 23, 0),
    "tlas_nodes4": (48, 43, 0),
    "tlas_nodes8": (96, 161, 0),
    "tlas_nodes8q": (153, 173, 0),
    "blas_nodes": (24, 23, 0),
    "instances": (51, 17, 3),
    "leaves": (12, 11, 0),
    "sbt_lookups": (0, 0, 0),      # Eq. 1 index arithmetic is integer
    "is_calls_0": (30, 3, 2),      # sphere
    "is_calls_1": (18, 31, 3),     # box / slab
    "is_calls_2": (48, 20, 6),     # pac-man
    "is_calls_3": (5, 0, 1),       # sphere-traced shaders: 1/|d| before the march
    "is_calls_4": (5, 0, 1),
    "is_calls_5": (5, 0, 1),
    "is_calls_6": (5, 0, 1),
    "is_calls_7": (5, 0, 1),
    "is_calls_8": (5, 0, 1),
    "is_calls_9": (5, 0, 1),
    "de_evals_3": (18, 6, 2),      # torus
    "de_evals_4": (22, 10, 1),     # rounded box
    "de_evals_5": (16, 6, 1),      # capsule
    "de_evals_6": (66, 16, 7),     # four balls + three polynomial smooth minima
    "de_evals_7": (18, 4, 3),      # Julia set-up + escape tail
    "de_evals_8": (12, 4, 3),      # Mandelbulb escape tail
    "de_evals_9": (24, 5, 3),      # cut Julia: Julia + plane distance
    "julia_iters": (24, 1, 0),
    "mandelbulb_iters": (52, 6, 3),
    "shaded": (112, 10, 5),
}


def _total(counters: dict, k: int) -> float:
    return float(sum(UNITS[name][k] * v for name, v in counters.items() if name in UNITS))


def frame_fma_flops(counters: dict) -> float:
    """FMA-pipe FLOPs of one launch (FFMA = 2, FADD / FMUL = 1)."""
    return _total(counters, 0)


def frame_alu_ops(counters: dict) -> float:
    """ALU-pipe FP32 operations (min / max, compares, selects) of one launch."""
    return _total(counters, 1)


def frame_special_ops(counters: dict) -> float:
    """Special-function operations (rcp, sqrt, rsqrt, log, sincos, div) of one launch."""
    return _total(counters, 2)


# the roofline's FLOPs are the FMA pipe's
frame_flops = frame_fma_flops


def fp32_peak_tflops(n_sm: int, sm_mhz: float) -> float:
    """SMs x 128 FP32 lanes x 2 FLOP (FMA) x clock."""
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
