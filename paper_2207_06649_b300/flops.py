"""Algorithmic floating-point operation counts of the rollout path.

The engine counts events per environment (pmbs_query_events); each event carries a fixed
cost, the average number of floating-point operations the plain double-precision
statement of the method (the FP64 oracle) spends on it.  The costs were measured with the
oracle's flop counter (its build with a counting scalar type: add, subtract, multiply,
divide and square root count 1 each, a multiply-add 2, compares, abs, min and max 0) on
48 seeded clutter scenes of the benchmark's distribution (4-40 boxes, one push of 240
substeps each) and fitted per phase by least squares over the environments
(oracle/fit_flop_costs.py); on held-out scenes the fitted costs reproduce the counted
flops of every phase within 0.2 % (tests/test_flop_model.py checks 2 %).  As in the
oracle and the CUDA kernel, a static body's terms (plane, pusher: zero velocity and
inverse mass) are evaluated and counted, and the separating-axis test stops at the first
separating axis, so its cost per test is the distribution's average.  Per-event costs:

  box_steps      194  gravity, rotation matrix (twice: body frames and the pair predicate),
                      world inverse inertia, AABB, integration
  sat             75  one separating-axis test (most pairs separate on an early axis)
  face           762  reference/incident face set-up and four Sutherland-Hodgman passes
  clip_verts      70  depth test and the four-point reduction per clipped vertex
  edge          1435  edge-edge test: all 15 axes, supporting edges, closest points
  plane          167  box-plane: eight vertices R h + c and the deepest four
  pusher         132  capsule segment clipped to the box height, closest points
  points          98  per contact point: effective masses along n, t1, t2, bias
  bb_points       93  second dynamic body of a box-box point
  manifolds       27  tangent basis and pair friction
  pgs_points     162  per point and iteration: normal row and 2-D friction row with the
                      disk clamp, both bodies' velocity terms
  pgs_bb_points   73  the second dynamic body's impulse updates

Cylinder pairs are counted as separating-axis tests at the box cost (their 9 + 9 face
and 81 edge axes are not), so rates on cylinder batches are lower bounds.
"""
import numpy as np

FLOPS_PER_EVENT = {
    "box_steps": 194.3,
    "sat": 74.8,
    "face": 762.0,
    "clip_verts": 70.4,
    "edge": 1435.3,
    "plane": 166.8,
    "pusher": 132.1,
    "points": 97.8,
    "bb_points": 93.4,
    "manifolds": 27.3,
    "pgs_points": 162.2,
    "pgs_bb_points": 73.0,
}


def algorithmic_flops(events, names) -> float:
    """Total flops of an events array [..., n_events] with column names `names`."""
    ev = np.asarray(events, np.float64).reshape(-1, len(names)).sum(0)
    return float(sum(FLOPS_PER_EVENT.get(k, 0) * v for k, v in zip(names, ev)))


def fp32_peak_tflops(sms: int, clock_mhz: float) -> float:
    """FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 (FMA) x clock."""
    return sms * 128 * 2 * clock_mhz * 1e6 / 1e12


PHASES = {
    "per_body": ("box_steps",),
    "narrowphase": ("sat", "face", "clip_verts", "edge", "plane", "pusher"),
    "contact_prep": ("points", "bb_points", "manifolds"),
    "contact_solve": ("pgs_points", "pgs_bb_points"),
}


def flops_by_phase(events, names) -> dict:
    """Algorithmic flops of an events array split by phase of the substep."""
    ev = dict(zip(names, np.asarray(events, np.float64).reshape(-1, len(names)).sum(0)))
    return {ph: float(sum(FLOPS_PER_EVENT[k] * ev.get(k, 0.0) for k in keys)) for ph, keys in PHASES.items()}
