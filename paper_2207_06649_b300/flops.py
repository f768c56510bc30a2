"""Algorithmic floating-point operation counts of the rollout path.

The engine counts events per environment (pmbs_query_events); each event has a fixed
hand-counted cost taken from the algorithm's formulas (multiply, add, subtract, divide
and square root count 1 each, a fused multiply-add counts 2, compares, min/max and abs
count 0).  Work on a static body (plane, pusher) is not counted: it is multiplication by
zero inverse mass that the algorithm does not need.  Per-event costs:

  box_steps      158  gravity 6, rotation matrix 30, world inverse inertia 48, AABB 27,
                      integration (position 6, quaternion update and renormalise 41)
  sat            723  15 separating axes: D 3, |A^T B| 45, 6 face axes 72, 9 edge axes
                      (cross 9, |L|^2 5, sqrt 1, two support radii 40, |D.L| 5, 2, divide 1,
                      normalise 4)
  face           460  reference/incident face set-up 58, four Sutherland-Hodgman passes
  clip_verts       8  depth of each clipped vertex
  edge            95  supporting edges, closest points, midpoint
  plane          128  eight vertices R h + c_z
  pusher         107  capsule segment clipped to the box height, two closest points
  points          99  per contact point: effective masses along n, t1, t2 for one body
                      (cross 9, inertia product 15, dot 5, add 2, reciprocal 1) and bias
  bb_points      105  second dynamic body of a box-box point, offsets rA and rB
  manifolds       30  tangent basis and pair friction
  pgs_points     128  normal row (relative velocity 12, projection and clamp 8, impulse
                      on one body 33) and 2-D friction row with the disk clamp (75)
  pgs_bb_points  102  the second dynamic body's velocity terms and impulses
"""
import numpy as np

FLOPS_PER_EVENT = {
    "box_steps": 158,
    "sat": 723,
    "face": 460,
    "clip_verts": 8,
    "edge": 95,
    "plane": 128,
    "pusher": 107,
    "points": 99,
    "bb_points": 105,
    "manifolds": 30,
    "pgs_points": 128,
    "pgs_bb_points": 102,
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
