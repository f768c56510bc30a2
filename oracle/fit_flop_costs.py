"""Per-event flop costs of the rollout path, measured with the oracle's flop counter.

TEST INFRASTRUCTURE: runs only the flop-counting build of the FP64 oracle
(liboracle_flops.so) on seeded clutter scenes of the benchmark's uneven distribution
(4-40 boxes, one valid push, one push of 240 substeps each), and fits, phase by phase, the
non-negative cost per event that reproduces the counted flops (least squares over the
environments).  The counter counts every add, subtract, multiply, divide and square root
of the plain double engine (compares, abs, min and max count 0), including the terms of a
static body (plane, pusher), whose velocity and inverse mass are zero; the separating-axis
test stops at the first separating axis, so its cost per test is an average over the
distribution.  Prints the costs as JSON; the benchmark's flop model transcribes them.

    python oracle/fit_flop_costs.py [--seed 21] [--envs 48] [--substeps 240]
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# events that carry each phase's work (the oracle's event counters)
PHASE_EVENTS = {
    "per_body": ("box_steps",),
    "narrowphase": ("sat", "face", "clip_verts", "edge", "plane", "pusher"),
    "contact_prep": ("points", "bb_points", "manifolds"),
    "contact_solve": ("pgs_points", "pgs_bb_points"),
}


def counted(seed, n_envs, substeps):
    """Counted flops [envs, phases] and event counters [envs, events]."""
    import oracle
    from paper_2207_06649_b300 import scenegen as sg
    scn, pushes, _ = sg.config_uneven(seed=seed, n_envs=n_envs, n_lo=5, n_hi=40, workers=1)
    st = sg.state13(scn).astype(np.float64)
    F, E = [], []
    for e in range(scn.n_scenes):
        a, b = scn.box_offset[e], scn.box_offset[e + 1]
        f, ev = oracle.count_flops(st[a:b], scn.half[a:b], scn.mass[a:b], scn.mu[a:b], pushes[e].astype(np.float64),
                                   substeps)
        F.append([f[p] for p in PHASE_EVENTS])
        E.append(ev.astype(np.float64))
    return np.array(F), np.array(E)


def fit(F, E):
    import oracle
    from scipy.optimize import nnls
    idx = {n: i for i, n in enumerate(oracle.EVENT_NAMES)}
    costs = {}
    for pi, (ph, keys) in enumerate(PHASE_EVENTS.items()):
        X = np.stack([E[:, idx[k]] for k in keys], 1)
        coef, _ = nnls(X, F[:, pi])
        costs.update({k: float(c) for k, c in zip(keys, coef)})
    return costs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seed", type=int, default=21)
    ap.add_argument("--envs", type=int, default=48)
    ap.add_argument("--substeps", type=int, default=240)
    a = ap.parse_args()
    F, E = counted(a.seed, a.envs, a.substeps)
    print(json.dumps({k: round(v, 1) for k, v in fit(F, E).items()}))


if __name__ == "__main__":
    main()
