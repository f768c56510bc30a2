"""The benchmark's flop model against the oracle's flop counter (CPU only).

The roofline's numerator is the algorithmic flop count of a launch: the event counters
of the GPU times per-event costs (paper_2207_06649_b300/flops.py).  Those costs were
fitted to the oracle's flop counter; here they must reproduce the counter, phase by phase,
on clutter scenes the fit did not see (seeds other than the fit's) and on the tiny
workload.  The counter itself is pinned on a case counted by hand.
"""
import numpy as np
import pytest

PHASES = ["per_body", "narrowphase", "contact_prep", "contact_solve"]


def _model_by_phase(ev):
    import oracle
    from paper_2207_06649_b300 import flops
    return flops.flops_by_phase(np.asarray(ev, np.float64)[None], oracle.EVENT_NAMES)


def test_counter_counts_free_flight_by_hand(orc):
    """One box in free flight far above the table, no pusher: per substep the counted work
    is gravity (v + g dt: 3 multiplies, 3 adds), the body frame and the pair predicate's
    rotation, world inverse inertia, AABB and integration -- and nothing in the other
    phases (no contact).  Two substeps count exactly twice one substep."""
    st = np.array([[0, 0, 1.0, 1, 0, 0, 0, 0.1, 0, 0, 0, 0, 0]], np.float64)
    half = np.array([[0.02, 0.03, 0.01]], np.float32)
    m, mu = np.array([0.1], np.float32), np.array([0.5], np.float32)
    far = np.array([0.19, 0.19, 0.19, 0.19])
    f1, ev1 = orc.count_flops(st, half, m, mu, far, 1)
    f2, ev2 = orc.count_flops(st, half, m, mu, far, 2)
    assert f1["narrowphase"] == f1["contact_prep"] == f1["contact_solve"] == 0
    assert f1["per_body"] > 100
    assert f2["per_body"] == 2 * f1["per_body"]
    # the counter and the model agree on the body work of a free box to within 1 %
    assert abs(_model_by_phase(ev1)["per_body"] - f1["per_body"]) <= 0.01 * f1["per_body"]


@pytest.mark.parametrize("vx, clamped", [(0.0, False), (0.1, True)])
def test_counter_counts_the_solve_by_hand(orc, vx, clamped):
    """A box resting on the table (4 plane points, 10 iterations, one substep), counted by
    hand from the solve's formulas (Sec. III-A transition; the projected Gauss-Seidel
    reading), with the plane as the static body: normal row = relative velocity of the
    two bodies 27 (two cross products 9 + 9, two sums 3 + 3, difference 3), dot 5, target
    and projection 4 (difference, product, sum, difference), impulse n dl 3, one dynamic
    body's update 33 (v + P im: 6, r x P: 9, I^-1 (.): 15, sum 3) -- 72; friction pair =
    relative velocity 27, two dots 10, two candidates 4, limit 1, |c|^2 3, the clamp test
    1, two differences 2, impulse t1 d1 + t2 d2 9, body update 33 -- 90, plus 4 when the
    candidate is scaled onto the disk (a quotient, a square root, two products).  At rest
    the candidate is inside the disk; sliding (0.1 m/s) it is scaled every time."""
    st = np.array([[0.0, 0.0, 0.01, 1, 0, 0, 0, vx, 0, 0, 0, 0, 0]], np.float64)
    half = np.array([[0.01, 0.01, 0.01]], np.float32)
    f, ev = orc.count_flops(st, half, np.array([0.1], np.float32), np.array([0.5], np.float32),
                            np.array([0.19, 0.19, 0.19, 0.19]), 1)
    visits = 10 * 4
    assert int(ev[orc.EVENT_NAMES.index("pgs_points")]) == visits
    assert f["contact_solve"] == visits * (72 + 90 + (4 if clamped else 0))


@pytest.mark.parametrize("seed", [31, 32])
def test_model_reproduces_the_counter_on_held_out_clutter(orc, seed):
    from paper_2207_06649_b300 import scenegen as sg
    scn, pushes, _ = sg.config_uneven(seed=seed, n_envs=12, n_lo=5, n_hi=40, workers=1)
    st = sg.state13(scn).astype(np.float64)
    got = {p: 0.0 for p in PHASES}
    want = {p: 0.0 for p in PHASES}
    for e in range(scn.n_scenes):
        a, b = scn.box_offset[e], scn.box_offset[e + 1]
        f, ev = orc.count_flops(st[a:b], scn.half[a:b], scn.mass[a:b], scn.mu[a:b], pushes[e].astype(np.float64), 240)
        m = _model_by_phase(ev)
        for p in PHASES:
            got[p] += m[p]
            want[p] += f[p]
    rel = {p: (got[p] - want[p]) / want[p] for p in PHASES}
    print("model vs counter, relative: " + ", ".join(f"{p} {100 * r:+.2f} %" for p, r in rel.items()))
    for p in PHASES:
        assert abs(rel[p]) <= 0.02, p
    tot = (sum(got.values()) - sum(want.values())) / sum(want.values())
    assert abs(tot) <= 0.01


def test_model_reproduces_the_counter_on_the_tiny_workload(orc):
    from paper_2207_06649_b300 import scenegen as sg
    sc, pushes = sg.config_tiny(seed=5)
    st = sg.state13(sc).astype(np.float64)
    got = want = 0.0
    for e in range(len(pushes)):
        f, ev = orc.count_flops(st, sc.half, sc.mass, sc.mu, pushes[e].astype(np.float64), 120)
        got += sum(_model_by_phase(ev).values())
        want += sum(f[p] for p in PHASES)
    assert abs(got - want) <= 0.03 * want
