"""Diagnostics of the rollout kernel on the GPU: the bounds-checked library and the
per-phase timers.

The bounds-checked library (libpmbs_checked.so: the same source compiled with
PMBS_BOUNDS_CHECK=1, every shared and global index of the rollout kernel checked) must
meet no out-of-range index on small cases of every kind -- the tiny workload, a 64-box
scene, cylinders, warm start, several environments per warp -- over whole rollouts.  Its
arithmetic is the release library's, but it is a different compilation: nvcc may contract
a * b + c into a fused multiply-add at different places, so states agree to FP32 rounding
(checked after one substep: 1e-6 m, 1e-5 m/s, 3e-3 rad/s, the one-substep parity bounds'
order) rather than bit for bit, and long clutter trajectories may drift apart chaotically;
full rollouts must agree on at least 90 % of the costs, like the oracle parity.  Phase
timers change no code path and must leave results bit-identical.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _pm():
    from paper_2207_06649_b300 import pmbs
    return pmbs


def _sg():
    from paper_2207_06649_b300 import scenegen
    return scenegen


def _run(eng, scenes, pushes, depth, seeds=None):
    ids = eng.load(scenes)
    out = eng.rollout(ids, pushes, depth=depth, seeds=seeds)
    eng.free_scenes(ids)
    return out


def _cases():
    sg = _sg()
    out = []
    sc, pushes = sg.config_tiny(seed=3)
    envs = sc.gather([0] * len(pushes))
    out.append(("tiny", envs, pushes, 1, None, {}))
    rng = np.random.default_rng(3)
    big = sg.make_scene(rng, 64, half_lo=0.008, half_hi=0.012, region_half=0.19)
    bp = np.stack([sg._random_valid_push(rng, big, 0) for _ in range(2)])
    out.append(("64 boxes", big.gather([0, 0]), bp, 1, None, {}))
    cs, cp, cseeds = sg.config_cylinders(seed=5, n_envs=12, n_lo=4, n_hi=12, workers=1)
    out.append(("cylinders", cs, cp, 2, cseeds, {}))
    us, up, useeds = sg.config_uneven(seed=31, n_envs=24, n_lo=5, n_hi=30, workers=1)
    out.append(("warm start", us, up, 2, useeds, {"warm_start": 1}))
    out.append(("8 lanes per env", us, up, 2, useeds, {"lanes_per_env": 8, "smem_manifolds": 4}))
    return out


@pytest.mark.parametrize("case", range(5))
def test_bounds_checked_library_is_clean(case):
    name, scenes, pushes, depth, seeds, opts = _cases()[case]
    pm = _pm()
    rel = pm.Engine(device=0, mem_budget_bytes=1 << 30, **opts)
    chk = pm.Engine(device=0, mem_budget_bytes=1 << 30, checked=True, **opts)
    try:
        chk.check_status(reset=True)
        one = []
        for eng in (rel, chk):
            ids = eng.load(scenes)
            b = eng.rollout_pushes(ids, pushes, depth, seeds)
            eng.step(b, 1)
            one.append(eng.query_states(b)[0])
            eng.release_batch(b)
            eng.free_scenes(ids)
        a = _run(rel, scenes, pushes, depth, seeds)
        b = _run(chk, scenes, pushes, depth, seeds)
        status = chk.check_status(reset=True)
    finally:
        rel.close()
        chk.close()
    assert status == (0, 0, 0, 0), f"{name}: out-of-range index (count, array id, index, capacity) = {status}"
    d = np.abs(one[0] - one[1])
    assert d[:, :3].max() <= 1e-6 and d[:, 7:10].max() <= 1e-5 and d[:, 10:13].max() <= 3e-3, name
    assert np.array_equal(a["flags"] & 2, b["flags"] & 2), name
    assert np.mean(a["cost"] == b["cost"]) >= 0.9, name
    assert np.array_equal(a["events"][:, 0] > 0, b["events"][:, 0] > 0), name


def test_release_library_has_no_status_word():
    pm = _pm()
    eng = pm.Engine(device=0, mem_budget_bytes=64 << 20)
    try:
        with pytest.raises(pm.PmbsError) as ei:
            eng.check_status()
        assert ei.value.status == pm.PMBS_E_INVALID
    finally:
        eng.close()


def test_phase_timers_leave_results_unchanged_and_cover_every_phase():
    """With phase_timers = 1 the results are bit-identical; every simulated environment
    has cycles in every per-substep phase and in push set-up and end of push; the contact
    solve is the largest phase on clutter."""
    pm, sg = _pm(), _sg()
    scenes, pushes, seeds = sg.config_uneven(seed=33, n_envs=64, n_lo=5, n_hi=40, workers=1)
    plain = pm.Engine(device=0, mem_budget_bytes=1 << 30)
    timed = pm.Engine(device=0, mem_budget_bytes=1 << 30, phase_timers=1)
    try:
        a = _run(plain, scenes, pushes, 2, seeds)
        b = _run(timed, scenes, pushes, 2, seeds)
    finally:
        plain.close()
        timed.close()
    assert "phase_cycles" not in a
    assert np.array_equal(a["cost"], b["cost"])
    assert np.array_equal(a["state"].view(np.uint32), b["state"].view(np.uint32))
    ph = b["phase_cycles"].astype(np.float64)
    sim = (b["flags"] & 2) == 0
    assert sim.sum() > 50
    assert np.all(ph[sim] > 0), "a simulated environment with an empty phase"
    assert np.all(ph[~sim][:, 1:] == 0)
    share = ph[sim].sum(0) / ph[sim].sum()
    names = pm.PHASE_NAMES
    print("phase shares: " + ", ".join(f"{n} {100 * s:.1f} %" for n, s in zip(names, share)))
    assert share[names.index("contact_solve")] == share.max()
