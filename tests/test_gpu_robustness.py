"""Failure handling on the GPU without faulting it, and the fixed 1024-environment workload
at full size.

- The per-environment watchdog (a bounded run time per launch) stops environments after
  their current substep; the call reports PMBS_E_TIMEOUT, the context stays usable and
  stepping again resumes them, so the final results are bit-identical to an unlimited run.
- Scene validation refuses scenes whose boxes start interpenetrating (separating-axis test
  on the device) or that hold more boxes than the context allows, without leaking arena.
- The serving loop survives planners that submit and vanish: their work completes, device
  memory returns, and cancelled tickets release everything.
- 1024 clones of one 15-box scene, three pushes each (Sec. V-A style workload): graph
  stepping equals one persistent launch bit for bit, and every environment's flags, costs
  and rewards agree with what the oracle's exact predicates say about its states.
"""
import threading
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _pm():
    from paper_2207_06649_b300 import pmbs
    return pmbs


def _sg():
    from paper_2207_06649_b300 import scenegen
    return scenegen


@pytest.fixture(scope="module")
def work():
    return _sg().config_uneven(seed=41, n_envs=24, n_lo=5, n_hi=25, workers=1)


def _same(a, b):
    assert np.array_equal(a["cost"], b["cost"])
    assert np.array_equal(a["flags"], b["flags"])
    assert np.array_equal(a["reward"].view(np.uint32), b["reward"].view(np.uint32))
    assert np.array_equal(a["state"].view(np.uint32), b["state"].view(np.uint32))
    assert np.array_equal(a["steps"], b["steps"])


def _results(eng, b):
    out = eng.query_cost(b)
    out["state"], out["steps"] = eng.query_states(b)
    return out


def _resume(eng, b, limit=5000):
    """pmbs_step until the batch finishes; returns the number of watchdog reports."""
    pm = _pm()
    timeouts = 0
    for _ in range(limit):
        st = eng.lib.pmbs_step(eng.ctx, b, 1 << 20)
        if st == pm.PMBS_OK:
            return timeouts
        assert st == pm.PMBS_E_TIMEOUT, eng.lib.pmbs_last_error(eng.ctx)
        timeouts += 1
    raise AssertionError("batch did not finish")


# ------------------------------------------------------------------ watchdog
def test_watchdog_stops_and_resumes_with_identical_results(work):
    pm = _pm()
    scenes, pushes, seeds = work
    ref_eng = pm.Engine(device=0, mem_budget_bytes=1 << 30)
    ids = ref_eng.load(scenes)
    ref = ref_eng.rollout(ids, pushes, depth=2, seeds=seeds)
    ref_eng.close()

    # 1e-6 ms = 2 SM cycles: every environment stops after one substep of each launch
    eng = pm.Engine(device=0, mem_budget_bytes=1 << 30, watchdog_ms=1e-6)
    ids = eng.load(scenes)
    b = eng.rollout_pushes(ids, pushes, 2, seeds)
    assert eng.lib.pmbs_step(eng.ctx, b, 0) == pm.PMBS_OK   # enqueue only
    with pytest.raises(pm.PmbsError) as ei:
        eng.query_cost(b)
    assert ei.value.status == pm.PMBS_E_TIMEOUT
    _, steps = eng.query_states(b)
    assert (steps == 1).all()
    n = _resume(eng, b)
    # one launch per substep, plus the launches that only evaluate the end of a push
    assert n >= int(ref["steps"].max()) - 1
    _same(_results(eng, b), ref)
    eng.release_batch(b)

    # graph stepping: the captured launches stop early as well, the query says so, and
    # pmbs_step finishes the batch with the same results
    b = eng.rollout_pushes(ids, pushes, 2, seeds)
    eng.step_graph(b, 240)
    with pytest.raises(pm.PmbsError) as ei:
        eng.query_cost(b)
    assert ei.value.status == pm.PMBS_E_TIMEOUT
    _resume(eng, b)
    _same(_results(eng, b), ref)
    eng.release_batch(b)

    # the context keeps working for other calls
    off = np.array([0, 2], np.int32)
    st = np.zeros((2, 13), np.float32)
    st[:, 3] = 1
    st[0, :3] = (0, 0, 0.02)
    st[1, :3] = (0.2, 0, 0.02)
    assert eng.eval_pairs(off, st, np.full((2, 3), 0.02, np.float32))[0][0].shape[0] == 0
    eng.close()


def test_watchdog_inside_the_server_resumes_transparently(work):
    pm = _pm()
    scenes, pushes, seeds = work
    ref_eng = pm.Engine(device=0, mem_budget_bytes=1 << 30)
    ids = ref_eng.load(scenes)
    ref = ref_eng.rollout(ids, pushes, depth=1, seeds=seeds)
    ref_eng.close()
    eng = pm.Engine(device=0, mem_budget_bytes=1 << 30, watchdog_ms=1e-6)
    ids = eng.load(scenes)
    sv = pm.Server(eng, n_streams=2, max_inflight=4)
    out = sv.wait(sv.submit(ids, pushes, 1, seeds), timeout_ms=120000)
    assert out is not None
    for k in ("cost", "flags", "steps"):
        assert np.array_equal(out[k], ref[k]), k
    st = sv.stats()
    assert st["resumes"] >= int(ref["steps"].max()) - 1 and st["completed"] == 1
    sv.close()
    eng.close()


# ------------------------------------------------------------------ scene validation
def _pair_scene(dx, dz=0.0, yaw=0.0):
    sg = _sg()
    h = 0.03
    pose = np.zeros((2, 7), np.float32)
    pose[:, 3] = 1
    pose[0, :3] = (0, 0, h)
    pose[1, :3] = (dx, 0, h + dz)
    pose[1, 3:] = (np.cos(yaw / 2), 0, 0, np.sin(yaw / 2))
    return sg.Scenes(np.array([0, 2], np.int32), pose, np.zeros((2, 6), np.float32), np.full((2, 3), h, np.float32),
                     np.full(2, 0.1, np.float32), np.full(2, 0.5, np.float32), np.array([0], np.int32))


def test_scene_validation_refuses_penetration_and_size():
    pm = _pm()
    eng = pm.Engine(device=0, mem_budget_bytes=256 << 20, max_boxes_per_env=8)
    sv = pm.Server(eng, n_streams=1, max_inflight=1)   # only for its arena-usage figure
    base = sv.stats()["arena_used_bytes"]
    # 0.5 mm overlap (below the 1 mm limit), exact face contact, a box resting on another
    for sc in (_pair_scene(0.06 - 5e-4), _pair_scene(0.06), _pair_scene(0.0, dz=0.06)):
        ids = eng.load(sc)
        eng.free_scenes(ids)
    assert sv.stats()["arena_used_bytes"] == base
    # 2 mm overlap along x; a 45-degree box whose corner reaches 5 mm into its neighbour
    corner = 0.03 + 0.03 * np.sqrt(2) - 0.005
    for sc in (_pair_scene(0.06 - 2e-3), _pair_scene(corner, yaw=np.pi / 4)):
        with pytest.raises(pm.PmbsError) as ei:
            eng.load(sc)
        assert ei.value.status == pm.PMBS_E_INVALID and "penetration" in str(ei.value)
    # the penetration test looks at every scene of a call: one bad scene refuses the call
    good, bad = _pair_scene(0.2), _pair_scene(0.05)
    with pytest.raises(pm.PmbsError):
        eng.load(_sg().concat([good, good, bad]))
    # more boxes than the context holds
    sg = _sg()
    sc9 = sg.make_scene(np.random.default_rng(0), 9, region_half=0.15)
    with pytest.raises(pm.PmbsError) as ei:
        eng.load(sc9)
    assert ei.value.status == pm.PMBS_E_INVALID
    assert sv.stats()["arena_used_bytes"] == base
    # nothing leaked: the context still loads and simulates
    ids = eng.load(sg.concat([good, good]))
    out = eng.rollout(ids, np.array([[0.19, 0.19, 0.19, 0.19]] * 2, np.float32), depth=1)
    assert (out["steps"] == 240).all()
    sv.close()
    eng.close()


def test_penetration_limit_is_configurable():
    pm = _pm()
    eng = pm.Engine(device=0, mem_budget_bytes=64 << 20, max_initial_penetration=0.01)
    eng.free_scenes(eng.load(_pair_scene(0.06 - 8e-3)))
    with pytest.raises(pm.PmbsError):
        eng.load(_pair_scene(0.06 - 2e-2))
    eng.close()
    eng = pm.Engine(device=0, mem_budget_bytes=64 << 20, max_initial_penetration=1e-4)
    with pytest.raises(pm.PmbsError):
        eng.load(_pair_scene(0.06 - 5e-4))
    eng.close()


# ------------------------------------------------------------------ serving
def test_server_survives_planners_that_vanish(work):
    pm = _pm()
    scenes, pushes, seeds = work
    eng = pm.Engine(device=0, mem_budget_bytes=1 << 30)
    ids = eng.load(scenes)
    sv = pm.Server(eng, n_streams=2, max_inflight=2)
    base = sv.stats()["arena_used_bytes"]
    rng = np.random.default_rng(9)
    tickets = []

    def planner():
        # submits and leaves without waiting
        for _ in range(6):
            pick = rng.integers(0, len(ids), size=150)
            tickets.append(sv.submit(ids[pick], pushes[pick], 2, seeds[pick]))

    th = threading.Thread(target=planner)
    th.start()
    th.join()
    t0 = time.time()
    while sv.stats()["outstanding"] > 0 and time.time() - t0 < 120:
        time.sleep(0.01)
    st = sv.stats()
    assert st["outstanding"] == 0 and st["completed"] == 6 and st["held_results"] == 6
    assert st["arena_used_bytes"] == base          # device memory came back without a wait
    for t in tickets:
        sv.cancel(t)                               # a supervisor drops the orphaned results
    assert sv.stats()["held_results"] == 0

    # cancelled while pending or on the device: nothing is held, nothing leaks
    more = []
    for _ in range(8):
        pick = rng.integers(0, len(ids), size=300)
        more.append(sv.submit(ids[pick], pushes[pick], 2, seeds[pick]))
    for t in more:
        sv.cancel(t)
    t0 = time.time()
    while sv.stats()["outstanding"] > 0 and time.time() - t0 < 120:
        time.sleep(0.01)
    st = sv.stats()
    assert st["outstanding"] == 0 and st["held_results"] == 0 and st["arena_used_bytes"] == base
    assert eng.lib.pmbs_server_wait(sv.sv, more[0], 0, None, None, None, None, None) == pm.PMBS_E_INVALID

    # a waiter whose ticket is cancelled from another thread returns instead of blocking
    t = sv.submit(np.repeat(ids, 100)[:2000], np.repeat(pushes, 100, 0)[:2000], 3, np.repeat(seeds, 100)[:2000])
    res = {}

    def waiter():
        res["st"] = eng.lib.pmbs_server_wait(sv.sv, t, 120000, None, None, None, None, None)

    w = threading.Thread(target=waiter)
    w.start()
    time.sleep(0.05)
    sv.lib.pmbs_server_cancel(sv.sv, t)
    w.join(timeout=150)
    assert not w.is_alive() and res["st"] in (pm.PMBS_E_INVALID, pm.PMBS_OK)

    # and the server still serves
    pick = rng.integers(0, len(ids), size=64)
    out = sv.wait(sv.submit(ids[pick], pushes[pick], 2, seeds[pick]))
    direct = eng.rollout(ids[pick], pushes[pick], depth=2, seeds=seeds[pick])
    assert np.array_equal(out["cost"], direct["cost"])
    sv.close()
    eng.close()


# ------------------------------------------------------------------ full-size fixed workload
def test_fixed_1024_envs_graph_equals_launch_and_oracle_predicates(orc):
    pm = _pm()
    sg = _sg()
    sc, pushes, seeds = sg.config_fixed()
    n_envs, depth = len(pushes), 3
    eng = pm.Engine(device=0, mem_budget_bytes=2 << 30)
    ids = eng.load(sc)
    scene_ids = np.repeat(ids, n_envs)
    ref = eng.rollout(scene_ids, pushes, depth=depth, seeds=seeds)
    b = eng.rollout_pushes(scene_ids, pushes, depth, seeds)
    eng.step_graph(b, 240)
    _same(_results(eng, b), ref)
    eng.release_batch(b)

    st0 = sg.state13(sc)
    prm = orc.params()
    inv = (ref["flags"] & pm.FLAG_INVALID_START) != 0
    # the invalid-start flag is the oracle's exact start test on the first push
    want = np.array([orc.start_blocked(st0, sc.half, p[0], p[1], f32=True) for p in pushes])
    assert np.array_equal(inv, want) and 0 < inv.sum() < n_envs
    assert (ref["cost"][inv] == depth + 1).all() and (ref["steps"][inv] == 0).all()
    # reward is gamma^(cost-1) for a grasp, else 0
    g = np.float64(prm.gamma)
    rw = np.where(ref["cost"] <= depth, g ** (ref["cost"] - 1.0), 0.0)
    assert np.abs(ref["reward"] - rw).max() <= 1e-6
    # the grasp decision on every final state, evaluated by the oracle's exact test,
    # matches the outcome (graspable iff the rollout stopped with cost <= depth)
    out_ws = (ref["flags"] & pm.FLAG_OUT_OF_WORKSPACE) != 0
    nb = sc.box_offset[1]
    for e in np.flatnonzero(~inv & ~out_ws):
        fin = ref["state"][e * nb:(e + 1) * nb]
        assert orc.grasp(fin, sc.half, int(sc.target[0]), f32=True) == (ref["cost"][e] <= depth), e
    # every environment did work proportional to its pushes
    done = ~inv & ~out_ws
    assert (ref["steps"][done] == 240 * np.minimum(ref["cost"][done], depth)).all()
    eng.close()
