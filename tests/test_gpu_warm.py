"""Warm-started contact solve on the GPU (cfg.warm_start = 1) against the oracle with the
same option: non-chaotic scenes within the trajectory tolerance, the six-cube stack that
stands only when impulses are carried over, momentum conservation, and resumable
stepping (the per-environment caches survive launch boundaries bit for bit)."""
import numpy as np
import pytest

from tests import _geom as G

pytestmark = pytest.mark.gpu


def _pm():
    from paper_2207_06649_b300 import pmbs
    return pmbs


def _sg():
    from paper_2207_06649_b300 import scenegen
    return scenegen


@pytest.fixture(scope="module")
def warm():
    e = _pm().Engine(device=0, mem_budget_bytes=2 << 30, warm_start=1)
    yield e
    e.close()


def _scene(rows, halves, mass=0.1, mu=0.5):
    sg = _sg()
    st = np.stack(rows).astype(np.float32)
    n = len(rows)
    return sg.Scenes(np.array([0, n], np.int32), st[:, :7].copy(), st[:, 7:].copy(), np.asarray(halves, np.float32),
                     np.full(n, mass, np.float32), np.full(n, mu, np.float32), np.array([0], np.int32))


def _run(eng, sc, count, push=(0.19, 0.19, 0.19, 0.19)):
    ids = eng.load(sc)
    b = eng.rollout_pushes(ids, np.array([push], np.float32), 1)
    eng.step(b, count)
    st, steps = eng.query_states(b)
    eng.release_batch(b)
    eng.free_scenes(ids)
    return st.astype(np.float64)


def _stack(nb, h=0.01):
    return [G.box_row(0.0005 * k, -0.0003 * k, h + 2 * h * k) for k in range(nb)], np.full((nb, 3), h)


def test_warm_six_cube_stack_stands_and_matches_oracle(warm, orc):
    rows, half = _stack(6)
    sc = _scene(rows, half)
    st = _run(warm, sc, 240)
    gap = np.diff(st[:, 2]) - 0.02
    assert np.abs(gap).max() <= 5e-4 and np.abs(st[:, :2] - np.stack(rows)[:, :2]).max() <= 2e-3
    ref, _, _ = orc.run_substeps(np.stack(rows), half, np.full(6, 0.1), np.full(6, 0.5),
                                 push=np.array([0.19, 0.19, 0.19, 0.19]), count=240, prm=orc.params(warm_start=1))
    assert np.abs(st[:, :3] - ref[:, :3]).max() <= 1e-3
    # without warm start the same stack falls
    cold = _pm().Engine(device=0, mem_budget_bytes=256 << 20)
    st_c = _run(cold, sc, 480)
    cold.close()
    assert np.abs(np.diff(st_c[:, 2]) - 0.02).max() > 5e-3


@pytest.mark.parametrize("case", ["rest", "push", "stack"])
def test_warm_non_chaotic_parity(warm, orc, case):
    if case == "rest":
        rows, half, push = [G.box_row(0.05, -0.02, 0.015)], [[0.02, 0.03, 0.015]], (0.19, 0.19, 0.19, 0.19)
    elif case == "push":
        rows, half, push = [G.box_row(0, 0, 0.02)], [[0.02, 0.02, 0.02]], (-0.05, 0.0, 0.05, 0.0)
    else:
        rows, half, push = ([G.box_row(0, 0, 0.02), G.box_row(0.005, -0.004, 0.055)],
                            [[0.03, 0.03, 0.02], [0.02, 0.02, 0.015]], (0.19, 0.19, 0.19, 0.19))
    sc = _scene(rows, half)
    st = _run(warm, sc, 240, push)
    ref, _, _ = orc.run_substeps(np.stack(rows), np.asarray(half), np.full(len(rows), 0.1), np.full(len(rows), 0.5),
                                 push=np.asarray(push, np.float64), count=240, prm=orc.params(warm_start=1))
    assert np.abs(st[:, :3] - ref[:, :3]).max() <= 1e-3


def test_warm_collisions_conserve_momentum():
    pm = _pm()
    eng = pm.Engine(device=0, mem_budget_bytes=256 << 20, warm_start=1, gravity=(0.0, 0.0, 0.0))
    rows = [G.box_row(-0.021, 0.0, 1.5, v=(0.3, 0.0, 0.0), w=(0.0, 0.0, 1.0)),
            G.box_row(0.021, 0.002, 1.5, v=(-0.2, 0.0, 0.0), w=(0.5, 0.0, 0.0))]
    sg = _sg()
    st0 = np.stack(rows).astype(np.float32)
    sc = sg.Scenes(np.array([0, 2], np.int32), st0[:, :7].copy(), st0[:, 7:].copy(), np.full((2, 3), 0.02, np.float32),
                   np.array([0.1, 0.2], np.float32), np.full(2, 0.5, np.float32), np.array([0], np.int32))
    st = _run(eng, sc, 120)
    eng.close()
    m = np.array([0.1, 0.2])
    p0 = (m[:, None] * st0[:, 7:10].astype(np.float64)).sum(0)
    p1 = (m[:, None] * st[:, 7:10]).sum(0)
    assert np.abs(st[:, 7:10] - st0[:, 7:10]).max() > 0.05
    assert np.abs(p1 - p0).max() <= 1e-6 * np.abs(m[:, None] * st0[:, 7:10]).sum()


def test_warm_caches_survive_launch_boundaries(warm):
    """Graph stepping (one launch per push) and 97-substep steps equal one persistent
    launch bit for bit with warm start on."""
    sg = _sg()
    scenes, pushes, seeds = sg.config_uneven(seed=61, n_envs=64, n_lo=5, n_hi=30, workers=1)
    ids = warm.load(scenes)
    ref = warm.rollout(ids, pushes, depth=2, seeds=seeds)
    for k in (240, 97):
        b = warm.rollout_pushes(ids, pushes, 2, seeds)
        if k == 240:
            warm.step_graph(b, k)
        else:
            while not warm.step(b, k):
                pass
        r = warm.query_cost(b)
        st, steps = warm.query_states(b)
        warm.release_batch(b)
        assert np.array_equal(r["cost"], ref["cost"]) and np.array_equal(steps, ref["steps"])
        assert np.array_equal(st.view(np.uint32), ref["state"].view(np.uint32))
    warm.free_scenes(ids)


@pytest.mark.parametrize("seed", [0, 1])
def test_warm_clutter_two_substeps_all_state(orc, seed):
    """Two substeps of 48 squeezed clutter scenes with warm start (the second substep
    starts from the impulses carried over from the first) against the oracle with the same
    option: every box's position within 2e-4 m and rotation within 2e-3 rad (twice the
    one-substep bounds); linear velocity within 2e-5 m/s and angular velocity within
    6e-3 rad/s (twice the one-substep FP32-rounding bounds of the parity tests) for at least
    99 % of the boxes -- a point whose match in the previous substep lies at the 2 mm
    tolerance may be carried over in FP64 and not in FP32 or the reverse, so a few bodies
    may differ by more -- and every box within the bound the position check implies
    (2e-4 m over two substeps of 1/240 s: 0.048 m/s)."""
    import math
    sg = _sg()
    rng = np.random.default_rng(seed)
    parts = []
    for e in range(48):
        n = int(rng.integers(3, 25))
        sc = sg.make_scene(rng, n, half_lo=0.01, half_hi=0.035, yaw_hi=math.pi / 2,
                           density_scale=rng.uniform(0.3, 0.6))
        sc.pose[:, :2] *= 0.95
        parts.append(sc)
    sc = sg.concat(parts)
    pushes = np.stack([sg._random_valid_push(rng, sc, e) for e in range(sc.n_scenes)])
    eng = _pm().Engine(device=0, mem_budget_bytes=1 << 30, warm_start=1, max_initial_penetration=0.01)
    try:
        ids = eng.load(sc)
        b = eng.rollout_pushes(ids, pushes, 1)
        eng.step(b, 2)
        st, steps = eng.query_states(b)
        eng.release_batch(b)
    finally:
        eng.close()
    s0 = sg.state13(sc)
    dx, dq, dv, dw = [], [], [], []
    for e in range(sc.n_scenes):
        a, z = sc.box_offset[e], sc.box_offset[e + 1]
        ref, _, _ = orc.run_substeps(s0[a:z], sc.half[a:z], sc.mass[a:z], sc.mu[a:z], push=pushes[e].astype(float),
                                     count=2, prm=orc.params(warm_start=1))
        assert steps[e] == 2
        dx.extend(np.abs(st[a:z, :3] - ref[:, :3]).max(1))
        dq.extend(G.rotation_angle_between(st[a:z, 3:7], ref[:, 3:7]))
        dv.extend(np.abs(st[a:z, 7:10] - ref[:, 7:10]).max(1))
        dw.extend(np.abs(st[a:z, 10:13] - ref[:, 10:13]).max(1))
    dx, dq, dv, dw = map(np.array, (dx, dq, dv, dw))
    ok = (dv <= 2e-5) & (dw <= 6e-3)
    print(f"warm start, two substeps, seed {seed}: x {dx.max():.2e} m, rotation {dq.max():.2e} rad; "
          f"{ok.mean() * 100:.2f} % of {len(dv)} boxes within the velocity bounds, max {dv.max():.2e} m/s, "
          f"{dw.max():.2e} rad/s")
    assert dx.max() <= 2e-4 and dq.max() <= 2e-3
    assert ok.mean() >= 0.99
    assert dv.max() <= 0.048 and dw.max() <= 0.048 * 212
