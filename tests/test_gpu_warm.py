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
