"""Rollout outcome rules of the oracle (cost-to-go, reward, flags), CPU only."""
import math

import numpy as np
import pytest

from tests import _geom as G


def _one_env(rows, halves, target=0, mass=0.1, mu=0.5):
    st = np.stack([G.box_row(*r) for r in rows]).astype(np.float32)
    n = len(rows)
    return (np.array([0, n], np.int32), st, np.array(halves, np.float32), np.full(n, mass, np.float32),
            np.full(n, mu, np.float32), np.array([target], np.int32))


def test_isolated_target_costs_one_push(orc):
    off, st, h, m, mu, t = _one_env([(0, 0, 0.02), (0.12, 0.1, 0.02)], [[0.02, 0.02, 0.02]] * 2)
    push = np.array([[-0.1, 0.15, 0.0, 0.15]], np.float32)   # far from every box
    r = orc.rollout(off, st, h, m, mu, t, push, depth=3)
    assert r.cost[0] == 1 and r.reward[0] == 1.0
    assert r.flags[0] & orc.F_GRASP1
    assert r.steps[0] == 240


def test_blocked_start_is_flagged_and_not_simulated(orc):
    off, st, h, m, mu, t = _one_env([(0, 0, 0.02)], [[0.02, 0.02, 0.02]])
    push = np.array([[0.025, 0.0, 0.125, 0.0]], np.float32)   # inside the box footprint + r
    r = orc.rollout(off, st, h, m, mu, t, push, depth=3)
    assert r.flags[0] & orc.F_INVALID_START
    assert r.cost[0] == 4 and r.reward[0] == 0 and r.steps[0] == 0


def test_box_pushed_off_the_table_fails(orc):
    off, st, h, m, mu, t = _one_env([(0, 0, 0.02), (0.16, 0.0, 0.02)], [[0.05, 0.05, 0.02], [0.02, 0.02, 0.02]])
    push = np.array([[0.11, 0.0, 0.21, 0.0]], np.float32)
    r = orc.rollout(off, st, h, m, mu, t, push, depth=2)
    assert r.flags[0] & orc.F_OUT_OF_WS
    assert r.cost[0] == 3 and r.reward[0] == 0


def test_ungraspable_until_depth_gives_sentinel_cost(orc):
    # target wider than the opening can never be grasped
    off, st, h, m, mu, t = _one_env([(0, 0, 0.02)], [[0.05, 0.05, 0.02]])
    push = np.array([[-0.15, 0.15, -0.15, 0.05]], np.float32)
    r = orc.rollout(off, st, h, m, mu, t, push, depth=3, seeds=np.array([7], np.uint64))
    assert r.cost[0] == 4 and r.reward[0] == 0 and r.steps[0] == 3 * 240


def test_tiny_config_rollouts_are_thread_independent(orc):
    from paper_2207_06649_b300 import scenegen
    sc, pushes = scenegen.config_tiny(seed=1)
    envs = sc.gather([0] * len(pushes))
    args = (envs.box_offset, scenegen.state13(envs), envs.half, envs.mass, envs.mu, envs.target, pushes)
    a = orc.rollout(*args, depth=1, threads=1)
    b = orc.rollout(*args, depth=1, threads=4)
    assert np.array_equal(a.cost, b.cost) and np.array_equal(a.state, b.state)
    assert set(a.cost.tolist()) <= {1, 2}
    assert (a.steps[(a.flags & orc.F_INVALID_START) == 0] == 240).all()


def test_discounted_reward_follows_cost(orc):
    from paper_2207_06649_b300 import scenegen
    sc, pushes, seeds = scenegen.config_fixed(seed=2, n_boxes=15, n_envs=64)
    envs = sc.gather([0] * 64)
    r = orc.rollout(envs.box_offset, scenegen.state13(envs), envs.half, envs.mass, envs.mu, envs.target,
                    pushes, depth=3, seeds=seeds, threads=8)
    for c, rw in zip(r.cost, r.reward):
        if c <= 3:
            assert rw == pytest.approx(0.8 ** (c - 1), rel=1e-6)
        else:
            assert rw == 0
