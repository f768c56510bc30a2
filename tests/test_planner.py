"""PMBS planner (Alg. 1, Alg. 2, Eq. 1, Eq. 2) on CPU with the oracle as rollout backend."""
import itertools
import math

import numpy as np
import pytest

from paper_2207_06649_b300 import planner as P
from paper_2207_06649_b300 import scenegen as sg
from tests import _geom as G


def test_ucb_closed_forms():
    # Eq. 1 (no virtual counts) and Eq. 2
    assert P.ucb_virtual(3.0, 4, 0, 10, 0, 1.4) == pytest.approx(3 / 4 + 1.4 * math.sqrt(2 * math.log(10) / 4))
    assert P.ucb_virtual(3.0, 4, 2, 10, 5, 0.3) == pytest.approx(3 / 6 + 0.3 * math.sqrt(2 * math.log(15) / 6))
    assert P.ucb_virtual(0.0, 0, 0, 7, 0, 1.0) == math.inf
    # virtual visits lower a child's score: selected-but-unexpanded nodes are penalised
    assert P.ucb_virtual(2.0, 3, 1, 10, 1, 1.4) < P.ucb_virtual(2.0, 3, 0, 10, 0, 1.4)


def test_contour_candidates_start_clear_and_aim_inward():
    sc = sg.make_scene(np.random.default_rng(4), 8, region_half=0.09, yaw_hi=1.0)
    st = sg.state13(sc)
    cand = P.contour_candidates(st, sc.half, 0)
    assert len(cand) > 0
    import oracle
    for p in cand[:40]:
        assert not oracle.start_blocked(st, sc.half, p[0], p[1], f32=False)
        assert abs(np.hypot(p[2] - p[0], p[3] - p[1]) - 0.1) < 1e-5


class _FakeBackend:
    """Deterministic toy backend: a push's rollout cost is read from a table."""

    def __init__(self, costs):
        self.costs = costs
        self.calls = []

    def rollout(self, handles, pushes, depth, seeds):
        self.calls.append(len(handles))
        cost = np.array([self.costs.get(round(float(p[0]), 4), depth + 1) for p in pushes], np.int32)
        flags = (cost == 1).astype(np.uint8)
        n = len(handles)
        return dict(cost=cost, flags=flags, child_handles=np.arange(100, 100 + n),
                    child_states=np.zeros((n, 1, 13), np.float32))

    def release(self, handles):
        pass


def test_selection_returns_unique_pairs_and_resets_virtual_counts():
    be = _FakeBackend({})
    pl = P.Planner(be, np.full((1, 3), 0.02, np.float32), 0, n_envs=8, max_iterations=1)
    root = P.Node(0, np.zeros((1, 13), np.float32), 0)
    root.sampled = True
    root.untried = [np.array([0.1 * i, 0, 0.1 * i + 0.1, 0], np.float32) for i in range(5)]
    pairs = pl._select(root)
    assert len(pairs) == 5                                  # all unique, fewer than n_envs
    assert len({round(float(a[0]), 4) for _, a in pairs}) == 5
    assert root.Nv == 5


def _tiny_world():
    rows = [(0, 0, 0.02), (0.05, 0.0, 0.02), (-0.05, 0.0, 0.02), (0.0, 0.05, 0.02), (0.0, -0.05, 0.02)]
    st = np.stack([G.box_row(*r) for r in rows]).astype(np.float32)
    half = np.array([[0.02, 0.02, 0.02]] + [[0.02, 0.025, 0.02]] * 4, np.float32)
    mass = np.full(5, 0.1, np.float32)
    mu = np.full(5, 0.5, np.float32)
    return st, half, mass, mu


def test_fully_explored_tiny_tree_picks_a_brute_force_optimal_first_action():
    import oracle
    from tests._oracle_backend import OracleBackend
    st, half, mass, mu = _tiny_world()
    assert not oracle.grasp(st, half, 0, f32=False)
    # four candidate pushes: slide the +x or -x neighbour out along +y, slide the +y
    # neighbour along +x, or push nothing; clearing both x sides takes two pushes
    acts = np.array([[0.05, -0.04, 0.05, 0.06], [-0.05, -0.04, -0.05, 0.06], [-0.04, 0.05, 0.06, 0.05],
                     [0.18, 0.18, 0.18, 0.08]], np.float32)
    prm = oracle.params(substeps_per_push=120)
    be = OracleBackend(half, mass, mu, 0, prm=prm)

    # brute force: minimal number of pushes (depth <= 2) over the fixed action set
    def cost_of(seq):
        s = st
        for k, a in enumerate(seq):
            h = be.load_state(s, half, 0)
            r = be.rollout([h], a[None], 1, np.zeros(1, np.uint64))
            s = r["child_states"][0]
            if r["flags"][0] & 6:
                return 99
            if oracle.grasp(s, half, 0, f32=False):
                return k + 1
        return 99

    best = min(cost_of(seq) for L in (1, 2) for seq in itertools.product(acts, repeat=L))
    firsts = {i for i in range(4) if min(cost_of((acts[i],) + rest) for L in (0, 1)
                                         for rest in itertools.product(acts, repeat=L)) == best}

    class FixedActions(P.Planner):
        def _candidates(self, node):
            if not node.sampled:
                node.sampled = True
                if not node.terminal and not node.failed and node.depth < self.d_T:
                    node.untried = [a.copy() for a in acts[::-1]]
            return node.untried

    pl = FixedActions(be, half, 0, n_envs=16, d_T=2, d_s=0, t_max=120, seed=1)
    h = be.load_state(st, half, 0)
    action, info = pl.plan(h, st)
    assert best < 99
    chosen = [i for i in range(4) if np.allclose(acts[i], action)]
    assert chosen and chosen[0] in firsts, (chosen, firsts, best)


def test_planning_scene_is_buried_and_not_graspable():
    import oracle
    sc = sg.config_planning(seed=0)
    st = sg.state13(sc)
    assert sc.box_offset[-1] == 30
    assert sg._buried(sc.pose.astype(float), sc.half.astype(float))
    assert not oracle.grasp(st, sc.half, 0, f32=False)
