"""Host planner: parallel MCTS with batched simulation (PMBS, Alg. 1 and Alg. 2) and the
serial MCTS baseline (Sec. IV-A, Eq. 1) over the batched rollout engine.

The tree lives on the host; every node's state is a scene id in the engine's
device-resident scene store (batch expansion registers each child state as a scene,
Sec. IV-C), so states never leave the device except for the host-side contour sampler of
expansion candidates (Sec. IV-B).  A backend object supplies rollouts; `GpuBackend` wraps
the C ABI.  Serial MCTS is the same loop with one environment per iteration (then the
virtual counts are always zero and Eq. 2 reduces to Eq. 1).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

# ------------------------------------------------------------------ UCB (Eq. 1, Eq. 2)


def ucb_virtual(q, n, n_virt, n_parent, n_parent_virt, c):
    """Eq. 2: Q/(N + N^) + c sqrt(2 ln(N_p + N^_p) / (N + N^)).  With N^ = 0 this is Eq. 1.
    A child with N + N^ = 0 scores +inf (unvisited first)."""
    d = n + n_virt
    if d <= 0:
        return math.inf
    return q / d + c * math.sqrt(2.0 * math.log(max(n_parent + n_parent_virt, 1)) / d)


# ------------------------------------------------------------------ host contour sampler


def footprints(state13, half):
    """Top-down footprint per box or cylinder: centre, unit axis u (horizontal part of the
    body's x axis, or y axis when x is vertical), v = perp(u), support half widths along u
    and v."""
    st = np.asarray(state13, np.float64)
    h = np.asarray(half, np.float64)
    w, x, y, z = st[:, 3], st[:, 4], st[:, 5], st[:, 6]
    R = np.empty((len(st), 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    e = R[:, :2, 0].copy()
    small = np.einsum("ij,ij->i", e, e) < 1e-12
    e[small] = R[small, :2, 1]
    u = e / np.linalg.norm(e, axis=1, keepdims=True)
    v = np.stack([-u[:, 1], u[:, 0]], 1)
    pu = np.einsum("ikj,ik->ij", R[:, :2, :], u)   # u on the body axes
    pv = np.einsum("ikj,ik->ij", R[:, :2, :], v)
    su = (np.abs(pu) * np.abs(h)).sum(1)
    sv = (np.abs(pv) * np.abs(h)).sum(1)
    cyl = h[:, 1] < 0
    if cyl.any():
        # a cylinder (row (r, -r, h)): r times the 16-gon's radial support plus h |.z_b|
        ang = np.arange(8) * np.pi / 8
        c, s = np.cos(ang), np.sin(ang)
        for sup, pp in ((su, pu), (sv, pv)):
            rad = np.abs(pp[cyl, 0:1] * c + pp[cyl, 1:2] * s).max(1)
            sup[cyl] = rad * h[cyl, 0] + np.abs(pp[cyl, 2]) * h[cyl, 2]
    return st[:, :2], u, v, su, sv


def contour_candidates(state13, half, target, radius=0.01, clearance=0.005, n_points=16, near=0.1,
                       length=0.1):
    """Expansion candidates (Sec. IV-B): n_points start points spaced by arc length around
    the footprint (grown by radius + clearance) of every box whose centre is within `near`
    of the target's, each pushing toward that box's centre for `length`; starts whose
    pusher disc meets a footprint are discarded.  Returns [k, 4] pushes (x_s, y_s, x_e, y_e)."""
    c, u, v, su, sv = footprints(state13, half)
    t = int(target)
    out = []
    for j in range(len(c)):
        if np.linalg.norm(c[j] - c[t]) > near + 1e-12:
            continue
        A, B = su[j] + radius + clearance, sv[j] + radius + clearance
        per = 4 * (A + B)
        for p in range(n_points):
            ell = per * p / n_points
            if ell < B:
                lu, lv = A, ell
            elif ell < B + 2 * A:
                lu, lv = A - (ell - B), B
            elif ell < 3 * B + 2 * A:
                lu, lv = -A, B - (ell - B - 2 * A)
            elif ell < 3 * B + 4 * A:
                lu, lv = ell - 3 * B - 2 * A - A, -B
            else:
                lu, lv = A, ell - 3 * B - 4 * A - B
            s = c[j] + lu * u[j] + lv * v[j]
            d = c[j] - s
            d = d / np.linalg.norm(d)
            rel = s - c
            pu = np.maximum(np.abs(np.einsum("ij,ij->i", rel, u)) - su, 0.0)
            pv = np.maximum(np.abs(np.einsum("ij,ij->i", rel, v)) - sv, 0.0)
            if np.any(pu * pu + pv * pv < radius * radius):
                continue
            out.append([s[0], s[1], s[0] + d[0] * length, s[1] + d[1] * length])
    return np.array(out, np.float32).reshape(-1, 4)


# ------------------------------------------------------------------ tree


@dataclass
class Node:
    handle: int                     # scene id of this node's state
    state: np.ndarray               # [n, 13] host copy (for the contour sampler)
    depth: int
    parent: "Node | None" = None
    action: np.ndarray | None = None
    terminal: bool = False          # target graspable here
    failed: bool = False            # workspace left (or the start was blocked): dead end
    exhausted: bool = False         # every node below is terminal, failed or fully expanded
    N: int = 0
    Q: float = 0.0
    Nv: int = 0                     # virtual count of this selection round
    children: list = field(default_factory=list)
    untried: list = field(default_factory=list)
    sampled: bool = False


@dataclass
class PlanInfo:
    iterations: int = 0
    rollouts: int = 0
    nodes: int = 0
    seconds: float = 0.0
    best_value: float = 0.0
    found_depth: int | None = None


class Planner:
    """PMBS (n_envs > 1) or serial MCTS (n_envs == 1) over a rollout backend.

    backend.rollout(handles, pushes, depth, seeds) -> dict(cost, flags, child_handles,
    child_states); backend.release(handles) frees child scenes.  half / target are the
    static box data of the scene being planned.
    """

    def __init__(self, backend, half, target, n_envs=512, c=1.4, gamma=0.8, d_T=7, d_s=3, t_max=60.0,
                 max_iterations=10 ** 9, seed=0, near=0.1):
        self.be = backend
        self.half = np.asarray(half, np.float32)
        self.target = int(target)
        self.n_envs = n_envs
        self.c = c
        self.gamma = gamma
        self.d_T0, self.d_s0 = d_T, d_s
        self.d_T, self.d_s = d_T, d_s
        self.t_max = t_max
        self.max_iterations = max_iterations
        self.rng = np.random.default_rng(seed)
        self.near = near

    # -- helpers
    def _candidates(self, node: Node):
        if not node.sampled:
            node.sampled = True
            if not node.terminal and not node.failed and node.depth < self.d_T:
                pushes = contour_candidates(node.state, self.half, self.target, near=self.near)
                order = self.rng.permutation(len(pushes))
                node.untried = [pushes[i] for i in order]
        return node.untried

    def _expandable(self, node: Node):
        return not node.terminal and not node.failed and node.depth < self.d_T and len(self._candidates(node)) > 0

    def _select(self, root: Node):
        """Alg. 2: traverse by Eq. 2 to a node with untried actions, take one, raise the
        virtual counts of that node and its ancestors; repeat until n_envs unique
        state-action pairs or nothing is left to expand."""
        pairs = []
        misses = 0
        while len(pairs) < self.n_envs and misses < 4:
            node = root
            path = [node]
            while not self._expandable(node):
                kids = [k for k in node.children if not k.terminal and not k.failed and not k.exhausted]
                if not kids:
                    node = None
                    break
                np_, nvp = node.N, node.Nv
                scores = [ucb_virtual(k.Q, k.N, k.Nv, np_, nvp, self.c) for k in kids]
                node = kids[int(np.argmax(scores))]
                path.append(node)
            if node is None:
                # fully explored branch: nothing below is left to expand; traversal skips
                # it from now on, while its statistics still rank it for the final action
                misses += 1
                if len(path) == 1:
                    break
                path[-1].exhausted = True
                continue
            action = node.untried.pop()
            pairs.append((node, action))
            for p in path:
                p.Nv += 1
        return pairs

    def _backprop(self, node: Node, value: float):
        g = value
        while node is not None:
            node.N += 1
            node.Q += g
            g *= self.gamma
            node = node.parent

    # -- Alg. 1
    def plan(self, root_handle, root_state):
        t0 = time.perf_counter()
        self.d_T, self.d_s = self.d_T0, self.d_s0
        root = Node(root_handle, np.asarray(root_state, np.float32), 0)
        info = PlanInfo()
        es_level = 1
        graspable_depths = []
        all_nodes = [root]
        created = []
        while time.perf_counter() - t0 < self.t_max and info.iterations < self.max_iterations:
            if graspable_depths and min(graspable_depths) <= es_level:
                break
            pairs = self._select(root)
            for n in all_nodes:
                n.Nv = 0
            if not pairs:
                break                   # tree fully explored
            # leaf parallelisation: spare environments repeat pairs with other seeds
            reps = [pairs[i % len(pairs)] for i in range(max(self.n_envs, len(pairs)))]
            handles = np.array([p[0].handle for p in reps], np.int32)
            pushes = np.stack([p[1] for p in reps]).astype(np.float32)
            depth = max(1, self.d_T + self.d_s - min(p[0].depth for p in reps))
            seeds = self.rng.integers(0, 2 ** 63, size=len(reps), dtype=np.uint64)
            out = self.be.rollout(handles, pushes, depth, seeds)
            info.rollouts += len(reps)
            cost, flags = out["cost"], out["flags"]
            # one child per unique pair; its value = max over its simulations
            child_of = {}
            spare = []
            for i, (node, action) in enumerate(reps):
                key = (id(node), i % len(pairs))
                horizon = self.d_T + self.d_s - node.depth
                k = int(cost[i])
                ok = k <= horizon and not (flags[i] & 4) and not (flags[i] & 2)
                # value seen from the child: k - 1 pushes after it, discounted
                v = self.gamma ** (k - 1) if ok else 0.0
                if key not in child_of:
                    child = Node(int(out["child_handles"][i]), out["child_states"][i], node.depth + 1, node, action,
                                 terminal=bool(flags[i] & 1), failed=bool(flags[i] & 6))
                    node.children.append(child)
                    child_of[key] = [child, v]
                    created.append(child.handle)
                    all_nodes.append(child)
                else:
                    child_of[key][1] = max(child_of[key][1], v)
                    spare.append(int(out["child_handles"][i]))
            self.be.release(spare)
            for child, v in child_of.values():
                if child.terminal:
                    graspable_depths.append(child.depth)
                    if child.depth < self.d_T:      # Sec. IV-A: tighten the depth limits
                        self.d_T, self.d_s = child.depth, 0
                    v = 1.0
                self._backprop(child, v)
            # Alg. 1: raise the early-stop level once a whole level is expanded or terminal
            while True:
                level = [n for n in all_nodes if n.depth == es_level - 1]
                if level and all(n.terminal or n.failed or not self._expandable(n) for n in level):
                    es_level += 1
                    if es_level > self.d_T + 1:
                        break
                else:
                    break
            info.iterations += 1
        # best root child by average value (Sec. III-B); ties go to the earlier child
        best, best_v = None, -1.0
        for k in root.children:
            if k.N > 0 and k.Q / k.N > best_v + 1e-12:
                best, best_v = k, k.Q / k.N
        info.seconds = time.perf_counter() - t0
        info.nodes = len(all_nodes)
        info.best_value = best_v
        info.found_depth = min(graspable_depths) if graspable_depths else None
        self.be.release(created)
        return (None if best is None else best.action), info


# ------------------------------------------------------------------ episodes


def run_episode(backend, scene_state, half, target, make_planner, max_actions=16):
    """Alg. 1 Main: while the target is not graspable, plan a push and execute it on the
    scene (here: the same engine stands in for the real scene).  Returns the number of
    actions to retrieval (pushes + the grasp), planning seconds per push and success."""
    state = np.asarray(scene_state, np.float32)
    pushes, plan_s = 0, []
    h = None  # the scene's handle; after a push, the state the engine registered for it
    while pushes < max_actions:
        if backend.graspable(state, half, target):
            if h is not None:
                backend.release([h])
            return dict(actions=pushes + 1, plan_s=plan_s, success=True)
        if h is None:
            h = backend.load_state(state, half, target)
        planner = make_planner()
        action, info = planner.plan(h, state)
        plan_s.append(info.seconds)
        if action is None:
            break
        res = backend.rollout(np.array([h], np.int32), action[None], 1, np.zeros(1, np.uint64))
        backend.release([h])
        h = None
        if res["flags"][0] & 6:
            backend.release(list(res["child_handles"]))
            break
        state = res["child_states"][0]
        h = int(res["child_handles"][0])
        pushes += 1
    if h is not None:
        backend.release([h])
    return dict(actions=max_actions + 1, plan_s=plan_s, success=False)


class GpuBackend:
    """Rollouts on the CUDA engine; node states are device-resident scene ids."""

    def __init__(self, engine, half, mass, mu):
        self.eng = engine
        self.half = np.asarray(half, np.float32)
        self.mass = np.asarray(mass, np.float32)
        self.mu = np.asarray(mu, np.float32)
        self.n = len(self.half)

    def load_state(self, state, half, target):
        off = np.array([0, self.n], np.int32)
        st = np.asarray(state, np.float32)
        return int(self.eng.load_scenes(off, st[:, :7], self.half, self.mass, self.mu,
                                        np.array([target], np.int32), vel=st[:, 7:])[0])

    def rollout(self, handles, pushes, depth, seeds):
        b = self.eng.rollout_pushes(handles, pushes, depth, seeds)
        self.eng.step(b, 0)
        r = self.eng.query_cost(b, child_states=True, child_scenes=True)
        self.eng.release_batch(b)
        ne = len(handles)
        r["child_handles"] = r.pop("child_scene_ids")
        r["child_states"] = r["child_states"].reshape(ne, self.n, 13)
        return r

    def release(self, handles):
        if len(handles):
            self.eng.free_scenes(np.asarray(handles, np.int32))

    def graspable(self, state, half, target):
        off = np.array([0, self.n], np.int32)
        return bool(self.eng.eval_grasp(off, np.asarray(state, np.float32), self.half, [target])[0])
