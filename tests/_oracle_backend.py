"""Planner backend on the FP64 oracle, for CPU tests of the planner only."""
import numpy as np

import oracle


class OracleBackend:
    def __init__(self, half, mass, mu, target, prm=None, threads=8):
        self.half = np.asarray(half, np.float32)
        self.mass = np.asarray(mass, np.float32)
        self.mu = np.asarray(mu, np.float32)
        self.target = int(target)
        self.prm = prm
        self.threads = threads
        self.states = {}
        self.next = 1
        self.rollouts = 0

    def load_state(self, state, half, target):
        h = self.next
        self.next += 1
        self.states[h] = np.asarray(state, np.float32).copy()
        return h

    def rollout(self, handles, pushes, depth, seeds):
        n = len(self.half)
        ne = len(handles)
        st = np.concatenate([self.states[int(h)] for h in handles])
        off = np.arange(ne + 1, dtype=np.int32) * n
        tile = lambda a: np.tile(a, (ne,) + (1,) * (a.ndim - 1))
        r = oracle.rollout(off, st, tile(self.half), tile(self.mass), tile(self.mu), np.full(ne, self.target, np.int32),
                           pushes, depth, seeds, prm=self.prm, threads=self.threads, child=True)
        self.rollouts += ne
        child = r.child.astype(np.float32).reshape(ne, n, 13)
        hs = [self.load_state(child[i], self.half, self.target) for i in range(ne)]
        return dict(cost=r.cost, reward=r.reward, flags=r.flags, child_handles=np.array(hs), child_states=child)

    def release(self, handles):
        for h in handles:
            self.states.pop(int(h), None)

    def graspable(self, state, half, target):
        return oracle.grasp(state, half, target, f32=False)
