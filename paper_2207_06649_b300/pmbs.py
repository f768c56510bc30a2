"""Thin Python binding of libpmbs.so (ctypes).  Argument marshalling only: every step of
the rollout path runs in the CUDA library.  The C entry points are exposed under the
same names (pmbs_create, pmbs_load_scenes, pmbs_rollout_pushes, pmbs_step,
pmbs_query_cost, ...); `Engine` wraps them for numpy arrays.  There is no CPU fallback:
loading fails loudly if the library is missing."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpmbs.so")

PMBS_OK, PMBS_E_INVALID, PMBS_E_OOM, PMBS_E_CUDA, PMBS_E_NOT_READY, PMBS_E_TIMEOUT, PMBS_E_BUSY = range(7)
FLAG_GRASP_AFTER_PUSH1, FLAG_INVALID_START, FLAG_OUT_OF_WORKSPACE, FLAG_CONTACT_OVERFLOW, FLAG_NOOP_PUSH = \
    1, 2, 4, 8, 16
NUM_EVENTS = 18
EVENT_NAMES = ["substeps", "box_steps", "pair_tests", "sat", "face", "edge", "plane",
               "pusher", "points", "manifolds", "pgs_manifolds", "pgs_points",
               "push_evals", "sample_attempts", "clip_verts", "colours", "bb_points", "pgs_bb_points"]
NUM_PHASES = 8
PHASE_NAMES = ["push_setup", "broadphase", "narrowphase", "contact_prep", "colouring", "contact_solve",
               "integrate", "push_end"]

EXPORTED = ["pmbs_default_config", "pmbs_create", "pmbs_create_with_arena", "pmbs_destroy",
            "pmbs_last_error", "pmbs_load_scenes", "pmbs_free_scenes", "pmbs_rollout_pushes",
            "pmbs_rollout_pushes_device", "pmbs_step", "pmbs_query_cost", "pmbs_query_cost_device",
            "pmbs_query_states", "pmbs_query_events", "pmbs_query_phase_cycles", "pmbs_batch_info", "pmbs_release_batch",
            "pmbs_eval_pairs", "pmbs_eval_grasp", "pmbs_eval_sample", "pmbs_eval_start_blocked",
            "pmbs_launch_shape", "pmbs_set_launch_shape", "pmbs_fp32_peak", "pmbs_check_status",
            "pmbs_rollout_noalloc",
            "pmbs_step_graph", "pmbs_autotune", "pmbs_server_create", "pmbs_server_submit",
            "pmbs_server_wait", "pmbs_server_stats", "pmbs_server_cancel", "pmbs_server_destroy",
            "pmbs_render_heightmaps", "pmbs_render_heightmaps_device", "pmbs_query_heightmaps",
            "pmbs_eval_grasp_heightmap"]


class pmbs_config(C.Structure):
    _fields_ = [("device", C.c_int), ("max_envs", C.c_int), ("max_boxes_per_env", C.c_int),
                ("mem_budget_bytes", C.c_size_t), ("dt", C.c_float), ("substeps_per_push", C.c_int),
                ("pgs_iters", C.c_int), ("gravity", C.c_float * 3), ("table_half", C.c_float * 2),
                ("table_mu", C.c_float), ("pusher_mu", C.c_float), ("pusher_radius", C.c_float),
                ("pusher_z0", C.c_float), ("pusher_z1", C.c_float), ("pusher_speed", C.c_float),
                ("push_length", C.c_float), ("gamma", C.c_float), ("grasp_opening", C.c_float),
                ("grasp_clearance", C.c_float), ("finger_depth", C.c_float), ("finger_width", C.c_float),
                ("grasp_angles", C.c_int), ("margin", C.c_float), ("slop", C.c_float),
                ("baumgarte", C.c_float), ("sample_clearance", C.c_float), ("sample_attempts", C.c_int),
                ("contour_points", C.c_int), ("contact_cap", C.c_int), ("manifold_cap", C.c_int),
                ("pair_cap", C.c_int), ("lanes_per_env", C.c_int), ("warps_per_block", C.c_int),
                ("smem_points", C.c_int),
                ("smem_manifolds", C.c_int), ("watchdog_ms", C.c_float),
                ("max_initial_penetration", C.c_float), ("warm_start", C.c_int),
                ("warm_tolerance", C.c_float), ("cylinders", C.c_int), ("phase_timers", C.c_int)]


class PmbsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"pmbs status {status}: {msg}")
        self.status = status


_libs = {}


def load(build_if_missing: bool = True, checked: bool = False):
    """Load libpmbs.so, or with checked=True its bounds-checked twin libpmbs_checked.so
    (building it if the sources are newer and nvcc is present)."""
    if checked in _libs:
        return _libs[checked]
    path = _build.LIB_CHECKED if checked else LIB_PATH
    if build_if_missing and _build.stale(checked) and os.path.exists(_build.NVCC):
        _build.build(checked=checked)
    if not os.path.exists(path):
        raise ImportError(f"{os.path.basename(path)} not built at {path}; run paper_2207_06649_b300/build.py")
    L = C.CDLL(path)
    vp, i32, i64, P = C.c_void_p, C.c_int, C.c_int64, C.POINTER
    sig = {
        "pmbs_default_config": ([P(pmbs_config)], None),
        "pmbs_create": ([P(pmbs_config), vp, P(vp)], i32),
        "pmbs_create_with_arena": ([P(pmbs_config), vp, vp, C.c_size_t, P(vp)], i32),
        "pmbs_destroy": ([vp], None),
        "pmbs_last_error": ([vp], C.c_char_p),
        "pmbs_load_scenes": ([vp, i32] + [vp] * 8, i32),
        "pmbs_free_scenes": ([vp, i32, vp], i32),
        "pmbs_rollout_pushes": ([vp, i32, vp, vp, i32, vp, vp], i32),
        "pmbs_rollout_pushes_device": ([vp, i32, vp, vp, i32, vp, vp], i32),
        "pmbs_step": ([vp, i64, i32], i32),
        "pmbs_step_graph": ([vp, i64, i32], i32),
        "pmbs_autotune": ([vp, i32, vp, vp, i32, vp, i32, vp, vp, vp, vp, vp], i32),
        "pmbs_query_cost": ([vp, i64, vp, vp, vp, vp, vp], i32),
        "pmbs_query_cost_device": ([vp, i64, vp, vp, vp], i32),
        "pmbs_query_states": ([vp, i64, vp, vp], i32),
        "pmbs_query_events": ([vp, i64, vp], i32),
        "pmbs_query_phase_cycles": ([vp, i64, vp], i32),
        "pmbs_batch_info": ([vp, i64, vp, vp], i32),
        "pmbs_release_batch": ([vp, i64], i32),
        "pmbs_eval_pairs": ([vp, i32] + [vp] * 10, i32),
        "pmbs_eval_grasp": ([vp, i32] + [vp] * 5, i32),
        "pmbs_eval_sample": ([vp, i32, vp, vp, vp, vp, i32, vp, vp], i32),
        "pmbs_eval_start_blocked": ([vp, i32] + [vp] * 5, i32),
        "pmbs_launch_shape": ([vp, i32, vp, vp, vp, vp, vp], i32),
        "pmbs_set_launch_shape": ([vp, i32, i32, i32, i32], i32),
        "pmbs_fp32_peak": ([vp, P(C.c_double)], i32),
        "pmbs_check_status": ([vp, vp, i32], i32),
        "pmbs_rollout_noalloc": ([P(pmbs_config), vp, i32, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp], i32),
        "pmbs_server_create": ([vp, i32, i32, P(vp)], i32),
        "pmbs_server_submit": ([vp, i32, vp, vp, i32, vp, P(C.c_int64)], i32),
        "pmbs_server_wait": ([vp, C.c_int64, i32, vp, vp, vp, vp, P(C.c_double)], i32),
        "pmbs_server_stats": ([vp, vp], i32),
        "pmbs_server_cancel": ([vp, C.c_int64], i32),
        "pmbs_render_heightmaps": ([vp, i32, vp, vp, vp, vp], i32),
        "pmbs_render_heightmaps_device": ([vp, i32, vp, vp, vp, vp], i32),
        "pmbs_query_heightmaps": ([vp, C.c_int64, vp], i32),
        "pmbs_eval_grasp_heightmap": ([vp, i32, vp, vp, vp, vp, C.c_float, vp], i32),
        "pmbs_server_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _libs[checked] = L
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def default_config(**overrides) -> pmbs_config:
    cfg = pmbs_config()
    load().pmbs_default_config(C.byref(cfg))
    for k, v in overrides.items():
        if k in ("gravity", "table_half"):
            arr = getattr(cfg, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(cfg, k, v)
    return cfg


def current_stream_handle():
    """cudaStream_t of torch's current stream on the current device (None if no torch)."""
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


class Engine:
    """A pmbs context with numpy-array methods (one C call each)."""

    def __init__(self, cfg: pmbs_config | None = None, stream=None, arena=None, checked: bool = False,
                 **overrides):
        """checked=True runs every call on the bounds-checked library (same results,
        slower; read its status word with check_status)."""
        self.lib = load(checked=checked)
        self.cfg = cfg or default_config(**overrides)
        self.ctx = C.c_void_p()
        if arena is not None:
            # a caller-owned device buffer, e.g. a torch.uint8 CUDA tensor
            ptr, nbytes = arena
            st = self.lib.pmbs_create_with_arena(C.byref(self.cfg), stream, C.c_void_p(ptr), nbytes,
                                                 C.byref(self.ctx))
        else:
            st = self.lib.pmbs_create(C.byref(self.cfg), stream, C.byref(self.ctx))
        if st != PMBS_OK:
            raise PmbsError(st, "pmbs_create failed")

    def close(self):
        if self.ctx:
            self.lib.pmbs_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != PMBS_OK:
            raise PmbsError(st, f"{what}: {self.lib.pmbs_last_error(self.ctx).decode()}")

    # ---- scenes and batches
    def load_scenes(self, box_offset, pose, half, mass, mu, target, vel=None):
        box_offset = np.ascontiguousarray(box_offset, np.int32)
        pose = np.ascontiguousarray(pose, np.float32)
        half = np.ascontiguousarray(half, np.float32)
        mass = np.ascontiguousarray(mass, np.float32)
        mu = np.ascontiguousarray(mu, np.float32)
        target = np.ascontiguousarray(target, np.int32)
        vel = None if vel is None else np.ascontiguousarray(vel, np.float32)
        ns = box_offset.shape[0] - 1
        ids = np.zeros(ns, np.int32)
        self._check(self.lib.pmbs_load_scenes(self.ctx, ns, _p(box_offset), _p(pose), _p(vel), _p(half),
                                              _p(mass), _p(mu), _p(target), _p(ids)), "pmbs_load_scenes")
        return ids

    def load(self, sc):
        """Load a scenegen.Scenes object."""
        return self.load_scenes(sc.box_offset, sc.pose, sc.half, sc.mass, sc.mu, sc.target, vel=sc.vel)

    def free_scenes(self, ids):
        ids = np.ascontiguousarray(ids, np.int32)
        self._check(self.lib.pmbs_free_scenes(self.ctx, ids.shape[0], _p(ids)), "pmbs_free_scenes")

    def rollout_pushes(self, scene_ids, first_push, depth, seeds=None) -> int:
        scene_ids = np.ascontiguousarray(scene_ids, np.int32)
        first_push = np.ascontiguousarray(first_push, np.float32)
        n = scene_ids.shape[0]
        seeds = np.ascontiguousarray(np.zeros(n, np.uint64) if seeds is None else seeds, np.uint64)
        b = C.c_int64()
        self._check(self.lib.pmbs_rollout_pushes(self.ctx, n, _p(scene_ids), _p(first_push), depth, _p(seeds),
                                                 C.byref(b)), "pmbs_rollout_pushes")
        return b.value

    def rollout_pushes_device(self, n_envs, d_scene_ids, d_first_push, depth, d_seeds) -> int:
        b = C.c_int64()
        self._check(self.lib.pmbs_rollout_pushes_device(self.ctx, n_envs, C.c_void_p(d_scene_ids),
                                                        C.c_void_p(d_first_push), depth, C.c_void_p(d_seeds),
                                                        C.byref(b)), "pmbs_rollout_pushes_device")
        return b.value

    def step(self, batch, max_substeps=0) -> bool:
        st = self.lib.pmbs_step(self.ctx, batch, max_substeps)
        if st == PMBS_E_NOT_READY:
            return False
        self._check(st, "pmbs_step")
        return True

    def step_graph(self, batch, substeps_per_launch=240):
        self._check(self.lib.pmbs_step_graph(self.ctx, batch, substeps_per_launch), "pmbs_step_graph")

    def autotune(self, scene_ids, first_push, depth, seeds=None, substeps=240):
        scene_ids = np.ascontiguousarray(scene_ids, np.int32)
        first_push = np.ascontiguousarray(first_push, np.float32)
        n = scene_ids.shape[0]
        seeds = np.ascontiguousarray(np.zeros(n, np.uint64) if seeds is None else seeds, np.uint64)
        g, w, m, t, k = C.c_int32(), C.c_int32(), C.c_int32(), C.c_float(), C.c_int32()
        self._check(self.lib.pmbs_autotune(self.ctx, n, _p(scene_ids), _p(first_push), depth, _p(seeds), substeps,
                                           C.byref(g), C.byref(w), C.byref(m), C.byref(t), C.byref(k)),
                    "pmbs_autotune")
        return dict(lanes_per_env=g.value, warps_per_block=w.value, smem_manifolds=m.value, ms=t.value,
                    substeps_per_launch=k.value)

    def batch_info(self, batch):
        ne, nb = C.c_int32(), C.c_int32()
        self._check(self.lib.pmbs_batch_info(self.ctx, batch, C.byref(ne), C.byref(nb)), "pmbs_batch_info")
        return ne.value, nb.value

    def query_cost(self, batch, child_states=False, child_scenes=False):
        ne, nb = self.batch_info(batch)
        cost = np.zeros(ne, np.int32)
        reward = np.zeros(ne, np.float32)
        flags = np.zeros(ne, np.uint8)
        child = np.zeros((max(nb, 1), 13), np.float32) if child_states else None
        cids = np.zeros(ne, np.int32) if child_scenes else None
        self._check(self.lib.pmbs_query_cost(self.ctx, batch, _p(cost), _p(reward), _p(flags), _p(child), _p(cids)),
                    "pmbs_query_cost")
        out = dict(cost=cost, reward=reward, flags=flags)
        if child_states:
            out["child_states"] = child[:nb]
        if child_scenes:
            out["child_scene_ids"] = cids
        return out

    def query_cost_device(self, batch, d_cost, d_reward, d_flags):
        self._check(self.lib.pmbs_query_cost_device(self.ctx, batch, C.c_void_p(d_cost), C.c_void_p(d_reward),
                                                    C.c_void_p(d_flags)), "pmbs_query_cost_device")

    def query_states(self, batch):
        ne, nb = self.batch_info(batch)
        st = np.zeros((max(nb, 1), 13), np.float32)
        steps = np.zeros(ne, np.int32)
        self._check(self.lib.pmbs_query_states(self.ctx, batch, _p(st), _p(steps)), "pmbs_query_states")
        return st[:nb], steps

    def query_events(self, batch):
        ne, _ = self.batch_info(batch)
        ev = np.zeros((ne, NUM_EVENTS), np.uint64)
        self._check(self.lib.pmbs_query_events(self.ctx, batch, _p(ev)), "pmbs_query_events")
        return ev

    def check_status(self, reset=True):
        """Bounds-checked library only: (violations, first array id, index, capacity)."""
        out = np.zeros(4, np.uint32)
        self._check(self.lib.pmbs_check_status(self.ctx, _p(out), 1 if reset else 0), "pmbs_check_status")
        return tuple(int(v) for v in out)

    def query_phase_cycles(self, batch):
        """[n_envs, NUM_PHASES] SM clock cycles per phase (PHASE_NAMES order); zeros unless
        the engine was created with phase_timers=1."""
        ne, _ = self.batch_info(batch)
        ph = np.zeros((ne, NUM_PHASES), np.uint64)
        self._check(self.lib.pmbs_query_phase_cycles(self.ctx, batch, _p(ph)), "pmbs_query_phase_cycles")
        return ph

    def release_batch(self, batch):
        self._check(self.lib.pmbs_release_batch(self.ctx, batch), "pmbs_release_batch")

    # ---- snapshot predicates
    @staticmethod
    def _csr(box_offset, states, half):
        """CSR arrays for the snapshot calls; refuses ranges the arrays do not hold (the C
        calls trust the sizes)."""
        off = np.ascontiguousarray(box_offset, np.int32)
        st = np.ascontiguousarray(states, np.float32).reshape(-1, 13)
        h = np.ascontiguousarray(half, np.float32).reshape(-1, 3)
        if off.ndim != 1 or off.shape[0] < 1 or off[0] < 0 or np.any(np.diff(off) < 0) or \
                st.shape[0] < off[-1] or h.shape[0] < off[-1]:
            raise ValueError("box_offset does not describe the given state and half-extent arrays")
        return off, st, h

    def eval_pairs(self, box_offset, states, half, pusher_xy=None):
        off, st, h = self._csr(box_offset, states, half)
        ne = off.shape[0] - 1
        B = int(off[-1] - off[0])
        cap = self.cfg.pair_cap
        pairs = np.zeros((max(ne, 1), cap, 2), np.int32)
        npairs = np.zeros(max(ne, 1), np.int32)
        plane = np.zeros(max(B, 1), np.int32)
        nplane = np.zeros(max(ne, 1), np.int32)
        pusher = np.zeros(max(B, 1), np.int32)
        npusher = np.zeros(max(ne, 1), np.int32)
        pxy = None if pusher_xy is None else np.ascontiguousarray(pusher_xy, np.float32)
        self._check(self.lib.pmbs_eval_pairs(self.ctx, ne, _p(off), _p(st), _p(h), _p(pxy), _p(pairs), _p(npairs),
                                             _p(plane), _p(nplane), _p(pusher), _p(npusher)), "pmbs_eval_pairs")
        out = []
        for e in range(ne):
            b0 = int(off[e] - off[0])
            out.append((pairs[e, :npairs[e]].copy(), plane[b0:b0 + nplane[e]].copy(),
                        pusher[b0:b0 + npusher[e]].copy()))
        return out

    def eval_grasp(self, box_offset, states, half, target):
        off, st, h = self._csr(box_offset, states, half)
        ne = off.shape[0] - 1
        t = np.ascontiguousarray(target, np.int32)
        out = np.zeros(max(ne, 1), np.uint8)
        self._check(self.lib.pmbs_eval_grasp(self.ctx, ne, _p(off), _p(st), _p(h), _p(t), _p(out)), "pmbs_eval_grasp")
        return out[:ne].astype(bool)

    def eval_sample(self, box_offset, states, half, seeds, k):
        off, st, h = self._csr(box_offset, states, half)
        ne = off.shape[0] - 1
        sd = np.ascontiguousarray(seeds, np.uint64)
        push = np.zeros((max(ne, 1), 4), np.float32)
        att = np.zeros(max(ne, 1), np.int32)
        self._check(self.lib.pmbs_eval_sample(self.ctx, ne, _p(off), _p(st), _p(h), _p(sd), k, _p(push), _p(att)),
                    "pmbs_eval_sample")
        return att[:ne], push[:ne]

    def eval_start_blocked(self, box_offset, states, half, starts):
        off, st, h = self._csr(box_offset, states, half)
        ne = off.shape[0] - 1
        s2 = np.ascontiguousarray(starts, np.float32)
        out = np.zeros(max(ne, 1), np.uint8)
        self._check(self.lib.pmbs_eval_start_blocked(self.ctx, ne, _p(off), _p(st), _p(h), _p(s2), _p(out)),
                    "pmbs_eval_start_blocked")
        return out[:ne].astype(bool)

    # ---- launch shape and probes
    HM_CELLS = 144

    def render_heightmaps(self, box_offset, states, half):
        """Top-down workspace heightmaps [n_envs, 144 (y), 144 (x)] of a state snapshot."""
        box_offset, states, half = self._csr(box_offset, states, half)
        ne = box_offset.shape[0] - 1
        out = np.zeros((max(ne, 1), self.HM_CELLS, self.HM_CELLS), np.float32)
        self._check(self.lib.pmbs_render_heightmaps(self.ctx, ne, _p(box_offset), _p(states), _p(half), _p(out)),
                    "pmbs_render_heightmaps")
        return out[:ne]

    def render_heightmaps_device(self, n_envs, d_box_offset, d_states, d_half, d_out):
        self._check(self.lib.pmbs_render_heightmaps_device(self.ctx, n_envs, C.c_void_p(d_box_offset),
                                                           C.c_void_p(d_states), C.c_void_p(d_half),
                                                           C.c_void_p(d_out)), "pmbs_render_heightmaps_device")

    def eval_grasp_heightmap(self, box_offset, states, half, target, depth=0.02):
        box_offset, states, half = self._csr(box_offset, states, half)
        target = np.ascontiguousarray(target, np.int32)
        ne = box_offset.shape[0] - 1
        out = np.zeros(max(ne, 1), np.uint8)
        self._check(self.lib.pmbs_eval_grasp_heightmap(self.ctx, ne, _p(box_offset), _p(states), _p(half), _p(target),
                                                       float(depth), _p(out)), "pmbs_eval_grasp_heightmap")
        return out[:ne].astype(bool)

    def query_heightmaps(self, batch):
        ne, _ = self.batch_info(batch)
        out = np.zeros((max(ne, 1), self.HM_CELLS, self.HM_CELLS), np.float32)
        self._check(self.lib.pmbs_query_heightmaps(self.ctx, batch, _p(out)), "pmbs_query_heightmaps")
        return out[:ne]

    def launch_shape(self, max_boxes):
        g, w, ps, ms, sm = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        self._check(self.lib.pmbs_launch_shape(self.ctx, max_boxes, C.byref(g), C.byref(w), C.byref(ps),
                                               C.byref(ms), C.byref(sm)), "pmbs_launch_shape")
        return dict(lanes_per_env=g.value, warps_per_block=w.value, smem_points=ps.value,
                    smem_manifolds=ms.value, smem_bytes=sm.value)

    def set_launch_shape(self, lanes_per_env=0, warps_per_block=0, smem_points=-1, smem_manifolds=-1):
        self._check(self.lib.pmbs_set_launch_shape(self.ctx, lanes_per_env, warps_per_block, smem_points,
                                                   smem_manifolds), "pmbs_set_launch_shape")

    def fp32_peak(self) -> float:
        t = C.c_double()
        self._check(self.lib.pmbs_fp32_peak(self.ctx, C.byref(t)), "pmbs_fp32_peak")
        return t.value

    # ---- convenience
    def rollout(self, scene_ids, first_push, depth, seeds=None, child=False):
        b = self.rollout_pushes(scene_ids, first_push, depth, seeds)
        self.step(b, 0)
        out = self.query_cost(b, child_states=child)
        st, steps = self.query_states(b)
        out["state"], out["steps"] = st, steps
        out["events"] = self.query_events(b)
        if self.cfg.phase_timers:
            out["phase_cycles"] = self.query_phase_cycles(b)
        self.release_batch(b)
        return out


class Server:
    """Continuous-batching request server on an Engine (pmbs_server_* calls)."""

    def __init__(self, engine: Engine, n_streams: int = 8, max_inflight: int = 64):
        self.engine = engine
        self.lib = engine.lib
        self.sv = C.c_void_p()
        st = self.lib.pmbs_server_create(engine.ctx, n_streams, max_inflight, C.byref(self.sv))
        if st != PMBS_OK:
            raise PmbsError(st, "pmbs_server_create failed")
        self._n = {}

    def submit(self, scene_ids, first_push, depth, seeds=None) -> int:
        scene_ids = np.ascontiguousarray(scene_ids, np.int32)
        first_push = np.ascontiguousarray(first_push, np.float32)
        n = scene_ids.shape[0]
        seeds = np.ascontiguousarray(np.zeros(n, np.uint64) if seeds is None else seeds, np.uint64)
        t = C.c_int64()
        st = self.lib.pmbs_server_submit(self.sv, n, _p(scene_ids), _p(first_push), depth, _p(seeds), C.byref(t))
        if st != PMBS_OK:
            raise PmbsError(st, "pmbs_server_submit")
        self._n[t.value] = n
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        n = self._n[ticket]
        cost = np.zeros(max(n, 1), np.int32)
        reward = np.zeros(max(n, 1), np.float32)
        flags = np.zeros(max(n, 1), np.uint8)
        steps = np.zeros(max(n, 1), np.int32)
        lat = C.c_double()
        st = self.lib.pmbs_server_wait(self.sv, ticket, timeout_ms, _p(cost), _p(reward), _p(flags), _p(steps),
                                       C.byref(lat))
        if st in (PMBS_E_NOT_READY, PMBS_E_TIMEOUT):
            return None
        self._n.pop(ticket, None)
        if st != PMBS_OK:
            raise PmbsError(st, "pmbs_server_wait")
        return dict(cost=cost[:n], reward=reward[:n], flags=flags[:n], steps=steps[:n], latency_ms=lat.value)

    def cancel(self, ticket: int):
        """Drop a ticket that will never be waited for."""
        st = self.lib.pmbs_server_cancel(self.sv, ticket)
        self._n.pop(ticket, None)
        if st != PMBS_OK:
            raise PmbsError(st, "pmbs_server_cancel")

    def stats(self):
        out = np.zeros(11, np.float64)
        self.lib.pmbs_server_stats(self.sv, _p(out))
        keys = ["completed", "env_steps", "span_s", "p50_ms", "p99_ms", "mean_ms", "peak_bytes", "outstanding",
                "held_results", "resumes", "arena_used_bytes"]
        return dict(zip(keys, out.tolist()))

    def close(self):
        if self.sv:
            self.lib.pmbs_server_destroy(self.sv)
            self.sv = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# Module-level names matching the C ABI, for callers that manage handles themselves.
def __getattr__(name):
    if name.startswith("pmbs_"):
        return getattr(load(), name)
    raise AttributeError(name)
