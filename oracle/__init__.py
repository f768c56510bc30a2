"""FP64 CPU oracle of the batched push-rollout hot path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this package; the product library never does.  The oracle
shares no code with the CUDA engine: it is a separate C++ source (pmbs_oracle.cpp),
compiled with g++ -O2 -ffp-contract=off, with its own parameter struct.

Parity status: pinned by closed forms, invariants and brute force in the CPU tests,
except long multi-contact clutter trajectories (chaotic), whose parity is unpinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pmbs_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_FLOPS = os.path.join(_HERE, "liboracle_flops.so")
PHASES = ["per_body", "narrowphase", "contact_prep", "contact_solve", "other"]

EVENT_NAMES = ["substeps", "box_steps", "pair_tests", "sat", "face", "edge", "plane",
               "pusher", "points", "manifolds", "pgs_manifolds", "pgs_points",
               "push_evals", "sample_attempts", "clip_verts", "colours", "bb_points", "pgs_bb_points"]
F_GRASP1, F_INVALID_START, F_OUT_OF_WS, F_OVERFLOW, F_NOOP = 1, 2, 4, 8, 16


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("gravity", C.c_double * 3), ("table_half", C.c_double * 2),
                ("table_mu", C.c_double), ("pusher_mu", C.c_double),
                ("pusher_radius", C.c_double), ("pusher_z0", C.c_double), ("pusher_z1", C.c_double),
                ("pusher_speed", C.c_double), ("push_length", C.c_double), ("gamma", C.c_double),
                ("grasp_opening", C.c_double), ("grasp_clearance", C.c_double),
                ("finger_depth", C.c_double), ("finger_width", C.c_double),
                ("margin", C.c_double), ("slop", C.c_double), ("baumgarte", C.c_double),
                ("sample_clearance", C.c_double),
                ("substeps_per_push", C.c_int32), ("pgs_iters", C.c_int32),
                ("point_cap", C.c_int32), ("manifold_cap", C.c_int32), ("pair_cap", C.c_int32),
                ("grasp_angles", C.c_int32), ("sample_attempts", C.c_int32),
                ("contour_points", C.c_int32), ("warm_start", C.c_int32), ("warm_tolerance", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle shared library next to its source (idempotent)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fPIC", "-shared",
                               "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def build_flops(force: bool = False) -> str:
    """Compile the flop-counting build of the oracle (-DORACLE_COUNT_FLOPS)."""
    if force or not os.path.exists(_LIB_FLOPS) or os.path.getmtime(_LIB_FLOPS) < os.path.getmtime(_SRC):
        tmp = _LIB_FLOPS + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fPIC", "-shared",
                               "-pthread", "-DORACLE_COUNT_FLOPS", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_FLOPS)
    return _LIB_FLOPS


_lib = None
_lib_flops = None


def count_flops(state13, half, mass, mu, push, count, prm=None):
    """Run `count` substeps of one environment under `push` in the flop-counting build.
    Returns (flops by phase as a dict over PHASES, event counters [NEV])."""
    global _lib_flops
    if _lib_flops is None:
        L = C.CDLL(build_flops())
        L.oracle_count_flops.argtypes = [C.POINTER(Params), C.c_int] + [C.c_void_p] * 5 + \
            [C.c_int, C.c_void_p, C.c_void_p]
        _lib_flops = L
    prm = prm or params()
    st = np.ascontiguousarray(state13, np.float64)
    h, m, u = (np.ascontiguousarray(a, np.float32) for a in (half, mass, mu))
    p = np.ascontiguousarray(push, np.float64)
    f = np.zeros(5, np.uint64)
    ev = np.zeros(len(EVENT_NAMES), np.uint64)
    _lib_flops.oracle_count_flops(C.byref(prm), st.shape[0], _ptr(st), _ptr(h), _ptr(m), _ptr(u), _ptr(p), int(count),
                                  _ptr(f), _ptr(ev))
    return dict(zip(PHASES, f.astype(np.float64))), ev


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.POINTER
        vp = C.c_void_p
        L.oracle_default_params.argtypes = [P(Params)]
        L.oracle_splitmix64.argtypes = [P(C.c_uint64)]
        L.oracle_splitmix64.restype = C.c_uint64
        L.oracle_rollout.argtypes = [P(Params), C.c_int] + [vp] * 7 + [C.c_int, vp, C.c_int] + [vp] * 7
        L.oracle_run_substeps.argtypes = [P(Params), C.c_int, vp, vp, vp, vp, vp, C.c_int, C.c_int,
                                          C.c_int, vp]
        L.oracle_contacts.argtypes = [P(Params), C.c_int, vp, vp, vp, vp, vp, C.c_int, C.c_int, vp, vp, vp]
        L.oracle_box_box.argtypes = [vp, vp, vp, vp, C.c_double, vp, vp, vp, vp, vp]
        L.oracle_pairs.argtypes = [P(Params), C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_grasp.argtypes = [P(Params), C.c_int, C.c_int, vp, vp, C.c_int]
        L.oracle_sample_push.argtypes = [P(Params), C.c_int, C.c_int, vp, vp, C.c_uint64, C.c_int, vp]
        L.oracle_start_blocked.argtypes = [P(Params), C.c_int, C.c_int, vp, vp, C.c_float, C.c_float]
        L.oracle_heightmap.argtypes = [C.c_int, C.c_int, vp, vp, C.c_int, C.c_int, C.c_double, C.c_double,
                                       C.c_double, vp]
        L.oracle_heightmap.restype = None
        L.oracle_grasp_heightmap.argtypes = [P(Params), C.c_int, C.c_int, vp, vp, C.c_int, C.c_double]
        L.oracle_footprints.argtypes = [C.c_int, C.c_int, vp, vp, vp]
        _lib = L
    return _lib


def params(**overrides) -> Params:
    p = Params()
    lib().oracle_default_params(C.byref(p))
    for k, v in overrides.items():
        if k in ("gravity", "table_half"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a if shape is None else a.reshape(shape)


def splitmix64(state: int, count: int):
    s = C.c_uint64(state)
    return [int(lib().oracle_splitmix64(C.byref(s))) for _ in range(count)]


@dataclass
class RolloutResult:
    cost: np.ndarray
    reward: np.ndarray
    flags: np.ndarray
    steps: np.ndarray
    state: np.ndarray
    child: np.ndarray | None
    events: np.ndarray


def rollout(box_offset, state13, half, mass, mu, target, first_push, depth, seeds=None,
            prm: Params | None = None, threads: int = 1, child=False) -> RolloutResult:
    """Per-env rollouts; env e owns rows box_offset[e]:box_offset[e+1]."""
    prm = prm or params()
    box_offset = np.ascontiguousarray(box_offset, np.int32)
    ne = box_offset.shape[0] - 1
    B = int(box_offset[-1])
    state13, half, mass, mu = _f32(state13), _f32(half), _f32(mass), _f32(mu)
    target = np.ascontiguousarray(target, np.int32)
    first_push = _f32(first_push)
    seeds = np.ascontiguousarray(np.zeros(ne, np.uint64) if seeds is None else seeds, np.uint64)
    cost = np.zeros(ne, np.int32)
    reward = np.zeros(ne, np.float32)
    flags = np.zeros(ne, np.uint8)
    steps = np.zeros(ne, np.int32)
    st = np.zeros((B, 13), np.float64)
    ch = np.zeros((B, 13), np.float64) if child else None
    ev = np.zeros((ne, len(EVENT_NAMES)), np.uint64)
    lib().oracle_rollout(C.byref(prm), ne, _ptr(box_offset), _ptr(state13), _ptr(half), _ptr(mass),
                         _ptr(mu), _ptr(target), _ptr(first_push), depth, _ptr(seeds), threads,
                         _ptr(cost), _ptr(reward), _ptr(flags), _ptr(steps), _ptr(st), _ptr(ch), _ptr(ev))
    return RolloutResult(cost, reward, flags, steps, st, ch, ev)


def run_substeps(state13, half, mass, mu, push=None, s0=0, count=1, reverse=False,
                 prm: Params | None = None):
    """Advance one env `count` substeps; returns (state[n,13] float64, events, overflow)."""
    prm = prm or params()
    st = np.ascontiguousarray(state13, np.float64).copy()
    n = st.shape[0]
    half, mass, mu = _f32(half), _f32(mass), _f32(mu)
    pu = None if push is None else np.ascontiguousarray(push, np.float64)
    ev = np.zeros(len(EVENT_NAMES), np.uint64)
    ov = lib().oracle_run_substeps(C.byref(prm), n, _ptr(st), _ptr(half), _ptr(mass), _ptr(mu), _ptr(pu),
                                   s0, count, 1 if reverse else 0, _ptr(ev))
    return st, ev, bool(ov)


def contacts(state13, half, mass, mu, push=None, s=0, prm: Params | None = None, max_m=512):
    """Manifolds of one state: (info[m,4] = A,B,npts,colour; normal[m,3]; pts[m,4,4])."""
    prm = prm or params()
    st = np.ascontiguousarray(state13, np.float64)
    n = st.shape[0]
    half, mass, mu = _f32(half), _f32(mass), _f32(mu)
    pu = None if push is None else np.ascontiguousarray(push, np.float64)
    info = np.zeros((max_m, 4), np.int32)
    nrm = np.zeros((max_m, 3), np.float64)
    pts = np.zeros((max_m, 4, 4), np.float64)
    nm = lib().oracle_contacts(C.byref(prm), n, _ptr(st), _ptr(half), _ptr(mass), _ptr(mu), _ptr(pu),
                               s, max_m, _ptr(info), _ptr(nrm), _ptr(pts))
    nm = min(nm, max_m)
    return info[:nm], nrm[:nm], pts[:nm]


def box_box(sA, hA, sB, hB, margin=1e-3):
    sA = np.ascontiguousarray(sA, np.float64)
    sB = np.ascontiguousarray(sB, np.float64)
    hA, hB = _f32(hA), _f32(hB)
    sep = np.zeros(1)
    ax = np.zeros(1, np.int32)
    nrm = np.zeros(3)
    p = np.zeros((4, 3))
    d = np.zeros(4)
    npts = lib().oracle_box_box(_ptr(sA), _ptr(hA), _ptr(sB), _ptr(hB), margin, _ptr(sep), _ptr(ax),
                                _ptr(nrm), _ptr(p), _ptr(d))
    if npts < 0:
        return None
    return dict(sep=float(sep[0]), axis=int(ax[0]), n=nrm, pts=p[:npts], depth=d[:npts])


def pairs(state13, half, pusher_xy=None, f32=True, prm: Params | None = None):
    """(box-box pairs [k,2], plane boxes, pusher boxes, overflow) at one state."""
    prm = prm or params()
    st, half = _f32(state13), _f32(half)
    n = st.shape[0]
    cap = max(prm.pair_cap, 1)
    bb = np.zeros((cap, 2), np.int32)
    nb = np.zeros(1, np.int32)
    pl = np.zeros(max(n, 1), np.int32)
    npl = np.zeros(1, np.int32)
    pu = np.zeros(max(n, 1), np.int32)
    npu = np.zeros(1, np.int32)
    pxy = None if pusher_xy is None else _f32(pusher_xy)
    ov = lib().oracle_pairs(C.byref(prm), 1 if f32 else 0, n, _ptr(st), _ptr(half), _ptr(pxy), _ptr(bb),
                            _ptr(nb), _ptr(pl), _ptr(npl), _ptr(pu), _ptr(npu))
    return bb[:nb[0]].copy(), pl[:npl[0]].copy(), pu[:npu[0]].copy(), bool(ov)


def grasp(state13, half, target, f32=True, prm: Params | None = None) -> bool:
    prm = prm or params()
    st, half = _f32(state13), _f32(half)
    return bool(lib().oracle_grasp(C.byref(prm), 1 if f32 else 0, st.shape[0], _ptr(st), _ptr(half),
                                   int(target)))


def sample_push(state13, half, seed, k, f32=True, prm: Params | None = None):
    """(attempt index or -1, push[4] float32)."""
    prm = prm or params()
    st, half = _f32(state13), _f32(half)
    out = np.zeros(4, np.float32)
    a = lib().oracle_sample_push(C.byref(prm), 1 if f32 else 0, st.shape[0], _ptr(st), _ptr(half),
                                 C.c_uint64(int(seed)), int(k), _ptr(out))
    return a, out


def start_blocked(state13, half, sx, sy, f32=True, prm: Params | None = None) -> bool:
    prm = prm or params()
    st, half = _f32(state13), _f32(half)
    return bool(lib().oracle_start_blocked(C.byref(prm), 1 if f32 else 0, st.shape[0], _ptr(st),
                                           _ptr(half), C.c_float(sx), C.c_float(sy)))


# Workspace grid of Sec. V-A: 0.288 m x 0.288 m centred on the table, 144 x 144 cells.
HM_CELLS, HM_CELL, HM_X0 = 144, 0.002, -0.144


def heightmap(state13, half, f32=True, cells=HM_CELLS, cell=HM_CELL, x0=HM_X0, y0=HM_X0):
    """Top-down heightmap [rows y][cols x] of one state (binary32 twin when f32)."""
    st, half = _f32(state13), _f32(half)
    out = np.zeros((cells, cells), np.float32)
    lib().oracle_heightmap(1 if f32 else 0, st.shape[0], _ptr(st), _ptr(half), cells, cells, x0, y0, cell,
                           _ptr(out))
    return out


def grasp_heightmap(state13, half, target, depth=0.02, f32=True, prm: Params | None = None) -> bool:
    """Heightmap form of the grasp test: finger tips `depth` below the target's top."""
    prm = prm or params()
    st, half = _f32(state13), _f32(half)
    return bool(lib().oracle_grasp_heightmap(C.byref(prm), 1 if f32 else 0, st.shape[0], _ptr(st), _ptr(half),
                                             int(target), float(depth)))


def footprints(state13, half, f32=True):
    st, half = _f32(state13), _f32(half)
    out = np.zeros((st.shape[0], 8), np.float64)
    lib().oracle_footprints(1 if f32 else 0, st.shape[0], _ptr(st), _ptr(half), _ptr(out))
    return out
