"""The allocation-free rollout entry point (pmbs_rollout_noalloc), called through the C
ABI with caller-owned device buffers, against the context-based entry points.

This file is collected last so that a run stopping at the first failure has already run
every other test.  It must pass alone in a fresh process and after the other tests: the
entry point's per-device set-up happens on its first call in the process, whichever test
runs first.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_rollout_matches_context_rollout_on_two_calls():
    import torch
    from paper_2207_06649_b300 import pmbs, scenegen as sg
    lib = pmbs.load()
    scenes, pushes, seeds = sg.config_uneven(seed=21, n_envs=96, workers=1)
    eng = pmbs.Engine(device=0, mem_budget_bytes=1 << 30)
    ids = eng.load(scenes)
    ref = eng.rollout(ids, pushes, depth=3, seeds=seeds)
    eng.close()

    dev = torch.device("cuda", 0)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rec = np.concatenate([scenes.pose, scenes.vel, scenes.half, scenes.mass[:, None], scenes.mu[:, None]],
                         1).astype(np.float32)
    d_off, d_rec, d_tgt = to(scenes.box_offset), to(rec), to(scenes.target)
    d_push, d_seed = to(pushes.astype(np.float32)), to(seeds.view(np.int64))
    B, n = rec.shape[0], scenes.n_scenes
    cfg = pmbs.default_config(device=0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        # outputs start as garbage so that stale values cannot pass for results
        d_state = torch.full((B, 13), float("nan"), device=dev)
        d_cost = torch.full((n,), -7, dtype=torch.int32, device=dev)
        d_rew = torch.full((n,), -1.0, device=dev)
        d_flags = torch.full((n,), 255, dtype=torch.uint8, device=dev)
        st = lib.pmbs_rollout_noalloc(ctypes.byref(cfg), stream, n, _ptr(d_off), _ptr(d_rec), _ptr(d_tgt),
                                      _ptr(d_push), _ptr(d_seed), 3, _ptr(d_state), _ptr(d_cost), _ptr(d_rew),
                                      _ptr(d_flags))
        torch.cuda.synchronize()
        assert st == pmbs.PMBS_OK, f"call {call}: status {st}"
        assert np.array_equal(d_cost.cpu().numpy(), ref["cost"])
        assert np.array_equal(d_flags.cpu().numpy(), ref["flags"])
        # the same kernel on the same inputs: identical bits, whatever the launch shape
        assert np.array_equal(d_rew.cpu().numpy().view(np.uint32), ref["reward"].view(np.uint32))
        assert np.array_equal(d_state.cpu().numpy().view(np.uint32), ref["state"].view(np.uint32))


def test_noalloc_rejects_requests_beyond_its_scratch():
    from paper_2207_06649_b300 import pmbs
    lib = pmbs.load()
    cfg = pmbs.default_config(device=0)
    null = ctypes.c_void_p()
    st = lib.pmbs_rollout_noalloc(ctypes.byref(cfg), null, 16385, null, null, null, null, null, 1, null, null,
                                  null, null)
    assert st == pmbs.PMBS_E_INVALID
    big = pmbs.default_config(device=0, max_boxes_per_env=65)
    st = lib.pmbs_rollout_noalloc(ctypes.byref(big), null, 1, null, null, null, null, null, 1, null, null, null,
                                  null)
    assert st == pmbs.PMBS_E_INVALID


def test_noalloc_with_cylinders_matches_context_rollout():
    """cfg.cylinders = 1 runs the solver with the cylinder contact paths: the cylinder
    workload's results equal the context entry point's."""
    import torch
    from paper_2207_06649_b300 import pmbs, scenegen as sg
    lib = pmbs.load()
    scenes, pushes, seeds = sg.config_cylinders(seed=23, n_envs=64, workers=1)
    eng = pmbs.Engine(device=0, mem_budget_bytes=1 << 30)
    ids = eng.load(scenes)
    ref = eng.rollout(ids, pushes, depth=2, seeds=seeds)
    eng.close()
    dev = torch.device("cuda", 0)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    rec = np.concatenate([scenes.pose, scenes.vel, scenes.half, scenes.mass[:, None], scenes.mu[:, None]],
                         1).astype(np.float32)
    B, n = rec.shape[0], scenes.n_scenes
    d_state = torch.full((B, 13), float("nan"), device=dev)
    d_cost = torch.full((n,), -7, dtype=torch.int32, device=dev)
    d_rew = torch.full((n,), -1.0, device=dev)
    d_flags = torch.full((n,), 255, dtype=torch.uint8, device=dev)
    cfg = pmbs.default_config(device=0, cylinders=1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = [to(scenes.box_offset), to(rec), to(scenes.target), to(pushes.astype(np.float32)), to(seeds.view(np.int64))]
    st = lib.pmbs_rollout_noalloc(ctypes.byref(cfg), stream, n, *[_ptr(a) for a in args], 2, _ptr(d_state),
                                  _ptr(d_cost), _ptr(d_rew), _ptr(d_flags))
    torch.cuda.synchronize()
    assert st == pmbs.PMBS_OK
    assert np.array_equal(d_cost.cpu().numpy(), ref["cost"])
    assert np.array_equal(d_flags.cpu().numpy(), ref["flags"])
    assert np.array_equal(d_state.cpu().numpy().view(np.uint32), ref["state"].view(np.uint32))


def test_noalloc_refuses_cylinder_rows_without_the_cylinder_solver():
    """cfg.cylinders = 0 with a cylinder row, or a cylinder row whose radii differ, makes
    that environment invalid: the call returns PMBS_E_INVALID and the other environments
    are simulated as usual."""
    import torch
    from paper_2207_06649_b300 import pmbs, scenegen as sg
    lib = pmbs.load()
    scenes, pushes, seeds = sg.config_uneven(seed=25, n_envs=8, n_lo=5, n_hi=10, workers=1)
    eng = pmbs.Engine(device=0, mem_budget_bytes=1 << 30)
    ref = eng.rollout(eng.load(scenes), pushes, depth=1)
    eng.close()
    dev = torch.device("cuda", 0)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    half = scenes.half.copy()
    a0 = scenes.box_offset[3]
    half[a0] = (0.02, -0.02, 0.02)   # env 3 holds a cylinder
    rec = np.concatenate([scenes.pose, scenes.vel, half, scenes.mass[:, None], scenes.mu[:, None]], 1).astype(np.float32)
    B, n = rec.shape[0], scenes.n_scenes
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for cyl_flag, row in ((0, (0.02, -0.02, 0.02)), (1, (0.02, -0.01, 0.02))):
        rec[a0, 13:16] = row
        d_state = torch.zeros((B, 13), device=dev)
        d_cost = torch.zeros((n,), dtype=torch.int32, device=dev)
        d_rew = torch.zeros((n,), device=dev)
        d_flags = torch.zeros((n,), dtype=torch.uint8, device=dev)
        cfg = pmbs.default_config(device=0, cylinders=cyl_flag)
        args = [to(scenes.box_offset), to(rec), to(scenes.target), to(pushes.astype(np.float32)), to(seeds.view(np.int64))]
        st = lib.pmbs_rollout_noalloc(ctypes.byref(cfg), stream, n, *[_ptr(a) for a in args], 1, _ptr(d_state),
                                      _ptr(d_cost), _ptr(d_rew), _ptr(d_flags))
        torch.cuda.synchronize()
        assert st == pmbs.PMBS_E_INVALID
        got = d_cost.cpu().numpy()
        ok = np.arange(n) != 3
        assert np.array_equal(got[ok], ref["cost"][ok])


def _records(scenes, half=None):
    h = scenes.half if half is None else half
    return np.concatenate([scenes.pose, scenes.vel, h, scenes.mass[:, None], scenes.mu[:, None]], 1).astype(np.float32)


def _call(lib, cfg, scenes, rec, pushes, seeds, depth):
    import torch
    from paper_2207_06649_b300 import pmbs
    dev = torch.device("cuda", 0)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    B, n = rec.shape[0], scenes.n_scenes
    out = dict(state=torch.full((B, 13), float("nan"), device=dev), cost=torch.full((n,), -7, dtype=torch.int32, device=dev),
               reward=torch.full((n,), -1.0, device=dev), flags=torch.full((n,), 255, dtype=torch.uint8, device=dev))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = [to(scenes.box_offset), to(rec), to(scenes.target), to(pushes.astype(np.float32)), to(seeds.view(np.int64))]
    st = lib.pmbs_rollout_noalloc(ctypes.byref(cfg), stream, scenes.n_scenes, *[_ptr(a) for a in args], depth,
                                  _ptr(out["state"]), _ptr(out["cost"]), _ptr(out["reward"]), _ptr(out["flags"]))
    torch.cuda.synchronize()
    return st, {k: v.cpu().numpy() for k, v in out.items()}


def test_noalloc_refuses_rows_that_scene_loading_refuses():
    """An environment with a zero-mass row, one with a NaN first push, one with a
    non-unit quaternion and one with a negative friction coefficient are not simulated
    (PMBS_E_INVALID, their outputs untouched); every other environment equals the context
    entry point's result bit for bit."""
    from paper_2207_06649_b300 import pmbs, scenegen as sg
    lib = pmbs.load()
    scenes, pushes, seeds = sg.config_uneven(seed=27, n_envs=12, n_lo=5, n_hi=12, workers=1)
    eng = pmbs.Engine(device=0, mem_budget_bytes=1 << 30)
    ref = eng.rollout(eng.load(scenes), pushes, depth=2, seeds=seeds)
    eng.close()
    rec = _records(scenes)
    pushes = pushes.astype(np.float32).copy()
    off = scenes.box_offset
    rec[off[2] + 1, 16] = 0.0            # env 2: zero mass
    pushes[5, 1] = np.nan                # env 5: NaN push
    rec[off[7], 3] = 0.9                 # env 7: |q| = 0.9 (with zero vector part)
    rec[off[7], 4:7] = 0.0
    rec[off[9] + 2, 17] = -0.1           # env 9: negative mu
    bad = np.zeros(scenes.n_scenes, bool)
    bad[[2, 5, 7, 9]] = True
    st, out = _call(lib, pmbs.default_config(device=0), scenes, rec, pushes, seeds, 2)
    assert st == pmbs.PMBS_E_INVALID
    assert np.all(out["cost"][bad] == -7) and np.all(out["flags"][bad] == 255)
    assert np.array_equal(out["cost"][~bad], ref["cost"][~bad])
    assert np.array_equal(out["flags"][~bad], ref["flags"][~bad])
    for e in np.nonzero(~bad)[0]:
        a, z = off[e], off[e + 1]
        assert np.array_equal(out["state"][a:z].view(np.uint32), ref["state"][a:z].view(np.uint32))
    for e in np.nonzero(bad)[0]:
        assert np.isnan(out["state"][off[e]:off[e + 1]]).all()


def test_noalloc_reports_the_watchdog():
    """A run-time limit of a few SM cycles stops every environment after its first
    substep: the call returns PMBS_E_TIMEOUT (no hang, no fault) and the library stays
    usable: the next call with the default limit equals the context entry point's."""
    from paper_2207_06649_b300 import pmbs, scenegen as sg
    lib = pmbs.load()
    scenes, pushes, seeds = sg.config_uneven(seed=29, n_envs=16, n_lo=5, n_hi=12, workers=1)
    rec = _records(scenes)
    st, _ = _call(lib, pmbs.default_config(device=0, watchdog_ms=1e-6), scenes, rec, pushes, seeds, 2)
    assert st == pmbs.PMBS_E_TIMEOUT
    eng = pmbs.Engine(device=0, mem_budget_bytes=1 << 30)
    ref = eng.rollout(eng.load(scenes), pushes, depth=2, seeds=seeds)
    eng.close()
    st, out = _call(lib, pmbs.default_config(device=0), scenes, rec, pushes, seeds, 2)
    assert st == pmbs.PMBS_OK
    assert np.array_equal(out["cost"], ref["cost"])
    assert np.array_equal(out["state"].view(np.uint32), ref["state"].view(np.uint32))
