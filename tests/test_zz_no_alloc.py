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
        assert np.allclose(d_rew.cpu().numpy(), ref["reward"], rtol=1e-6, atol=0)
        assert np.allclose(d_state.cpu().numpy(), ref["state"], atol=1e-6, rtol=0)


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
