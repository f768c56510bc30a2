"""PMBS planner on the CUDA engine (GPU backend over the C ABI)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_gpu_planner_plans_and_frees_its_scenes():
    from paper_2207_06649_b300 import pmbs, planner as P, scenegen as sg
    eng = pmbs.Engine(device=0, mem_budget_bytes=1 << 30)
    sc = sg.config_planning(0)
    st = sg.state13(sc)
    be = P.GpuBackend(eng, sc.half, sc.mass, sc.mu)
    assert not be.graspable(st, sc.half, 0)
    root = be.load_state(st, sc.half, 0)
    pl = P.Planner(be, sc.half, 0, n_envs=128, t_max=30.0, max_iterations=3, seed=0)
    action, info = pl.plan(root, st)
    assert action is not None and action.shape == (4,)
    # the early-stop rule of Alg. 1 may end planning before the iteration cap
    assert 1 <= info.iterations <= 3 and info.rollouts == info.iterations * 128 and info.nodes > 1
    # every child scene the planner registered has been released: freeing them again fails
    ids = eng.load(sc)
    assert ids[0] != root
    with pytest.raises(pmbs.PmbsError):
        eng.free_scenes(np.array([int(root) + 1], np.int32) if int(ids[0]) != int(root) + 1
                        else np.array([int(root) + 2], np.int32))
    be.release([root])
    eng.free_scenes(ids)
    eng.close()


def test_serial_and_parallel_planners_share_one_engine():
    from paper_2207_06649_b300 import pmbs, planner as P, scenegen as sg
    eng = pmbs.Engine(device=0, mem_budget_bytes=1 << 30)
    sc = sg.config_planning(1)
    st = sg.state13(sc)
    be = P.GpuBackend(eng, sc.half, sc.mass, sc.mu)
    root = be.load_state(st, sc.half, 0)
    serial = P.Planner(be, sc.half, 0, n_envs=1, t_max=30.0, max_iterations=4, seed=0)
    a1, i1 = serial.plan(root, st)
    par = P.Planner(be, sc.half, 0, n_envs=64, t_max=30.0, max_iterations=2, seed=0)
    a2, i2 = par.plan(root, st)
    assert i1.rollouts == i1.iterations and 1 <= i1.iterations <= 4
    assert i2.rollouts == 64 * i2.iterations and 1 <= i2.iterations <= 2
    assert a1 is not None and a2 is not None
    be.release([root])
    eng.close()


def test_planner_retrieves_a_cylinder_target():
    """A cylinder target ringed by six slabs (not graspable at the start): the planner's
    host contour sampler works on the cylinder footprint, PMBS plans on the cylinder
    solver, and the episode either retrieves the target or exhausts its pushes."""
    import math
    from paper_2207_06649_b300 import pmbs, planner as P, scenegen as sg
    eng = pmbs.Engine(device=0, mem_budget_bytes=1 << 30)
    rows = [(0.0, 0.0, 0.03)]
    half = [sg.cylinder_half(0.025, 0.03)]
    # a ring of tall slabs around the target leaves no room for the fingers
    for k in range(6):
        a = k * math.pi / 3
        rows.append((0.05 * math.cos(a), 0.05 * math.sin(a), 0.04, a))
        half.append(np.array([0.008, 0.02, 0.04], np.float32))
    st = np.zeros((len(rows), 13), np.float32)
    for i, r in enumerate(rows):
        st[i, :3] = r[:3]
        yaw = r[3] if len(r) > 3 else 0.0
        st[i, 3], st[i, 6] = math.cos(yaw / 2), math.sin(yaw / 2)
    half = np.stack(half).astype(np.float32)
    mass = np.full(len(rows), 0.1, np.float32)
    mu = np.full(len(rows), 0.5, np.float32)
    be = P.GpuBackend(eng, half, mass, mu)
    assert not be.graspable(st, half, 0)
    cands = P.contour_candidates(st, half, 0)
    assert len(cands) > 0 and np.isfinite(cands).all()
    res = P.run_episode(be, st, half, 0, lambda: P.Planner(be, half, 0, n_envs=128, t_max=20.0, max_iterations=2,
                                                           seed=0), max_actions=3)
    assert 1 <= res["actions"] <= 4 and len(res["plan_s"]) >= 1
    eng.close()
