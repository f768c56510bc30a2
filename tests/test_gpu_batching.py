"""Batching and serving on the GPU (through the C ABI): graph stepping, autotuning and the
continuous-batching server produce exactly the results of a plain launch; the server admits
by memory and reports latency statistics."""
import threading

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _pm():
    from paper_2207_06649_b300 import pmbs
    return pmbs


@pytest.fixture(scope="module")
def work():
    from paper_2207_06649_b300 import scenegen as sg
    scenes, pushes, seeds = sg.config_uneven(seed=31, n_envs=160, workers=1)
    return scenes, pushes, seeds


def test_graph_stepping_equals_one_launch(work):
    pm = _pm()
    scenes, pushes, seeds = work
    eng = pm.Engine(device=0, mem_budget_bytes=1 << 30)
    ids = eng.load(scenes)
    ref = eng.rollout(ids, pushes, depth=3, seeds=seeds)
    for k in (240, 97):
        b = eng.rollout_pushes(ids, pushes, 3, seeds)
        eng.step_graph(b, k)
        r = eng.query_cost(b)
        st, steps = eng.query_states(b)
        eng.release_batch(b)
        assert np.array_equal(r["cost"], ref["cost"]) and np.array_equal(r["flags"], ref["flags"])
        assert np.array_equal(st.view(np.uint32), ref["state"].view(np.uint32))
        assert np.array_equal(steps, ref["steps"])
    eng.close()


def test_autotune_picks_a_shape_and_keeps_results(work):
    pm = _pm()
    scenes, pushes, seeds = work
    eng = pm.Engine(device=0, mem_budget_bytes=1 << 30)
    ids = eng.load(scenes)
    ref = eng.rollout(ids, pushes, depth=2, seeds=seeds)
    best = eng.autotune(ids, pushes, 2, seeds, substeps=60)
    assert best["lanes_per_env"] in (8, 16, 32) and best["warps_per_block"] in (1, 2, 4) and best["ms"] > 0
    assert 0 <= best["smem_manifolds"] <= 40 and best["substeps_per_launch"] in (0, 240, 60)
    shape = eng.launch_shape(int(scenes.counts().max()))
    assert shape["lanes_per_env"] == best["lanes_per_env"]
    out = eng.rollout(ids, pushes, depth=2, seeds=seeds)
    assert np.array_equal(out["state"].view(np.uint32), ref["state"].view(np.uint32))
    eng.close()


def _requests(scenes, pushes, seeds, sizes, seed=0):
    rng = np.random.default_rng(seed)
    reqs = []
    for n in sizes:
        pick = rng.integers(0, scenes.n_scenes, size=n)
        reqs.append((pick, pushes[pick], rng.integers(0, 2 ** 63, size=n, dtype=np.uint64)))
    return reqs


def test_server_results_identical_alone_and_in_mix(work):
    pm = _pm()
    scenes, pushes, seeds = work
    eng = pm.Engine(device=0, mem_budget_bytes=2 << 30)
    ids = eng.load(scenes)
    sv = pm.Server(eng, n_streams=4, max_inflight=16)
    reqs = _requests(scenes, pushes, seeds, [32, 300, 64, 500, 40, 128, 33, 250])
    alone = []
    for pick, pu, sd in reqs:
        t = sv.submit(ids[pick], pu, 3, sd)
        alone.append(sv.wait(t))
    # all at once, from several threads
    tickets = [None] * len(reqs)

    def go(i):
        pick, pu, sd = reqs[i]
        tickets[i] = sv.submit(ids[pick], pu, 3, sd)

    th = [threading.Thread(target=go, args=(i,)) for i in range(len(reqs))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    mixed = [sv.wait(t) for t in tickets]
    for a, m in zip(alone, mixed):
        for k in ("cost", "flags", "steps"):
            assert np.array_equal(a[k], m[k]), k
        assert np.array_equal(a["reward"].view(np.uint32), m["reward"].view(np.uint32))
    # the same as the context's own entry points
    pick, pu, sd = reqs[1]
    direct = eng.rollout(ids[pick], pu, depth=3, seeds=sd)
    assert np.array_equal(direct["cost"], alone[1]["cost"])
    st = sv.stats()
    assert st["completed"] == 2 * len(reqs) and st["p50_ms"] <= st["p99_ms"]
    assert st["env_steps"] == sum(int(a["steps"].sum()) for a in alone + mixed)
    sv.close()
    eng.close()


def test_server_admits_by_memory(work):
    pm = _pm()
    scenes, pushes, seeds = work
    # a small arena: only a few batches fit at once; the rest wait for memory
    budget = 160 << 20
    eng = pm.Engine(device=0, mem_budget_bytes=budget)
    ids = eng.load(scenes)
    sv = pm.Server(eng, n_streams=4, max_inflight=64)
    reqs = _requests(scenes, pushes, seeds, [400] * 10, seed=3)
    tickets = [sv.submit(ids[p], pu, 2, sd) for p, pu, sd in reqs]
    outs = [sv.wait(t, timeout_ms=120000) for t in tickets]
    assert all(o is not None for o in outs)
    st = sv.stats()
    assert st["peak_bytes"] <= budget
    assert st["completed"] == len(reqs)
    # a request that can never fit is refused, not queued forever
    big = np.repeat(ids[:1], 60000)
    with pytest.raises(pm.PmbsError) as ei:
        t = sv.submit(big, np.repeat(pushes[:1], 60000, 0), 2, np.zeros(60000, np.uint64))
        sv.wait(t, timeout_ms=60000)
    assert ei.value.status in (pm.PMBS_E_OOM, pm.PMBS_E_INVALID)
    sv.close()
    eng.close()
