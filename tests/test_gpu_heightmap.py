"""Top-down workspace heightmaps on the GPU (through the C ABI) against the oracle's
binary32 twin, bit for bit: random tilted snapshots, generated clutter, empty and 64-box
environments, a finished batch's final states, and the 4096-environment workload."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    from paper_2207_06649_b300 import pmbs
    e = pmbs.Engine(device=0, mem_budget_bytes=4 << 30)
    yield e
    e.close()


def _sg():
    from paper_2207_06649_b300 import scenegen
    return scenegen


def _bits_equal(a, b):
    return np.array_equal(np.ascontiguousarray(a, np.float32).view(np.uint32),
                          np.ascontiguousarray(b, np.float32).view(np.uint32))


def _tilted_snapshots(seed, n_envs, n_lo=1, n_hi=40):
    sg = _sg()
    rng = np.random.default_rng(seed)
    sts, hs, off = [], [], [0]
    for _ in range(n_envs):
        n = int(rng.integers(n_lo, n_hi + 1))
        pose, vel, half = sg.random_state_snapshot(rng, n, spread=0.02 + 0.004 * n, tilt=0.6)
        sts.append(np.concatenate([pose, vel], 1))
        hs.append(half)
        off.append(off[-1] + n)
    return np.array(off, np.int32), np.concatenate(sts).astype(np.float32), np.concatenate(hs).astype(np.float32)


@pytest.mark.parametrize("seed", [0, 1])
def test_heightmaps_bit_exact_on_tilted_snapshots(eng, orc, seed):
    off, st, h = _tilted_snapshots(seed, 48)
    got = eng.render_heightmaps(off, st, h)
    for e in range(len(off) - 1):
        a, b = off[e], off[e + 1]
        want = orc.heightmap(st[a:b], h[a:b], f32=True)
        assert _bits_equal(got[e], want), f"env {e}"
    assert (got > 0).any() and (got == 0).any()


def test_heightmaps_of_clutter_empty_and_64_boxes(eng, orc):
    sg = _sg()
    rng = np.random.default_rng(3)
    sc = sg.make_scene(rng, 64, half_lo=0.008, half_hi=0.02, region_half=0.19)
    st64 = sg.state13(sc).astype(np.float32)
    assert len(st64) == 64
    empty = np.zeros((0, 13), np.float32)
    off = np.array([0, 0, 64], np.int32)
    got = eng.render_heightmaps(off, np.concatenate([empty, st64]), sc.half)
    assert (got[0] == 0).all()
    assert _bits_equal(got[1], orc.heightmap(st64, sc.half, f32=True))
    # upright boxes: every covered cell shows a box top (centre height + half height)
    tops = set(np.round(st64[:, 2] + sc.half[:, 2], 6).tolist())
    assert set(np.round(np.unique(got[1][got[1] > 0]), 6).tolist()) <= tops


def test_batch_final_states_and_device_entry(eng, orc):
    import torch
    sg = _sg()
    scenes, pushes, seeds = sg.config_uneven(seed=51, n_envs=40, n_lo=5, n_hi=30, workers=1)
    ids = eng.load(scenes)
    b = eng.rollout_pushes(ids, pushes, 2, seeds)
    eng.step(b, 0)
    hm = eng.query_heightmaps(b)
    st, _ = eng.query_states(b)
    eng.release_batch(b)
    eng.free_scenes(ids)
    ref = eng.render_heightmaps(scenes.box_offset, st, scenes.half)
    assert _bits_equal(hm, ref)
    for e in (0, 17, 39):
        a, c = scenes.box_offset[e], scenes.box_offset[e + 1]
        assert _bits_equal(hm[e], orc.heightmap(st[a:c], scenes.half[a:c], f32=True))
    # device entry point on the same snapshot
    dev = torch.device("cuda", 0)
    d_off = torch.from_numpy(scenes.box_offset.astype(np.int32)).to(dev)
    d_st = torch.from_numpy(np.ascontiguousarray(st, np.float32)).to(dev)
    d_h = torch.from_numpy(np.ascontiguousarray(scenes.half, np.float32)).to(dev)
    d_out = torch.zeros((40, 144, 144), dtype=torch.float32, device=dev)
    eng.render_heightmaps_device(40, d_off.data_ptr(), d_st.data_ptr(), d_h.data_ptr(), d_out.data_ptr())
    torch.cuda.synchronize()
    assert _bits_equal(d_out.cpu().numpy(), ref)


def test_heightmaps_full_workload_sampled(eng, orc):
    """The 4096-environment uneven workload in one device call; sampled environments are
    compared with the oracle bit for bit, and every map is finite and non-negative."""
    import torch
    sg = _sg()
    scenes, _, _ = sg.config_uneven(seed=3, n_envs=4096)
    st = sg.state13(scenes).astype(np.float32)
    dev = torch.device("cuda", 0)
    d_off = torch.from_numpy(scenes.box_offset.astype(np.int32)).to(dev)
    d_st = torch.from_numpy(st).to(dev)
    d_h = torch.from_numpy(np.ascontiguousarray(scenes.half, np.float32)).to(dev)
    d_out = torch.empty((4096, 144, 144), dtype=torch.float32, device=dev)
    eng.render_heightmaps_device(4096, d_off.data_ptr(), d_st.data_ptr(), d_h.data_ptr(), d_out.data_ptr())
    torch.cuda.synchronize()
    out = d_out.cpu().numpy()
    assert np.isfinite(out).all() and (out >= 0).all()
    for e in np.random.default_rng(0).choice(4096, size=24, replace=False):
        a, c = scenes.box_offset[e], scenes.box_offset[e + 1]
        assert _bits_equal(out[e], orc.heightmap(st[a:c], scenes.half[a:c], f32=True)), e


@pytest.mark.parametrize("depth", [0.005, 0.02, 0.06])
def test_heightmap_grasp_decisions_bit_exact(eng, orc, depth):
    """Decisions of the heightmap grasp test on clutter (a random box of each scene as the
    target, poses jittered) equal the oracle's binary32 twin, and both outcomes occur."""
    sg = _sg()
    rng = np.random.default_rng(int(depth * 1000))
    parts = []
    for _ in range(96):
        n = int(rng.integers(3, 20))
        parts.append(sg.make_scene(rng, n, half_lo=0.01, half_hi=0.035, yaw_hi=np.pi / 2,
                                   density_scale=rng.uniform(0.3, 0.6)))
    sc = sg.concat(parts)
    st = sg.state13(sc).astype(np.float32)
    st[:, :2] += rng.normal(scale=0.002, size=(len(st), 2)).astype(np.float32)
    tgt = np.array([rng.integers(0, sc.box_offset[e + 1] - sc.box_offset[e]) for e in range(sc.n_scenes)], np.int32)
    got = eng.eval_grasp_heightmap(sc.box_offset, st, sc.half, tgt, depth=depth)
    want = [orc.grasp_heightmap(st[sc.box_offset[e]:sc.box_offset[e + 1]], sc.half[sc.box_offset[e]:sc.box_offset[e + 1]],
                                int(tgt[e]), depth=depth, f32=True) for e in range(sc.n_scenes)]
    assert got.tolist() == want
    assert 0 < sum(want) < len(want)
