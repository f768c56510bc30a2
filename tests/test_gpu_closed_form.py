"""GPU engine (through the C ABI) against closed forms and conservation laws, independent of
the oracle.

- Free flight under gravity (Sec. IV-C's rollouts integrate rigid bodies semi-implicitly):
  after k substeps v_k = v0 + k g dt and x_k = x0 + k dt v0 + g dt^2 k(k+1)/2; a cube's
  angular velocity stays constant and its orientation turns by 2 atan(|w| dt / 2) per
  substep about w (renormalised first-order quaternion update).
- Collisions without gravity or table contact: every contact impulse acts with opposite
  signs on two boxes at one point, so total linear momentum sum m v and, for cubes
  (isotropic inertia, so free rotation conserves I w), total angular momentum
  sum (x cross m v + I w) about the origin are conserved up to FP32 rounding.  A wrong
  sign, lever arm or inertia term in the solver breaks these at order one.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

DT = 1.0 / 240.0


def _pm():
    from paper_2207_06649_b300 import pmbs
    return pmbs


def _sg():
    from paper_2207_06649_b300 import scenegen
    return scenegen


def _scenes(rows_per_env, half_per_env, mass_per_env):
    """Scenes from per-env lists of 13-float rows (pose, velocity)."""
    sg = _sg()
    rows = np.concatenate(rows_per_env).astype(np.float32)
    off = np.concatenate([[0], np.cumsum([len(r) for r in rows_per_env])]).astype(np.int32)
    n = len(rows)
    return sg.Scenes(off, rows[:, :7].copy(), rows[:, 7:].copy(),
                     np.concatenate(half_per_env).astype(np.float32),
                     np.concatenate(mass_per_env).astype(np.float32), np.full(n, 0.5, np.float32),
                     np.zeros(len(rows_per_env), np.int32))


def _run(eng, sc, count):
    ids = eng.load(sc)
    far = np.tile(np.array([[0.19, 0.19, 0.19, 0.19]], np.float32), (sc.n_scenes, 1))  # no pusher motion
    b = eng.rollout_pushes(ids, far, 1)
    eng.step(b, count)
    st, steps = eng.query_states(b)
    ev = eng.query_events(b)
    eng.release_batch(b)
    eng.free_scenes(ids)
    assert (steps == count).all()
    return st.astype(np.float64), ev


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def test_free_flight_closed_form():
    pm = _pm()
    rng = np.random.default_rng(5)
    n_envs, k = 64, 120
    rows, halves, masses = [], [], []
    for _ in range(n_envs):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        x = [rng.uniform(-0.12, 0.12), rng.uniform(-0.12, 0.12), rng.uniform(1.5, 2.0)]
        v = [rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1), rng.uniform(0.0, 1.0)]
        w = rng.uniform(-6, 6, size=3)
        rows.append(np.array([x + list(q) + v + list(w)]))
        h = rng.uniform(0.01, 0.03)
        halves.append(np.full((1, 3), h))
        masses.append(np.array([rng.uniform(0.05, 0.3)]))
    sc = _scenes(rows, halves, masses)
    eng = pm.Engine(device=0, mem_budget_bytes=256 << 20)
    st, ev = _run(eng, sc, k)
    eng.close()
    s0 = np.concatenate(rows).astype(np.float32).astype(np.float64)
    g = np.array([0.0, 0.0, -9.81])
    v_want = s0[:, 7:10] + k * DT * g
    x_want = s0[:, :3] + k * DT * s0[:, 7:10] + g * DT * DT * k * (k + 1) / 2
    # FP32: ~k roundings of |x| <= 2.5 m at 2^-24 each
    assert np.abs(st[:, 7:10] - v_want).max() <= 2e-5
    assert np.abs(st[:, :3] - x_want).max() <= 4e-5
    assert np.abs(st[:, 10:13] - s0[:, 10:13]).max() <= 1e-6 * 6
    for i in range(n_envs):
        w = s0[i, 10:13]
        wn = np.linalg.norm(w)
        ang = k * 2 * math.atan(wn * DT / 2)
        r = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * w / wn])
        q_want = _qmul(r, s0[i, 3:7] / np.linalg.norm(s0[i, 3:7]))
        # angle of the relative rotation from its vector part (well conditioned near zero);
        # FP32 rounding of ~k quaternion updates: ~1e-6 rad
        q = st[i, 3:7] / np.linalg.norm(st[i, 3:7])
        rel = _qmul(q_want * np.array([1, -1, -1, -1]), q)
        assert 2 * math.asin(min(1.0, float(np.linalg.norm(rel[1:])))) <= 2e-5, i
    # no contact of any kind was generated
    names = list(pm.EVENT_NAMES)
    assert ev[:, names.index("sat")].sum() == 0 and ev[:, names.index("plane")].sum() == 0


def _cube_pairs(rng, n_envs):
    rows, halves, masses = [], [], []
    for _ in range(n_envs):
        ha, hb = rng.uniform(0.015, 0.03, size=2)
        qa, qb = rng.normal(size=4), rng.normal(size=4)
        qa /= np.linalg.norm(qa)
        qb /= np.linalg.norm(qb)
        # bounding spheres 5 mm apart along a random direction, approaching with an offset
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        sep = math.sqrt(3) * (ha + hb) + 0.005
        c = np.array([0.0, 0.0, 2.0])   # far above the table and the pusher for the whole second
        xa = c - d * sep / 2
        xb = c + d * sep / 2
        off = rng.normal(size=3) * 0.3 * min(ha, hb)
        speed = rng.uniform(0.5, 1.5)
        va = d * speed * 0.5 + rng.normal(size=3) * 0.05
        vb = -d * speed * 0.5 + rng.normal(size=3) * 0.05
        rows.append(np.array([list(xa + off) + list(qa) + list(va) + list(rng.uniform(-3, 3, 3)),
                              list(xb - off) + list(qb) + list(vb) + list(rng.uniform(-3, 3, 3))]))
        halves.append(np.array([[ha] * 3, [hb] * 3]))
        masses.append(rng.uniform(0.05, 0.3, size=2))
    return rows, halves, masses


def _momenta(st, half, mass):
    m = mass[:, None]
    p = (m * st[:, 7:10]).reshape(-1, 2, 3).sum(1)
    inertia = (2.0 / 3.0) * mass * half[:, 0] ** 2
    ang = np.cross(st[:, :3], m * st[:, 7:10]) + inertia[:, None] * st[:, 10:13]
    return p, ang.reshape(-1, 2, 3).sum(1)


def test_collisions_conserve_linear_and_angular_momentum():
    pm = _pm()
    rng = np.random.default_rng(11)
    n_envs, k = 96, 240
    rows, halves, masses = _cube_pairs(rng, n_envs)
    sc = _scenes(rows, halves, masses)
    eng = pm.Engine(device=0, mem_budget_bytes=256 << 20, gravity=(0.0, 0.0, 0.0))
    st, ev = _run(eng, sc, k)
    eng.close()
    s0 = np.concatenate(rows).astype(np.float32).astype(np.float64)
    half = sc.half.astype(np.float64)
    mass = sc.mass.astype(np.float64)
    p0, l0 = _momenta(s0, half, mass)
    p1, l1 = _momenta(st, half, mass)
    # every pair collided: velocities changed at order one
    dv = np.abs(st[:, 7:10] - s0[:, 7:10]).reshape(-1, 2, 3).max(axis=(1, 2))
    names = list(pm.EVENT_NAMES)
    assert (dv > 0.05).mean() > 0.9 and ev[:, names.index("pgs_bb_points")].sum() > 0
    # scale of the momenta: sum of |m v| (and |x m v| + |I w|) over both boxes
    pscale = (mass[:, None] * np.abs(s0[:, 7:10])).reshape(-1, 2, 3).sum(1).max(1)
    lscale = (np.linalg.norm(s0[:, :3], axis=1) * mass * np.linalg.norm(s0[:, 7:10], axis=1)
              + (2.0 / 3.0) * mass * half[:, 0] ** 2 * np.linalg.norm(s0[:, 10:13], axis=1)).reshape(-1, 2).sum(1)
    ep = (np.abs(p1 - p0).max(1) / pscale)
    el = (np.abs(l1 - l0).max(1) / lscale)
    print(f"momentum relative error: linear max {ep.max():.3g} median {np.median(ep):.3g}; "
          f"angular max {el.max():.3g} median {np.median(el):.3g}")
    # measured on a B300: linear max 1.1e-6, angular max 4.8e-6 (FP32 rounding of ~10^4
    # impulse applications per pair); the bounds leave a factor of ten
    assert ep.max() <= 2e-5
    assert el.max() <= 5e-5
    # no box touched the plane (no gravity, boxes stay above z = 1)
    assert ev[:, names.index("plane")].sum() == 0
