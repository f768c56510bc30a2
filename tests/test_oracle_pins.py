"""Pins of the FP64 oracle against closed forms, invariants and brute force (CPU only).

Each test fixes a property the method's definition implies, computed independently of
the oracle's code, so that a dropped term, a wrong sign or a transposed operand in the
oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from tests import _geom as G

G_ACC = 9.81
DT = 1.0 / 240.0


def one_box(half=(0.02, 0.02, 0.02), mass=0.1, mu=0.5):
    return (np.array([half], np.float32), np.array([mass], np.float32), np.array([mu], np.float32))


# ---------------------------------------------------------------- random numbers
def test_splitmix64_published_vectors(orc):
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")
    lines = [l.split("#")[0].strip() for l in open(path)]
    lines = [l for l in lines if l]
    seed = int(lines[0].split()[1])
    want = [int(x) for x in lines[1:]]
    assert orc.splitmix64(seed, len(want)) == want


# ---------------------------------------------------------------- integration
def test_free_flight_matches_discrete_closed_form(orc):
    """Semi-implicit Euler under gravity: z_k = z0 + v0 k dt - g dt^2 k(k+1)/2 exactly
    (the continuous parabola differs by g dt^2 k / 2)."""
    h, m, mu = one_box()
    s = G.box_row(0.01, -0.02, 5.0, v=(0.3, -0.1, 0.5))[None]
    for k in (1, 7, 240):
        st, _, _ = orc.run_substeps(s, h, m, mu, count=k)
        z = 5.0 + 0.5 * k * DT - G_ACC * DT * DT * k * (k + 1) / 2
        assert abs(st[0, 2] - z) < 1e-12
        assert abs(st[0, 0] - (0.01 + 0.3 * k * DT)) < 1e-12
        assert abs(st[0, 1] - (-0.02 - 0.1 * k * DT)) < 1e-12
        assert abs(st[0, 9] - (0.5 - G_ACC * DT * k)) < 1e-12


@pytest.mark.parametrize("axis", [(0, 0, 1), (1, 2, -0.5)])
def test_rotation_update_closed_form(orc, axis):
    """q <- normalize(q + dt/2 (0,w) x q) about a fixed axis advances the angle by exactly
    2 atan(|w| dt / 2) per substep and keeps the axis."""
    h, m, mu = one_box()
    a = np.array(axis, float) / np.linalg.norm(axis)
    wmag = 3.0
    s = G.box_row(0, 0, 1.0, w=tuple(a * wmag))[None]
    k = 100
    st, _, _ = orc.run_substeps(s, h, m, mu, count=k, prm=orc.params(gravity=(0, 0, 0)))
    ang = k * 2 * math.atan(wmag * DT / 2)
    want = G.quat_from_rotvec(a * ang)
    assert np.allclose(st[0, 3:7], want, atol=1e-12)
    assert np.allclose(st[0, 10:13], a * wmag, atol=1e-12)


# ---------------------------------------------------------------- contact behaviour
def test_resting_box_stays_at_rest(orc):
    h, m, mu = one_box((0.02, 0.03, 0.015), 0.12)
    s = G.box_row(0.05, -0.02, 0.015)[None]
    p = orc.params()
    st, _, _ = orc.run_substeps(s, h, m, mu, count=240)
    pen = 0.015 - st[0, 2]
    assert pen <= p.slop + 1e-4
    assert np.linalg.norm(st[0, 7:10]) <= 1e-3
    ang = 2 * math.acos(min(1.0, abs(st[0, 3])))
    assert ang <= 1e-3
    assert abs(st[0, 0] - 0.05) < 1e-4 and abs(st[0, 1] + 0.02) < 1e-4


def test_stack_of_two_boxes_rests(orc):
    half = np.array([[0.03, 0.03, 0.02], [0.02, 0.02, 0.015]], np.float32)
    mass = np.array([0.2, 0.1], np.float32)
    mu = np.array([0.5, 0.5], np.float32)
    s = np.stack([G.box_row(0, 0, 0.02), G.box_row(0.005, -0.004, 0.04 + 0.015)])
    st, _, _ = orc.run_substeps(s, half, mass, mu, count=240)
    p = orc.params()
    assert 0.02 - st[0, 2] <= 2 * p.slop + 1e-4
    assert (0.055 - st[1, 2]) <= 2 * (2 * p.slop + 1e-4)
    assert np.abs(st[:, 7:10]).max() <= 1e-3
    # Inside the slop band contacts push back with zero Baumgarte velocity, so a box may
    # rock by up to (accumulated slop) / (contact span): 2 slop over the top box's width.
    assert 2 * math.acos(min(1.0, abs(st[0, 3]))) <= 1e-3
    assert 2 * math.acos(min(1.0, abs(st[1, 3]))) <= 2 * p.slop / (2 * 0.02) + 1e-3


@pytest.mark.parametrize("v0", [0.1, 0.5])
@pytest.mark.parametrize("mu_v", [0.3, 0.5, 0.8])
def test_sliding_box_stop_distance(orc, v0, mu_v):
    """Coulomb sliding on the plane with an isotropic friction disk: v_k = max(v0 -
    mu g dt k, 0), distance dt * sum v_k, close to v0^2/(2 mu g) - v0 dt / 2, in any
    direction."""
    for yaw in (0.0, 0.7):
        h, m, mu = one_box((0.02, 0.02, 0.02), 0.1, mu_v)
        s = G.box_row(0, 0, 0.02, v=(v0 * math.cos(yaw), v0 * math.sin(yaw), 0))[None]
        st, _, _ = orc.run_substeps(s, h, m, mu, count=480, prm=orc.params(table_mu=mu_v))
        d_disc = DT * sum(max(v0 - mu_v * G_ACC * DT * k, 0.0) for k in range(1, 2000))
        d_cont = v0 ** 2 / (2 * mu_v * G_ACC) - v0 * DT / 2
        d = math.hypot(st[0, 0], st[0, 1])
        assert abs(d - d_disc) <= 0.02 * d_disc + 1e-4
        assert abs(d_disc - d_cont) <= 0.01 * d_cont + 1e-5
        lateral = -st[0, 0] * math.sin(yaw) + st[0, 1] * math.cos(yaw)
        assert abs(lateral) < 1e-4
        assert np.linalg.norm(st[0, 7:10]) < 1e-3


def test_head_on_impact_conserves_momentum(orc):
    """g = 0, two boxes meet head-on: linear momentum conserved, common velocity
    (m1 v1 + m2 v2)/(m1 + m2) after a perfectly inelastic contact, no spin."""
    half = np.array([[0.02, 0.02, 0.02], [0.025, 0.02, 0.02]], np.float32)
    mass = np.array([0.1, 0.3], np.float32)
    mu = np.array([0.5, 0.5], np.float32)
    s = np.stack([G.box_row(-0.03, 0, 1.0, v=(0.4, 0, 0)), G.box_row(0.03, 0, 1.0, v=(-0.1, 0, 0))])
    prm = orc.params(gravity=(0, 0, 0))
    p0 = mass.astype(float) @ s[:, 7:10]
    st, ev, _ = orc.run_substeps(s, half, mass, mu, count=120, prm=prm)
    assert ev[orc.EVENT_NAMES.index("manifolds")] > 0
    p1 = mass.astype(float) @ st[:, 7:10]
    assert np.linalg.norm(p1 - p0) <= 1e-12 * np.linalg.norm(p0)
    vc = p0[0] / mass.sum()
    assert abs(st[0, 7] - vc) < 1e-3 and abs(st[1, 7] - vc) < 1e-3
    assert np.abs(st[:, 10:13]).max() < 1e-6


def test_push_displacement_through_centre(orc):
    """A push along a face normal through the centre: the box ends L - gap ahead, plus the
    discrete post-push slide, without turning."""
    h, m, mu = one_box((0.02, 0.02, 0.02), 0.1, 0.5)
    s = G.box_row(0, 0, 0.02)[None]
    push = np.array([-0.05, 0.0, 0.05, 0.0])
    st, _, _ = orc.run_substeps(s, h, m, mu, push=push, count=240)
    st2, _, _ = orc.run_substeps(st, h, m, mu, count=240)
    gap = 0.05 - 0.02 - 0.01
    slide = DT * sum(max(0.1 - 0.5 * G_ACC * DT * k, 0.0) for k in range(1, 100))
    assert abs(st2[0, 0] - (0.1 - gap + slide)) < 1e-3
    yaw = 2 * math.atan2(st2[0, 6], st2[0, 3])
    assert abs(yaw) < 2e-3
    assert abs(st2[0, 1]) < 1e-3


# ---------------------------------------------------------------- broadphase
def _snapshot(seed, n):
    from paper_2207_06649_b300 import scenegen
    rng = np.random.default_rng(seed)
    pose, vel, half = scenegen.random_state_snapshot(rng, n)
    return np.concatenate([pose, vel], axis=1), half


@pytest.mark.parametrize("seed", range(6))
def test_pairs_equal_vertex_aabb_brute_force(orc, seed):
    st, half = _snapshot(seed, 12)
    pusher = np.array([0.01, -0.02], np.float32)
    for f32 in (True, False):
        bb, plane, pu, ov = orc.pairs(st, half, pusher_xy=pusher, f32=f32)
        assert not ov
        m = 1e-3
        lo = np.array([G.vertices(st[i].astype(float), half[i]).min(0) - m for i in range(len(st))])
        hi = np.array([G.vertices(st[i].astype(float), half[i]).max(0) + m for i in range(len(st))])
        want, amb = [], []
        for i in range(len(st)):
            for j in range(i + 1, len(st)):
                gap = max(np.max(lo[i] - hi[j]), np.max(lo[j] - hi[i]))
                if abs(gap) < 1e-6:
                    amb.append((i, j))
                elif gap <= 0:
                    want.append((i, j))
        got = [tuple(p) for p in bb]
        assert got == sorted(got), "pairs must be lexicographic"
        assert set(want) <= set(got) and set(got) <= set(want) | set(amb)
        plane_want = {i for i in range(len(st)) if lo[i, 2] < -1e-6}
        assert plane_want <= set(plane.tolist()) <= {i for i in range(len(st)) if lo[i, 2] < 1e-6}
        r = 0.01 + m
        plo = np.array([pusher[0] - r, pusher[1] - r, 0.01 - r])
        phi = np.array([pusher[0] + r, pusher[1] + r, 0.20 + r])
        pu_want = {i for i in range(len(st)) if np.all(lo[i] <= phi - 1e-6) and np.all(plo <= hi[i] - 1e-6)}
        assert pu_want <= set(pu.tolist())


@pytest.mark.parametrize("seed", range(4))
def test_pairs_superset_of_touching_boxes(orc, seed):
    st, half = _snapshot(100 + seed, 10)
    bb, _, _, _ = orc.pairs(st, half, f32=False)
    got = {tuple(p) for p in bb}
    for i in range(len(st)):
        for j in range(i + 1, len(st)):
            r = orc.box_box(st[i], half[i], st[j], half[j])
            if r is not None:
                assert (i, j) in got


# ---------------------------------------------------------------- narrowphase
@pytest.mark.parametrize("seed", range(8))
def test_sat_separation_is_complete_and_exact(orc, seed):
    """For penetrating or touching boxes the chosen axis's separation equals the
    vertex-support gap along the returned normal, and no sampled direction separates
    the boxes more than the tie-break tolerance allows."""
    rng = np.random.default_rng(seed)
    hits = 0
    for trial in range(40):
        hA = rng.uniform(0.01, 0.04, 3).astype(np.float32)
        hB = rng.uniform(0.01, 0.04, 3).astype(np.float32)
        qA = G.quat_from_rotvec(rng.normal(size=3))
        qB = G.quat_from_rotvec(rng.normal(size=3))
        d = G.random_unit_vectors(rng, 1)[0] * rng.uniform(0.01, 0.06)
        sA = G.box_row(0, 0, 0, q=qA)
        sB = G.box_row(*d, q=qB)
        r = orc.box_box(sA, hA, sB, hB)
        if r is None:
            # separated by at least the margin along some direction
            gaps = [G.support_gap(sA, hA, sB, hB, L) for L in G.random_unit_vectors(rng, 2000)]
            continue
        hits += 1
        n = r["n"]
        assert abs(np.linalg.norm(n) - 1) < 1e-12
        assert abs(G.support_gap(sA, hA, sB, hB, n) - r["sep"]) < 1e-9
        L = G.random_unit_vectors(rng, 10000)
        vA = G.vertices(sA, hA)
        vB = G.vertices(sB, hB)
        gaps = (vB @ L.T).min(0) - (vA @ L.T).max(0)
        s = r["sep"]
        assert gaps.max() <= s + 1e-4 + 0.05 * abs(s) + 1e-5 + 1e-9
    assert hits > 5


def test_face_contact_overhanging_stack(orc):
    """Small box resting on a big one, overhanging: contact points are the corners of
    the footprint intersection at the top face, with the known depth."""
    hA = np.array([0.03, 0.03, 0.02], np.float32)
    hB = np.array([0.02, 0.015, 0.01], np.float32)
    pen = 4e-4
    sA = G.box_row(0, 0, 0)
    sB = G.box_row(0.025, -0.01, 0.02 + 0.01 - pen)
    r = orc.box_box(sA, hA, sB, hB)
    assert r["axis"] == 2 and np.allclose(r["n"], [0, 0, 1])
    xs = [0.025 - 0.02, 0.03]   # overlap in x clipped at A's side
    ys = [-0.01 - 0.015, -0.01 + 0.015]
    want = np.array(sorted((float(np.float32(x)), float(np.float32(y))) for x in xs for y in ys))
    got = np.array(sorted((p[0], p[1]) for p in r["pts"]))
    assert got.shape == want.shape and np.allclose(got, want, atol=1e-8)
    assert np.allclose(r["depth"], -pen, atol=1e-12)
    assert np.allclose(r["pts"][:, 2], 0.02 - pen, atol=1e-12)


def test_edge_edge_crossing_point(orc):
    """Two cubes standing on edges (rotated 45 deg about x and about y) crossing at the
    top: edge axis z, separation -delta, one point midway between the edges."""
    h = np.array([0.02, 0.02, 0.02], np.float32)
    r2 = math.sqrt(2) * 0.02
    delta = 3e-4
    sA = G.box_row(0, 0, 0, q=G.quat_from_rotvec([math.pi / 4, 0, 0]))
    sB = G.box_row(0, 0, 2 * r2 - delta, q=G.quat_from_rotvec([0, math.pi / 4, 0]))
    r = orc.box_box(sA, h, sB, h)
    assert r["axis"] == 6 + 3 * 0 + 1
    assert np.allclose(r["n"], [0, 0, 1], atol=1e-7)
    assert abs(r["sep"] + delta) < 1e-6
    assert len(r["pts"]) == 1
    assert np.allclose(r["pts"][0], [0, 0, r2 - delta / 2], atol=1e-7)


def test_box_plane_deepest_four(orc):
    """A tilted box touching the plane: contact vertices are those below the margin,
    deepest first, at most four, with normal +z."""
    half = np.array([[0.03, 0.02, 0.01]], np.float32)
    q = G.quat_from_rotvec([0.0, 0.2, 0.0])
    verts = G.vertices(G.box_row(0, 0, 0, q=q), half[0])
    zc = -verts[:, 2].min() - 2e-4
    st = G.box_row(0, 0, zc, q=q)[None]
    info, nrm, pts = orc.contacts(st, half, np.ones(1, np.float32), np.full(1, 0.5, np.float32))
    assert info.shape[0] == 1 and info[0, 0] == -1 and info[0, 1] == 0
    assert np.allclose(nrm[0], [0, 0, 1])
    vz = np.sort(verts[:, 2] + zc)
    below = vz[vz < 1e-3]
    k = min(len(below), 4)
    assert info[0, 2] == k
    assert np.allclose(np.sort(pts[0, :k, 3]), below[:k], atol=1e-12)


# ---------------------------------------------------------------- colouring
def _clutter_state(seed, n=14):
    from paper_2207_06649_b300 import scenegen
    rng = np.random.default_rng(seed)
    sc = scenegen.make_scene(rng, n, region_half=0.07)
    st = scenegen.state13(sc).astype(np.float64)
    # squeeze the clutter so that neighbouring boxes touch
    st[:, :2] *= 0.93
    return st, sc


@pytest.mark.parametrize("seed", range(5))
def test_colouring_is_greedy_independent_sets(orc, seed):
    st, sc = _clutter_state(seed)
    info, _, _ = orc.contacts(st, sc.half, sc.mass, sc.mu, push=np.array([-0.15, 0, 0.15, 0.0]), s=0)
    assert len(info) > 0
    nb = len(st)
    used = [set() for _ in range(nb)]
    deg = np.zeros(nb, int)
    for A, B, npts, c in info:
        bodies = [b for b in (A, B) if b >= 0]
        for b in bodies:
            deg[b] += 1
        want = 0
        taken = set().union(*[used[b] for b in bodies]) if bodies else set()
        while want in taken:
            want += 1
        assert c == want
        for b in bodies:
            used[b].add(c)
    assert info[:, 3].max() + 1 <= deg.max() + 1
    # independent sets: no dynamic body appears twice within a colour
    for c in range(info[:, 3].max() + 1):
        sel = info[info[:, 3] == c]
        bodies = [b for row in sel for b in row[:2] if b >= 0]
        assert len(bodies) == len(set(bodies))


@pytest.mark.parametrize("seed", range(3))
def test_solve_order_within_colour_is_irrelevant(orc, seed):
    """Manifolds of one colour touch disjoint bodies, so any order inside a colour gives
    bit-identical results."""
    st, sc = _clutter_state(10 + seed)
    push = np.array([-0.15, 0.0, 0.15, 0.0])
    a, _, _ = orc.run_substeps(st, sc.half, sc.mass, sc.mu, push=push, count=5, reverse=False)
    b, _, _ = orc.run_substeps(st, sc.half, sc.mass, sc.mu, push=push, count=5, reverse=True)
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- grasp test
def _scene(rows, halves, target=0):
    st = np.stack([G.box_row(*r) for r in rows]).astype(np.float32)
    return st, np.array(halves, np.float32), target


@pytest.mark.parametrize("f32", [True, False])
def test_isolated_target_is_graspable(orc, f32):
    st, half, t = _scene([(0, 0, 0.02), (0.15, 0.1, 0.02)], [[0.02, 0.03, 0.02], [0.02, 0.02, 0.02]])
    assert orc.grasp(st, half, t, f32=f32)


@pytest.mark.parametrize("f32", [True, False])
def test_ringed_target_is_not_graspable(orc, f32):
    ht = 0.02
    rows, halves = [(0, 0, ht)], [[ht, ht, ht]]
    for k in range(8):
        a = k * math.pi / 4
        d = ht + 0.005 + 0.012
        rows.append((d * math.cos(a) * (1.4 if k % 2 else 1), d * math.sin(a) * (1.4 if k % 2 else 1), 0.012,
                     G.yaw_q(a)))
        halves.append([0.012, 0.02, 0.012])
    st, half, t = _scene(rows, halves)
    assert not orc.grasp(st, half, t, f32=f32)


def test_too_wide_target_is_not_graspable(orc):
    st, half, t = _scene([(0, 0, 0.02)], [[0.045, 0.045, 0.02]])
    assert not orc.grasp(st, half, t)


def test_footprint_of_upright_box_is_its_rectangle(orc):
    rng = np.random.default_rng(3)
    for _ in range(20):
        yaw = rng.uniform(-3, 3)
        h = rng.uniform(0.01, 0.04, 3)
        st = G.box_row(0.1, -0.05, h[2], q=G.yaw_q(yaw))[None].astype(np.float32)
        fp = orc.footprints(st, h[None].astype(np.float32), f32=False)[0]
        assert np.allclose(fp[:2], [0.1, -0.05], atol=1e-7)
        assert np.allclose(fp[2:4], [math.cos(yaw), math.sin(yaw)], atol=1e-7)
        assert np.allclose(fp[6:8], h[:2], atol=1e-7)


@pytest.mark.parametrize("f32", [False, True])
def test_footprint_of_tilted_box_bounds_its_corners(orc, f32):
    """Sec. IV-B footprints under any 3-D rotation: u is the horizontal part of the box's
    x axis (of its y axis when x is vertical), v = perp(u), and the support half widths
    su, sv equal the largest projection of the 8 corners (scipy rotation, independent of
    the oracle's quaternion algebra) on u and v.  A dropped or misplaced third term
    |(R e_2)_xy . u| h_2, or a transposed rotation, moves su or sv by up to h_2."""
    rng = np.random.default_rng(11)
    cases = [G.quat_from_rotvec(rng.normal(size=3) * rng.uniform(0.2, 2.0)) for _ in range(40)]
    # the box's x axis vertical (rotation about y by -90 degrees, then a yaw about the world
    # z axis): u falls back to the horizontal part of its y axis
    for yaw in (0.0, 0.7, -2.1):
        q_tilt = np.array([math.cos(-math.pi / 4), 0.0, math.sin(-math.pi / 4), 0.0])
        w1, x1, y1, z1 = G.yaw_q(yaw)
        w2, x2, y2, z2 = q_tilt
        cases.append(np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                               w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2]))
    tol = 2e-7 if f32 else 1e-9
    n_fallback = 0
    for q in cases:
        h = rng.uniform(0.01, 0.04, 3)
        row = G.box_row(0.03, -0.07, 0.05, q=tuple(q))
        st = row[None].astype(np.float32)
        hh = h[None].astype(np.float32)
        cx, cy, ux, uy, vx, vy, su, sv = orc.footprints(st, hh, f32=f32)[0]
        Rm = G.rotmat(st[0, 3:7].astype(np.float64))
        ax = Rm[:2, 0] if np.hypot(*Rm[:2, 0]) > 1e-6 else Rm[:2, 1]
        n_fallback += np.hypot(*Rm[:2, 0]) <= 1e-6
        ax = ax / np.linalg.norm(ax)
        assert np.allclose([cx, cy], st[0, :2], atol=0)
        assert np.allclose([ux, uy], ax, atol=tol * 10)
        assert np.allclose([vx, vy], [-ax[1], ax[0]], atol=tol * 10)
        V = G.vertices(st[0].astype(np.float64), hh[0].astype(np.float64))
        d = V[:, :2] - st[0, :2].astype(np.float64)
        assert abs(su - np.abs(d @ ax).max()) <= tol * 10 + 1e-12
        assert abs(sv - np.abs(d @ np.array([-ax[1], ax[0]])).max()) <= tol * 10 + 1e-12
    assert n_fallback == 3


def _raster_overlap(rect, foot, cell=1e-4):
    """Cells of a 0.1 mm grid whose centres are inside both rectangles.
    rect/foot = (cx, cy, ux, uy, hu, hv) with v = perp(u)."""
    cx, cy, ux, uy, hu, hv = rect
    R = math.hypot(hu, hv)
    xs = np.arange(cx - R, cx + R, cell) + cell / 2
    ys = np.arange(cy - R, cy + R, cell) + cell / 2
    X, Y = np.meshgrid(xs, ys)

    def inside(r, X, Y):
        dx, dy = X - r[0], Y - r[1]
        a = np.abs(dx * r[2] + dy * r[3])
        b = np.abs(-dx * r[3] + dy * r[2])
        return (a < r[4]) & (b < r[5])

    return int(np.count_nonzero(inside(rect, X, Y) & inside(foot, X, Y)))


def _signed_overlap_depth(rect, foot):
    """Largest separating gap over the four rectangle axes (negative = overlap depth)."""
    def corners(r):
        u = np.array([r[2], r[3]])
        v = np.array([-r[3], r[2]])
        c = np.array([r[0], r[1]])
        return np.array([c + su * r[4] * u + sv * r[5] * v for su in (-1, 1) for sv in (-1, 1)])

    A, B = corners(rect), corners(foot)
    best = -1e9
    for r in (rect, foot):
        for ax in (np.array([r[2], r[3]]), np.array([-r[3], r[2]])):
            pa, pb = A @ ax, B @ ax
            best = max(best, max(pb.min() - pa.max(), pa.min() - pb.max()))
    return best


@pytest.mark.parametrize("seed", range(6))
def test_grasp_matches_rasterised_fingers(orc, seed):
    """Brute force: finger sweep rectangles and footprints rasterised on a 0.1 mm grid
    give the same decision wherever no overlap is within 0.3 mm of touching."""
    from paper_2207_06649_b300 import scenegen
    rng = np.random.default_rng(200 + seed)
    p = orc.params()
    checked = 0
    for trial in range(10):
        sc = scenegen.make_scene(rng, 8, region_half=0.075, yaw_hi=math.pi / 2, half_lo=0.01, half_hi=0.03)
        st = scenegen.state13(sc)
        fp = orc.footprints(st, sc.half, f32=False)
        t = 0
        W, c, f, fw = p.grasp_opening, p.grasp_clearance, p.finger_depth, p.finger_width
        decision, robust = False, True
        ft = fp[t]
        for k in range(p.grasp_angles):
            th = k * math.pi / p.grasp_angles
            a = np.array([math.cos(th), math.sin(th)])
            # width of the target footprint rectangle along a, from its corners
            u, v = ft[2:4], ft[4:6]
            corners = [ft[:2] + su * ft[6] * u + sv * ft[7] * v for su in (-1, 1) for sv in (-1, 1)]
            wa = max(np.dot(cc - ft[:2], a) for cc in corners)
            if 2 * (wa + c) > W:
                continue
            ok = True
            for s in (1, -1):
                centre = ft[:2] + s * a * (wa + W / 2 + f) / 2
                rect = (centre[0], centre[1], a[0], a[1], (W / 2 + f - wa) / 2, fw / 2)
                for o in range(1, len(st)):
                    foot = (fp[o, 0], fp[o, 1], fp[o, 2], fp[o, 3], fp[o, 6], fp[o, 7])
                    depth = _signed_overlap_depth(rect, foot)
                    if abs(depth) < 3e-4:
                        robust = False
                    if _raster_overlap(rect, foot) > 0:
                        ok = False
            if ok:
                decision = True
        if robust:
            checked += 1
            assert orc.grasp(st, sc.half, t, f32=False) == decision
            assert orc.grasp(st, sc.half, t, f32=True) == decision
    assert checked >= 3


# ---------------------------------------------------------------- push sampler
def _splitmix_draws(seed, k, a, n, npts):
    M = (1 << 64) - 1
    s = (seed ^ ((k << 32) | a)) & M
    out = []
    for _ in range(2):
        s = (s + 0x9E3779B97F4A7C15) & M
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        out.append(z ^ (z >> 31))
    return ((out[0] >> 32) * n) >> 32, ((out[1] >> 32) * npts) >> 32


def _contour_point(f, j_pt, npts, grow):
    """Point j_pt of npts spaced by arc length on the footprint rectangle f grown by
    `grow`, counter-clockwise from (+A, 0) in the (u, v) frame."""
    A, B = f[6] + grow, f[7] + grow
    ell = 4 * (A + B) * j_pt / npts
    path = [((A, 0), (A, B)), ((A, B), (-A, B)), ((-A, B), (-A, -B)), ((-A, -B), (A, -B)), ((A, -B), (A, 0))]
    for (a0, a1) in path:
        seg = math.hypot(a1[0] - a0[0], a1[1] - a0[1])
        if ell < seg or a1 == (A, 0):
            t = ell / seg
            lu, lv = a0[0] + t * (a1[0] - a0[0]), a0[1] + t * (a1[1] - a0[1])
            break
        ell -= seg
    return f[:2] + lu * f[2:4] + lv * f[4:6]


def _check_sampler(orc, st, half, sd, k):
    p = orc.params()
    fp = orc.footprints(st, half, f32=False)
    a, push = orc.sample_push(st, half, sd, k, f32=False)
    a32, push32 = orc.sample_push(st, half, sd, k, f32=True)
    assert a == a32
    last = a if a >= 0 else p.sample_attempts
    for prev in range(last):
        j, pp = _splitmix_draws(sd, k, prev, len(st), p.contour_points)
        q = _contour_point(fp[j], pp, p.contour_points, p.pusher_radius + p.sample_clearance)
        assert orc.start_blocked(st, half, q[0], q[1], f32=False), "rejected attempt must be blocked"
    if a < 0:
        return a
    assert np.allclose(push, push32, atol=1e-6)
    j, pp = _splitmix_draws(sd, k, a, len(st), p.contour_points)
    q = _contour_point(fp[j], pp, p.contour_points, p.pusher_radius + p.sample_clearance)
    assert np.allclose(push[:2], q, atol=1e-6)
    d = push[2:].astype(float) - push[:2]
    assert abs(np.linalg.norm(d) - p.push_length) < 1e-6
    to_c = fp[j, :2] - push[:2]
    assert np.dot(d, to_c) / (np.linalg.norm(d) * np.linalg.norm(to_c)) > 1 - 1e-6
    assert not orc.start_blocked(st, half, push[0], push[1], f32=False)
    return a


@pytest.mark.parametrize("seed", range(5))
def test_sampled_push_on_grown_contour_towards_centre(orc, seed):
    from paper_2207_06649_b300 import scenegen
    rng = np.random.default_rng(300 + seed)
    sc = scenegen.make_scene(rng, 10, region_half=0.08, yaw_hi=math.pi / 2)
    st = scenegen.state13(sc)
    for k in (2, 3, 7):
        _check_sampler(orc, st, sc.half, int(rng.integers(0, 2 ** 63)), k)


def test_dense_grid_sampler_rejections_and_noop(orc):
    rows, halves = [], []
    for i in range(6):
        for j in range(6):
            rows.append((-0.1 + 0.04 * i, -0.1 + 0.04 * j, 0.02))
            halves.append([0.0195, 0.0195, 0.02])
    st, half, _ = _scene(rows, halves)
    seen = set()
    for sd in range(400):
        a = _check_sampler(orc, st, half, sd * 7919 + 1, 2)
        seen.add(a)
    assert -1 in seen and 0 in seen and max(seen) >= 3


# ------------------------------------------------------------------ heightmap (Sec. V-A grid)
def _cell_centres():
    c = -0.144 + (np.arange(144) + 0.5) * 0.002
    return np.meshgrid(c, c)  # X[j, i], Y[j, i]


def test_heightmap_of_yawed_upright_boxes_is_their_rectangles(orc):
    """Upright boxes (yaw only): height c_z + h_z exactly where the cell centre lies in
    the rotated rectangle (independent point-in-rectangle test), 0 elsewhere; several boxes
    give the cell-wise maximum."""
    X, Y = _cell_centres()
    rng = np.random.default_rng(4)
    rows, halves, want = [], [], np.zeros((144, 144))
    for b in range(5):
        yaw = rng.uniform(0, math.pi)
        h = rng.uniform(0.01, 0.03, 3)
        # quarter-cell offsets keep cell centres off the rectangle edges
        c = np.array([rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1), h[2] + 0.01 * b]) + 0.0005
        rows.append(G.box_row(*c, q=(math.cos(yaw / 2), 0, 0, math.sin(yaw / 2))))
        halves.append(h)
        u = np.array([math.cos(yaw), math.sin(yaw)])
        v = np.array([-u[1], u[0]])
        du = (X - c[0]) * u[0] + (Y - c[1]) * u[1]
        dv = (X - c[0]) * v[0] + (Y - c[1]) * v[1]
        inside = (np.abs(du) <= h[0]) & (np.abs(dv) <= h[1])
        want = np.maximum(want, np.where(inside, c[2] + h[2], 0.0))
    st = np.stack(rows)
    got = orc.heightmap(st, np.array(halves), f32=False)
    assert np.abs(got - want).max() <= 1e-8  # double result stored as float32
    assert (got > 0).sum() > 1000
    # the binary32 twin agrees to rounding
    assert np.abs(orc.heightmap(st, np.array(halves), f32=True) - want).max() <= 1e-6


def test_heightmap_of_tilted_boxes_matches_convex_hull_and_linear_programme(orc):
    """Tilted boxes: a cell is covered iff its centre lies inside the convex hull of the
    box's projected vertices, and the stored height is the maximum z of the box on the
    vertical line, found by a linear programme (scipy), independent of the slab formula."""
    from scipy.optimize import linprog
    from scipy.spatial import ConvexHull
    X, Y = _cell_centres()
    rng = np.random.default_rng(7)
    for trial in range(3):
        q = G.quat_from_rotvec(rng.normal(size=3) * 0.8)
        h = rng.uniform(0.015, 0.035, 3)
        c = np.array([rng.uniform(-0.05, 0.05), rng.uniform(-0.05, 0.05), 0.08])
        row = G.box_row(*c, q=tuple(q))
        got = orc.heightmap(row[None], h[None], f32=False)
        V = G.vertices(row, h)
        hull = ConvexHull(V[:, :2])
        eq = hull.equations  # a x + b y + d <= 0 inside
        dist = (eq[:, :1, None] * X[None] + eq[:, 1:2, None] * Y[None] + eq[:, 2:3, None]).max(0)
        inside, outside = dist < -1e-6, dist > 1e-6
        assert (got[inside] > 0).all() and (got[outside] == 0).all()
        R = G.rotmat(q)
        idx = np.argwhere(inside)
        for j, i in idx[rng.choice(len(idx), size=40, replace=False)]:
            # maximise z subject to -h <= R^T (p - c) <= h with p = (x, y, z)
            A = np.vstack([R.T, -R.T])
            p0 = np.array([X[j, i], Y[j, i], 0.0]) - c
            b_ub = np.concatenate([h - R.T @ p0, h + R.T @ p0])
            res = linprog(c=[-1.0], A_ub=A[:, 2:3], b_ub=b_ub, bounds=[(None, None)], method="highs")
            assert res.status == 0
            # inputs enter the oracle as float32 (a quaternion off unit length by ~1e-8)
            assert abs(got[j, i] - res.x[0]) <= 1e-7


def test_heightmap_clamps_at_the_table_and_is_empty_without_boxes(orc):
    st = np.stack([G.box_row(0.0, 0.0, -0.05)])      # entirely below the table
    assert (orc.heightmap(st, np.array([[0.02, 0.02, 0.02]])) == 0).all()
    assert (orc.heightmap(np.zeros((0, 13)), np.zeros((0, 3))) == 0).all()
    st = np.stack([G.box_row(0.0, 0.0, 0.005)])      # half sunk: top at 0.025
    m = orc.heightmap(st, np.array([[0.02, 0.02, 0.02]]), f32=False)
    assert abs(m.max() - 0.025) <= 2e-9  # stored as float32


# ------------------------------------------------------------------ heightmap grasp test
def _ring(target_h, ring_h):
    rows, halves = [(0, 0, target_h)], [[0.02, 0.02, target_h]]
    for k in range(8):
        a = k * math.pi / 4
        d = 0.02 + 0.005 + 0.012
        rows.append((d * math.cos(a) * (1.4 if k % 2 else 1), d * math.sin(a) * (1.4 if k % 2 else 1), ring_h,
                     G.yaw_q(a)))
        halves.append([0.012, 0.02, ring_h])
    return _scene(rows, halves)


@pytest.mark.parametrize("f32", [True, False])
def test_heightmap_grasp_isolated_and_ringed(orc, f32):
    st, half, t = _scene([(0, 0, 0.02)], [[0.02, 0.02, 0.02]])
    assert orc.grasp_heightmap(st, half, t, f32=f32)
    # a ring as tall as the target blocks every finger path (tips 2 cm below its top)
    st, half, t = _ring(0.02, 0.02)
    assert not orc.grasp_heightmap(st, half, t, f32=f32) and not orc.grasp(st, half, t, f32=f32)


@pytest.mark.parametrize("f32", [True, False])
def test_heightmap_grasp_passes_over_low_neighbours(orc, f32):
    """A tall target (top 0.06 m) ringed by flat boxes (top 0.01 m): the footprint test
    sees the ring and refuses, the heightmap test lets fingers that stop 2 cm below the
    target's top pass over it; with tips 5.5 cm down the ring blocks again."""
    st, half, t = _ring(0.03, 0.005)
    assert not orc.grasp(st, half, t, f32=f32)
    assert orc.grasp_heightmap(st, half, t, depth=0.02, f32=f32)
    assert not orc.grasp_heightmap(st, half, t, depth=0.055, f32=f32)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_heightmap_grasp_is_monotone(orc, seed):
    """Deeper finger tips can only block more, and removing other boxes can only free
    paths (random clutter, every box as target)."""
    sg = _sg_mod()
    rng = np.random.default_rng(seed)
    sc = sg.make_scene(rng, 12, half_lo=0.01, half_hi=0.03, yaw_hi=math.pi / 2, region_half=0.09)
    st, half = sg.state13(sc), sc.half
    n = len(st)
    changed = 0
    for t in range(n):
        d1 = orc.grasp_heightmap(st, half, t, depth=0.005)
        d2 = orc.grasp_heightmap(st, half, t, depth=0.02)
        d3 = orc.grasp_heightmap(st, half, t, depth=0.06)
        assert (d3 <= d2 <= d1)
        changed += int(d1 != d3)
        keep = [t] + [o for o in range(n) if o != t and rng.random() < 0.5]
        sub = orc.grasp_heightmap(st[keep], half[keep], 0, depth=0.02)
        assert sub >= d2
    assert changed > 0


def _sg_mod():
    from paper_2207_06649_b300 import scenegen
    return scenegen


# ------------------------------------------------------------------ warm start (option)
def _stack(nb, h=0.01):
    rows = [G.box_row(0.0005 * k, -0.0003 * k, h + 2 * h * k) for k in range(nb)]
    return np.stack(rows), np.full((nb, 3), h), np.full(nb, 0.1), np.full(nb, 0.5)


def test_warm_start_first_substep_is_unchanged(orc):
    """With nothing to carry over, the first substep equals the cold solve exactly."""
    st, half, m, mu = _stack(4)
    a, _, _ = orc.run_substeps(st, half, m, mu, count=1, prm=orc.params(warm_start=0))
    b, _, _ = orc.run_substeps(st, half, m, mu, count=1, prm=orc.params(warm_start=1))
    assert np.array_equal(a, b)


def test_warm_start_holds_a_tall_stack(orc):
    """Six 2 cm cubes, each offset by a fraction of a millimetre: carrying the impulses
    over keeps the stack standing for two seconds (every gap within 0.5 mm of contact),
    while ten cold Gauss-Seidel iterations per substep let it collapse."""
    st, half, m, mu = _stack(6)
    warm, _, _ = orc.run_substeps(st, half, m, mu, count=480, prm=orc.params(warm_start=1))
    cold, _, _ = orc.run_substeps(st, half, m, mu, count=480, prm=orc.params(warm_start=0))
    gap = lambda s: np.diff(s[:, 2]) - 0.02
    assert np.abs(gap(warm)).max() <= 5e-4 and np.abs(warm[:, :2] - st[:, :2]).max() <= 2e-3
    assert np.abs(gap(cold)).max() > 5e-3


def test_warm_start_conserves_momentum_in_impacts(orc):
    """Carried impulses act in equal and opposite pairs: two boxes colliding in free space
    (no gravity) keep their total momentum."""
    prm = orc.params(warm_start=1, gravity=(0.0, 0.0, 0.0))
    st = np.stack([G.box_row(-0.021, 0.0, 0.5, v=(0.3, 0.0, 0.0), w=(0.0, 0.0, 1.0)),
                   G.box_row(0.021, 0.002, 0.5, v=(-0.2, 0.0, 0.0), w=(0.5, 0.0, 0.0))])
    half = np.full((2, 3), 0.02)
    m = np.array([0.1, 0.2])
    out, _, _ = orc.run_substeps(st, half, m, np.full(2, 0.5), count=120, prm=prm)
    p0 = (m[:, None] * st[:, 7:10]).sum(0)
    p1 = (m[:, None] * out[:, 7:10]).sum(0)
    assert np.abs(out[:, 7:10] - st[:, 7:10]).max() > 0.05      # they did collide
    assert np.abs(p1 - p0).max() <= 1e-12


def test_pusher_box_contact_closed_form(orc):
    """Capsule pusher (radius 0.01 m, z in [0.01, 0.20]) beside an upright box: the two
    contact points sit on the box face at the ends of the overlapping height range
    [0.01, 2 h_z], separation = centre distance - h_x - r, normal from the box to the
    pusher; a pusher level with a box corner meets it at the corner edge."""
    hx, hy, hz, rp = 0.03, 0.02, 0.025, 0.01
    half = np.array([[hx, hy, hz]], np.float32)
    st = G.box_row(0, 0, hz)[None]
    gap = 4e-4
    px = -(hx + rp + gap)
    info, nrm, pts = orc.contacts(st, half, np.ones(1, np.float32), np.full(1, 0.5, np.float32),
                                  push=np.array([px, 0.0, px + 0.1, 0.0]), s=0)
    m = [k for k in range(len(info)) if info[k, 1] == -2][0]
    assert info[m, 2] == 2
    assert np.allclose(nrm[m], [-1, 0, 0], atol=1e-12)
    zs = np.sort(pts[m, :2, 2])
    assert np.allclose(zs, [0.01, 2 * hz], atol=1e-7)
    assert np.allclose(pts[m, :2, 0], -hx, atol=1e-7) and np.allclose(pts[m, :2, 3], gap, atol=1e-7)
    # diagonal approach to the (-x, -y) corner edge: distance to the edge minus the radius
    d = rp + gap
    p = np.array([-hx, -hy]) - d * np.array([1, 1]) / math.sqrt(2)
    info, nrm, pts = orc.contacts(st, half, np.ones(1, np.float32), np.full(1, 0.5, np.float32),
                                  push=np.array([p[0], p[1], p[0] + 0.1, p[1]]), s=0)
    m = [k for k in range(len(info)) if info[k, 1] == -2][0]
    assert np.allclose(pts[m, :info[m, 2], 3], gap, atol=1e-7)
    assert np.allclose(nrm[m], [-1 / math.sqrt(2), -1 / math.sqrt(2), 0], atol=1e-7)
    assert np.allclose(pts[m, :info[m, 2], :2], [-hx, -hy], atol=1e-7)


def test_speculative_contact_closes_the_gap_exactly(orc):
    """A separated contact (gap d < margin) allows an approach speed of d/dt and no more:
    a box falling at 0.5 m/s onto the table from d = 0.8 mm (0.5 m/s x dt = 2.1 mm would
    overshoot by 1.3 mm) lands within the Gauss-Seidel residual of z = h_z after one
    substep with v_z = -d/dt to 1 %, never penetrates by more than 1 um, and rests."""
    h, m, mu = one_box((0.02, 0.02, 0.02), 0.1, 0.5)
    d0 = 8e-4
    st = G.box_row(0.01, -0.01, 0.02 + d0, v=(0.0, 0.0, -0.5))[None]
    st1, _, _ = orc.run_substeps(st, h, m, mu, count=1)
    assert -1e-6 <= st1[0, 2] - 0.02 <= 1e-3 * d0
    assert abs(st1[0, 9] / (-d0 / DT) - 1) < 1e-2
    cur = st1
    for k in range(1, 40):
        cur, _, _ = orc.run_substeps(cur, h, m, mu, s0=k, count=1)
        assert cur[0, 2] - 0.02 >= -1e-6
    assert abs(cur[0, 9]) < 1e-4
