"""Pins of the FP64 oracle's cylinders (CPU only).

A cylinder (half-extent row (r, -r, h)) collides as the right prism over the regular
16-gon inscribed in its circle and carries the solid cylinder's mass properties.  The
checks below derive what that definition implies from the prism's corners (scipy hulls,
brute force over vertices), from closed forms and from impulse ratios at known lever
arms, independently of the oracle's support functions and slab formulas.
"""
import math

import numpy as np
import pytest

from tests import _geom as G

DT = 1.0 / 240.0
G_ACC = 9.81
APO = math.cos(math.pi / 16)       # apothem of the unit-radius 16-gon
HALF_EDGE = math.sin(math.pi / 16)


def cyl(r, h):
    return np.array([r, -r, h], np.float32)


def qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


# ---------------------------------------------------------------- separating axes
def _hull_axes(V):
    """Facet normals and edge directions of the convex hull of V (unique up to sign)."""
    from scipy.spatial import ConvexHull
    hull = ConvexHull(V)
    faces = hull.equations[:, :3]
    edges = []
    for simplex in hull.simplices:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            e = V[simplex[b]] - V[simplex[a]]
            n = np.linalg.norm(e)
            if n > 1e-9:
                edges.append(e / n)
    return faces, np.array(edges)


@pytest.mark.parametrize("seed", range(6))
def test_cylinder_sat_separation_is_exact_and_complete(orc, seed):
    """Box-cylinder and cylinder-cylinder pairs: the separation equals the corner-support
    gap along the returned normal, and neither any hull facet normal nor any cross
    product of hull edges separates more than the tie-break tolerance allows."""
    rng = np.random.default_rng(100 + seed)
    hits = 0
    for trial in range(25):
        hA = (cyl(rng.uniform(0.01, 0.03), rng.uniform(0.01, 0.04)) if trial % 2
              else rng.uniform(0.01, 0.04, 3).astype(np.float32))
        hB = cyl(rng.uniform(0.01, 0.03), rng.uniform(0.01, 0.04))
        sA = G.box_row(0, 0, 0, q=G.quat_from_rotvec(rng.normal(size=3)))
        d = G.random_unit_vectors(rng, 1)[0] * rng.uniform(0.01, 0.06)
        sB = G.box_row(*d, q=G.quat_from_rotvec(rng.normal(size=3)))
        r = orc.box_box(sA, hA, sB, hB)
        if r is None:
            continue
        hits += 1
        n, s = r["n"], r["sep"]
        assert abs(np.linalg.norm(n) - 1) < 1e-12
        assert abs(G.body_gap(sA, hA, sB, hB, n) - s) < 1e-9
        VA, VB = G.body_vertices(sA, hA), G.body_vertices(sB, hB)
        fA, eA = _hull_axes(VA)
        fB, eB = _hull_axes(VB)
        cand = [fA, fB]
        X = np.cross(eA[:, None, :], eB[None, :, :]).reshape(-1, 3)
        ln = np.linalg.norm(X, axis=1)
        cand.append(X[ln > 1e-6] / ln[ln > 1e-6, None])
        L = np.concatenate(cand)
        gaps = (VB @ L.T).min(0) - (VA @ L.T).max(0)
        assert gaps.max() <= s + 1e-4 + 0.05 * abs(s) + 1e-5 + 1e-9
    assert hits > 8


@pytest.mark.parametrize("psi", [0.0, 0.1, math.pi / 16])
def test_cylinder_box_gap_closed_form(orc, psi):
    """Upright cylinder beside a box along x: the gap is d - h_x - r (cos of the angle
    from the nearest corner direction) -- r at a corner (yaw 0), r cos(pi/16) facing a side."""
    r, h = 0.02, 0.03
    hb = np.array([0.02, 0.02, 0.02], np.float32)
    dx = 0.0445
    sB = G.box_row(dx, 0, 0.1, q=G.yaw_q(psi))
    res = orc.box_box(G.box_row(0, 0, 0.1), hb, sB, cyl(r, h), margin=0.01)
    # angular distance from the -x direction to the nearest corner direction k pi/8
    ang = (math.pi - psi) % (math.pi / 8)
    delta = min(ang, math.pi / 8 - ang)
    assert abs(res["sep"] - (dx - 0.02 - r * math.cos(delta))) < 1e-8
    assert np.allclose(res["n"], [1, 0, 0], atol=1e-9)


def test_cylinder_cap_on_box_face_contact(orc):
    """Upright cylinder on a box top: the 16 cap corners are all in contact and reduce to
    four -- the first corner (deepest, earliest), the one opposite, then the two at right
    angles -- at the known depth."""
    r, h, pen = 0.02, 0.03, 3e-4
    hb = np.array([0.04, 0.04, 0.02], np.float32)
    res = orc.box_box(G.box_row(0, 0, 0), hb, G.box_row(0, 0, 0.02 + h - pen), cyl(r, h))
    assert np.allclose(res["n"], [0, 0, 1])
    want = np.array([[r, 0], [-r, 0], [0, r], [0, -r]])
    got = res["pts"][:, :2]
    assert got.shape == (4, 2)
    assert np.allclose(np.sort(got, axis=0), np.sort(want, axis=0), atol=2e-9)
    assert np.allclose(res["depth"], -pen, atol=1e-9)


def test_stacked_cylinders_cap_contact(orc):
    """Two coaxial cylinders of different radii: the smaller cap's corners all lie inside
    the larger cap, so the contact corners are the smaller cylinder's."""
    pen = 2e-4
    res = orc.box_box(G.box_row(0, 0, 0), cyl(0.03, 0.02), G.box_row(0, 0, 0.02 + 0.015 - pen), cyl(0.018, 0.015))
    assert np.allclose(res["n"], [0, 0, 1])
    assert np.allclose(np.hypot(res["pts"][:, 0], res["pts"][:, 1]), 0.018, atol=1e-8)
    assert np.allclose(res["depth"], -pen, atol=1e-9)


def test_cylinder_plane_contacts(orc):
    """Tilted cylinder: contact corners are those below the margin, deepest first (a
    brute-force minimum over the 32 corners); flat on its cap: four of the 16 corners."""
    half = cyl(0.025, 0.03)[None]
    q = G.quat_from_rotvec([0.0, 0.3, 0.0])
    V = G.cyl_vertices(G.box_row(0, 0, 0, q=q), 0.025, 0.03)
    zc = -V[:, 2].min() - 2e-4
    info, nrm, pts = orc.contacts(G.box_row(0, 0, zc, q=q)[None], half, np.ones(1, np.float32),
                                  np.full(1, 0.5, np.float32))
    vz = np.sort(V[:, 2] + zc)
    below = vz[vz < 1e-3]
    assert info[0, 2] == min(len(below), 4)
    assert abs(pts[0, 0, 3] - below[0]) < 1e-8   # half extents enter as binary32
    info, nrm, pts = orc.contacts(G.box_row(0.01, 0, 0.03 - 1e-4)[None], half, np.ones(1, np.float32),
                                  np.full(1, 0.5, np.float32))
    assert info[0, 2] == 4
    assert np.allclose(np.hypot(pts[0, :4, 0] - 0.01, pts[0, :4, 1]), 0.025, atol=1e-9)
    assert np.allclose(pts[0, :4, 3], -1e-4, atol=1e-12)


@pytest.mark.parametrize("where", ["corner", "side"])
def test_pusher_cylinder_distance(orc, where):
    """Capsule pusher beside an upright cylinder: separation = distance between the axes
    minus the pusher radius minus r (facing a corner) or r cos(pi/16) (facing a side)."""
    r, h, rp = 0.02, 0.03, 0.01
    yaw = 0.0 if where == "corner" else math.pi / 16
    dist = r + rp + 5e-4
    st = G.box_row(0, 0, h, q=G.yaw_q(yaw))[None]
    push = np.array([-dist, 0.0, -dist + 0.1, 0.0])
    info, nrm, pts = orc.contacts(st, cyl(r, h)[None], np.ones(1, np.float32), np.full(1, 0.5, np.float32),
                                  push=push, s=0)
    pm = [m for m in range(len(info)) if info[m, 1] == -2]
    assert len(pm) == 1
    m = pm[0]
    reach = r if where == "corner" else r * APO
    assert np.allclose(pts[m, :info[m, 2], 3], dist - reach - rp, atol=1e-12)
    assert np.allclose(nrm[m], [-1, 0, 0], atol=1e-12)


# ---------------------------------------------------------------- dynamics
def test_upright_and_lying_cylinders_rest(orc):
    r, h = 0.02, 0.03
    st, _, _ = orc.run_substeps(G.box_row(0.01, -0.02, h)[None], cyl(r, h)[None], [0.1], [0.5], count=480)
    assert abs(st[0, 2] - h) < 1e-6 and np.abs(st[0, 7:]).max() < 1e-6
    # lying on a side face (a side normal turned to -z): rests at the apothem
    q = qmul(G.quat_from_rotvec([0, math.pi / 2, 0]), G.quat_from_rotvec([0, 0, -math.pi / 16]))
    st, _, _ = orc.run_substeps(G.box_row(0, 0, r * APO, q=tuple(q))[None], cyl(r, h)[None], [0.1], [0.5], count=480)
    assert abs(st[0, 2] - r * APO) < 1e-5 and np.hypot(st[0, 0], st[0, 1]) < 1e-4


@pytest.mark.parametrize("v0,mu_v", [(0.3, 0.5), (0.2, 0.3)])
def test_sliding_cylinder_stop_distance(orc, v0, mu_v):
    """An upright cylinder slides like any flat-bottomed body: v_k = max(v0 - mu g dt k, 0),
    distance dt * sum v_k, without tipping."""
    r, h = 0.02, 0.03
    st, _, _ = orc.run_substeps(G.box_row(0, 0, h, v=(v0, 0, 0))[None], cyl(r, h)[None], [0.1], [mu_v], count=480,
                                prm=orc.params(table_mu=mu_v))
    d_disc = DT * sum(max(v0 - mu_v * G_ACC * DT * k, 0.0) for k in range(1, 2000))
    assert abs(st[0, 0] - d_disc) <= 0.02 * d_disc + 1e-4
    assert abs(st[0, 2] - h) < 1e-5 and np.linalg.norm(st[0, 7:]) < 1e-3


def _first_impulse(orc, st, half, mass, mu, push, prm, nmax=200):
    cur = st.copy()
    for s in range(nmax):
        nxt, _, _ = orc.run_substeps(cur, half, mass, mu, push=push, s0=s, count=1, prm=prm)
        if np.abs(nxt[-1, 7:10] - cur[-1, 7:10]).max() > 1e-9:
            return cur, nxt
        cur = nxt
    raise AssertionError("no contact")


def test_cylinder_inertia_about_a_diameter(orc):
    """g = 0, mu = 0: a pusher moving along +x meets a floating cylinder lying along y at
    axial offset delta.  Every contact impulse P (normals in the xz plane) acts at y offset
    delta, so dw_z / dv_x = -delta m / I_d with I_d = m (3 r^2 + 4 h^2) / 12."""
    r, h, m, delta = 0.02, 0.03, 0.1, 0.012
    q = qmul(G.quat_from_rotvec([-math.pi / 2, 0, 0]), G.quat_from_rotvec([0, 0, math.pi / 16]))
    st = G.box_row(0, 0, 0.1, q=tuple(q))[None]
    x0 = -(r * APO + 0.01 + 0.003)
    push = np.array([x0, delta, x0 + 0.1, delta])
    prm = orc.params(gravity=(0, 0, 0), pusher_mu=0.0)
    a, b = _first_impulse(orc, st, cyl(r, h)[None], [m], [0.0], push, prm)
    dv, dw = b[0, 7:10] - a[0, 7:10], b[0, 10:13] - a[0, 10:13]
    I_d = m * (3 * r * r + 4 * h * h) / 12
    assert dv[0] > 1e-4 and abs(dv[1]) < 1e-12
    assert abs(dw[2] / dv[0] - (-delta * m / I_d)) < 1e-6 * abs(delta * m / I_d)  # r, h enter as binary32


def test_cylinder_inertia_about_its_axis(orc):
    """g = 0, mu = 0: a heavy box moving along +x strikes a floating upright cylinder
    yawed by psi on its leading corner edge (corner 8, at (-r cos psi, -r sin psi)).  The
    box face's impulse P along x gives dw_z / dv_x = m r sin(psi) / I_a with
    I_a = m r^2 / 2, i.e. 2 sin(psi) / r."""
    r, h, psi = 0.02, 0.03, 0.03
    half = np.stack([np.array([0.02, 0.05, 0.05], np.float32), cyl(r, h)])
    st = np.stack([G.box_row(-(r + 0.02 + 0.003), 0, 0.1, v=(0.2, 0, 0)), G.box_row(0, 0, 0.1, q=G.yaw_q(psi))])
    prm = orc.params(gravity=(0, 0, 0))
    a, b = _first_impulse(orc, st, half, [5.0, 0.1], [0.0, 0.0], None, prm)
    dv, dw = b[1, 7:10] - a[1, 7:10], b[1, 10:13] - a[1, 10:13]
    yaw = 2 * math.atan2(a[1, 6], a[1, 3])
    assert dv[0] > 1e-4 and abs(dv[1]) < 1e-12
    assert abs(dw[2] / dv[0] - 2 * math.sin(yaw) / r) < 1e-6 * (2 * math.sin(yaw) / r)


# ---------------------------------------------------------------- footprints, heightmaps
def test_cylinder_footprint_bounds_its_corners(orc):
    """Footprint support half widths equal the brute-force maximum of the corners'
    projections on u and v, upright and tilted."""
    rng = np.random.default_rng(5)
    for trial in range(6):
        r, h = rng.uniform(0.01, 0.03), rng.uniform(0.01, 0.04)
        q = G.quat_from_rotvec(rng.normal(size=3) * (0.0 if trial < 2 else 0.5) + np.array([0, 0, rng.uniform(0, 3)]))
        row = G.box_row(0.01, -0.02, 0.05, q=tuple(q))
        f = orc.footprints(row[None], cyl(r, h)[None], f32=False)[0]
        cx, cy, ux, uy, vx, vy, su, sv = f
        V = G.cyl_vertices(row, r, h)
        assert abs(su - np.abs((V[:, 0] - cx) * ux + (V[:, 1] - cy) * uy).max()) < 1e-8  # binary32 inputs
        assert abs(sv - np.abs((V[:, 0] - cx) * vx + (V[:, 1] - cy) * vy).max()) < 1e-8


def _cell_centres():
    c = -0.144 + (np.arange(144) + 0.5) * 0.002
    return np.meshgrid(c, c)


@pytest.mark.parametrize("pose", ["upright", "lying", "tilted"])
def test_cylinder_heightmap_matches_hull_and_linear_programme(orc, pose):
    """A cell is covered iff its centre lies in the convex hull of the projected prism
    corners, and its height is the largest z on the vertical line inside the prism (a
    linear programme over the 3-D hull's facets), independent of the slab formula."""
    from scipy.optimize import linprog
    from scipy.spatial import ConvexHull
    r, h = 0.025, 0.035
    q = {"upright": G.yaw_q(0.3), "lying": tuple(G.quat_from_rotvec([math.pi / 2, 0, 0.2])),
         "tilted": tuple(G.quat_from_rotvec([0.4, -0.7, 0.2]))}[pose]
    row = G.box_row(0.0107, -0.0093, 0.06, q=q)
    got = orc.heightmap(row[None], cyl(r, h)[None], f32=False)
    V = G.cyl_vertices(row, r, h)
    X, Y = _cell_centres()
    hull2 = ConvexHull(V[:, :2])
    eq = hull2.equations
    dist = (eq[:, :1, None] * X[None] + eq[:, 1:2, None] * Y[None] + eq[:, 2:3, None]).max(0)
    inside, outside = dist < -1e-6, dist > 1e-6
    assert (got[inside] > 0).all() and (got[outside] == 0).all()
    hull3 = ConvexHull(V)
    A, bvec = hull3.equations[:, :3], -hull3.equations[:, 3]
    rng = np.random.default_rng(1)
    idx = np.argwhere(inside)
    for j, i in idx[rng.choice(len(idx), size=30, replace=False)]:
        # maximise z subject to A (x, y, z) <= b at fixed (x, y)
        res = linprog(c=[-1.0], A_ub=A[:, 2:3], b_ub=bvec - A[:, 0] * X[j, i] - A[:, 1] * Y[j, i],
                      bounds=[(None, None)], method="highs")
        assert res.status == 0
        assert abs(got[j, i] - res.x[0]) <= 1e-7
    # binary32 twin within rounding
    assert np.abs(orc.heightmap(row[None], cyl(r, h)[None], f32=True) - got).max() <= 2e-6


def test_heightmap_grasp_of_cylinder_target(orc):
    """An isolated upright cylinder (diameter below the opening) is graspable; ringed by
    tall boxes it is not."""
    from paper_2207_06649_b300 import scenegen as sg
    st = [G.box_row(0, 0, 0.03)]
    half = [cyl(0.02, 0.03)]
    assert orc.grasp_heightmap(np.stack(st), np.stack(half), 0, f32=False)
    for k in range(8):
        a = k * math.pi / 4
        st.append(G.box_row(0.045 * math.cos(a), 0.045 * math.sin(a), 0.04, q=G.yaw_q(a)))
        half.append(np.array([0.008, 0.012, 0.04], np.float32))
    assert not orc.grasp_heightmap(np.stack(st), np.stack(half), 0, f32=False)
    assert sg.is_cylinder(np.stack(half)).tolist() == [True] + [False] * 8


def test_crossed_cylinder_edges_meet_at_one_point(orc):
    """Two lying cylinders crossing at right angles, the lower with a corner edge up and
    the upper with one down: edge-edge axis (the two cylinder axes, id 200), separation =
    the gap, one point midway between the edges above their crossing."""
    r, h, gap = 0.02, 0.04, 4e-4
    qA = G.quat_from_rotvec([0, math.pi / 2, 0])    # axis along x, corner 8 up
    qB = G.quat_from_rotvec([-math.pi / 2, 0, 0])   # axis along y, corner 4 down
    sA = G.box_row(0, 0, 0, q=tuple(qA))
    sB = G.box_row(0.003, -0.002, 2 * r + gap, q=tuple(qB))
    res = orc.box_box(sA, cyl(r, h), sB, cyl(r, h))
    assert res["axis"] == 200
    assert np.allclose(res["n"], [0, 0, 1], atol=1e-9)
    assert abs(res["sep"] - gap) < 1e-8
    assert len(res["pts"]) == 1
    assert np.allclose(res["pts"][0], [0.003, 0.0, r + gap / 2], atol=1e-8)
