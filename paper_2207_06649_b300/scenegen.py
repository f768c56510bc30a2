"""Seeded synthetic inputs for the batched push-rollout engine.

These generators stand in for the paper's evaluation scenes (Sec. V-A: 20 clutter
cases that are not available here).  They produce boxes (and, on request, upright
cylinders) resting on a table plane at non-overlapping, seeded positions and straight
push actions a^p = (x_s, y_s, x_e, y_e)
(Sec. III-A, action space).  The module is input data only: it holds none of the
engine's physics, contact, grasp or sampling arithmetic, and both the CUDA path and
the CPU oracle consume its output.

Scene arrays (CSR over boxes, all little-endian, C-contiguous):
  box_offset int32[S+1]   boxes of scene s are rows box_offset[s]:box_offset[s+1]
  pose       float32[B,7] x, y, z, qw, qx, qy, qz
  vel        float32[B,6] linear xyz, angular xyz (zeros: boxes start at rest)
  half       float32[B,3] half-extents (m); a row (r, -r, h) is an upright cylinder of
                          radius r and half height h about its body z axis
  mass       float32[B]   kg
  mu         float32[B]   Coulomb friction coefficient
  target     int32[S]     local index of the target box in its scene
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

TABLE_HALF = 0.2          # 0.4 x 0.4 m table
PUSHER_RADIUS = 0.01
PUSH_LENGTH = 0.1
PLACEMENT_GAP = 1e-3      # footprints at least 1 mm apart


@dataclass
class Scenes:
    box_offset: np.ndarray
    pose: np.ndarray
    vel: np.ndarray
    half: np.ndarray
    mass: np.ndarray
    mu: np.ndarray
    target: np.ndarray

    @property
    def n_scenes(self) -> int:
        return int(self.box_offset.shape[0] - 1)

    def counts(self) -> np.ndarray:
        return np.diff(self.box_offset).astype(np.int32)

    def scene(self, s: int) -> "Scenes":
        a, b = int(self.box_offset[s]), int(self.box_offset[s + 1])
        return Scenes(np.array([0, b - a], np.int32), self.pose[a:b].copy(),
                      self.vel[a:b].copy(), self.half[a:b].copy(), self.mass[a:b].copy(),
                      self.mu[a:b].copy(), self.target[s:s + 1].copy())

    def gather(self, scene_ids) -> "Scenes":
        """Per-env copy of the selected scenes (env e gets scene scene_ids[e])."""
        parts = [self.scene(int(s)) for s in scene_ids]
        return concat(parts)


def concat(parts) -> Scenes:
    offs, base = [np.zeros(1, np.int64)], 0
    for p in parts:
        offs.append(np.asarray(p.box_offset[1:], np.int64) + base)
        base += int(p.box_offset[-1])
    off = np.concatenate(offs).astype(np.int32)
    cat =lambda name, shape: (np.concatenate([getattr(p, name) for p in parts])
                               if parts else np.zeros(shape, np.float32))
    return Scenes(off, cat("pose", (0, 7)).astype(np.float32),
                  cat("vel", (0, 6)).astype(np.float32), cat("half", (0, 3)).astype(np.float32),
                  cat("mass", (0,)).astype(np.float32), cat("mu", (0,)).astype(np.float32),
                  (np.concatenate([p.target for p in parts]) if parts
                   else np.zeros(0, np.int32)).astype(np.int32))


def cylinder_half(r: float, h: float) -> np.ndarray:
    """Half-extent row of a cylinder of radius r and half height h."""
    return np.array([r, -r, h], np.float32)


def is_cylinder(half) -> np.ndarray:
    """Cylinder mask of half-extent rows (negative second entry)."""
    return np.asarray(half)[..., 1] < 0


def _corners(cx, cy, hx, hy, yaw):
    """Corners [..., 4, 2] of yawed rectangles (broadcast over leading dims)."""
    c, s = np.cos(yaw), np.sin(yaw)
    sx = np.array([1, -1, -1, 1], np.float64)
    sy = np.array([1, 1, -1, -1], np.float64)
    lx = sx * np.asarray(hx)[..., None]
    ly = sy * np.asarray(hy)[..., None]
    x = np.asarray(cx)[..., None] + np.asarray(c)[..., None] * lx - np.asarray(s)[..., None] * ly
    y = np.asarray(cy)[..., None] + np.asarray(s)[..., None] * lx + np.asarray(c)[..., None] * ly
    return np.stack([x, y], -1)


def _overlaps(cand, placed, gap):
    """Placement test: candidate rectangles [K] (cx, cy, hx, hy, yaw) against placed
    rectangles [P], each grown by gap/2.  Pairs whose circumscribed circles are apart
    are free, pairs whose inscribed circles meet overlap, the rest go through the
    separating-axis test over the four edge normals.  Returns bool [K, P] (True =
    overlap).  Used only to place boxes."""
    K, P = cand.shape[0], placed.shape[0]
    g2 = gap / 2
    d = np.hypot(cand[:, None, 0] - placed[None, :, 0], cand[:, None, 1] - placed[None, :, 1])
    Rc = np.hypot(cand[:, 2] + g2, cand[:, 3] + g2)
    Rp = np.hypot(placed[:, 2] + g2, placed[:, 3] + g2)
    rc = np.minimum(cand[:, 2], cand[:, 3]) + g2
    rp = np.minimum(placed[:, 2], placed[:, 3]) + g2
    out = d < (rc[:, None] + rp[None, :])
    amb = ~out & (d <= (Rc[:, None] + Rp[None, :]))
    ki, pi = np.nonzero(amb)
    if ki.size:
        a, b = cand[ki], placed[pi]
        ca = _corners(a[:, 0], a[:, 1], a[:, 2] + g2, a[:, 3] + g2, a[:, 4])
        cb = _corners(b[:, 0], b[:, 1], b[:, 2] + g2, b[:, 3] + g2, b[:, 4])
        sep = np.zeros(ki.size, bool)
        for yaw in (a[:, 4], b[:, 4]):
            for ax in ((np.cos(yaw), np.sin(yaw)), (-np.sin(yaw), np.cos(yaw))):
                pa = ca[..., 0] * ax[0][:, None] + ca[..., 1] * ax[1][:, None]
                pb = cb[..., 0] * ax[0][:, None] + cb[..., 1] * ax[1][:, None]
                sep |= (pa.max(-1) <= pb.min(-1)) | (pb.max(-1) <= pa.min(-1))
        out[ki, pi] = ~sep
    return out


def _yaw_quat(yaw):
    return (math.cos(yaw / 2), 0.0, 0.0, math.sin(yaw / 2))


def make_scene(rng: np.random.Generator, n: int, *, half_lo=0.015, half_hi=0.03,
               mass_lo=0.05, mass_hi=0.2, mu_lo=0.5, mu_hi=0.5, yaw_hi=0.0,
               region_half=0.08, density_scale=None, attempts=1000,
               target_at_centre=False, cyl_frac=0.0, target_cylinder=False) -> Scenes:
    """One scene of up to n boxes placed by rejection sampling inside a centred square
    clutter region; boxes rest on the plane (z = h_z) with zero velocity.  Boxes that
    fail `attempts` placements are dropped (so the final count may be below n).
    Box 0 is the target.  With cyl_frac > 0 each object is an upright cylinder with that
    probability (radius min(h_x, h_y) of its drawn extents, half height h_z), and
    target_cylinder makes object 0 one; these draws follow all the others, so scenes
    without cylinders are unchanged."""
    halves = rng.uniform(half_lo, half_hi, size=(n, 3))
    masses = rng.uniform(mass_lo, mass_hi, size=n) if mass_hi > mass_lo else np.full(n, mass_lo)
    mus = rng.uniform(mu_lo, mu_hi, size=n) if mu_hi > mu_lo else np.full(n, mu_lo)
    yaws = rng.uniform(0.0, yaw_hi, size=n) if yaw_hi > 0 else np.zeros(n)
    cyl = np.zeros(n, bool)
    if cyl_frac > 0 or target_cylinder:
        cyl = rng.uniform(size=n) < cyl_frac
        cyl[0] |= target_cylinder
        r = np.minimum(halves[:, 0], halves[:, 1])
        halves[cyl, 0] = r[cyl]
        halves[cyl, 1] = r[cyl]
    if density_scale is not None:
        area = float(np.sum(4 * halves[:, 0] * halves[:, 1]))
        region_half = min(math.sqrt(area / density_scale) / 2, TABLE_HALF)
    placed = []
    arr = np.zeros((0, 5))
    for i in range(n):
        hx, hy = halves[i, 0], halves[i, 1]
        # conservative footprint radius, so the footprint stays inside the region
        rad = math.hypot(hx, hy) if yaws[i] != 0 else max(hx, hy)
        lim = region_half - rad
        if i == 0:
            lim = max(lim, 1e-3)   # the target always fits, even in a tiny dense region
        ok = False
        tried = 0
        while lim > 0 and tried < attempts and not ok:
            k = min(250, attempts - tried)
            xy = rng.uniform(-lim, lim, size=(k, 2))
            if i == 0 and target_at_centre and tried == 0:
                xy[0] = 0.0
            tried += k
            cand = np.column_stack([xy, np.full(k, hx), np.full(k, hy), np.full(k, yaws[i])])
            free = ~_overlaps(cand, arr, PLACEMENT_GAP).any(1) if len(arr) else np.ones(k, bool)
            if free.any():
                j = int(np.argmax(free))
                cx, cy = xy[j]
                placed.append((cx, cy, hx, hy, yaws[i], halves[i, 2], masses[i], mus[i], bool(cyl[i])))
                arr = np.vstack([arr, [cx, cy, hx, hy, yaws[i]]])
                ok = True
        if not ok and i == 0:
            raise RuntimeError("target could not be placed")
    m = len(placed)
    pose = np.zeros((m, 7), np.float64)
    half = np.zeros((m, 3), np.float64)
    for k, p in enumerate(placed):
        pose[k, :3] = (p[0], p[1], p[5])
        pose[k, 3:] = _yaw_quat(p[4])
        half[k] = (p[2], p[3], p[5])
        if p[8]:
            half[k, 1] = -p[2]
    return Scenes(np.array([0, m], np.int32), pose.astype(np.float32),
                  np.zeros((m, 6), np.float32), half.astype(np.float32),
                  np.array([p[6] for p in placed], np.float32),
                  np.array([p[7] for p in placed], np.float32), np.array([0], np.int32))


def _support_half_width(half, quat, d):
    """Half-width of an upright yawed box's footprint along the unit 2-D direction d (a
    cylinder's radius)."""
    if half[1] < 0:
        return float(half[0])
    yaw = 2 * math.atan2(quat[3], quat[0])
    u = (math.cos(yaw), math.sin(yaw))
    v = (-u[1], u[0])
    return abs(d[0] * u[0] + d[1] * u[1]) * half[0] + abs(d[0] * v[0] + d[1] * v[1]) * half[1]


def push_through_target(sc: Scenes, theta: float, offset: float, standoff=0.05,
                        length=PUSH_LENGTH, radius=PUSHER_RADIUS):
    """Push along direction theta through the target centre shifted by `offset` along the
    left normal; it starts standoff + radius beyond the target's support half-width."""
    t = int(sc.target[0])
    d = (math.cos(theta), math.sin(theta))
    perp = (-d[1], d[0])
    c = sc.pose[t, :2].astype(np.float64)
    w = _support_half_width(sc.half[t].astype(np.float64), sc.pose[t, 3:].astype(np.float64), d)
    back = w + radius + standoff
    sx = c[0] + offset * perp[0] - d[0] * back
    sy = c[1] + offset * perp[1] - d[1] * back
    return np.array([sx, sy, sx + d[0] * length, sy + d[1] * length], np.float32)


def config_tiny(seed: int = 1, n_boxes: int = 5):
    """16 envs of one 5-box scene (axis-aligned, half-extents U[0.015,0.03], mass
    U[0.05,0.2], mu 0.5); env e runs push e of 8 directions x 2 offsets (+-0.01 m)."""
    rng = np.random.default_rng(seed)
    sc = make_scene(rng, n_boxes, region_half=0.08)
    pushes = []
    for k in range(8):
        for off in (-0.01, 0.01):
            pushes.append(push_through_target(sc, k * math.pi / 4, off))
    return sc, np.stack(pushes)


def config_fixed(seed: int = 2, n_boxes: int = 15, n_envs: int = 1024):
    """One 15-box scene cloned to 1024 envs; push e = direction floor(e/16) of 64 times
    offset (e mod 16) in {-0.075 .. 0.075} step 0.01 m.  Seeds 1000+e drive the
    device-sampled pushes 2..D."""
    rng = np.random.default_rng(seed)
    # a 0.28 m clutter square: large enough that all 15 boxes find a place
    sc = make_scene(rng, n_boxes, region_half=0.14)
    pushes = []
    for e in range(n_envs):
        k, o = e // 16, e % 16
        pushes.append(push_through_target(sc, 2 * math.pi * k / 64, -0.075 + 0.01 * o))
    seeds = (1000 + np.arange(n_envs)).astype(np.uint64)
    return sc, np.stack(pushes), seeds


def _random_valid_push(rng, sc: Scenes, s: int, attempts=200):
    """A random push toward one box centre whose start disk (pusher radius + 1 mm)
    clears every footprint; falls back to a push from outside the clutter."""
    a, b = int(sc.box_offset[s]), int(sc.box_offset[s + 1])
    pose, half = sc.pose[a:b].astype(np.float64), sc.half[a:b].astype(np.float64)
    n = b - a
    for _ in range(attempts):
        j = int(rng.integers(n))
        th = rng.uniform(0, 2 * math.pi)
        d = (math.cos(th), math.sin(th))
        w = _support_half_width(half[j], pose[j, 3:], d)
        back = w + PUSHER_RADIUS + rng.uniform(0.002, 0.03)
        sx, sy = pose[j, 0] - d[0] * back, pose[j, 1] - d[1] * back
        clear = True
        for i in range(n):
            yaw = 2 * math.atan2(pose[i, 6], pose[i, 3])
            c, sn = math.cos(yaw), math.sin(yaw)
            dx, dy = sx - pose[i, 0], sy - pose[i, 1]
            lu, lv = c * dx + sn * dy, -sn * dx + c * dy
            qu = max(abs(lu) - half[i, 0], 0.0)
            qv = max(abs(lv) - abs(half[i, 1]), 0.0)
            if qu * qu + qv * qv < (PUSHER_RADIUS + 1e-3) ** 2:
                clear = False
                break
        if clear:
            return np.array([sx, sy, sx + d[0] * PUSH_LENGTH, sy + d[1] * PUSH_LENGTH], np.float32)
    return np.array([0.19, 0.19, 0.19, 0.09], np.float32)


def _uneven_scene(args):
    ss, n_lo, n_hi = args
    rng = np.random.default_rng(ss)
    n = int(rng.integers(n_lo, n_hi + 1))
    rho = rng.uniform(0.2, 0.6)
    sc = make_scene(rng, n, half_lo=0.01, half_hi=0.04, mu_lo=0.3, mu_hi=0.8,
                    yaw_hi=math.pi / 2, density_scale=rho, attempts=1000)
    return sc, _random_valid_push(rng, sc, 0)


def config_uneven(seed: int = 3, n_envs: int = 4096, n_lo=5, n_hi=40, workers: int = 0):
    """4096 independent scenes: n ~ U{5..40}, half-extents U[0.01,0.04], mu U[0.3,0.8],
    yaw U[0, pi/2), mass U[0.05,0.2], clutter density rho ~ U[0.2,0.6] (sum of footprint
    areas over the area of a centred square region, clipped to the table); one random
    valid push per env; seeds for the device-sampled pushes.  Scene e draws from its own
    child stream of `seed`, so the result does not depend on `workers` (processes used
    to generate; 0 = all cores for large batches)."""
    root = np.random.SeedSequence(seed)
    children = root.spawn(n_envs + 1)
    jobs = [(children[e], n_lo, n_hi) for e in range(n_envs)]
    if workers == 0:
        import os
        workers = (os.cpu_count() or 1) if n_envs >= 256 else 1
    if workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_uneven_scene, jobs, chunksize=max(1, n_envs // (8 * workers)))
    else:
        res = [_uneven_scene(j) for j in jobs]
    scenes = concat([r[0] for r in res])
    pushes = np.stack([r[1] for r in res]) if res else np.zeros((0, 4), np.float32)
    seeds = np.random.default_rng(children[-1]).integers(0, 2 ** 63, size=n_envs, dtype=np.uint64)
    return scenes, pushes, seeds


def _cyl_scene(args):
    ss, n_lo, n_hi, frac = args
    rng = np.random.default_rng(ss)
    n = int(rng.integers(n_lo, n_hi + 1))
    rho = rng.uniform(0.2, 0.6)
    sc = make_scene(rng, n, half_lo=0.01, half_hi=0.04, mu_lo=0.3, mu_hi=0.8,
                    yaw_hi=math.pi / 2, density_scale=rho, attempts=1000,
                    cyl_frac=frac, target_cylinder=True)
    return sc, _random_valid_push(rng, sc, 0)


def config_cylinders(seed: int = 5, n_envs: int = 4096, n_lo=5, n_hi=40, cyl_frac=0.3, workers: int = 0):
    """The uneven workload with cylinders: per scene the same distributions as
    config_uneven, each object an upright cylinder with probability cyl_frac and the
    target always one (the paper's target object is a small cylinder)."""
    root = np.random.SeedSequence(seed)
    children = root.spawn(n_envs + 1)
    jobs = [(children[e], n_lo, n_hi, cyl_frac) for e in range(n_envs)]
    if workers == 0:
        import os
        workers = (os.cpu_count() or 1) if n_envs >= 256 else 1
    if workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_cyl_scene, jobs, chunksize=max(1, n_envs // (8 * workers)))
    else:
        res = [_cyl_scene(j) for j in jobs]
    scenes = concat([r[0] for r in res])
    pushes = np.stack([r[1] for r in res]) if res else np.zeros((0, 4), np.float32)
    seeds = np.random.default_rng(children[-1]).integers(0, 2 ** 63, size=n_envs, dtype=np.uint64)
    return scenes, pushes, seeds


def _buried(pose, half, gap=0.03, rays=16, samples=7):
    """True when, on every one of `rays` rays leaving the target (box 0) footprint, some
    other footprint lies within `gap` of the target's boundary (sampled along the ray)."""
    t = pose[0]
    yaw_t = 2 * math.atan2(t[6], t[3])
    for k in range(rays):
        th = 2 * math.pi * k / rays
        d = np.array([math.cos(th), math.sin(th)])
        w = _support_half_width(half[0], pose[0, 3:], d)
        hit = False
        for s_ in np.linspace(0.0, gap, samples):
            p = pose[0, :2] + d * (w + s_)
            for i in range(1, len(pose)):
                yaw = 2 * math.atan2(pose[i, 6], pose[i, 3])
                c, sn = math.cos(yaw), math.sin(yaw)
                rel = p - pose[i, :2]
                if abs(c * rel[0] + sn * rel[1]) <= half[i, 0] and abs(-sn * rel[0] + c * rel[1]) <= half[i, 1]:
                    hit = True
                    break
            if hit:
                break
        if not hit:
            return False
    return True


def config_planning(seed: int, n_boxes: int = 30, attempts: int = 50):
    """Planning scene: the target (box 0) at the table centre buried in clutter: every one
    of 16 rays from its boundary meets another box within 0.03 m.  For each ray not yet
    covered a box is placed on it just outside the target, aligned with the ray; the
    remaining boxes are placed anywhere on the table by rejection sampling (a box that
    finds no room is redrawn, which favours smaller late boxes).  Sizes, friction and
    masses follow the uneven workload (half extents U[0.01, 0.04], mu U[0.3, 0.8], mass
    U[0.05, 0.2])."""
    rng = np.random.default_rng(seed)
    for _ in range(attempts):
        ht = rng.uniform(0.015, 0.025, size=3)
        yaw_t = rng.uniform(0, math.pi / 2)
        rows = [(0.0, 0.0, ht[0], ht[1], yaw_t, ht[2])]
        arr = np.array([[0.0, 0.0, ht[0], ht[1], yaw_t]])
        tq = np.array(_yaw_quat(yaw_t))
        for k in range(16):
            th = 2 * math.pi * k / 16
            d = np.array([math.cos(th), math.sin(th)])
            pose = np.array([[r[0], r[1], 0, *_yaw_quat(r[4])] for r in rows])
            half = np.array([[r[2], r[3], r[5]] for r in rows])
            w = _support_half_width(ht, tq, d)
            covered = False
            for s_ in np.linspace(0.0, 0.03, 7):
                p = d * (w + s_)
                for r in rows[1:]:
                    c, sn = math.cos(r[4]), math.sin(r[4])
                    rel = p - np.array(r[:2])
                    if abs(c * rel[0] + sn * rel[1]) <= r[2] and abs(-sn * rel[0] + c * rel[1]) <= r[3]:
                        covered = True
                        break
                if covered:
                    break
            if covered:
                continue
            perp = np.array([-d[1], d[0]])
            for _a in range(400):
                hr = rng.uniform(0.01, 0.03)          # radial half extent
                htg = rng.uniform(0.012, 0.035)       # tangential half extent
                gap = rng.uniform(0.0015, 0.02)
                # the box only has to cross the ray: shift it sideways within its width
                ctr = d * (w + gap + hr) + perp * rng.uniform(-(htg - 0.003), htg - 0.003)
                cand = np.array([[ctr[0], ctr[1], hr, htg, th]])
                if not _overlaps(cand, arr, PLACEMENT_GAP).any():
                    rows.append((ctr[0], ctr[1], hr, htg, th, rng.uniform(0.01, 0.04)))
                    arr = np.vstack([arr, cand])
                    break
        redraws = 0
        while len(rows) < n_boxes and redraws < 60:
            h = rng.uniform(0.01, 0.04, size=3)
            yaw = rng.uniform(0, math.pi / 2)
            lim = TABLE_HALF - math.hypot(h[0], h[1]) - 0.005
            ok = False
            for _a in range(8):
                xy = rng.uniform(-lim, lim, size=(250, 2))
                cand = np.column_stack([xy, np.full(250, h[0]), np.full(250, h[1]), np.full(250, yaw)])
                free = ~_overlaps(cand, arr, PLACEMENT_GAP).any(1)
                if free.any():
                    q = int(np.argmax(free))
                    rows.append((xy[q, 0], xy[q, 1], h[0], h[1], yaw, h[2]))
                    arr = np.vstack([arr, cand[q:q + 1]])
                    ok = True
                    break
            if not ok:
                redraws += 1       # no room for this size: draw another box
        if len(rows) != n_boxes:
            continue
        m = n_boxes
        pose = np.zeros((m, 7))
        half = np.zeros((m, 3))
        for k, r in enumerate(rows):
            pose[k, :3] = (r[0], r[1], r[5])
            pose[k, 3:] = _yaw_quat(r[4])
            half[k] = (r[2], r[3], r[5])
        if _buried(pose, half):
            return Scenes(np.array([0, m], np.int32), pose.astype(np.float32), np.zeros((m, 6), np.float32),
                          half.astype(np.float32), rng.uniform(0.05, 0.2, size=m).astype(np.float32),
                          rng.uniform(0.3, 0.8, size=m).astype(np.float32), np.array([0], np.int32))
    raise RuntimeError("no buried scene found")


def random_state_snapshot(rng: np.random.Generator, n: int, spread=0.06, tilt=0.3):
    """Generic box state (arbitrary orientations, small velocities) for snapshot tests
    of pair lists, grasp decisions and sampling; boxes may touch or overlap."""
    pose = np.zeros((n, 7))
    pose[:, :2] = rng.uniform(-spread, spread, size=(n, 2))
    half = rng.uniform(0.01, 0.035, size=(n, 3))
    pose[:, 2] = half[:, 2] + rng.uniform(-0.003, 0.01, size=n)
    axis = rng.normal(size=(n, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    ang = rng.uniform(-tilt, tilt, size=n)
    yaw = rng.uniform(0, 2 * math.pi, size=n)
    for i in range(n):
        qa = np.array([math.cos(ang[i] / 2), *(axis[i] * math.sin(ang[i] / 2))])
        qy = np.array([math.cos(yaw[i] / 2), 0, 0, math.sin(yaw[i] / 2)])
        w1, x1, y1, z1 = qy
        w2, x2, y2, z2 = qa
        q = np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                      w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                      w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                      w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
        pose[i, 3:] = q / np.linalg.norm(q)
    vel = rng.normal(scale=0.02, size=(n, 6))
    return pose.astype(np.float32), vel.astype(np.float32), half.astype(np.float32)


def state13(sc: Scenes) -> np.ndarray:
    """[B,13] rows: x y z qw qx qy qz vx vy vz wx wy wz."""
    return np.concatenate([sc.pose, sc.vel], axis=1).astype(np.float32)
