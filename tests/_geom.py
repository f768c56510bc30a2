"""Independent geometry helpers for the tests (scipy rotations, vertex enumeration).

Written separately from both the oracle and the CUDA engine so that pins computed here
do not re-use either side's formulas.
"""
import math

import numpy as np
from scipy.spatial.transform import Rotation


def rotmat(q_wxyz):
    w, x, y, z = [float(v) for v in q_wxyz]
    return Rotation.from_quat([x, y, z, w]).as_matrix()


def quat_from_rotvec(rv):
    x, y, z, w = Rotation.from_rotvec(rv).as_quat()
    return np.array([w, x, y, z])


def vertices(state_row, half):
    R = rotmat(state_row[3:7])
    c = np.asarray(state_row[:3], np.float64)
    out = []
    for v in range(8):
        l = np.array([(1 if v & 1 else -1) * half[0], (1 if v & 2 else -1) * half[1],
                      (1 if v & 4 else -1) * half[2]], np.float64)
        out.append(c + R @ l)
    return np.array(out)


def support_gap(stA, hA, stB, hB, L):
    """min over B's vertices of L.x minus max over A's vertices of L.x."""
    vA = vertices(stA, hA) @ L
    vB = vertices(stB, hB) @ L
    return vB.min() - vA.max()


def random_unit_vectors(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def box_row(x, y, z, q=(1, 0, 0, 0), v=(0, 0, 0), w=(0, 0, 0)):
    return np.array([x, y, z, *q, *v, *w], np.float64)


def yaw_q(yaw):
    return (math.cos(yaw / 2), 0.0, 0.0, math.sin(yaw / 2))


def cyl_vertices(state_row, r, h):
    """The 32 corners of the right prism over the regular 16-gon inscribed in a cylinder
    of radius r and half height h: cap vertex k at angle k pi/8 in the body xy plane,
    bottom cap (k = 0..15) then top cap."""
    R = rotmat(state_row[3:7])
    c = np.asarray(state_row[:3], np.float64)
    ang = np.arange(16) * np.pi / 8
    out = []
    for z in (-h, h):
        for a in ang:
            out.append(c + R @ np.array([r * math.cos(a), r * math.sin(a), z]))
    return np.array(out)


def body_vertices(state_row, half):
    """Corners of a box, or of a cylinder's prism when half = (r, -r, h)."""
    half = np.asarray(half, np.float64)
    if half[1] < 0:
        return cyl_vertices(state_row, half[0], half[2])
    return vertices(state_row, half)


def body_gap(stA, hA, stB, hB, L):
    """min over B's corners of L.x minus max over A's corners of L.x."""
    return (body_vertices(stB, hB) @ L).min() - (body_vertices(stA, hA) @ L).max()


def rotation_angle_between(qa, qb):
    """Angle of the relative rotation between unit quaternions (w, x, y, z), row-wise:
    2 atan2(|vec(conj(qa) qb)|, |w(conj(qa) qb)|).  Well conditioned for small angles,
    unlike 2 arccos(|qa . qb|), which turns a norm error eps of a binary32 quaternion into
    an apparent angle of 2 sqrt(2 eps) (about 7e-4 rad at eps = 6e-8)."""
    qa = np.asarray(qa, np.float64)
    qb = np.asarray(qb, np.float64)
    qa = qa / np.linalg.norm(qa, axis=-1, keepdims=True)
    qb = qb / np.linalg.norm(qb, axis=-1, keepdims=True)
    wa, va = qa[..., :1], qa[..., 1:]
    wb, vb = qb[..., :1], qb[..., 1:]
    w = wa[..., 0] * wb[..., 0] + np.sum(va * vb, axis=-1)
    v = wa * vb - wb * va - np.cross(va, vb)
    return 2 * np.arctan2(np.linalg.norm(v, axis=-1), np.abs(w))
