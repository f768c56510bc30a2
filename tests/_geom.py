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
