"""The seeded scenes hold the geometry their descriptions state (the input
recipe of the box-feature workload and of the two closed-form supports).
Box corners and edges are computed here with scipy rotations, independently
of both the oracle and the CUDA path.  No GPU."""
import numpy as np
from scipy.spatial.transform import Rotation

from paper_2604_17513_gb300 import scenes


def _world(pose, pts):
    return Rotation.from_quat([pose[4], pose[5], pose[6], pose[3]]).apply(pts) + pose[:3]


def _corners(d):
    return np.array([[s0 * d[0], s1 * d[1], s2 * d[2]] for s2 in (-1, 1) for s1 in (-1, 1) for s0 in (-1, 1)])


def test_bar_drop_geometry():
    """Environment 0: the bar runs along x midway between vertex rows n/4 and
    n/4 + 1 and is narrower than the gap to them; the post's top face lies
    strictly inside one triangle; both tops at 5 cm; the cloth starts flat
    2-6 mm above them; other environments turn the bar by at most 4 degrees."""
    sc = scenes.cloth_bar_drop(n_envs=6, steps=2)
    n_side, side = 16, 0.25
    sp = side / (n_side - 1)
    ys = np.unique(np.round(sc.rest[:, 1], 12))
    bar, post = sc.poses[0, 0, 1], sc.poses[0, 0, 2]
    jb = n_side // 4
    assert abs(bar[1] - 0.5 * (ys[jb] + ys[jb + 1])) < 1e-12
    assert sc.obs_dims[0, 1, 1] < 0.5 * sp - sc.thickness - 1e-3   # vertices pass beside the bar
    top_bar = _world(bar, _corners(sc.obs_dims[0, 1]))[:, 2].max()
    top_post = _world(post, _corners(sc.obs_dims[0, 2]))[:, 2].max()
    assert abs(top_bar - 0.05) < 1e-12 and abs(top_post - 0.05) < 1e-12
    # the post's top corners inside a triangle by barycentric coordinates
    top = _world(post, _corners(sc.obs_dims[0, 2]))[4:, :2]
    inside = []
    for t in sc.elems:
        P = sc.rest[t][:, :2]
        T = np.c_[P[1] - P[0], P[2] - P[0]]
        w = np.linalg.solve(T, (top - P[0]).T).T
        bary = np.c_[1 - w.sum(1), w]
        inside.append((bary > 0).all())
    assert sum(inside) == 1
    for e in range(sc.n_envs):
        gap = sc.q0[e][:, 2].min() - 0.05 - sc.thickness
        assert 0.002 <= gap <= 0.006 and np.ptp(sc.q0[e][:, 2]) < 1e-12
        yaw = Rotation.from_quat(sc.poses[e, 0, 1, [4, 5, 6, 3]]).as_euler("xyz")
        assert abs(yaw[0]) < 1e-12 and abs(yaw[1]) < 1e-12 and abs(yaw[2]) <= np.deg2rad(4) + 1e-12
        assert (e == 0) == (abs(yaw[2]) < 1e-15)


def test_support_scene_geometry():
    """corner_support: the cube's corner 7 is the top, directly under the
    triangle's centroid one thickness below it, and every other corner is
    out of reach (thickness + margin).  edge_support: the bar's edge 3 is the
    top, along x under the square's middle line one thickness below it, and
    every other long edge is out of reach."""
    sc = scenes.corner_support()
    C = _world(sc.poses[0, 0, 0], _corners(sc.obs_dims[0, 0]))
    cen = sc.q0[0].mean(0)
    assert np.argmax(C[:, 2]) == 7
    assert np.abs(C[7, :2] - cen[:2]).max() < 1e-12 and abs(cen[2] - C[7, 2] - sc.thickness) < 1e-12
    others = np.delete(C, 7, axis=0)
    assert (cen[2] - others[:, 2] > sc.thickness + sc.margin).all()
    sc = scenes.edge_support()
    d = sc.obs_dims[0, 0]
    z = []
    for m in range(4):   # the four long edges (along x): signs of (y, z) from bits 0 and 1
        p = np.array([0.0, d[1] if m & 1 else -d[1], d[2] if m & 2 else -d[2]])
        z.append(_world(sc.poses[0, 0, 0], p[None])[0])
    z = np.array(z)
    assert np.argmax(z[:, 2]) == 3 and abs(z[3, 1]) < 1e-12
    zq = sc.q0[0][:, 2]
    assert np.ptp(zq) < 1e-12 and abs(zq[0] - z[3, 2] - sc.thickness) < 1e-12
    assert (zq[0] - np.delete(z, 3, axis=0)[:, 2] > sc.thickness + sc.margin).all()
