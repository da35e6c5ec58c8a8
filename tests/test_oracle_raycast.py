"""Pins of the FP64 ray-casting oracle (appendix, depth rendering: depth maps,
instance segmentation and point clouds ray cast from the simulation state)
against closed forms and geometric facts computed independently of it
(scipy rotations, 2D point-in-triangle, angular sphere silhouettes).
"""
import numpy as np
import pytest

import oracle

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation

W, H = 40, 30
INTR = (36.0, 34.0, 19.3, 14.6, 0.05, 10.0)   # fx, fy, cx, cy, z_near, z_far


def _pose(p, rot):
    x, y, z, w = rot.as_quat()
    return np.array([*p, w, x, y, z])


def _rays(rot):
    """World directions (d_cam z = 1) of every pixel through scipy's rotation."""
    u, v = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    dc = np.stack([(u - INTR[2]) / INTR[0], (v - INTR[3]) / INTR[1], np.ones_like(u)], -1)
    return rot.apply(dc.reshape(-1, 3)).reshape(H, W, 3)


NO_MESH = (np.zeros((0, 3)), np.zeros((0, 3), np.int32))
GROUND = ([1], np.zeros((1, 3)), [[0, 0, 0, 1, 0, 0, 0]])


@pytest.mark.parametrize("tilt", [0.0, 0.35])
def test_ground_plane_closed_form(tilt):
    """Camera 1.2 m above the ground looking down, tilted about its x axis:
    t = height / (-d_z) where the ray descends (and t <= z_far), else no hit;
    the hit points lie on z = 0."""
    rot = Rotation.from_euler("x", 180 + np.degrees(tilt), degrees=True)
    cam = _pose((0.1, -0.2, 1.2), rot)
    d, s, p = oracle.raycast(*NO_MESH, *GROUND, cam, INTR, W, H)
    dw = _rays(rot)
    t = np.where(dw[..., 2] < 0, 1.2 / np.maximum(-dw[..., 2], 1e-300), 0.0)
    t = np.where(t <= INTR[5], t, 0.0)
    assert np.allclose(d, t, rtol=1e-12, atol=0)
    assert ((s == 2) == (t > 0)).all()
    assert np.abs(p[s == 2][:, 2]).max() < 1e-12
    assert np.isnan(p[s == 0]).all()


def test_triangle_parallel_to_image_plane():
    """A triangle at depth 0.8 facing the camera: pixel hit iff the image point
    scaled to that depth lies inside the 2D triangle; depth exactly 0.8."""
    Z = 0.8
    tri2 = np.array([[-0.31, -0.17], [0.27, -0.21], [0.05, 0.29]])
    x = np.c_[tri2, np.full(3, Z)]
    d, s, p = oracle.raycast(x, [[0, 1, 2]], [], [], [], _pose((0, 0, 0), Rotation.identity()), INTR, W, H)
    u, v = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    X = (u - INTR[2]) / INTR[0] * Z
    Y = (v - INTR[3]) / INTR[1] * Z
    inside = np.ones((H, W), bool)
    for i in range(3):
        a, b, c = tri2[i], tri2[(i + 1) % 3], tri2[(i + 2) % 3]
        side = (b[0] - a[0]) * (Y - a[1]) - (b[1] - a[1]) * (X - a[0])
        ref = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
        assert np.abs(side).min() > 1e-9          # no pixel on an edge
        inside &= np.sign(side) == np.sign(ref)
    assert inside.sum() > 50 and (~inside).sum() > 50
    assert ((s == 1) == inside).all() and (s[~inside] == 0).all()
    assert np.allclose(d[inside], Z, rtol=1e-14) and (d[~inside] == 0).all()


def test_sphere_silhouette_and_surface():
    """Sphere of radius 0.1 at 1 m: a ray hits iff its angle to the centre is
    below asin(r/|c|); the hit point is on the sphere and on its near side."""
    c = np.array([0.05, -0.02, 1.0])
    r = 0.1
    rot = Rotation.from_euler("y", 3, degrees=True)
    d, s, p = oracle.raycast(*NO_MESH, [2], [[r, 0, 0]], [[*c, 1, 0, 0, 0]], _pose((0, 0, 0), rot), INTR, W, H)
    dw = _rays(rot)
    cosang = (dw @ c) / (np.linalg.norm(dw, axis=-1) * np.linalg.norm(c))
    hit = cosang > np.cos(np.arcsin(r / np.linalg.norm(c)))
    assert hit.sum() > 20 and ((s == 2) == hit).all()
    q = p[hit]
    assert np.abs(np.linalg.norm(q - c, axis=1) - r).max() < 1e-12
    assert ((dw[hit] * (q - c)).sum(1) < 0).all()


def test_box_top_face_from_above():
    """Camera straight above a yawed box on the ground: pixels whose ray meets
    the top face's footprint see depth height - 2 h_z, the rest the ground."""
    hx, hy, hz = 0.12, 0.07, 0.05
    yaw = Rotation.from_euler("z", 25, degrees=True)
    box_pose = _pose((0.03, 0.02, hz), yaw)
    rot = Rotation.from_euler("x", 180, degrees=True)
    Hc = 0.9
    d, s, p = oracle.raycast(*NO_MESH, [1, 3], [[0, 0, 0], [hx, hy, hz]], [[0, 0, 0, 1, 0, 0, 0], box_pose],
                             _pose((0, 0, Hc), rot), INTR, W, H)
    dw = _rays(rot)
    t_top = (Hc - 2 * hz) / -dw[..., 2]
    xy = t_top[..., None] * dw[..., :2] - np.array([0.03, 0.02])
    local = yaw.inv().apply(np.c_[xy.reshape(-1, 2), np.zeros(H * W)])[:, :2].reshape(H, W, 2)
    top = (np.abs(local[..., 0]) < hx) & (np.abs(local[..., 1]) < hy)
    assert top.sum() > 20
    assert ((s == 3) == top).all()
    assert np.allclose(d[top], Hc - 2 * hz, rtol=1e-12)
    assert np.allclose(d[~top], Hc, rtol=1e-12) and (s[~top] == 2).all()


def test_nearest_of_single_primitive_renders():
    """The combined render is the per-pixel nearest of rendering each
    primitive alone, and does not depend on the triangle order."""
    g = np.random.default_rng(5)
    x = g.uniform(-0.4, 0.4, (30, 3)) + [0, 0, 1.2]
    tris = g.permutation(30).reshape(10, 3)
    ot, od, op = [2, 3], [[0.15, 0, 0], [0.1, 0.2, 0.05]], [[0.55, 0.35, 1.5, 1, 0, 0, 0], [-0.1, 0, 1.1, 0.9, 0.1, 0.3, 0.2]]
    op[1][3:] = list(np.array(op[1][3:]) / np.linalg.norm(op[1][3:]))
    cam = _pose((0, 0, 0), Rotation.identity())
    d, s, p = oracle.raycast(x, tris, ot, od, op, cam, INTR, W, H)
    best = np.full((H, W), np.inf)
    inst = np.zeros((H, W), int)
    for f in range(len(tris)):
        df, sf, _ = oracle.raycast(x, tris[f:f + 1], [], [], [], cam, INTR, W, H)
        m = (sf == 1) & (df < best)
        best[m], inst[m] = df[m], 1
    for k in range(2):
        dk, sk, _ = oracle.raycast(*NO_MESH, ot[k:k + 1], od[k:k + 1], op[k:k + 1], cam, INTR, W, H)
        m = (sk == 2) & (dk < best)
        best[m], inst[m] = dk[m], 2 + k
    assert (inst == s).all() and len(np.unique(s)) == 4
    assert np.allclose(np.where(s > 0, best, 0), d, rtol=1e-15)
    d2, s2, p2 = oracle.raycast(x, tris[::-1], ot, od, op, cam, INTR, W, H)
    assert (s2 == s).all() and np.array_equal(d2, d)


def test_points_reproject_to_pixel_centres():
    """World hit points map back through the camera model to their pixel
    centres and their depth."""
    rot = Rotation.from_euler("xyz", [170, 8, -20], degrees=True)
    cam_p = np.array([0.2, 0.1, 1.0])
    d, s, p = oracle.raycast(*NO_MESH, [1, 2], [[0, 0, 0], [0.2, 0, 0]],
                             [[0, 0, 0, 1, 0, 0, 0], [0.25, 0.05, 0.1, 1, 0, 0, 0]], _pose(cam_p, rot), INTR, W, H)
    v, u = np.nonzero(s > 0)
    pc = rot.inv().apply(p[v, u] - cam_p)
    assert np.allclose(pc[:, 2], d[v, u], rtol=1e-12)
    assert np.allclose(INTR[0] * pc[:, 0] / pc[:, 2] + INTR[2], u + 0.5, atol=1e-9)
    assert np.allclose(INTR[1] * pc[:, 1] / pc[:, 2] + INTR[3], v + 0.5, atol=1e-9)
    assert (s == 3).sum() > 10 and (s == 2).sum() > 10


def test_dilation_decides_rays_through_shared_edges():
    """Two triangles sharing a diagonal that passes exactly through pixel
    centres (corners on pixel centres too): a shrunk test loses those pixels
    to the ground behind, a grown test keeps them; pixels away from the
    edges are the same either way."""
    # camera at the origin looking along +z; the square's diagonal from
    # image point (0.5, 0.5) to (W - 0.5, H - 0.5) scaled to depth Z
    Z = 0.5
    def at(u, v):
        return [(u - INTR[2]) / INTR[0] * Z, (v - INTR[3]) / INTR[1] * Z, Z]
    x = np.array([at(0.5, 0.5), at(W - 0.5, 0.5), at(0.5, H - 0.5), at(W - 0.5, H - 0.5)])
    tris = [[0, 1, 3], [0, 3, 2]]
    cam = _pose((0, 0, 0), Rotation.identity())
    ground = ([1], np.zeros((1, 3)), [[0, 0, 2.0, 1, 0, 0, 0]])   # plane z = 2 behind the square
    diag = [(v, u) for v in range(H) for u in range(W) if abs((u - 0.0) * (H - 1) - v * (W - 1)) == 0]
    assert len(diag) >= 2
    d0, s0, _ = oracle.raycast(x, tris, *ground, cam, INTR, W, H, dil=0.0)
    dm, sm, _ = oracle.raycast(x, tris, *ground, cam, INTR, W, H, dil=-1e-6)
    dp, sp, _ = oracle.raycast(x, tris, *ground, cam, INTR, W, H, dil=1e-6)
    for v, u in diag:   # undilated, the FP64 decision on the edge itself is rounding's
        assert sp[v, u] == 1 and sm[v, u] == 2
    inner = np.zeros((H, W), bool)
    inner[1:-1, 1:-1] = True
    for v, u in diag:
        inner[v, u] = False
    assert (s0[inner] == 1).all() and (sm[inner] == 1).all()


def test_near_and_far_clip():
    """Surfaces before z_near or beyond z_far are not seen."""
    x = np.array([[-1, -1, 0.03], [1, -1, 0.03], [0, 1.5, 0.03]])
    cam = _pose((0, 0, 0), Rotation.identity())
    d, s, _ = oracle.raycast(x, [[0, 1, 2]], [1], [[0, 0, 0]], [[0, 0, 12.0, 1, 0, 0, 0]], cam, INTR, W, H)
    assert (s == 0).all() and (d == 0).all()
    intr = INTR[:5] + (20.0,)
    d, s, _ = oracle.raycast(x, [[0, 1, 2]], [1], [[0, 0, 0]], [[0, 0, 12.0, 1, 0, 0, 0]], cam, intr, W, H)
    assert (s == 2).all() and np.allclose(d, 12.0, rtol=1e-14)
