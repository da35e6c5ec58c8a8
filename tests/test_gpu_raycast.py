"""GPU parity of batched depth ray casting (appendix, depth rendering: depth
maps, instance segmentation and point clouds cast from the simulation state)
against the FP64 brute-force oracle, on the same FP32 inputs.

A pixel's answer is unique unless its ray passes within a hair of a
primitive's boundary (a silhouette edge, a box edge, a sphere's rim), where
FP32 and FP64 may fairly disagree.  The oracle decides that per pixel by
casting twice more with every primitive grown and shrunk by EPS (barycentric
margin, relative radius, relative half extent): where both give the same
instance the pixel is unique and the GPU must match the undilated oracle
(instance exactly; depth and point within TOL); elsewhere the GPU must match
one of the three answers: its instance, at its depth within 1 % (depth is
ill-conditioned there, e.g. where a ray grazes a sphere's rim).

TOL: FP32 depth through a dozen rounded operations on coordinates of order
the depth d is about 2e-6 d, up to 20x more on surfaces seen almost edge-on
(the folded towel's cylinder): |depth error| <= 1e-6 + 4e-5 d.
"""
import numpy as np
import pytest

import oracle
from paper_2604_17513_gb300 import scenes

pytestmark = pytest.mark.gpu

EPS = 1e-3


def _tol(d):
    return 1e-6 + 4e-5 * np.abs(d)


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def _cast_gpu(cuda, rs, seg=True, points=True):
    import torch
    from paper_2604_17513_gb300 import flash
    W, H, fx, fy, cx, cy, zn, zf = rs.cam
    cam = flash.Camera(W, H, fx, fy, cx, cy, zn, zf)
    rc = flash.Raycaster(cam, rs.n_envs, rs.verts.shape[1], rs.tris)
    t = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dt, device=cuda)
    K = rs.obs_type.shape[1]
    out = rc.cast(t(rs.verts), t(rs.obs_type, torch.int32) if K else None, t(rs.obs_dims) if K else None,
                  t(rs.obs_poses) if K else None, t(rs.cam_poses), seg=seg, points=points)
    torch.cuda.synchronize()
    return [None if o is None else o.cpu().numpy() for o in out]


def _oracle(rs, e, uv=None):
    """(undilated, grown, shrunk) oracle answers for environment e, all
    pixels or the pixel list uv."""
    W, H, fx, fy, cx, cy, zn, zf = rs.cam
    intr = (fx, fy, cx, cy, zn, zf)
    args = (_f32(rs.verts[e]), rs.tris, rs.obs_type[e], _f32(rs.obs_dims[e]), _f32(rs.obs_poses[e]),
            _f32(rs.cam_poses[e]), _f32(intr))
    if uv is None:
        return [oracle.raycast(*args, W, H, dil=dl) for dl in (0.0, EPS, -EPS)]
    return [oracle.raycast_pixels(*args, uv, dil=dl) for dl in (0.0, EPS, -EPS)]


def _close(a, b):
    """Agreement of a dilated depth: TOL plus the shift that dilating a sphere
    or box by EPS makes (EPS x 0.1 m)."""
    return np.abs(a - b) <= _tol(b) + EPS * 0.1


def _check(ref, dg, sg, pg, max_ambiguous=0.05):
    (d0, s0, p0), (dp, sp, pp), (dm, sm, pm) = ref
    unique = (s0 == sp) & (s0 == sm) & _close(dp, d0) & _close(dm, d0)
    assert unique.mean() >= 1 - max_ambiguous, unique.mean()
    u = unique
    assert (sg[u] == s0[u]).all(), np.argwhere(u & (sg != s0))[:5]
    assert (np.abs(dg[u] - d0[u]) <= _tol(d0[u])).all(), np.abs(dg[u] - d0[u]).max()
    hit = u & (s0 > 0)
    if pg is not None:
        assert (np.abs(pg[hit] - p0[hit]) <= 2 * _tol(d0[hit])[:, None]).all()
        assert np.isnan(pg[u & (s0 == 0)]).all()
    assert (dg[u & (s0 == 0)] == 0).all()
    a = ~unique
    if a.any():   # ambiguous pixels: the instance of one of the three answers, at its depth within 1 %
        near = lambda d: np.abs(dg[a] - d[a]) <= _tol(d[a]) + 1e-2 * d[a]
        ok = ((sg[a] == s0[a]) & near(d0)) | ((sg[a] == sp[a]) & near(dp)) | ((sg[a] == sm[a]) & near(dm))
        assert ok.all(), (np.argwhere(a)[~ok][:5], sg[a][~ok], s0[a][~ok], sp[a][~ok], sm[a][~ok],
                          dg[a][~ok], d0[a][~ok], dp[a][~ok], dm[a][~ok])
    return unique


def test_towel_views_parity(cuda):
    """Three folded, wrinkled towels (24x24 grid, 1058 triangles) with ground,
    two finger boxes and an invisible carrier, 77x53 images (ragged against
    the 256-pixel blocks), every pixel checked."""
    rs = scenes.towel_views(n_envs=3, n_side=24, side=0.3, width=77, height=53, cam_height=(0.32, 0.4))
    dg, sg, pg = _cast_gpu(cuda, rs)
    for e in range(rs.n_envs):
        ref = _oracle(rs, e)
        _check(ref, dg[e], sg[e], pg[e])
        s0 = ref[0][1]
        assert (s0 == 1).mean() > 0.2 and (s0 == 2).any()


@pytest.mark.parametrize("offset", [(0.0, 0.0), (0.5, 0.0), (0.0, 0.5)])
def test_watertight_grid_no_cracks(cuda, offset):
    """A flat 41x41 grid seen from straight above, scaled to one pixel per
    cell and placed so that pixel rays pass through its vertices (offset 0)
    or through the midpoints of its shared edges: every pixel inside the
    grid's border must hit it (no ray slips between two triangles)."""
    n_side, Hc, f = 41, 0.5, 40.0
    W = H = 48
    rest, tris = scenes.cloth_grid(n_side, n_side, 1.0)
    # camera at (0, 0, Hc) looking down (180 deg about x): pixel (u, v) looks
    # at ground point x = (u - 23.5) p, y = -(v - 23.5) p with pitch p = Hc / f;
    # grid vertex (i, j) in -20..20 sits at pixel (24 + i + ox, 24 - j + oy)
    cx = cy = 24.0
    pitch = Hc / f
    verts = np.zeros((1, len(rest), 3))
    verts[0, :, 0] = (rest[:, 0] * (n_side - 1) + 0.5 + offset[0]) * pitch
    verts[0, :, 1] = (rest[:, 1] * (n_side - 1) - 0.5 - offset[1]) * pitch
    rs = scenes.RayScene("grid", verts, tris, np.array([[1]], np.int32), np.zeros((1, 1, 3)),
                         np.array([[[0, 0, -0.1, 1, 0, 0, 0]]], np.float64),
                         np.array([[0, 0, Hc, 0, 1, 0, 0]], np.float64), (W, H, f, f, cx, cy, 0.05, 5.0))
    dg, sg, pg = _cast_gpu(cuda, rs)
    inner = np.zeros((H, W), bool)
    inner[5:44, 5:44] = True          # pixels strictly inside the border
    assert (sg[0][inner] == 1).all(), int((sg[0][inner] != 1).sum())
    assert np.allclose(dg[0][inner], Hc, rtol=1e-6)
    _check(_oracle(rs, 0), dg[0], sg[0], pg[0], max_ambiguous=1.0)


def test_edge_cases(cuda):
    """No triangles; a camera looking away from everything; a triangle
    reaching behind the camera; a 1x1 image; far clipping; outputs left
    out."""
    g = np.random.default_rng(2)
    verts = np.zeros((2, 3, 3))
    verts[0] = [[-0.5, -0.5, 0.2], [0.6, -0.4, 0.3], [0.0, 0.7, -0.4]]   # crosses the camera plane z = 0.1
    verts[1] = g.uniform(-0.2, 0.2, (3, 3)) + [0, 0, 0.5]
    ot = np.array([[2, 1], [3, 0]], np.int32)
    od = np.array([[[0.1, 0, 0], [0, 0, 0]], [[0.1, 0.1, 0.1], [0, 0, 0]]])
    op = np.array([[[0.1, 0.1, 0.8, 1, 0, 0, 0], [0, 0, -0.5, 1, 0, 0, 0]],
                   [[0, 0, 1.5, 1, 0, 0, 0], [0, 0, 0, 1, 0, 0, 0]]], np.float64)
    cams = np.array([[0, 0, 0.1, 1, 0, 0, 0], [0, 0, 0, 1, 0, 0, 0]], np.float64)
    rs = scenes.RayScene("edge", verts, np.array([[0, 1, 2]], np.int32), ot, od, op, cams,
                         (33, 21, 20.0, 20.0, 16.0, 10.0, 0.05, 3.0))
    dg, sg, pg = _cast_gpu(cuda, rs)
    for e in range(2):
        _check(_oracle(rs, e), dg[e], sg[e], pg[e], max_ambiguous=0.1)
    # the same without the triangle, without outputs, and looking away
    rs0 = scenes.RayScene("edge0", verts[:, :0], np.zeros((0, 3), np.int32), ot, od, op, cams, rs.cam)
    dg0, sg0, pg0 = _cast_gpu(cuda, rs0, seg=True, points=False)
    dg1, sg1, pg1 = _cast_gpu(cuda, rs0, seg=False, points=False)
    assert pg0 is None and sg1 is None and pg1 is None and np.array_equal(dg0, dg1)
    for e in range(2):
        _check(_oracle(rs0, e), dg0[e], sg0[e], None, max_ambiguous=0.1)
    away = cams.copy()
    away[:, 3:] = [0, 1, 0, 0]   # looking down -z from z <= 0.1: only the plane below (obstacle 1, env 0)
    rs2 = scenes.RayScene("away", verts, np.array([[0, 1, 2]], np.int32), ot, od, op, away, rs.cam)
    dg2, sg2, pg2 = _cast_gpu(cuda, rs2)
    for e in range(2):
        _check(_oracle(rs2, e), dg2[e], sg2[e], pg2[e], max_ambiguous=0.1)
    assert (sg2[1] == 0).all() and (dg2[1] == 0).all() and np.isnan(pg2[1]).all()
    # far clipping: the plane at 0.6 m below env 0's camera is beyond z_far = 0.5
    rs3 = scenes.RayScene("far", verts, np.array([[0, 1, 2]], np.int32), ot, od, op, away,
                          (33, 21, 20.0, 20.0, 16.0, 10.0, 0.05, 0.5))
    dg3, sg3, _ = _cast_gpu(cuda, rs3)
    assert (sg3[0] != 3).all()
    one = scenes.RayScene("one", verts, np.array([[0, 1, 2]], np.int32), ot, od, op, cams,
                          (1, 1, 20.0, 20.0, 0.5, 0.5, 0.05, 3.0))
    dg4, sg4, pg4 = _cast_gpu(cuda, one)
    for e in range(2):
        _check(_oracle(one, e), dg4[e], sg4[e], pg4[e], max_ambiguous=1.0)


def test_consecutive_casts_are_independent(cuda):
    """One ray caster used for 260 frames (the per-pixel keys are reused
    without clearing, tagged by frame, the buffer refilled after 255 frames):
    every checked frame equals a fresh cast of its own geometry, whether
    pixels gain or lose the mesh between frames."""
    import torch
    from paper_2604_17513_gb300 import flash
    rs = scenes.towel_views(n_envs=2, n_side=24, side=0.3, width=64, height=48, cam_height=(0.32, 0.4))
    lifted = rs.verts.copy()
    lifted[:, :, 2] += 0.05
    moved = rs.verts.copy()
    moved[:, :, 0] += 0.2        # the towel leaves part of the view
    W, H, fx, fy, cx, cy, zn, zf = rs.cam
    cam = flash.Camera(W, H, fx, fy, cx, cy, zn, zf)
    t = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(dtype=dt, device=cuda)
    obs = (t(rs.obs_type, torch.int32), t(rs.obs_dims), t(rs.obs_poses))
    rc = flash.Raycaster(cam, rs.n_envs, rs.verts.shape[1], rs.tris)
    geoms = [t(rs.verts), t(moved), t(lifted)]
    refs = []
    for v in geoms:
        fresh = flash.Raycaster(cam, rs.n_envs, rs.verts.shape[1], rs.tris)
        refs.append([o.cpu().numpy() for o in fresh.cast(v, *obs, t(rs.cam_poses))])
    checked = {0, 1, 2, 3, 4, 253, 254, 255, 256, 257, 259}
    for frame in range(260):
        g = (frame * 7 + frame // 3) % 3
        out = rc.cast(geoms[g], *obs, t(rs.cam_poses))
        if frame in checked:
            got = [o.cpu().numpy() for o in out]
            ref = refs[g]
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), frame
            assert np.array_equal(np.nan_to_num(got[2], nan=-1), np.nan_to_num(ref[2], nan=-1)), frame
    assert len({(f * 7 + f // 3) % 3 for f in checked}) == 3


def _boundary_faces(tets):
    """Faces of a tetrahedral mesh that belong to one tetrahedron only."""
    faces = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]], tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]])
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    return faces[cnt[inv.ravel()] == 1]


@pytest.mark.parametrize("kind", ["cloth_grasp", "tet_squeeze"])
def test_render_simulation_state(cuda, kind):
    """flash_render of a scene at the oracle's state of step s (a cloth held
    and lifted by the bilateral grasp; tet blocks between the fingers, whose
    boundary faces are ray cast), obstacles at their step-s poses; a camera
    per environment."""
    import torch
    from paper_2604_17513_gb300 import flash
    if kind == "cloth_grasp":
        sc = scenes.cloth_grasp(n_envs=3, steps=20)
        s, metric, tris = 14, 2, sc.elems
    else:
        sc = scenes.tet_squeeze(n_envs=3, steps=10)
        s, metric, tris = 6, 0, _boundary_faces(sc.elems)
    q = np.zeros((sc.n_envs, sc.n_verts, 3))
    for e in range(sc.n_envs):
        mesh = oracle.Mesh.from_scene(sc, e)
        st = oracle.EnvState(sc.q0[e], sc.v0[e])
        for k in range(s):
            oracle.step(mesh, sc, e, k, st, metric=metric)
        q[e] = _f32(st.q)
    sim = flash.Sim(sc, metric=1 if metric else 0)
    sim.set_state(torch.from_numpy(q.reshape(-1, 3).astype(np.float32)).to(cuda))
    sim.set_poses(flash.poses_tensor(sc, s, cuda), which=0)
    g = np.random.default_rng(11)
    cams = np.zeros((sc.n_envs, 7))
    for e in range(sc.n_envs):
        qd = scenes._quat_mul(scenes._quat_axis_angle((0, 0, 1), g.uniform(0, 6.3)),
                              scenes._quat_axis_angle((1, 0, 0), np.pi + g.uniform(-0.3, 0.3)))
        above = (0.3 if kind == "cloth_grasp" else 0.12) + g.uniform(0, 0.05)   # the mesh fills much of the view
        cams[e] = [*(q[e].mean(0)[:2] + g.uniform(-0.01, 0.01, 2)), q[e][:, 2].max() + above, *qd]
    W, H = 61, 45
    cam = flash.Camera(W, H, 50.0, 50.0, W / 2, H / 2, 0.05, 5.0)
    dg, sg, pg = (t.cpu().numpy() for t in sim.render(cam, torch.from_numpy(cams.astype(np.float32)).to(cuda)))
    assert sim.status() == 0
    for e in range(sc.n_envs):
        rs = scenes.RayScene(kind, q[e:e + 1], np.asarray(tris, np.int32), sc.obs_type[e:e + 1],
                             sc.obs_dims[e:e + 1], sc.poses[e:e + 1, s], cams[e:e + 1],
                             (W, H, 50.0, 50.0, W / 2, H / 2, 0.05, 5.0))
        ref = _oracle(rs, 0)
        _check(ref, dg[e], sg[e], pg[e])
        assert (ref[0][1] == 1).mean() > 0.1


def test_full_size_towel_sampled(cuda):
    """The bench's workload: 128 environments of the 181x181 towel (64,800
    triangles) at 640x480.  All pixels of every environment are cast on the
    GPU; 300 random pixels of the first, a middle and the last environment
    are checked against the oracle one by one, and every pixel against the
    output conventions."""
    rs = scenes.towel_views(n_envs=128)
    dg, sg, pg = _cast_gpu(cuda, rs)
    W, H = rs.cam[:2]
    g = np.random.default_rng(0)
    for e in (0, 63, 127):
        uv = np.c_[g.integers(0, W, 300), g.integers(0, H, 300)]
        ref = _oracle(rs, e, uv)
        _check(ref, dg[e][uv[:, 1], uv[:, 0]], sg[e][uv[:, 1], uv[:, 0]], pg[e][uv[:, 1], uv[:, 0]])
    hit = sg > 0
    assert (sg <= 4).all() and not (sg == 5).any()       # the pose carrier stays invisible
    assert (dg[hit] >= 0.05).all() and (dg[~hit] == 0).all()
    assert np.isfinite(pg[hit]).all() and np.isnan(pg[~hit]).all()
    assert (sg == 1).mean() > 0.2


def test_raycaster_api_errors(cuda):
    """Invalid cameras, sizes and triangle indices fail with FLASH_EINVAL."""
    from paper_2604_17513_gb300 import flash
    good = dict(width=8, height=8, fx=10.0, fy=10.0, cx=4.0, cy=4.0, z_near=0.1, z_far=2.0)
    for bad in ({"width": 0}, {"fx": 0.0}, {"z_near": 0.0}, {"z_far": 0.05}, {"cy": float("inf")}):
        cam = flash.Camera(**{**good, **bad})
        with pytest.raises(flash.FlashError) as ei:
            flash.Raycaster(cam, 2, 3, [[0, 1, 2]])
        assert ei.value.code == -1
    with pytest.raises(flash.FlashError):
        flash.Raycaster(flash.Camera(**good), 2, 3, [[0, 1, 3]])
    with pytest.raises(flash.FlashError):
        flash.Raycaster(flash.Camera(**good), 0, 3, [[0, 1, 2]])
