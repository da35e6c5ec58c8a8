"""GPU parity where features meet: ray casting a batch of many mesh groups,
the bilateral grasp on a cloth with self-collision, and self-collision in a
batch that mixes cloth and tetrahedral groups (self contacts for the cloths
only).  References are the oracle on the same inputs.
"""
import numpy as np
import pytest

import oracle
import parity
from paper_2604_17513_gb300 import scenes
from test_gpu_raycast import _check as raycast_check

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def _boundary_faces(tets):
    faces = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]], tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]])
    _, inv, cnt = np.unique(np.sort(faces, axis=1), axis=0, return_inverse=True, return_counts=True)
    return faces[cnt[inv.ravel()] == 1]


def _pick(scs, kind, k=0):
    """k-th smallest template of a kind: (scene index, scene)."""
    idx = sorted((sc.n_verts, i) for i, sc in enumerate(scs) if sc.elem_type == kind)
    i = idx[k][1]
    return i, scs[i]


def test_render_mixed_batch(cuda):
    """flash_render of the mixed batch (one group per template, cloths and
    tet blocks, boxes and spheres) at the initial state: sampled
    environments of two cloth and two tet templates against the oracle."""
    import torch
    from paper_2604_17513_gb300 import flash
    scs = scenes.mixed_batch(seed=3, n_envs=256, steps=4)
    sim = flash.Sim(scs)
    q0, v0 = flash.state_tensors(scs, cuda)
    sim.set_state(q0, v0)
    sim.set_poses(flash.poses_tensor(scs, 0, cuda), which=0)
    base = np.cumsum([0] + [sc.n_envs for sc in scs])
    W, H = 48, 36
    cam = flash.Camera(W, H, 30.0, 30.0, W / 2, H / 2, 0.05, 5.0)
    cams = np.zeros((sim.n_envs, 7))
    cams[:, 3:] = [0, 1, 0, 0]                       # looking down
    for si, sc in enumerate(scs):
        for e in range(sc.n_envs):
            c = sc.q0[e].mean(0)
            ext = np.ptp(sc.q0[e][:, :2], axis=0).max()
            cams[base[si] + e, :3] = [c[0], c[1], sc.q0[e][:, 2].max() + 1.2 * ext]   # the mesh fills much of the view
    dg, sg, pg = (t.cpu().numpy() for t in sim.render(cam, torch.from_numpy(cams.astype(np.float32)).to(cuda)))
    assert sim.status() == 0
    picks = [_pick(scs, scenes.TRI, 0), _pick(scs, scenes.TRI, 3), _pick(scs, scenes.TET, 0),
             _pick(scs, scenes.TET, 2)]
    for si, sc in picks:
        tris = sc.elems if sc.elem_type == scenes.TRI else _boundary_faces(sc.elems)
        e = sc.n_envs - 1
        g = base[si] + e
        intr = (30.0, 30.0, W / 2, H / 2, 0.05, 5.0)
        args = (_f32(sc.q0[e]), tris, sc.obs_type[e], _f32(sc.obs_dims[e]), _f32(sc.poses[e, 0]), _f32(cams[g]),
                intr, W, H)
        ref = [oracle.raycast(*args, dil=dl) for dl in (0.0, 1e-3, -1e-3)]
        assert (ref[0][1] == 1).mean() > 0.2
        # unique pixels exactly, the rest (edges seen edge-on, silhouettes) one of the answers
        raycast_check(ref, dg[g], sg[g], pg[g], max_ambiguous=0.4)


def test_grasp_with_self_collision(cuda):
    """The grasp scene with self-collision on (full metric): one step while
    the corner is lifted, from the oracle's state, the GPU re-activating the
    grasp; positions and contact lists (grasp and self rows) agree."""
    import torch
    from paper_2604_17513_gb300 import flash
    sc = scenes.cloth_grasp(n_envs=3, steps=30)
    sc.meta["self_collision"] = True
    s = 12
    q, v, meshes, refs = sc.q0.copy(), sc.v0.copy(), {}, {}
    for e in range(sc.n_envs):
        mesh = oracle.Mesh.from_scene(sc, e)
        st = oracle.EnvState(sc.q0[e], sc.v0[e])
        for k in range(s):
            oracle.step(mesh, sc, e, k, st, metric=2)
        q[e], v[e] = _f32(st.q), _f32(st.v)
        def step_fn(qq, vv, mesh=mesh, e=e, att=st.attached.copy()):
            x = oracle.EnvState(qq, vv)
            x.attached = att.copy()
            oracle.step(mesh, sc, e, s, x, metric=2)
            return x
        ref = step_fn(q[e], v[e])
        refs[e] = (ref, None)
    sim = flash.Sim(sc, solve=flash.SOLVE_F16X3, metric=flash.METRIC_FULL)
    sim.set_state(torch.from_numpy(q.reshape(-1, 3).astype(np.float32)).to(cuda),
                  torch.from_numpy(v.reshape(-1, 3).astype(np.float32)).to(cuda))
    sim.set_poses(flash.poses_tensor(sc, s, cuda), which=0)
    sim.set_poses(flash.poses_tensor(sc, s + 1, cuda), which=1)
    g = sc.meta["grasp"]
    sim.grasp(np.ones(sc.n_envs, np.int32), g["obstacle"], g["anchor"], g["radius"])
    sim.step(1)
    assert sim.status() == 0
    qg = sim.get_state()[0].cpu().numpy().reshape(sc.n_envs, sc.n_verts, 3)
    cnt, vert, obs, _ = (t.cpu().numpy() for t in sim.contacts())
    tri = sim.contact_tris().cpu().numpy()
    con = parity.gpu_contacts(sim)
    for e, (ref, spread) in refs.items():
        c = int(cnt[e])
        assert c == len(ref.cvert) and (obs[e, :c] == ref.cobs).all() and (tri[e, :c] == ref.ctri).all()
        assert (ref.cobs == oracle.GRASP_SLOT).sum() == 1
        err = np.abs(qg[e] - ref.q).max()
        assert err <= POS_TOL
        assert parity.impulse_check(con, e, ref, sc, e, s, err)[0]   # same lists


def test_self_collision_with_tet_groups(cuda):
    """Self-collision on in a batch of cloth and tet templates (one group
    each): self contacts for the cloths only; sampled environments of both
    kinds match the oracle after one full-metric step."""
    import torch
    from paper_2604_17513_gb300 import flash
    scs = scenes.mixed_batch(seed=3, n_envs=128, steps=12)
    for sc in scs:
        if sc.elem_type == scenes.TRI:
            sc.meta = dict(sc.meta or {}, self_collision=True)
    s = 6
    picks = [_pick(scs, scenes.TRI, 0), _pick(scs, scenes.TET, 0)]
    qs = [sc.q0.reshape(-1, 3).copy() for sc in scs]
    vs = [sc.v0.reshape(-1, 3).copy() for sc in scs]
    refs = []
    for si, sc in picks:
        e = 0
        mesh = oracle.Mesh.from_scene(sc, e)
        st = oracle.EnvState(sc.q0[e], sc.v0[e])
        for k in range(s):
            oracle.step(mesh, sc, e, k, st, metric=2)
        n = sc.n_verts
        qs[si][:n], vs[si][:n] = _f32(st.q), _f32(st.v)
        def step_fn(qq, vv, mesh=mesh, sc=sc):
            x = oracle.EnvState(qq, vv)
            oracle.step(mesh, sc, 0, s, x, metric=2)
            return x
        ref = step_fn(_f32(st.q), _f32(st.v))
        refs.append((ref, None))
    sim = flash.Sim(scs, solve=flash.SOLVE_F16X3, metric=flash.METRIC_FULL)
    sim.set_state(torch.from_numpy(np.concatenate(qs).astype(np.float32)).to(cuda),
                  torch.from_numpy(np.concatenate(vs).astype(np.float32)).to(cuda))
    sim.set_poses(flash.poses_tensor(scs, s, cuda), which=0)
    sim.set_poses(flash.poses_tensor(scs, s + 1, cuda), which=1)
    sim.step(1)
    assert sim.status() == 0
    q = sim.get_state()[0].cpu().numpy()
    base = np.cumsum([0] + [sc.n_envs for sc in scs])
    off = sim.offsets
    con = parity.gpu_contacts(sim)
    for (si, sc), (ref, spread) in zip(picks, refs):
        g = base[si]
        err = np.abs(q[off[g]:off[g + 1]] - ref.q).max()
        assert err <= POS_TOL
        assert parity.impulse_check(con, g, ref, sc, 0, s, err)[0]   # same lists
