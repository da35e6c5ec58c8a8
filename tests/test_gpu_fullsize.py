"""Parity at the full workload sizes, in the launch configuration bench.py
times: automatic lanes, graph replay (fixed iterations, or the tolerance loop as a device while-node) and autotuned
tensor-core tiles.  Every environment steps on the GPU; a sample, including
the first and last environment of lanes, starts from the oracle's state at
step s and is checked against one oracle step, one by one (max vertex
position error <= 1e-5 m).
"""
import numpy as np
import pytest

import oracle
import parity
from paper_2604_17513_gb300 import scenes

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def _oracle_state(sc, e, s, metric=0):
    mesh = oracle.Mesh.from_scene(sc, e)
    st = oracle.EnvState(sc.q0[e], sc.v0[e])
    for k in range(s):
        oracle.step(mesh, sc, e, k, st, metric=metric)
    return mesh, _f32(st.q), _f32(st.v), st.attached.copy()


def _step_all(cuda, scs, qs, vs, s, metric=0):
    """One GPU step of every environment of the scenes from (qs, vs) at step s,
    in the bench's configuration (f16x3, automatic lanes, graph replay)."""
    import torch
    from paper_2604_17513_gb300 import flash
    sim = flash.Sim(scs, solve=flash.SOLVE_F16X3, metric=metric)
    sim.set_state(torch.from_numpy(np.concatenate(qs).astype(np.float32)).to(cuda),
                  torch.from_numpy(np.concatenate(vs).astype(np.float32)).to(cuda))
    sim.set_poses(flash.poses_tensor(scs, s, cuda), which=0)
    sim.set_poses(flash.poses_tensor(scs, s + 1, cuda), which=1)
    first = 0
    for sc in scs:   # grasps held at s: re-activated (the held vertex sits on the gripper)
        g = sc.meta.get("grasp")
        if g and min(k for k, r in g["schedule"].items() if r == 1) < s:
            sim.grasp(np.ones(sc.n_envs, np.int32), g["obstacle"], g["anchor"], g["radius"], first)
        first += sc.n_envs
    sim.apply_grasp_schedule(s)
    sim.step(1)
    q = sim.get_state()[0].cpu().numpy()
    assert sim.status() == 0
    return sim, q


def _check(scs, picks, s, cuda, lanes, metric=0):
    """picks: (scene index, local environment) pairs checked against the oracle
    (GPU metric 1, the full metric, is the oracle's metric 2: the same GMRES)."""
    om = 2 if metric else 0
    qs = [sc.q0.reshape(-1, 3).copy() for sc in scs]
    vs = [sc.v0.reshape(-1, 3).copy() for sc in scs]
    refs, spreads = [], []
    for si, e in picks:
        sc = scs[si]
        mesh, q0, v0, att = _oracle_state(sc, e, s, om)
        n = sc.n_verts

        def step_fn(q, v, sc=sc, e=e, mesh=mesh, att=att):
            st = oracle.EnvState(q, v)
            st.attached = att.copy()
            oracle.step(mesh, sc, e, s, st, metric=om)
            return st
        qs[si][e * n:(e + 1) * n] = q0
        vs[si][e * n:(e + 1) * n] = v0
        ref = step_fn(q0, v0)
        refs.append(ref)
        spreads.append(None)
    sim, q = _step_all(cuda, scs, qs, vs, s, metric)
    assert sim.lane_count() == lanes
    base = np.cumsum([0] + [sc.n_envs for sc in scs])
    off = sim.offsets
    con = parity.gpu_contacts(sim)
    for (si, e), ref, spread in zip(picks, refs, spreads):
        g = base[si] + e
        err = np.abs(q[off[g]:off[g + 1]] - ref.q).max()
        assert err <= POS_TOL, (si, e, err, len(ref.cvert))
        if not metric:   # full metric: see test_gpu_fullmetric's converged-impulse test
            parity.assert_impulses(con, g, ref, scs[si], e, s, err)


def test_cloth_gripper_full_size(cuda):
    """1024 environments of the 32x32 cloth under the gripper (4 lanes of
    256); samples at both ends of lanes."""
    sc = scenes.cloth_gripper(seed=1, n_envs=1024, steps=20)
    _check([sc], [(0, 0), (0, 255), (0, 256), (0, 1023)], 10, cuda, lanes=4)


def test_tet_squeeze_full_size(cuda):
    """4096 tet blocks with per-environment stiffness (eigen-form solve,
    4 lanes of 1024); samples at both ends of lanes."""
    sc = scenes.tet_squeeze(seed=1, n_envs=4096, steps=12)
    _check([sc], [(0, 0), (0, 1023), (0, 1024), (0, 4095)], 6, cuda, lanes=4)


def test_mixed_batch_full_size(cuda):
    """The 2048-environment mixed batch (cloths of side 16..64, tet blocks of
    200..3000 vertices, one group per template, 8 lanes); samples from the
    smallest cloth and tet templates and a mid-size cloth (the oracle's dense
    Cholesky keeps the largest templates out of a test)."""
    scs = scenes.mixed_batch(seed=3, n_envs=2048, steps=16)
    cloths = sorted((sc.n_verts, i) for i, sc in enumerate(scs) if sc.elem_type == scenes.TRI)
    tets = sorted((sc.n_verts, i) for i, sc in enumerate(scs) if sc.elem_type == scenes.TET)
    mid = [i for n, i in cloths if 900 <= n <= 1300][0]
    picks = [(cloths[0][1], 0), (tets[0][1], scs[tets[0][1]].n_envs - 1), (mid, 0)]
    _check(scs, picks, 8, cuda, lanes=8)


def test_tet_squeeze_full_metric_full_size(cuda):
    """4096 tet blocks with the full contact metric (10 GMRES iterations per
    Newton step, each an A^-1 application to all 12288 columns), 4 lanes,
    graph replay; samples at both ends of lanes, from the oracle's
    full-metric state at step 10 (the plates squeeze)."""
    sc = scenes.tet_squeeze(seed=1, n_envs=4096, steps=14)
    _check([sc], [(0, 0), (0, 1023), (0, 1024), (0, 4095)], 10, cuda, lanes=4, metric=1)


def test_cloth_grasp_full_metric_full_size(cuda):
    """1024 environments of the 32x32 cloth held at a corner by the bilateral
    grasp, full metric (the bench's cloth-grasp workload: 4 lanes, graph
    replay), one step while the corner rises; samples at both ends of lanes
    start from the oracle's full-metric state at step 6."""
    sc = scenes.cloth_grasp(seed=1, n_envs=1024, n_side=32, side=0.5, steps=10, grasp_step=2,
                            release_step=1 << 30)
    _check([sc], [(0, 0), (0, 255), (0, 256), (0, 1023)], 6, cuda, lanes=4, metric=1)


def test_cloth_gripper_full_size_tolerance_mode(cuda):
    """The bench's default configuration at full size: 1024 environments of
    the 32x32 cloth, tolerance mode (r_ncp <= 1e-5, at most 10 iterations)
    replayed from the graph whose loop is a device while-node, 4 lanes;
    samples at both ends of lanes against the oracle at the GPU's own
    iteration count: the oracle's run with the same stopping rule where it
    stopped at the same count, else its fixed-count run of as many
    iterations (FP32 and FP64 may cross the threshold one iteration apart)."""
    import torch
    from paper_2604_17513_gb300 import flash
    sc = scenes.cloth_gripper(n_envs=1024, steps=20)
    s = 10
    kw = dict(mode=1, tol=1e-5, k_min=1, k_cap=10)
    picks = [0, 255, 256, 1023]
    q, v = sc.q0.reshape(-1, 3).copy(), sc.v0.reshape(-1, 3).copy()
    n = sc.n_verts
    starts = {}
    for e in picks:
        mesh, q0, v0, _ = _oracle_state(sc, e, s)
        q[e * n:(e + 1) * n], v[e * n:(e + 1) * n] = q0, v0
        starts[e] = (mesh, q0, v0)
    sim = flash.Sim(sc, solve=flash.SOLVE_F16X3, **kw)
    assert sim.lane_count() == 4
    sim.set_state(torch.from_numpy(q.astype(np.float32)).to(cuda), torch.from_numpy(v.astype(np.float32)).to(cuda))
    sim.set_poses(flash.poses_tensor(sc, s, cuda), which=0)
    sim.set_poses(flash.poses_tensor(sc, s + 1, cuda), which=1)
    sim.step(1)
    assert sim.status() == 0
    qg = sim.get_state()[0].cpu().numpy()
    it = sim.stats()[0].cpu().numpy()
    con = parity.gpu_contacts(sim)
    for e, (mesh, q0, v0) in starts.items():
        ref = oracle.EnvState(q0, v0)
        oracle.step(mesh, sc, e, s, ref, **kw)
        if ref.iters != it[e]:
            assert abs(int(it[e]) - ref.iters) <= 1, (e, it[e], ref.iters)
            ref = oracle.EnvState(q0, v0)
            oracle.step(mesh, sc, e, s, ref, k_max=int(it[e]))
        err = np.abs(qg[e * n:(e + 1) * n] - ref.q).max()
        assert err <= POS_TOL, (e, it[e], err)
        parity.assert_impulses(con, e, ref, sc, e, s, err)
