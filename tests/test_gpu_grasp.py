"""GPU parity of the bilateral grasp (appendix, Bilateral Constraint for Cloth
Control: C = x_i - p_grip(t+h) = 0 for the grasped set, activated by
proximity, released by emptying the set) against the oracle, through the
C-ABI's flash_grasp.  Environments start from the oracle's state at step s
(grasp set included: the GPU re-activates at s, which finds the same
vertices, the held vertex sitting on the gripper) and are compared after
one or two steps, max vertex error <= 1e-5 m; the contact lists carry the
same grasp rows.
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


def _oracle_states(sc, envs, s, metric, warm="cold"):
    """Oracle states (q, v rounded to FP32, grasp set) at the start of step s."""
    out = {}
    for e in envs:
        mesh = oracle.Mesh.from_scene(sc, e)
        st = oracle.EnvState(sc.q0[e], sc.v0[e])
        for k in range(s):
            oracle.step(mesh, sc, e, k, st, metric=metric, warm=warm)
        start = oracle.EnvState(_f32(st.q), _f32(st.v))   # no previous contacts, like a new Sim
        start.attached = st.attached.copy()
        out[e] = (mesh, start)
    return out


def _gpu_run(cuda, sc, starts, s, n_steps, activate, **kw):
    """GPU steps s .. s + n_steps - 1 of every environment of sc (sampled
    ones from the oracle's state), grasp requests from the scene's schedule;
    ``activate`` re-issues the activation at s for environments that hold."""
    import torch
    from paper_2604_17513_gb300 import flash
    q, v = sc.q0.copy(), sc.v0.copy()
    for e, (_, st) in starts.items():
        q[e], v[e] = st.q, st.v
    sim = flash.Sim(sc, solve=flash.SOLVE_F16X3, **kw)
    sim.set_state(torch.from_numpy(q.reshape(-1, 3).astype(np.float32)).to(cuda),
                  torch.from_numpy(v.reshape(-1, 3).astype(np.float32)).to(cuda))
    sim.set_poses(flash.poses_tensor(sc, s, cuda), which=0)
    g = sc.meta["grasp"]
    if activate:
        sim.grasp(np.ones(sc.n_envs, np.int32), g["obstacle"], g["anchor"], g["radius"])
    for k in range(s, s + n_steps):
        sim.set_poses(flash.poses_tensor(sc, k + 1, cuda), which=1)
        sim.apply_grasp_schedule(k)
        sim.step(1)
    assert sim.status() == 0
    qg = sim.get_state()[0].cpu().numpy().reshape(sc.n_envs, sc.n_verts, 3)
    cnt, vert, obs, _ = (t.cpu().numpy() for t in sim.contacts())
    _LAST["contacts"] = parity.gpu_contacts(sim)
    return sim, qg, cnt, vert, obs


def _compare(sc, starts, s, n_steps, metric_gpu, qg, cnt, vert, obs, warm="cold"):
    om = 2 if metric_gpu else 0
    for e, (mesh, st) in starts.items():
        ref = oracle.EnvState(st.q, st.v)
        ref.attached = st.attached.copy()
        for k in range(s, s + n_steps - 1):
            oracle.step(mesh, sc, e, k, ref, metric=om, warm=warm)
        q1, v1, att, prev = ref.q.copy(), ref.v.copy(), ref.attached.copy(), ref
        last = s + n_steps - 1

        def step_fn(q, v, mesh=mesh, e=e, att=att, prev=prev):
            x = oracle.EnvState(q, v)
            x.attached = att.copy()
            x.cvert, x.cobs, x.ctri, x.gamma = prev.cvert, prev.cobs, prev.ctri, prev.gamma
            oracle.step(mesh, sc, e, last, x, metric=om, warm=warm)
            return x
        ref = step_fn(q1, v1)
        err = np.abs(qg[e] - ref.q).max()
        assert err <= POS_TOL, (e, err, len(ref.cvert))
        c = int(cnt[e])
        assert c == len(ref.cvert) and (vert[e, :c] == ref.cvert).all() and (obs[e, :c] == ref.cobs).all(), e
        if not metric_gpu:   # full metric: GMRES iterates, impulses compared at convergence
            parity.assert_impulses(_LAST["contacts"], e, ref, sc, e, last, err)
    return ref


_LAST = {}


@pytest.mark.parametrize("metric", [0, 1])
def test_grasp_activation_step(cuda, metric):
    """Step 2 of the grasp scene (the activation: the corner within the radius
    joins S_grip, the gripper starts rising) and step 3, from the oracle's
    state at step 2, on 8 environments of the 16x16 cloth."""
    sc = scenes.cloth_grasp(n_envs=8, steps=20)
    starts = _oracle_states(sc, range(sc.n_envs), 2, 2 if metric else 0)
    _, qg, cnt, vert, obs = _gpu_run(cuda, sc, starts, 2, 2, activate=False, metric=metric)
    _compare(sc, starts, 2, 2, metric, qg, cnt, vert, obs)
    assert all((obs[e, :cnt[e]] == oracle.GRASP_SLOT).sum() == 1 for e in range(sc.n_envs))


@pytest.mark.parametrize("s", [12, 40])
def test_grasp_hold_full_metric(cuda, s):
    """One step with the corner held and lifted (s = 12) or held still
    (s = 40), full metric (the constraint is solved to ~1e-9 m), from the
    oracle's state; the GPU re-activates at s and finds the same vertex."""
    sc = scenes.cloth_grasp(n_envs=4, steps=60)
    starts = _oracle_states(sc, range(sc.n_envs), s, 2)
    for _, st in starts.values():
        assert st.attached.sum() == 1
    _, qg, cnt, vert, obs = _gpu_run(cuda, sc, starts, s, 1, activate=True, metric=1)
    ref = _compare(sc, starts, s, 1, 1, qg, cnt, vert, obs)
    p = oracle._to_world(sc.poses[sc.n_envs - 1, s + 1, 1], (0, 0, 0))
    assert np.abs(qg[sc.n_envs - 1][np.nonzero(ref.attached)[0][0]] - p).max() <= 1e-5


def test_grasp_release_full_metric(cuda):
    """The release: hold at step 29 (re-activated), release scheduled at 30;
    after step 30 no grasp rows remain and the cloth moves freely."""
    sc = scenes.cloth_grasp(n_envs=4, steps=40, release_step=30)
    starts = _oracle_states(sc, range(sc.n_envs), 29, 2)
    _, qg, cnt, vert, obs = _gpu_run(cuda, sc, starts, 29, 2, activate=True, metric=1)
    _compare(sc, starts, 29, 2, 1, qg, cnt, vert, obs)
    for e in range(sc.n_envs):
        assert (obs[e, :cnt[e]] != oracle.GRASP_SLOT).all()


def test_grasp_warm_prev_matches_by_slot(cuda):
    """Warm start from the previous step's multipliers: the grasp row of step
    3 starts from step 2's grasp multiplier (matched by (vertex, slot)), as in
    the oracle's warm="prev"."""
    from paper_2604_17513_gb300 import flash
    sc = scenes.cloth_grasp(n_envs=4, steps=20)
    starts = _oracle_states(sc, range(sc.n_envs), 2, 0)
    _, qg, cnt, vert, obs = _gpu_run(cuda, sc, starts, 2, 2, activate=False, metric=0, warm=flash.WARM_PREV)
    _compare(sc, starts, 2, 2, 0, qg, cnt, vert, obs, warm="prev")


def test_grasp_lanes_and_graph(cuda):
    """260 environments in 2 lanes with graph replay: the grasp requests
    (issued between replays) reach every lane; sampled environments at both
    ends of the lanes match the oracle over the activation and next step."""
    sc = scenes.cloth_grasp(n_envs=260, steps=20)
    picks = [0, 129, 130, 259]
    starts = _oracle_states(sc, picks, 2, 2)
    sim, qg, cnt, vert, obs = _gpu_run(cuda, sc, starts, 2, 2, activate=False, metric=1, lanes=2)
    assert sim.lane_count() == 2
    _compare(sc, starts, 2, 2, 1, qg, cnt, vert, obs)
    assert all((obs[e, :cnt[e]] == oracle.GRASP_SLOT).sum() == 1 for e in range(sc.n_envs))


def test_grasp_api_errors(cuda):
    """Invalid grasp calls fail with FLASH_EINVAL and change nothing."""
    from paper_2604_17513_gb300 import flash
    sc = scenes.cloth_grasp(n_envs=2, steps=4)
    sim = flash.Sim(sc)
    for kw in ({"request": [1, 1, 1]}, {"request": [2, 1]}, {"request": [1, 1], "obstacle": 8},
               {"request": [1, 1], "radius": -1.0}, {"request": [1, 1], "radius": float("nan")}):
        args = {"obstacle": 1, "radius": 0.01, **kw}
        with pytest.raises(flash.FlashError) as ei:
            sim.grasp(args["request"], args["obstacle"], radius=args["radius"])
        assert ei.value.code == -1
