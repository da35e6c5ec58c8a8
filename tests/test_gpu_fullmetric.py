"""GPU parity of the full contact metric Z = J A^-1 J^T + E (each Newton step:
lin_iters steps of block-Jacobi-preconditioned GMRES over all contacts of an
environment) against the oracle's metric 2, which runs the same GMRES in
FP64.  Per step from identical states, max vertex error <= 1e-5 m.
"""
import numpy as np
import pytest

import oracle
import parity
from paper_2604_17513_gb300 import scenes

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5
SOLVES = [0, 1]


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def _oracle_state(sc, e, s, **kw):
    mesh = oracle.Mesh.from_scene(sc, e)
    st = oracle.EnvState(sc.q0[e], sc.v0[e])
    for k in range(s):
        oracle.step(mesh, sc, e, k, st, metric=2, **kw)
    return mesh, _f32(st.q), _f32(st.v)


def _step_fn(mesh, sc, e, s, **kw):
    def f(q, v):
        st = oracle.EnvState(q, v)
        oracle.step(mesh, sc, e, s, st, **kw)
        return st
    return f


def _gpu_step(cuda, sc, q, v, s, **kw):
    import torch
    from paper_2604_17513_gb300 import flash
    sim = flash.Sim(sc, metric=flash.METRIC_FULL, **kw)
    sim.set_state(torch.from_numpy(np.asarray(q, np.float32).reshape(-1, 3)).to(cuda),
                  torch.from_numpy(np.asarray(v, np.float32).reshape(-1, 3)).to(cuda))
    sim.set_poses(flash.poses_tensor(sc, s, cuda), which=0)
    sim.set_poses(flash.poses_tensor(sc, s + 1, cuda), which=1)
    sim.step(1)
    it, r = sim.stats()
    assert sim.status() == 0
    _gpu_step.contacts = parity.gpu_contacts(sim)
    return sim.get_state()[0].cpu().numpy().reshape(sc.n_envs, sc.n_verts, 3), it.cpu().numpy(), r.cpu().numpy()


@pytest.mark.parametrize("solve", SOLVES)
def test_tet_squeeze_full_metric_one_step(cuda, solve):
    """Stiff tet blocks squeezed by the plates (where the lite metric stalls):
    one fixed step (k = 10, 10 linear iterations) from the oracle's own
    full-metric state at step 18, every environment checked."""
    sc = scenes.tet_squeeze(n_envs=3, steps=30)
    s = 18
    q, v, meshes = sc.q0.copy(), sc.v0.copy(), {}
    for e in range(sc.n_envs):
        meshes[e], q[e], v[e] = _oracle_state(sc, e, s)
    qg, _, rg = _gpu_step(cuda, sc, q, v, s, solve=solve)
    for e in range(sc.n_envs):
        step_fn = _step_fn(meshes[e], sc, e, s, metric=2)
        ref = step_fn(q[e], v[e])
        err = np.abs(qg[e] - ref.q).max()
        assert err <= POS_TOL, (e, err, len(ref.cvert))
        assert parity.impulse_check(_gpu_step.contacts, e, ref, sc, e, s, err)[0]   # same lists
        assert abs(rg[e] - ref.rncp) <= 1e-5 + 1e-2 * ref.rncp, (e, rg[e], ref.rncp)


@pytest.mark.parametrize("solve", SOLVES)
@pytest.mark.parametrize("s", [27, 40])
def test_cloth_drop_full_metric_one_step(cuda, s, solve):
    """16x16 cloth on the sphere: one fixed step with the full metric from the
    oracle's full-metric state at step s (in contact)."""
    sc = scenes.cloth_drop(steps=60)
    mesh, q0, v0 = _oracle_state(sc, 0, s)
    qg, _, _ = _gpu_step(cuda, sc, q0[None], v0[None], s, solve=solve)
    step_fn = _step_fn(mesh, sc, 0, s, metric=2)
    ref = step_fn(q0, v0)
    err = np.abs(qg[0] - ref.q).max()
    assert len(ref.cvert) > 0 and err <= POS_TOL, (s, err, len(ref.cvert))
    assert parity.impulse_check(_gpu_step.contacts, 0, ref, sc, 0, s, err)[0]   # same lists


def test_tet_squeeze_full_metric_tolerance_mode_lanes(cuda):
    """Tolerance mode with the full metric on 300 tet blocks in 2 lanes: every
    environment reaches r_ncp <= 1e-5.  Sampled environments start from the
    oracle's state; the inexact (10-step GMRES) Newton iterations approach
    the threshold slowly, so FP32 and FP64 may cross it a few iterations
    apart.  Each sample is compared with the oracle at the GPU's own
    iteration count: the oracle's run with the same stopping rule where it
    stopped at the same count, else its fixed-count run of as many
    iterations (the same iterate of the same iteration)."""
    sc = scenes.tet_squeeze(n_envs=300, steps=30)
    s = 12
    sample = [0, 149, 150, 299]
    q, v = sc.q0.copy(), sc.v0.copy()
    meshes = {}
    for e in sample:
        meshes[e], q[e], v[e] = _oracle_state(sc, e, s)
    qg, it, rg = _gpu_step(cuda, sc, q, v, s, solve=1, mode=1, tol=1e-5, k_cap=60, lanes=2)
    con = _gpu_step.contacts
    assert (rg <= 1e-5).all(), rg.max()
    for e in sample:
        ref = oracle.EnvState(q[e], v[e])
        oracle.step(meshes[e], sc, e, s, ref, metric=2, mode=1, tol=1e-5, k_cap=60)
        assert ref.rncp <= 1e-5 and abs(int(it[e]) - ref.iters) <= 3, (e, it[e], ref.iters)
        if ref.iters != it[e]:
            step_fn = _step_fn(meshes[e], sc, e, s, metric=2, k_max=int(it[e]))
        else:
            step_fn = _step_fn(meshes[e], sc, e, s, metric=2, mode=1, tol=1e-5, k_cap=60)
        ref = step_fn(q[e], v[e])
        err = np.abs(qg[e] - ref.q).max()
        # intermediate iterates of the inexact Newton steps amplify input
        # rounding: sqrt(k) FP32 ulps on the oracle's own input (k iterations
        # of FP32 rounding) move it by `moved`
        moved, _ = parity.oracle_spread(step_fn, q[e], v[e], ref, ulps=int(np.ceil(np.sqrt(it[e]))))
        assert err <= max(POS_TOL, 2.0 * moved), (e, it[e], err, moved)
        assert parity.impulse_check(con, e, ref, sc, e, s, err)[0]   # same lists


@pytest.mark.parametrize("scene", ["tet", "drop"])
def test_full_metric_converged_impulses(cuda, scene):
    """The full metric's Newton steps solve Z with 10 GMRES iterations, and
    their intermediate multipliers are not a well-conditioned function of
    the input (FP32 and FP64 Krylov bases part), so the one-step tests
    compare lists and positions only.  At convergence the multipliers are
    the NCP's solution, whatever the path: here both sides iterate to
    r_ncp <= 1e-7 m from the same state and the impulses are compared (with
    ``parity``'s rules)."""
    if scene == "tet":
        sc, s, envs = scenes.tet_squeeze(n_envs=4, steps=30), 12, range(4)
    else:
        sc, s, envs = scenes.cloth_drop(n_envs=1, steps=60), 40, range(1)
    kw = dict(mode=1, tol=1e-7, k_cap=200)
    q, v, meshes = sc.q0.copy(), sc.v0.copy(), {}
    for e in envs:
        meshes[e], q[e], v[e] = _oracle_state(sc, e, s)
    qg, it, rg = _gpu_step(cuda, sc, q, v, s, solve=0, **kw)
    con = _gpu_step.contacts
    for e in envs:
        ref = oracle.EnvState(q[e], v[e])
        oracle.step(meshes[e], sc, e, s, ref, metric=2, **kw)
        assert ref.rncp <= 1e-7 and rg[e] <= 1e-7, (e, ref.rncp, rg[e])
        err = np.abs(qg[e] - ref.q).max()
        assert err <= POS_TOL, (e, err)
        assert len(ref.cvert) > 0
        parity.assert_impulses(con, e, ref, sc, e, s, err)
