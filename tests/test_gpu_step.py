"""GPU parity of the batched step against the FP64 oracle (through the C ABI).

Per-step parity from identical states: the oracle and the CUDA path start
from the same float32-representable state and take one step; max vertex
position error <= 1e-5 m in FP32 (the tolerance the target states), the same
contact lists, and contact impulses within 1e-4 relative (with the FP32
allowances that ``parity`` states).
"""
import numpy as np
import pytest

import oracle
import parity
from paper_2604_17513_gb300 import scenes

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5


SOLVES = [0, 1]   # FLASH_SOLVE_F32, FLASH_SOLVE_F16X3


def _sim(sc, **kw):
    from paper_2604_17513_gb300 import flash
    return flash.Sim(sc, **kw)


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def gpu_step_from(sim, sc, s, q, v, n=1):
    """Set (q, v) [N][n][3] for all envs, take n steps starting at step index s."""
    import torch
    from paper_2604_17513_gb300 import flash
    dev = sim.dev
    sim.set_state(torch.from_numpy(np.asarray(q, np.float32).reshape(-1, 3)).to(dev),
                  torch.from_numpy(np.asarray(v, np.float32).reshape(-1, 3)).to(dev))
    sim.set_poses(flash.poses_tensor(sc, s, dev), which=0)
    for k in range(n):
        sim.set_poses(flash.poses_tensor(sc, s + k + 1, dev), which=1)
        sim.step(1)
    qg, vg = sim.get_state()
    torch.cuda.synchronize()
    return qg.cpu().numpy().reshape(sc.n_envs, sc.n_verts, 3), vg.cpu().numpy().reshape(sc.n_envs, sc.n_verts, 3)


def oracle_state_at(sc, env, s, **kw):
    mesh = oracle.Mesh.from_scene(sc, env)
    st = oracle.EnvState(sc.q0[env], sc.v0[env])
    for k in range(s):
        oracle.step(mesh, sc, env, k, st, **kw)
    return mesh, st


@pytest.mark.parametrize("solve", SOLVES)
def test_global_apply_matches_cholesky(cuda, solve):
    """The dense inverse apply equals the oracle's Cholesky solve A x = b
    (FP32 CUDA cores, or the tcgen05 f16 hi/lo split with FP32 accumulation)."""
    import torch
    sc = scenes.cloth_drop(n_envs=3)
    sim = _sim(sc, solve=solve)
    rng = np.random.default_rng(5)
    rhs = rng.normal(size=(3, sc.n_verts, 3)) * 1e-3
    out = sim.global_apply(0, 3, torch.from_numpy(rhs.astype(np.float32).reshape(-1, 3)).to(cuda))
    out = out.cpu().numpy().reshape(3, sc.n_verts, 3)
    mesh = oracle.Mesh.from_scene(sc)
    for e in range(3):
        ref = mesh.solve(_f32(rhs[e]))
        err = np.abs(out[e] - ref).max() / np.abs(ref).max()
        assert err < (2e-5 if solve == 0 else 1e-4), err


@pytest.mark.parametrize("solve", SOLVES)
def test_global_apply_tiny_and_zero_columns(cuda, solve):
    """Right-hand sides near the bottom of the float range (a contact update
    that has converged to ~1e-35, below the 2^-112 where the hi/lo split's
    power-of-two column scale reaches its cap) and exactly zero columns: the
    scale must stay finite and the result must still be A^-1 b.  Entries are
    normal floats; the step kernels flush subnormals to zero."""
    import torch
    sc = scenes.cloth_drop(n_envs=2)
    sim = _sim(sc, solve=solve)
    rng = np.random.default_rng(6)
    shape = (2, sc.n_verts, 3)
    rhs = rng.choice([-1.0, 1.0], size=shape) * rng.uniform(0.5, 2.0, size=shape) * 1e-35
    rhs[1, :, 2] = 0.0
    out = sim.global_apply(0, 2, torch.from_numpy(rhs.astype(np.float32).reshape(-1, 3)).to(cuda))
    out = out.cpu().numpy().reshape(2, sc.n_verts, 3)
    assert np.isfinite(out).all()
    assert (out[1, :, 2] == 0).all()
    mesh = oracle.Mesh.from_scene(sc)
    for e in range(2):
        ref = mesh.solve(_f32(rhs[e]).astype(np.float64) * 1e35) * 1e-35
        err = np.abs(out[e] - ref).max() / np.abs(ref).max()
        assert err < (2e-5 if solve == 0 else 1e-4), (e, err)


@pytest.mark.parametrize("solve", SOLVES)
@pytest.mark.parametrize("s", [0, 10, 27, 40])
def test_cloth_drop_one_step(cuda, s, solve):
    """16x16 cloth falling onto the sphere: one Mode-A step (k = 10) from the
    oracle's state at step s, free fall (s = 0, 10) and in contact (27, 40)."""
    sc = scenes.cloth_drop(steps=60)
    mesh, st = oracle_state_at(sc, 0, s)
    q0, v0 = _f32(st.q), _f32(st.v)
    sim = _sim(sc, solve=solve)
    qg, vg = gpu_step_from(sim, sc, s, q0[None], v0[None])
    ref = oracle.EnvState(q0, v0)
    oracle.step(mesh, sc, 0, s, ref)
    err = np.abs(qg[0] - ref.q).max()
    assert err <= POS_TOL, (s, err, len(ref.cvert))
    parity.assert_impulses(parity.gpu_contacts(sim), 0, ref, sc, 0, s, err)
    assert sim.status() == 0


@pytest.mark.parametrize("solve", SOLVES)
def test_cloth_gripper_one_step_sampled(cuda, solve):
    """32x32 cloths under the two-finger gripper: all 64 environments step on
    the GPU, a sample is checked against the oracle one by one."""
    sc = scenes.cloth_gripper(n_envs=64, steps=40)
    s = 12
    # start every env from the oracle's state of env e at step s for a sample,
    # and from the initial state elsewhere
    sample = [0, 17, 63]
    q = sc.q0.copy()
    v = sc.v0.copy()
    meshes = {}
    for e in sample:
        meshes[e], st = oracle_state_at(sc, e, s)
        q[e], v[e] = _f32(st.q), _f32(st.v)
    sim = _sim(sc, solve=solve)
    qg, _ = gpu_step_from(sim, sc, s, q, v)
    con = parity.gpu_contacts(sim)
    for e in sample:
        ref = oracle.EnvState(q[e], v[e])
        oracle.step(meshes[e], sc, e, s, ref)
        err = np.abs(qg[e] - ref.q).max()
        assert err <= POS_TOL, (e, err)
        parity.assert_impulses(con, e, ref, sc, e, s, err)


def test_rest_stays_at_rest(cuda):
    """Mesh in its rest shape, no gravity, no contact: q is unchanged."""
    sc = scenes.cloth_drop(n_envs=2, steps=5)
    sc.gravity = (0.0, 0.0, 0.0)
    sc.q0[:] = sc.rest[None] + np.array([0, 0, 0.6])
    sim = _sim(sc)
    qg, vg = gpu_step_from(sim, sc, 0, sc.q0, sc.v0, n=5)
    assert np.abs(qg - sc.q0).max() < 1e-6
    assert np.abs(vg).max() < 1e-4


@pytest.mark.parametrize("solve", SOLVES)
def test_tet_squeeze_one_step(cuda, solve):
    """Soft tet blocks squeezed by the parallel gripper; per-environment
    stiffness gives each environment its own system matrix (its own group)."""
    sc = scenes.tet_squeeze(n_envs=3, steps=30)
    s = 18
    q, v, meshes = sc.q0.copy(), sc.v0.copy(), {}
    for e in range(sc.n_envs):
        meshes[e], st = oracle_state_at(sc, e, s)
        q[e], v[e] = _f32(st.q), _f32(st.v)
    sim = _sim(sc, solve=solve)
    qg, _ = gpu_step_from(sim, sc, s, q, v)
    con = parity.gpu_contacts(sim)
    for e in range(sc.n_envs):
        ref = oracle.EnvState(q[e], v[e])
        oracle.step(meshes[e], sc, e, s, ref)
        err = np.abs(qg[e] - ref.q).max()
        assert err <= POS_TOL, (e, err, len(ref.cvert))
        parity.assert_impulses(con, e, ref, sc, e, s, err)


@pytest.mark.parametrize("theta", [0.2, 0.35])
def test_incline_coulomb_on_gpu(cuda, theta):
    """Tolerance mode on the GPU: a particle on an incline sticks iff
    tan(theta) <= mu and otherwise slides with x_n = a h^2 n(n+1)/2
    (mu swept in steps of 0.002 around tan(theta))."""
    from paper_2604_17513_gb300 import flash
    t = np.tan(theta)
    for dmu in (-0.004, -0.002, 0.002, 0.004):
        mu = t + dmu
        sc = scenes.incline_particle(theta, mu, steps=8)
        sim = _sim(sc, mode=flash.MODE_TOL, k_cap=50, tol=1e-7)
        qg, _ = gpu_step_from(sim, sc, 0, sc.q0, sc.v0, n=8)
        disp = np.linalg.norm(qg[0, 0] - sc.q0[0, 0])
        if mu >= t:
            assert disp < 1e-6, (mu, disp)
        else:
            a = 9.81 * (np.sin(theta) - mu * np.cos(theta))
            assert abs(disp - a * sc.h ** 2 * 36) < 2e-6, (mu, disp)
        it, r = sim.stats()
        assert r.max().item() <= 1e-7


def _corner_particle():
    """A particle pushed into the corner of three planes (x, y and z walls)."""
    rest = np.zeros((1, 3))
    tau = 1e-3
    q0 = np.full((1, 1, 3), tau)
    K = 3
    poses = np.zeros((1, 4, K, 7))
    # plane normals +z (identity), +x (rotate +z onto +x about y), +y (about x)
    c = np.cos(np.pi / 4)
    poses[0, :, 0] = (0, 0, 0, 1, 0, 0, 0)
    poses[0, :, 1] = (0, 0, 0, c, 0, c, 0)
    poses[0, :, 2] = (0, 0, 0, c, -c, 0, 0)
    sc = scenes.Scene("corner", scenes.TRI, rest, np.zeros((0, 3), np.int32), np.array([0.01]), 0.0, 0.0, q0,
                      np.zeros_like(q0), np.array([0.4]), np.ones(1),
                      np.array([[scenes.PLANE] * 3], np.int32), np.zeros((1, K, 3)), np.zeros((1, K)), poses,
                      thickness=tau, steps=3, gravity=(-3.0, -2.0, -9.81))
    return sc


def test_three_contacts_on_one_vertex(cuda):
    """General per-vertex block (three contacts): GPU vs oracle, and the
    particle stays in the corner."""
    sc = _corner_particle()
    mesh = oracle.Mesh.from_scene(sc)
    ref = oracle.EnvState(sc.q0[0], sc.v0[0])
    for s in range(3):
        oracle.step(mesh, sc, 0, s, ref)
    assert len(ref.cvert) == 3
    sim = _sim(sc)
    qg, _ = gpu_step_from(sim, sc, 0, sc.q0, sc.v0, n=3)
    err = np.abs(qg[0] - ref.q).max()
    assert err <= POS_TOL
    parity.assert_impulses(parity.gpu_contacts(sim), 0, ref, sc, 0, 2, err)
    assert np.abs(ref.q[0] - sc.q0[0, 0]).max() < 1e-4


@pytest.mark.parametrize("solve", SOLVES)
def test_mixed_meshes_one_step(cuda, solve):
    """Uneven batch in one scene: cloths and tet blocks of different sizes
    (one group per template) against random boxes and spheres; every
    environment is checked against the oracle after one step from its
    oracle state in contact."""
    import torch
    from paper_2604_17513_gb300 import flash
    scs = scenes.mixed_batch(n_envs=8, steps=40, side_choices=(16, 20), tet_targets=(250, 500))
    s = 22
    qs, vs, refs, who = [], [], [], []
    for sc in scs:
        for e in range(sc.n_envs):
            mesh, st = oracle_state_at(sc, e, s)
            q0, v0 = _f32(st.q), _f32(st.v)
            qs.append(q0)
            vs.append(v0)
            ref = oracle.EnvState(q0, v0)
            oracle.step(mesh, sc, e, s, ref)
            refs.append(ref)
            who.append((sc, e))
    assert sum(len(r.cvert) > 0 for r in refs) >= 4      # most environments touch something
    sim = flash.Sim(scs, solve=solve)
    sim.set_state(torch.from_numpy(np.concatenate(qs).astype(np.float32)).to(cuda),
                  torch.from_numpy(np.concatenate(vs).astype(np.float32)).to(cuda))
    sim.set_poses(flash.poses_tensor(scs, s, cuda), which=0)
    sim.set_poses(flash.poses_tensor(scs, s + 1, cuda), which=1)
    sim.step(1)
    qg, _ = sim.get_state()
    qg = qg.cpu().numpy()
    off = sim.offsets
    con = parity.gpu_contacts(sim)
    for i, ref in enumerate(refs):
        err = np.abs(qg[off[i]:off[i + 1]] - ref.q).max()
        assert err <= POS_TOL, (i, err, len(ref.cvert))
        parity.assert_impulses(con, i, ref, who[i][0], who[i][1], s, err)


@pytest.mark.parametrize("solve", SOLVES)
def test_mixed_meshes_tolerance_mode(cuda, solve):
    """Mode B on an uneven batch: every environment iterates until its NCP
    residual is <= 1e-5 (cap 60).  Every environment is compared with the
    oracle at the GPU's own iteration count: where the oracle's stopping rule
    stopped at the same count, with that run; where FP32 and FP64 crossed the
    threshold at different iterations, with the oracle's fixed-count run of
    as many iterations (the same iterate of the same iteration)."""
    import torch
    from paper_2604_17513_gb300 import flash
    scs = scenes.mixed_batch(n_envs=8, steps=40, side_choices=(16, 20), tet_targets=(250, 500))
    s = 22
    kw = dict(mode=1, tol=1e-5, k_min=1, k_cap=60)
    qs, vs, starts = [], [], []
    for sc in scs:
        for e in range(sc.n_envs):
            mesh, st = oracle_state_at(sc, e, s)
            q0, v0 = _f32(st.q), _f32(st.v)
            qs.append(q0)
            vs.append(v0)
            starts.append((sc, e, mesh, q0, v0))
    sim = flash.Sim(scs, solve=solve, **kw)
    sim.set_state(torch.from_numpy(np.concatenate(qs).astype(np.float32)).to(cuda),
                  torch.from_numpy(np.concatenate(vs).astype(np.float32)).to(cuda))
    sim.set_poses(flash.poses_tensor(scs, s, cuda), which=0)
    sim.set_poses(flash.poses_tensor(scs, s + 1, cuda), which=1)
    sim.step(1)
    it, r = sim.stats()
    it, r = it.cpu().numpy(), r.cpu().numpy()
    qg = sim.get_state()[0].cpu().numpy()
    off = sim.offsets
    con = parity.gpu_contacts(sim)
    same = 0
    for i, (sc, e, mesh, q0, v0) in enumerate(starts):
        if it[i] < 60:
            assert r[i] <= 1e-5, (i, it[i], r[i])
        ref = oracle.EnvState(q0, v0)
        oracle.step(mesh, sc, e, s, ref, **kw)
        if ref.iters == it[i]:
            same += 1
        else:
            assert abs(int(it[i]) - ref.iters) <= 2, (i, it[i], ref.iters)
            ref = oracle.EnvState(q0, v0)
            oracle.step(mesh, sc, e, s, ref, k_max=int(it[i]))
        err = np.abs(qg[off[i]:off[i + 1]] - ref.q).max()
        assert err <= POS_TOL, (i, err, it[i])
        parity.assert_impulses(con, i, ref, sc, e, s, err)
    assert same >= 6, (it,)


@pytest.mark.parametrize("solve", SOLVES)
def test_batched_groups_equal_separate_scenes(cuda, solve):
    """A scene of several mesh templates runs its per-environment kernels as
    table launches over all groups and its contractions on a stream pool;
    stepping it must give bit-identical states to stepping each template in a
    scene of its own."""
    import torch
    from paper_2604_17513_gb300 import flash
    scs = scenes.mixed_batch(n_envs=12, steps=12, side_choices=(16, 24), tet_targets=(250, 600))
    assert len(scs) >= 3
    big = flash.Sim(scs, solve=solve)
    q0, v0 = flash.state_tensors(scs, cuda)
    big.set_state(q0, v0)
    big.set_poses(flash.poses_tensor(scs, 0, cuda), which=0)
    for s in range(3):
        big.set_poses(flash.poses_tensor(scs, s + 1, cuda))
        big.step(1)
    qb = big.get_state()[0].cpu().numpy()
    off = big.offsets
    env0 = 0
    for sc in scs:
        one = flash.Sim(sc, solve=solve, contact_cap=big.desc.contact_cap)
        q1, v1 = flash.state_tensors(sc, cuda)
        one.set_state(q1, v1)
        one.set_poses(flash.poses_tensor(sc, 0, cuda), which=0)
        for s in range(3):
            one.set_poses(flash.poses_tensor(sc, s + 1, cuda))
            one.step(1)
        q = one.get_state()[0].cpu().numpy()
        part = qb[off[env0]:off[env0 + sc.n_envs]]
        assert np.array_equal(part, q), (sc.name, np.abs(part - q).max())
        env0 += sc.n_envs
    assert big.status() == 0


@pytest.mark.parametrize("solve", SOLVES)
@pytest.mark.parametrize("mode", [0, 1])
def test_lanes_do_not_change_results(cuda, solve, mode):
    """Environments partitioned into lanes that step concurrently on their own
    streams (each lane's contractions over its own column range), and fixed
    steps replayed from a captured CUDA graph, give bit-identical states to
    one lane launched kernel by kernel, in both stopping modes."""
    import torch
    from paper_2604_17513_gb300 import flash
    sc = scenes.cloth_gripper(n_envs=260, n_side=16, side=0.25, steps=30)
    kw = dict(mode=1, tol=1e-5, k_cap=40) if mode else {}
    out = []
    # 3 and 4 lanes split the 260 environments unevenly
    for lanes, eager in ((1, True), (1, False), (3, False), (4, True)):
        sim = flash.Sim(sc, solve=solve, lanes=lanes, eager=eager, **kw)
        q0, v0 = flash.state_tensors(sc, cuda)
        sim.set_state(q0, v0)
        sim.set_poses(flash.poses_tensor(sc, 0, cuda), which=0)
        for s in range(20):
            sim.set_poses(flash.poses_tensor(sc, s + 1, cuda))
            sim.step(1)
        it, r = sim.stats()
        out.append((sim.get_state()[0].cpu().numpy(), it.cpu().numpy(), sim.status()))
    for q, it, st in out[1:]:
        assert np.array_equal(q, out[0][0]) and np.array_equal(it, out[0][1]) and st == out[0][2]


def test_graphed_tolerance_loop_full_metric(cuda):
    """Tolerance mode replayed from a graph whose iteration loop is a device
    while-node (the device decides when every environment has stopped) gives
    bit-identical states, iteration counts and residuals to the eager host
    loop, on the full contact metric with two lanes.  Launch accounting: the
    kernels of one graphed step are a fixed part plus a fixed body per loop
    run, and the loop runs once per iteration after the first of the slowest
    environment."""
    from paper_2604_17513_gb300 import flash
    sc = scenes.tet_squeeze(n_envs=40, steps=12)
    out, deltas = [], []
    for eager in (True, False):
        sim = flash.Sim(sc, solve=flash.SOLVE_F16X3, metric=flash.METRIC_FULL, mode=flash.MODE_TOL, tol=1e-5,
                        k_cap=60, lanes=2, eager=eager)
        q0, v0 = flash.state_tensors(sc, cuda)
        sim.set_state(q0, v0)
        sim.set_poses(flash.poses_tensor(sc, 0, cuda), which=0)
        its = []
        for s in range(10):
            sim.set_poses(flash.poses_tensor(sc, s + 1, cuda))
            l0 = sim.launch_count()
            sim.step(1)
            it, r = sim.stats()
            its.append(it.cpu().numpy())
            deltas.append((eager, sim.launch_count() - l0, int(it.max().item())))
        out.append((sim.get_state()[0].cpu().numpy(), np.stack(its), r.cpu().numpy(), sim.status()))
    (qe, ite, re, se), (qg, itg, rg, sg) = out
    assert se == 0 and sg == 0
    assert np.array_equal(qe, qg) and np.array_equal(ite, itg) and np.array_equal(re, rg)
    pts = sorted({(m, d) for eager, d, m in deltas if not eager})
    assert len(pts) >= 2, pts
    (m0, d0), (m1, d1) = pts[0], pts[-1]
    assert m1 > m0 and (d1 - d0) % (m1 - m0) == 0, pts
    body = (d1 - d0) // (m1 - m0)
    assert body > 0 and all(d - d0 == body * (m - m0) for m, d in pts), pts


@pytest.mark.parametrize("solve", SOLVES)
def test_global_apply_eigen_form(cuda, solve):
    """Per-environment stiffness on one tet mesh: the library applies
    A_e^-1 = V diag(1/(1 + k_e lam)) V^T with one shared eigenbasis; each
    environment's result equals the oracle's Cholesky solve with its own A_e."""
    import torch
    sc = scenes.tet_squeeze(n_envs=5, steps=2)
    sim = _sim(sc, solve=solve)
    rng = np.random.default_rng(9)
    rhs = rng.normal(size=(5, sc.n_verts, 3)) * 1e-6
    out = sim.global_apply(0, 5, torch.from_numpy(rhs.astype(np.float32).reshape(-1, 3)).to(cuda))
    out = out.cpu().numpy().reshape(5, sc.n_verts, 3)
    for e in range(5):
        ref = oracle.Mesh.from_scene(sc, e).solve(_f32(rhs[e]))
        err = np.abs(out[e] - ref).max() / np.abs(ref).max()
        assert err < (5e-5 if solve == 0 else 2e-4), (e, sc.stiff[e], err)


@pytest.mark.parametrize("solve", SOLVES)
def test_largest_mixed_templates_one_step(cuda, solve):
    """The largest templates of the mixed batch: a 64x64 cloth (4096
    vertices) and a 17x17x8-cube tet block (2916 vertices, above the eigen
    form's limit, so its group has its own dense inverse), one fixed step in
    contact.  The common start comes from the oracle run with 2 iterations
    per step for the approach (any common state is a valid start)."""
    import torch
    from paper_2604_17513_gb300 import flash
    scs = scenes.mixed_batch(n_envs=2, steps=40, side_choices=(64,), tet_targets=(2900, 3000))
    assert sorted(sc.n_verts for sc in scs) == [2916, 4096]
    s = 24
    qs, vs, refs = [], [], []
    for sc in scs:
        mesh = oracle.Mesh.from_scene(sc, 0)
        st = oracle.EnvState(sc.q0[0], sc.v0[0])
        for k in range(s):
            oracle.step(mesh, sc, 0, k, st, k_max=2)
        q0, v0 = _f32(st.q), _f32(st.v)
        ref = oracle.EnvState(q0, v0)
        oracle.step(mesh, sc, 0, s, ref)
        assert len(ref.cvert) > 100
        qs.append(q0)
        vs.append(v0)
        refs.append(ref)
    sim = flash.Sim(scs, solve=solve)
    sim.set_state(torch.from_numpy(np.concatenate(qs).astype(np.float32)).to(cuda),
                  torch.from_numpy(np.concatenate(vs).astype(np.float32)).to(cuda))
    sim.set_poses(flash.poses_tensor(scs, s, cuda), which=0)
    sim.set_poses(flash.poses_tensor(scs, s + 1, cuda), which=1)
    sim.step(1)
    qg = sim.get_state()[0].cpu().numpy()
    off = sim.offsets
    con = parity.gpu_contacts(sim)
    for i, (sc, ref) in enumerate(zip(scs, refs)):
        err = np.abs(qg[off[i]:off[i + 1]] - ref.q).max()
        assert err <= POS_TOL, (sc.name, err)
        parity.assert_impulses(con, i, ref, sc, 0, s, err, what=sc.name)
    assert sim.status() == 0


def test_cloth_drop_rollout_invariants(cuda):
    """The 16x16 cloth dropped on the sphere, 200 steps in tolerance mode
    (r_ncp <= 1e-6, cap 200; the full metric, which reaches that residual in
    ~8 iterations where the lite metric needs more than the cap on most
    draped steps) on the GPU: trajectories of a chaotic drape are
    not compared, the NCP's invariants are.  After every step, every contact
    of every environment that converged satisfies lambda_n >= 0, gap >=
    -1e-6 m, |h lambda_n gap| <= 1e-8 (or, for impact forces, h lambda_n
    times the gap that the residual tolerance and an FP32 position resolve),
    |lambda_t| <= mu
    lambda_n (lambda_n and the cone within the residual's resolution
    m tol / h^2), with gaps
    evaluated in FP64 at the GPU's positions;
    at least 95 % of env-steps converge."""
    import torch
    from paper_2604_17513_gb300 import flash
    sc = scenes.cloth_drop(n_envs=4, steps=200)
    tol = 1e-6
    sim = flash.Sim(sc, solve=flash.SOLVE_F16X3, mode=flash.MODE_TOL, tol=tol, k_cap=200,
                    metric=flash.METRIC_FULL)
    q0, v0 = flash.state_tensors(sc, cuda)
    sim.set_state(q0, v0)
    sim.set_poses(flash.poses_tensor(sc, 0, cuda), which=0)
    h, n = sc.h, sc.n_verts
    conv = checked = 0
    for s in range(200):
        sim.set_poses(flash.poses_tensor(sc, s + 1, cuda))
        sim.step(1)
        it, r = (t.cpu().numpy() for t in sim.stats())
        q = sim.get_state()[0].cpu().numpy().astype(np.float64).reshape(sc.n_envs, n, 3)
        cnt, vert, obs, _, gam = parity.gpu_contacts(sim)
        for e in range(sc.n_envs):
            if r[e] > tol:
                continue
            conv += 1
            for j in range(int(cnt[e])):
                vtx, o, g = int(vert[e, j]), int(obs[e, j]), gam[e, j].astype(np.float64)
                sd, _ = oracle.sdf(sc.obs_type[e, o], sc.obs_dims[e, o], sc.poses[e, s + 1, o], q[e, vtx])
                gap = sd - sc.thickness
                m = sc.mass[vtx]
                lam_n, lam_t = g[0] / h ** 2, np.linalg.norm(g[1:]) / h ** 2
                # the residual bounds min(gap, y_n) by tol, y_n = gamma_n / m in metres
                assert lam_n >= -m * tol / h ** 2 and gap >= -1e-6, (s, e, j, lam_n, gap)
                # with lambda_n > 0 the FB residual bounds |gap| by tol, and an
                # FP32 position and the FP32 distance evaluated from it resolve
                # a gap to a few ulp(|x|): |h lambda_n gap| <= 1e-8, or
                # h lambda_n times the larger of tol and 4 ulp(|x|) (impacts)
                res = max(tol, 4.0 * float(np.spacing(np.float32(np.abs(q[e, vtx]).max()))))
                assert abs(h * lam_n * gap) <= max(1e-8, h * lam_n * res), (s, e, j, lam_n, gap)
                # sliding rows sit on the cone: FP32 rounding of the disk
                # projection and of the frame change between the last
                # linearisation and the end state, relative 1e-5
                assert lam_t <= sc.mu[e] * lam_n * (1 + 1e-5) + m * tol / h ** 2, (s, e, j, lam_t, lam_n)
                checked += 1
    assert sim.status() == 0
    assert conv >= 0.95 * 200 * sc.n_envs and checked > 1000, (conv, checked)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_grouped_solve_equals_per_template_launches(cuda, mode):
    """Uneven batch in two lanes of several mesh templates each: applying
    every template's dense inverse in one grouped tensor-core launch per lane
    gives bit-identical states and iteration counts to one launch per
    template (both stopping modes, and the full metric, whose Krylov applies
    write the grouped launch's third output table)."""
    import torch
    from paper_2604_17513_gb300 import flash
    scs = scenes.mixed_batch(n_envs=24, steps=12, side_choices=(16, 20, 24), tet_targets=(250, 600))
    assert len(scs) >= 4
    kw = [{}, dict(mode=1, tol=1e-5, k_cap=40), dict(metric=flash.METRIC_FULL)][mode]
    out = []
    for grouped in (flash.GROUPED_OFF, flash.GROUPED_ON):
        sim = flash.Sim(scs, solve=flash.SOLVE_F16X3, lanes=2, grouped=grouped, **kw)
        assert sim.grouped_solve() == (grouped == flash.GROUPED_ON)
        q0, v0 = flash.state_tensors(scs, cuda)
        sim.set_state(q0, v0)
        sim.set_poses(flash.poses_tensor(scs, 0, cuda), which=0)
        for s in range(8):
            sim.set_poses(flash.poses_tensor(scs, s + 1, cuda))
            sim.step(1)
        it, r = sim.stats()
        out.append((sim.get_state()[0].cpu().numpy(), it.cpu().numpy(), sim.status()))
    (q_off, it_off, st_off), (q_on, it_on, st_on) = out
    assert st_off == 0 and st_on == 0
    assert np.array_equal(q_on, q_off) and np.array_equal(it_on, it_off)


@pytest.mark.parametrize("mode", [0, 1])
def test_threads_per_environment_do_not_change_results(cuda, mode):
    """Cloth and tet templates in two lanes: the local pass with 256, 512 or
    1024 threads per environment, the NCP pass with 128, 256 or 512, and
    both timed on the first step (FLASH_THREADS_TUNE; graphed, and eager)
    give bit-identical states, iteration counts and residuals (one thread
    owns each vertex and each contact run, in a fixed order, and the block
    reductions are maxima), in both stopping modes.  The timed choice is
    one of the candidates for every local batch and every lane."""
    from paper_2604_17513_gb300 import flash
    scs = scenes.mixed_batch(n_envs=24, steps=12, side_choices=(16, 20, 24), tet_targets=(250, 600))
    kw = dict(mode=1, tol=1e-5, k_cap=40) if mode else {}
    runs = [(0, 0, False), (256, 128, False), (1024, 512, False), (512, 256, True),
            (flash.THREADS_TUNE, flash.THREADS_TUNE, False), (flash.THREADS_TUNE, flash.THREADS_TUNE, True)]
    out = []
    for lt, nt, eager in runs:
        sim = flash.Sim(scs, solve=flash.SOLVE_F16X3, lanes=2, eager=eager, local_threads=lt, ncp_threads=nt, **kw)
        q0, v0 = flash.state_tensors(scs, cuda)
        sim.set_state(q0, v0)
        sim.set_poses(flash.poses_tensor(scs, 0, cuda), which=0)
        for s in range(8):
            sim.set_poses(flash.poses_tensor(scs, s + 1, cuda))
            sim.step(1)
        it, r = sim.stats()
        out.append((sim.get_state()[0].cpu().numpy(), it.cpu().numpy(), r.cpu().numpy(), sim.status()))
        loc, ncp = sim.threads()
        assert len(ncp) == 2 and len(loc) >= 2
        if lt > 0:
            assert set(loc) == {lt} and set(ncp) == {nt}
        elif lt == flash.THREADS_TUNE:
            assert set(loc) <= {256, 512, 1024} and set(ncp) <= {128, 256, 512}
    q_ref, it_ref, r_ref, st_ref = out[0]
    assert st_ref == 0
    for (lt, nt, eager), (q, it, r, st) in zip(runs[1:], out[1:]):
        assert st == st_ref and np.array_equal(q, q_ref) and np.array_equal(it, it_ref) and np.array_equal(r, r_ref), \
            (lt, nt, eager)


@pytest.mark.parametrize("case", ["cloth_tol", "tet_eigen", "tet_bf16r"])
def test_split_k_does_not_change_results(cuda, case):
    """Every tensor-core apply sums the two K halves of each output tile
    separately and adds them last, on one CTA or, split-K, on two CTAs that
    meet through a scratch tile: both forms, and the autotuner's mix of them
    over lanes, give bit-identical states and iteration counts (dense
    inverse in tolerance mode, the eigen form's two contractions, the bf16
    solve with refinement)."""
    from paper_2604_17513_gb300 import flash
    if case == "cloth_tol":
        sc = scenes.cloth_gripper(n_envs=200, n_side=16, side=0.25, steps=12)
        kw = dict(solve=flash.SOLVE_F16X3, mode=flash.MODE_TOL, tol=1e-5, k_cap=20)
    else:
        sc = scenes.tet_squeeze(n_envs=96, steps=12)
        kw = dict(solve=flash.SOLVE_BF16R if case == "tet_bf16r" else flash.SOLVE_F16X3)
    out = []
    for split, lanes in ((flash.SPLITK_OFF, 1), (flash.SPLITK_ON, 1), (flash.SPLITK_ON, 3), (flash.SPLITK_AUTO, 2)):
        sim = flash.Sim(sc, lanes=lanes, split_k=split, **kw)
        if split != flash.SPLITK_AUTO:
            assert set(sim.tile_splits()) == {2 if split == flash.SPLITK_ON else 1}
        else:
            assert set(sim.tile_splits()) <= {1, 2}
        q0, v0 = flash.state_tensors(sc, cuda)
        sim.set_state(q0, v0)
        sim.set_poses(flash.poses_tensor(sc, 0, cuda), which=0)
        for s in range(8):
            sim.set_poses(flash.poses_tensor(sc, s + 1, cuda))
            sim.step(1)
        it, r = sim.stats()
        out.append((sim.get_state()[0].cpu().numpy(), it.cpu().numpy(), sim.status()))
    q0_, it0, st0 = out[0]
    assert st0 == 0 and np.isfinite(q0_).all()
    for q, it, st in out[1:]:
        assert st == st0 and np.array_equal(q, q0_) and np.array_equal(it, it0)


@pytest.mark.parametrize("steps_tol", [(0, 2e-2), (1, 3e-4), (2, 2e-5)])
@pytest.mark.parametrize("dense", [False, True])
def test_global_apply_bf16_refinement(cuda, steps_tol, dense):
    """The bf16 tensor-core solve with FP32 iterative refinement on tet
    blocks (condition 20-300): one bf16 product of the eigen form (per-
    environment stiffness) or of the dense inverse (one stiffness), then
    refine_steps corrections with the residual rhs - A w in FP32.  The
    error against the oracle's Cholesky solve falls by two orders a step, to
    the FP32 level after two (bounds from an FP64 emulation of the same
    arithmetic: 5e-3..1.3e-2, 2.5e-5..6.9e-5, 1e-7..7e-7)."""
    import torch
    from paper_2604_17513_gb300 import flash
    steps, tol = steps_tol
    sc = scenes.tet_squeeze(n_envs=4, steps=2)
    if dense:
        sc.stiff[:] = sc.stiff[0]
    sim = _sim(sc, solve=flash.SOLVE_BF16R, refine_steps=steps)
    rng = np.random.default_rng(10)
    rhs = rng.normal(size=(4, sc.n_verts, 3)) * 1e-6
    out = sim.global_apply(0, 4, torch.from_numpy(rhs.astype(np.float32).reshape(-1, 3)).to(cuda))
    out = out.cpu().numpy().reshape(4, sc.n_verts, 3)
    for e in range(4):
        ref = oracle.Mesh.from_scene(sc, e).solve(_f32(rhs[e]))
        err = np.abs(out[e] - ref).max() / np.abs(ref).max()
        assert err < tol, (e, sc.stiff[e], steps, err)


def test_tet_squeeze_one_step_bf16_refinement(cuda):
    """One fixed step of the squeezed tet blocks with the bf16 solve and two
    refinement steps: positions within 1e-5 m and impulses as the other
    solves (the correction form keeps the solve's error proportional to the
    small correction)."""
    from paper_2604_17513_gb300 import flash
    sc = scenes.tet_squeeze(n_envs=3, steps=30)
    s = 18
    q, v, meshes = sc.q0.copy(), sc.v0.copy(), {}
    for e in range(sc.n_envs):
        meshes[e], st = oracle_state_at(sc, e, s)
        q[e], v[e] = _f32(st.q), _f32(st.v)
    sim = _sim(sc, solve=flash.SOLVE_BF16R, refine_steps=2)
    qg, _ = gpu_step_from(sim, sc, s, q, v)
    con = parity.gpu_contacts(sim)
    for e in range(sc.n_envs):
        ref = oracle.EnvState(q[e], v[e])
        oracle.step(meshes[e], sc, e, s, ref)
        err = np.abs(qg[e] - ref.q).max()
        assert err <= POS_TOL, (e, err)
        parity.assert_impulses(con, e, ref, sc, e, s, err)
    assert sim.status() == 0


def test_bf16_refinement_refused_for_cloth(cuda):
    """A cloth's system (condition ~1e7) makes each bf16 refinement step grow
    the error, so the scene refuses the mode."""
    from paper_2604_17513_gb300 import flash
    with pytest.raises(flash.FlashError) as ei:
        _sim(scenes.cloth_drop(n_envs=1, steps=2), solve=flash.SOLVE_BF16R)
    assert ei.value.code == flash.ENOTIMPL
