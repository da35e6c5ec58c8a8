"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an invariant of the method, a library routine that a special case
reduces to, or brute-force enumeration.  No GPU.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2604_17513_gb300 import scenes


def rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


# ------------------------------------------------------------ local step
def test_closest_rotation_matches_svd_polar():
    """Closest 3x3 rotation = U diag(1,1,det UV^T) V^T from numpy's SVD;
    closest 3x2 orthonormal-column matrix = U V^T (thin SVD)."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        F = rng.normal(size=(3, 3))
        U, s, Vt = np.linalg.svd(F)
        d = np.sign(np.linalg.det(U @ Vt))
        ref = U @ np.diag([1, 1, d]) @ Vt
        assert np.abs(oracle.closest_rotation(F) - ref).max() < 1e-10
        F2 = rng.normal(size=(3, 2))
        U2, s2, Vt2 = np.linalg.svd(F2, full_matrices=False)
        assert np.abs(oracle.closest_rotation(F2) - U2 @ Vt2).max() < 1e-10


def test_closest_rotation_rest_and_equivariance():
    """A rotation projects to itself; R F projects to R p (Eq. internal's
    constitutive manifold is rotation invariant)."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        Q = rot(rng.normal(size=3), rng.uniform(0, np.pi))
        assert np.abs(oracle.closest_rotation(Q) - Q).max() < 1e-12
        F = rng.normal(size=(3, 3)) * 0.2 + np.eye(3)
        p = oracle.closest_rotation(F)
        assert np.abs(oracle.closest_rotation(Q @ F) - Q @ p).max() < 1e-10
        F2 = rng.normal(size=(3, 2))
        p2 = oracle.closest_rotation(F2)
        assert np.abs(oracle.closest_rotation(Q @ F2) - Q @ p2).max() < 1e-10


# ------------------------------------------------------------ system matrix
def test_cloth_topology_counts():
    """16x16 grid: 450 triangles and 645 interior edges (bending hinges)."""
    sc = scenes.cloth_drop()
    m = oracle.Mesh.from_scene(sc)
    assert m.ne == 450 and m.hinges == 645
    sc2 = scenes.cloth_gripper(n_envs=1, steps=1)
    assert len(sc2.elems) == 1922 and oracle.Mesh.from_scene(sc2).hinges == 2821
    sc3 = scenes.tet_squeeze(n_envs=1, steps=1)
    assert sc3.n_verts == 405 and len(sc3.elems) == 1280


@pytest.mark.parametrize("kind", ["tri", "tet"])
def test_system_matrix_spd_and_rigid_null_space(kind):
    """A = M + h^2 sum w G^T G is symmetric positive definite and G annihilates
    translations, so every row of A sums to the vertex mass."""
    sc = scenes.cloth_drop() if kind == "tri" else scenes.tet_squeeze(n_envs=1, steps=1)
    m = oracle.Mesh.from_scene(sc)
    A = m.matrix()
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0
    assert np.abs(A.sum(1) - sc.mass).max() < 1e-10 * np.abs(A).max()


def test_solve_residual():
    """Cholesky solve is backward stable: |A x - b| <= 1e-14 |A| |x| (FP64)."""
    sc = scenes.cloth_drop()
    m = oracle.Mesh.from_scene(sc)
    A = m.matrix()
    b = np.random.default_rng(2).normal(size=(sc.n_verts, 3))
    x = m.solve(b)
    assert np.linalg.norm(A @ x - b) <= 1e-14 * np.linalg.norm(A, 2) * np.linalg.norm(x)


def test_uniform_stretch_energy_closed_form():
    """A flat sheet stretched uniformly by (1+eps) along x: F = diag(1+eps, 1)
    in-plane, its closest rotation is I, so the stretch energy is
    w/2 * area * eps^2 and the flat bending energy is 0."""
    sc = scenes.cloth_drop()
    m = oracle.Mesh.from_scene(sc)
    eps = 0.013
    q = sc.rest.copy()
    q[:, 0] *= 1 + eps
    p = m.project(q)
    E = m.energy(q, q, p)
    area = 0.5 * 0.5
    assert abs(E - 0.5 * sc.w_stretch * area * eps ** 2) < 1e-10 * E


def test_bending_annihilates_affine_maps_and_energy_hessian():
    """Bending energy vanishes on any affine image of the flat rest mesh; the
    PD energy's Hessian (by central differences of the energy) equals A/h^2
    for fixed projections (A = M + h^2 sum w G^T G + bending)."""
    sc = scenes.cloth_drop()
    sc.w_stretch = 0.0
    m = oracle.Mesh.from_scene(sc)
    rng = np.random.default_rng(3)
    Aff = np.eye(3) + 0.3 * rng.normal(size=(3, 3))
    q = sc.rest @ Aff.T + rng.normal(size=3)
    p = np.zeros((m.ne, 9))
    assert m.energy(q, q, p) < 1e-18
    # Hessian along random directions
    sc2 = scenes.cloth_drop()
    m2 = oracle.Mesh.from_scene(sc2)
    A = m2.matrix()
    q0 = sc2.rest + 0.01 * rng.normal(size=sc2.rest.shape)
    p0 = m2.project(q0)
    for _ in range(3):
        d = rng.normal(size=q0.shape)
        t = 1e-3
        e_p, e_0, e_m = (m2.energy(q0 + t * d, q0, p0), m2.energy(q0, q0, p0), m2.energy(q0 - t * d, q0, p0))
        fd = (e_p - 2 * e_0 + e_m) / t ** 2
        exact = np.sum(d * (A @ d)) / sc2.h ** 2
        assert abs(fd - exact) < 1e-6 * abs(exact)


# ------------------------------------------------------------ whole step
def test_rest_shape_stays_at_rest():
    sc = scenes.cloth_drop(steps=5)
    sc.gravity = (0.0, 0.0, 0.0)
    sc.q0[0] = sc.rest + [0, 0, 0.6]
    st = oracle.rollout(sc, 0, 5)
    # rounding only: cond(A) ~ 7e5 for this mesh, so ~1e-16 * 7e5 * |q| per solve
    assert np.abs(st.q - sc.q0[0]).max() < 1e-9
    assert np.abs(st.v).max() < 1e-7


def test_free_fall_closed_form():
    """Rigid translation under gravity with implicit Euler: z_n = z_0 - g h^2 n(n+1)/2."""
    sc = scenes.cloth_drop(steps=12)
    sc.q0[0] = sc.rest + [0, 0, 2.0]
    st = oracle.rollout(sc, 0, 12)
    n = 12
    z = 2.0 - 9.81 * sc.h ** 2 * n * (n + 1) / 2
    # rounding of the solves (cond(A) ~ 7e5) is ~1e-10 per step; a dropped or
    # misplaced h^2 g term would show at 1e-3
    assert np.abs(st.q[:, 2] - z).max() < 1e-8
    assert np.abs(st.q[:, :2] - sc.rest[:, :2]).max() < 1e-8


def test_local_global_energy_monotone():
    """Without contact each local step (fixed q) and each global step (fixed p)
    does not increase E(q, p) = |M^1/2 (q - q~)|^2 / 2h^2 + sum w/2 |Gq - p|^2."""
    sc = scenes.cloth_drop()
    m = oracle.Mesh.from_scene(sc)
    rng = np.random.default_rng(4)
    qt = sc.rest + [0, 0, 0.5] + 0.02 * rng.normal(size=sc.rest.shape)
    q = qt.copy()
    p = m.project(q)
    E = m.energy(q, qt, p)
    for _ in range(15):
        q = m.solve(m.assemble_b(qt, p))
        E1 = m.energy(q, qt, p)
        p = m.project(q)
        E2 = m.energy(q, qt, p)
        assert E1 <= E * (1 + 1e-12) and E2 <= E1 * (1 + 1e-12)
        E = E2


def test_particle_resting_on_plane():
    """Normal contact: gamma_n = m g h^2, impulse m g h, zero gap."""
    sc = scenes.incline_particle(0.0, 0.3, steps=5)
    st = oracle.rollout(sc, 0, 5, mode=1, tol=1e-12, k_cap=50)
    m, g, h = sc.mass[0], 9.81, sc.h
    assert abs(st.gamma[0, 0] - m * g * h * h) < 1e-12
    assert abs(st.q[0, 2] - sc.thickness) < 1e-12
    assert np.abs(st.v).max() < 1e-12


@pytest.mark.parametrize("theta", [0.2, 0.35])
def test_coulomb_incline_stick_slide(theta):
    """A particle on an incline sticks iff tan(theta) <= mu; sliding follows
    x_n = a h^2 n(n+1)/2 with a = g (sin theta - mu cos theta).  mu is swept
    in steps of 0.001 around tan(theta)."""
    t = np.tan(theta)
    for dmu in (-0.003, -0.002, -0.001, 0.001, 0.002, 0.003):
        mu = t + dmu
        sc = scenes.incline_particle(theta, mu, steps=8)
        st = oracle.rollout(sc, 0, 8, mode=1, tol=1e-13, k_cap=100)
        disp = np.linalg.norm(st.q[0] - sc.q0[0, 0])
        if mu >= t:
            assert disp < 1e-12, (mu, disp)
        else:
            a = 9.81 * (np.sin(theta) - mu * np.cos(theta))
            n = 8
            assert abs(disp - a * sc.h ** 2 * n * (n + 1) / 2) < 1e-10, (mu, disp)


def _particle_scene(obs, poses, mu, steps, x0, h=0.01, mass=0.01):
    """One free particle (no elements) among kinematic obstacles.
    obs: list of (type, half-extents); poses: [S+1][K][7]."""
    K = len(obs)
    return scenes.Scene("particle", scenes.TRI, np.zeros((1, 3)), np.zeros((0, 3), np.int32), np.array([mass]),
                        0.0, 0.0, np.array([[x0]], float), np.zeros((1, 1, 3)), np.array([mu]), np.ones(1),
                        np.array([[t for t, _ in obs]], np.int32), np.array([[d for _, d in obs]], float),
                        np.zeros((1, K)), np.asarray(poses, float)[None], h=h, thickness=1e-3, steps=steps)


@pytest.mark.parametrize("mu", [0.8, 0.2])
def test_friction_on_translating_plane(mu):
    """The ground translates along x at V: the slip u_t is measured against
    the obstacle's own displacement over the step.  With mu g h >= V the
    particle sticks from the first step on (x_n = n V h); otherwise it slides
    with the Coulomb acceleration mu g toward the plane's velocity,
    x_n = mu g h^2 n(n+1)/2 while n mu g h < V."""
    V, h, n = 0.3 if mu < 0.5 else 0.05, 0.01, 8
    poses = np.array([[[V * h * s, 0, 0, 1, 0, 0, 0]] for s in range(n + 1)])
    sc = _particle_scene([(scenes.PLANE, (0, 0, 0))], poses, mu, n, (0, 0, 1e-3), h=h)
    st = oracle.rollout(sc, 0, n, mode=1, tol=1e-13, k_cap=100)
    if mu * 9.81 * h >= V:
        assert abs(st.q[0, 0] - n * V * h) < 1e-12 and abs(st.v[0, 0] - V) < 1e-10
    else:
        assert n * mu * 9.81 * h < V
        assert abs(st.q[0, 0] - mu * 9.81 * h * h * n * (n + 1) / 2) < 1e-12
        assert abs(st.v[0, 0] - n * mu * 9.81 * h) < 1e-10
    assert abs(st.q[0, 1]) < 1e-14 and abs(st.q[0, 2] - 1e-3) < 1e-12


def test_box_pushes_particle_on_frictionless_ground():
    """A 2 cm box sliding along x at V pushes a particle resting on the
    frictionless ground: two contacts on one vertex (ground normal z, box
    face normal x), and at convergence the particle stays exactly one
    thickness in front of the moving face and on the ground."""
    V, h, n, half = 0.1, 0.01, 10, 0.01
    poses = np.array([[[0, 0, 0, 1, 0, 0, 0], [V * h * s, 0, half, 1, 0, 0, 0]] for s in range(n + 1)])
    x0 = (half + 1e-3, 0.0, 1e-3)
    sc = _particle_scene([(scenes.PLANE, (0, 0, 0)), (scenes.BOX, (half, half, half))], poses, 0.0, n, x0, h=h)
    st = oracle.EnvState(sc.q0[0], sc.v0[0])
    mesh = oracle.Mesh.from_scene(sc, 0)
    for s in range(n):
        oracle.step(mesh, sc, 0, s, st, mode=1, tol=1e-13, k_cap=100)
        assert len(st.cvert) == 2
        assert abs(st.q[0, 0] - (x0[0] + (s + 1) * V * h)) < 1e-12, s
        assert abs(st.q[0, 2] - 1e-3) < 1e-12 and abs(st.q[0, 1]) < 1e-14
    assert abs(st.v[0, 0] - V) < 1e-10


def test_complementarity_at_convergence():
    """Converged contacts: lambda_n >= 0, gap >= -1e-6 m, |h lambda_n gap| <= 1e-8,
    |lambda_t| <= mu lambda_n, sliding contacts oppose the slip."""
    sc = scenes.cloth_drop(steps=40)
    mesh = oracle.Mesh.from_scene(sc)
    st = oracle.EnvState(sc.q0[0], sc.v0[0])
    for s in range(30):
        oracle.step(mesh, sc, 0, s, st)
    qt = st.q.copy()
    oracle.step(mesh, sc, 0, 30, st, mode=1, metric=1, tol=1e-10, k_cap=200)
    assert st.rncp <= 1e-10 and len(st.cvert) > 0
    for v, o, g in zip(st.cvert, st.cobs, st.gamma):
        sd, nrm = oracle.sdf(sc.obs_type[0, o], sc.obs_dims[0, o], sc.poses[0, 31, o], st.q[v])
        gap = sd - sc.thickness
        lam_n = g[0] / sc.h ** 2
        lam_t = np.linalg.norm(g[1:]) / sc.h ** 2
        assert lam_n >= -1e-9 and gap >= -1e-6
        assert abs(sc.h * lam_n * gap) <= 1e-8
        assert lam_t <= sc.mu[0] * lam_n + 1e-9
        slip = st.q[v] - qt[v]
        slip_t = slip - nrm * np.dot(nrm, slip)
        if np.linalg.norm(slip_t) > 1e-7:
            assert np.dot(g[1:], slip_t) <= 1e-12


def test_lite_and_full_metric_share_the_fixed_point():
    """The lite metric Z = J M^-1 J^T + E changes the Newton path, not the
    converged NCP solution (Sec. IV-B.1).  With a quadratic energy (bending
    only, so the local step is exact) a converged contact residual means a
    converged step, and both metrics must land on the same state."""
    sc = _small_bending_cloth(0.05)
    sc.mu[:] = 0.3
    mesh = oracle.Mesh.from_scene(sc)
    a = oracle.EnvState(sc.q0[0], sc.v0[0])
    b = oracle.EnvState(sc.q0[0], sc.v0[0])
    oracle.step(mesh, sc, 0, 0, a, mode=1, metric=0, tol=1e-11, k_cap=5000)
    oracle.step(mesh, sc, 0, 0, b, mode=1, metric=1, tol=1e-11, k_cap=500)
    assert a.rncp <= 1e-11 and b.rncp <= 1e-11 and len(a.cvert) > 0
    assert np.abs(a.q - b.q).max() < 1e-9
    assert b.iters < a.iters


def test_gmres_full_metric_exhausted_space_equals_exact_solve():
    """Full metric with the iterative Z solve (metric 2): when the linear
    iterations reach the dimension 3C of the contact system, GMRES has
    searched the whole space and every Newton step equals the exact dense
    solve of metric 1, in every local-global iterate."""
    sc = _small_bending_cloth(0.05)
    sc.mu[:] = 0.3
    mesh = oracle.Mesh.from_scene(sc)
    a = oracle.EnvState(sc.q0[0], sc.v0[0])
    b = oracle.EnvState(sc.q0[0], sc.v0[0])
    oracle.step(mesh, sc, 0, 0, a, k_max=6, metric=1)
    oracle.step(mesh, sc, 0, 0, b, k_max=6, metric=2, lin_iters=3 * 9)
    assert len(a.cvert) == 9
    assert np.abs(a.q - b.q).max() < 1e-10 and np.abs(a.gamma - b.gamma).max() < 1e-10 * np.abs(a.gamma).max()


def test_gmres_full_metric_shares_the_fixed_point():
    """With 10 linear iterations (fewer than the 3C = 27 unknowns) each Newton
    step is inexact, but run to convergence the full metric lands on the
    same state as the lite metric and the exact full metric."""
    sc = _small_bending_cloth(0.05)
    sc.mu[:] = 0.3
    mesh = oracle.Mesh.from_scene(sc)
    a = oracle.EnvState(sc.q0[0], sc.v0[0])
    c = oracle.EnvState(sc.q0[0], sc.v0[0])
    oracle.step(mesh, sc, 0, 0, a, mode=1, metric=0, tol=1e-11, k_cap=5000)
    oracle.step(mesh, sc, 0, 0, c, mode=1, metric=2, lin_iters=10, tol=1e-11, k_cap=500)
    assert c.rncp <= 1e-11
    assert np.abs(a.q - c.q).max() < 1e-9


def _small_bending_cloth(tilt):
    rest, tris = scenes.cloth_grid(3, 3, 0.2)
    n = len(rest)
    q0 = rest.copy()
    q0[:, 2] = 1e-3 + 2e-4 + tilt * rest[:, 0]
    v0 = np.zeros((1, n, 3))
    v0[0, :, 2] = -0.05
    sc = scenes.Scene("bb", scenes.TRI, rest, tris, np.full(n, 0.01), 0.0, 0.05, q0[None], v0,
                      np.array([0.0]), np.ones(1), np.array([[scenes.PLANE]], np.int32), np.zeros((1, 1, 3)),
                      np.zeros((1, 1)), np.tile(np.array(scenes.IDENTITY_POSE), (1, 3, 1, 1)), thickness=1e-3,
                      margin=0.05, steps=2)
    return sc


@pytest.mark.parametrize("tilt", [0.02, 0.05])
def test_brute_force_active_sets(tilt):
    """Frictionless plane contact with a quadratic (bending-only) energy: the
    converged NCP solution is the unique KKT point of
    min 1/2 q^T A q - b^T q  s.t.  z_v >= tau, found by enumerating all 2^C
    active sets."""
    sc = _small_bending_cloth(tilt)
    mesh = oracle.Mesh.from_scene(sc)
    st = oracle.EnvState(sc.q0[0], sc.v0[0])
    qt = sc.q0[0] + sc.h * sc.v0[0] + sc.h ** 2 * np.array(sc.gravity)
    oracle.step(mesh, sc, 0, 0, st, mode=1, tol=1e-13, k_cap=500)
    A = mesh.matrix()
    n = sc.n_verts
    b = mesh.assemble_b(qt, np.zeros((len(sc.elems), 9)))
    # only z couples to the plane; x, y are unconstrained
    bz = b[:, 2]
    found = []
    for act in itertools.product([0, 1], repeat=n):
        idx = [i for i in range(n) if act[i]]
        k = len(idx)
        K = np.zeros((n + k, n + k))
        K[:n, :n] = A
        rhs = np.zeros(n + k)
        rhs[:n] = bz
        for j, i in enumerate(idx):
            K[i, n + j] = -1.0
            K[n + j, i] = 1.0
            rhs[n + j] = sc.thickness
        sol = np.linalg.solve(K, rhs)
        z, lam = sol[:n], sol[n:]
        if np.all(z >= sc.thickness - 1e-12) and np.all(lam >= -1e-14):
            found.append(z)
    assert len(found) >= 1
    for z in found[1:]:
        assert np.abs(z - found[0]).max() < 1e-12
    assert np.abs(st.q[:, 2] - found[0]).max() < 1e-9
    assert 0 < sum(np.isclose(found[0], sc.thickness, atol=1e-12)) < n


# ------------------------------------------------------------ warm-start MLP
def test_mlp_gradient_finite_differences():
    """FP64 backward of the 10-128-128-6 network vs central differences."""
    rng = np.random.default_rng(6)
    n_par = 128 * 10 + 128 + 128 * 128 + 128 + 6 * 128 + 6
    p = rng.normal(size=n_par) * 0.1
    x = rng.normal(size=(7, 10))
    t = rng.normal(size=(7, 6))
    loss, g = oracle.mlp_loss_grad(p, x, t)
    assert abs(loss - 0.5 * np.mean(np.sum((oracle.mlp_forward(p, x) - t) ** 2, 1))) < 1e-12
    for i in rng.choice(n_par, 40, replace=False):
        e = np.zeros(n_par)
        e[i] = 1e-6
        fd = (oracle.mlp_loss_grad(p + e, x, t)[0] - oracle.mlp_loss_grad(p - e, x, t)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


# ---------------------------------------------------------------------------
# bilateral grasp (appendix, Bilateral Constraint for Cloth Control)
# ---------------------------------------------------------------------------
def _grasp_scene(release_step=45):
    """6x6 cloth of side 10 cm, a corner grasped at step 2 and lifted 40 cm in
    0.3 s (13 mm per step), released at ``release_step``."""
    return scenes.cloth_grasp(n_envs=1, n_side=6, side=0.1, steps=50, lift=(0.4, 0.4), inward=(0.0, 0.0),
                              rise_time=0.3, release_step=release_step)


def _world_force(st):
    """Sum over the contact list of the world-frame multiplier R^T gamma:
    normal along +z for the ground plane, along world x for a grasp row
    (frame = world axes); gamma[1:] is already the world tangential part."""
    F = np.zeros(3)
    for o, g in zip(st.cobs, st.gamma):
        n = np.array([1.0, 0.0, 0.0]) if o == oracle.GRASP_SLOT else np.array([0.0, 0.0, 1.0])
        F += n * g[0] + g[1:]
    return F


def test_grasp_activation_and_constraint():
    """Activation attaches exactly the vertices within the radius of the anchor
    (the corner: its neighbours are 20 mm away, the radius 6 mm), and, with
    the full metric, every step ends with the grasped vertex on the gripper
    at t+h (C = x - p_grip(t+h) ~ 0) while the gripper rises 13 mm per step;
    the constraint is one row of the contact list, after every obstacle row."""
    sc = _grasp_scene()
    mesh = oracle.Mesh.from_scene(sc, 0)
    st = oracle.EnvState(sc.q0[0], sc.v0[0])
    corner = None
    for s in range(20):
        oracle.step(mesh, sc, 0, s, st, metric=2)
        att = np.nonzero(st.attached)[0]
        if s < 2:
            assert len(att) == 0 and (st.cobs != oracle.GRASP_SLOT).all()
            continue
        p_t = oracle._to_world(sc.poses[0, 2, 1], (0, 0, 0))
        d = np.linalg.norm(sc.q0[0] - p_t, axis=1)
        if corner is None:
            corner = int(np.argmin(d))
            assert list(att) == [corner] and np.sort(d)[1] > 3 * sc.meta["grasp"]["radius"]
        assert list(att) == [corner]
        rows = np.nonzero(st.cobs == oracle.GRASP_SLOT)[0]
        assert len(rows) == 1 and st.cvert[rows[0]] == corner
        assert rows[0] == len(st.cvert) - 1 or st.cvert[rows[0] + 1] > corner
        p_th = oracle._to_world(sc.poses[0, s + 1, 1], (0, 0, 0))
        assert np.abs(st.q[corner] - p_th).max() <= 1e-8, (s, st.q[corner] - p_th)
    # the cloth left the ground with the corner
    assert st.q[:, 2].min() > 0.1


def test_grasp_momentum_balance_and_release():
    """Every global solve keeps sum_i m_i (q_i - q~_i) = sum of the contact
    multipliers in world axes (A has zero row sums apart from M), for ground
    and grasp rows alike and at any iteration count: while the cloth hangs
    from the corner rising at constant speed that sum is the grasp force
    (about the weight impulse M g h^2 upwards); after the release the contact list is empty and the
    centre of mass falls freely (sum = 0)."""
    sc = _grasp_scene(release_step=40)
    mesh = oracle.Mesh.from_scene(sc, 0)
    st = oracle.EnvState(sc.q0[0], sc.v0[0])
    m = sc.mass[:, None]
    weight = sc.mass.sum() * 9.81 * sc.h ** 2
    for s in range(46):
        qt, vt = st.q.copy(), st.v.copy()
        for metric in ([0, 2] if s in (2, 12) else [2]):
            trial = oracle.EnvState(qt, vt)
            trial.attached = st.attached.copy()
            oracle.step(mesh, sc, 0, s, trial, metric=metric)
            qtil = qt + sc.h * vt + sc.h ** 2 * np.asarray(sc.gravity)
            lhs = (m * (trial.q - qtil)).sum(0)
            assert np.abs(lhs - _world_force(trial)).max() <= 1e-12, (s, metric, lhs, _world_force(trial))
        st = trial
        if 10 <= s < 40:
            assert list(st.cobs) == [oracle.GRASP_SLOT]
        if 10 <= s < 30:   # gripper rising at constant speed: the force carries the weight
            assert 0.8 * weight < lhs[2] < 1.2 * weight, (s, lhs[2], weight)
        if s >= 40:
            assert len(st.cvert) == 0 and not st.attached.any()
            assert np.abs(lhs).max() <= 1e-12


# ---------------------------------------------------------------------------
# cloth self-collision (vertex against triangle; the paper disables it and
# describes no method, so these pin the reading's geometry and mechanics)
# ---------------------------------------------------------------------------
def _stack(self_collision=True, n_envs=1, n_side=16):
    sc = scenes.cloth_stack_drop(n_envs=n_envs, n_side=n_side, steps=30)
    if not self_collision:
        sc.meta = {}
    return sc


def _self_candidates_numpy(sc, q0, q1, reach):
    """Independent detection: each triangle's plane by SVD of its centred
    corners, barycentric coordinates of the projection by pseudo-inverse,
    topological neighbours as sets, both configurations, the first SELF_MAX
    triangles per vertex."""
    tris = sc.elems
    ring = [set() for _ in range(sc.n_verts)]
    for t in tris:
        for a in t:
            ring[a].update(int(x) for x in t)
    hit = np.zeros((sc.n_verts, len(tris)), bool)
    for x in (q0, q1):
        P = x[tris]                                        # [T][3][3]
        nrm = np.linalg.svd(P - P.mean(1, keepdims=True))[2][:, 2]   # [T][3]
        E = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]], -1)      # [T][3][2]
        pinv = np.linalg.pinv(E)                           # [T][2][3]
        rel = x[:, None, :] - P[None, :, 0]                # [n][T][3]
        d = (rel * nrm[None]).sum(-1)
        y = rel - d[..., None] * nrm[None]
        w12 = np.einsum("tij,ntj->nti", pinv, y)
        w = np.concatenate([1 - w12.sum(-1, keepdims=True), w12], -1)
        hit |= (np.abs(d) < reach) & (w.min(-1) >= -0.1)
    out = set()
    for p in range(sc.n_verts):
        found = [f for f in np.nonzero(hit[p])[0] if not any(int(v) in ring[p] for v in tris[f])]
        out.update((p, int(f)) for f in found[:oracle.SELF_MAX])
    return out


def test_self_detection_matches_brute_force():
    """Self-contact candidates at the step start equal an independent
    computation of the rule (plane distance < tau + margin, projection inside
    the triangle up to 0.1, no triangle touching the vertex's own triangles,
    at q_t or q~, at most SELF_MAX per vertex in triangle order)."""
    sc = _stack()
    mesh = oracle.Mesh.from_scene(sc, 0)
    st = oracle.EnvState(sc.q0[0], sc.v0[0])
    for s in range(3):
        oracle.step(mesh, sc, 0, s, st, metric=2)
    dp = oracle.params(sc, 0)[0]
    cv, co, ct = oracle.detect(mesh, sc, 0, 3, st.q, st.v, dp)
    got = {(int(v), int(t)) for v, o, t in zip(cv, co, ct) if o == oracle.SELF_SLOT}
    qp = st.q + sc.h * st.v + sc.h ** 2 * np.asarray(sc.gravity)
    ref = _self_candidates_numpy(sc, st.q, qp, sc.thickness + sc.margin)
    assert len(got) > 100 and got == ref
    assert all(t == -1 for o, t in zip(co, ct) if o not in (oracle.SELF_SLOT, oracle.EE_SLOT))


@pytest.mark.parametrize("metric", [0, 2])
def test_self_contact_forces_are_internal(metric):
    """Self contacts push their two sides equally and oppositely (weights 1
    and -w for vertex-triangle, 1 - s, s, -(1 - t), -t for edge-edge: sum
    zero): sum_i m_i (q_i - q~_i) equals
    the world-frame sum of the ground multipliers alone (to 1e-12), at any
    iteration count, while self contacts carry force."""
    sc = _stack()
    mesh = oracle.Mesh.from_scene(sc, 0)
    st = oracle.EnvState(sc.q0[0], sc.v0[0])
    m = sc.mass[:, None]
    carried = 0
    for s in range(8):
        qt, vt = st.q.copy(), st.v.copy()
        oracle.step(mesh, sc, 0, s, st, metric=metric)
        qtil = qt + sc.h * vt + sc.h ** 2 * np.asarray(sc.gravity)
        lhs = (m * (st.q - qtil)).sum(0)
        ground = st.cobs == 0
        F = st.gamma[ground, 0].sum() * np.array([0, 0, 1.0]) + st.gamma[ground, 1:].sum(0)
        assert np.abs(lhs - F).max() <= 1e-12, (s, lhs, F)
        carried += (st.gamma[st.cobs >= oracle.SELF_SLOT, 0] > 0).sum()
    if metric == 2:   # (the lite metric lets the layers pass through; the identity holds all the same)
        assert carried > 100


def test_stacked_cloth_rests_on_the_base():
    """With self-collision (full metric, 10 GMRES iterations) the dropped
    piece comes to rest one thickness tau above the base; without it the
    piece falls through to the ground."""
    nb = 256
    for on in (True, False):
        sc = _stack(self_collision=on)
        mesh = oracle.Mesh.from_scene(sc, 0)
        st = oracle.EnvState(sc.q0[0], sc.v0[0])
        for s in range(15):
            oracle.step(mesh, sc, 0, s, st, metric=2)
        zb, zt = st.q[:nb, 2], st.q[nb:, 2]
        if on:
            assert np.abs(zb - sc.thickness).max() < 2e-4
            assert np.abs(zt - 2 * sc.thickness).max() < 2e-4, (zt.min(), zt.max())
        else:
            assert np.abs(zt - sc.thickness).max() < 2e-4


def test_self_contact_complementarity_at_convergence():
    """Full-metric Newton steps (GMRES to 32 iterations) to r_ncp <= 1e-9 on a
    10x10 base with a 5x5 piece: every self contact
    has gap >= -1e-8, lambda_n >= 0 and |lambda_n gap| tiny, and the friction
    multiplier lies in the cone."""
    sc = _stack(n_side=10)
    mesh = oracle.Mesh.from_scene(sc, 0)
    st = oracle.EnvState(sc.q0[0], sc.v0[0])
    for s in range(6):
        oracle.step(mesh, sc, 0, s, st, metric=2, lin_iters=32, mode=1, tol=1e-9, k_cap=300)
    assert st.rncp <= 1e-9
    sel = np.nonzero(st.cobs == oracle.SELF_SLOT)[0]
    assert len(sel) > 20
    tri = sc.elems
    for i in sel:
        p, f = st.cvert[i], st.ctri[i]
        a, b, c = st.q[tri[f]]
        nrm = np.cross(b - a, c - a)
        nrm /= np.linalg.norm(nrm)
        gap = abs(nrm @ (st.q[p] - a)) - sc.thickness
        g = st.gamma[i]
        assert gap >= -1e-8 and g[0] >= -1e-15 and abs(g[0] * gap) <= 1e-14
        assert np.linalg.norm(g[1:]) <= sc.mu[0] * max(g[0], 0) + 1e-13   # 1e-9 m x effective mass


def _ee_candidates_numpy(sc, q0, q1, reach):
    """Independent edge-edge detection: unique edges by numpy, closest points
    of the two lines by least squares, topological exclusion by sets, both
    configurations, the first EE_MAX pairs per owner vertex in edge order."""
    tris = sc.elems
    E = np.unique(np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]]), axis=1), axis=0)
    tri_sets = [set(int(x) for x in t) for t in tris]
    out = set()
    for i in range(sc.n_verts):
        found = []
        for e1 in np.nonzero(E[:, 0] == i)[0]:
            a, b = E[e1]
            for e2, (c, d) in enumerate(E):
                if e2 <= e1 or len({a, b, c, d}) < 4:
                    continue
                if any(({a, b} & ts) and ({int(c), int(d)} & ts) for ts in tri_sets):
                    continue
                hit = False
                for x in (q0, q1):
                    M = np.c_[x[b] - x[a], -(x[d] - x[c])]
                    if np.linalg.matrix_rank(M, tol=1e-9) < 2:
                        continue
                    st = np.linalg.lstsq(M, x[c] - x[a], rcond=None)[0]
                    if not (0 < st[0] < 1 and 0 < st[1] < 1):
                        continue
                    pa = x[a] + st[0] * (x[b] - x[a])
                    pc = x[c] + st[1] * (x[d] - x[c])
                    hit = hit or np.linalg.norm(pa - pc) < reach
                if hit:
                    found.append(int(e1) * len(E) + e2)
        out.update((i, f) for f in found[:oracle.EE_MAX])
    return out


def test_edge_edge_detection_matches_brute_force():
    """Edge-edge self-contact candidates of the stacked cloth equal an
    independent brute force over all edge pairs."""
    sc = _stack(n_side=10)
    mesh = oracle.Mesh.from_scene(sc, 0)
    st = oracle.EnvState(sc.q0[0], sc.v0[0])
    for s in range(3):
        oracle.step(mesh, sc, 0, s, st, metric=2)
    dp = oracle.params(sc, 0)[0]
    cv, co, ct = oracle.detect(mesh, sc, 0, 3, st.q, st.v, dp)
    got = {(int(v), int(t)) for v, o, t in zip(cv, co, ct) if o == oracle.EE_SLOT}
    qp = st.q + sc.h * st.v + sc.h ** 2 * np.asarray(sc.gravity)
    ref = _ee_candidates_numpy(sc, st.q, qp, sc.thickness + sc.margin)
    assert len(got) > 20 and got == ref


def test_crossing_strips_meet_edge_to_edge():
    """Two narrow strips crossing with no vertex over the other strip: only
    edge-edge rows can hold them apart.  With self-collision (full metric)
    the top strip comes to rest on the bottom one, its edges one thickness
    above the bottom's where they cross, and the rows are edge-edge only;
    without self-collision it falls through to the ground."""
    for on in (True, False):
        sc = scenes.strips_cross_drop(n_envs=1, steps=40)
        if not on:
            sc.meta = {}
        mesh = oracle.Mesh.from_scene(sc, 0)
        st = oracle.EnvState(sc.q0[0], sc.v0[0])
        for s in range(25):
            oracle.step(mesh, sc, 0, s, st, metric=2, mode=1, tol=1e-8, k_cap=200)
        top = st.q[8:]
        centre = top[np.abs(top[:, 1]) < 0.05]     # the top strip's vertices next to the crossing
        if on:
            assert (st.cobs == oracle.SELF_SLOT).sum() == 0 and (st.cobs == oracle.EE_SLOT).sum() >= 4
            ee = st.cobs == oracle.EE_SLOT
            assert (st.gamma[ee, 0] > 0).any()
            # where the edges cross, the top strip lies 2 tau above the ground (1 tau above the bottom strip)
            assert centre[:, 2].min() > 1.5 * sc.thickness, centre[:, 2]
        else:
            assert centre[:, 2].max() < 1.2 * sc.thickness


# ------------------------------------------------------------ box features against cloth
def test_corner_support_closed_form():
    """A triangle whose centroid rests one thickness above the top corner of
    a cube standing on a vertex is in equilibrium: the corner pushes each
    vertex up by a third of its weight through the barycentric weights
    (1/3 each), so one tolerance-mode step leaves it at rest and the corner
    row's normal impulse is the triangle's weight times h; every other row
    carries nothing."""
    sc = scenes.corner_support()
    mesh = oracle.Mesh.from_scene(sc, 0)
    for metric in (1, 2):
        st = oracle.EnvState(sc.q0[0], sc.v0[0])
        oracle.step(mesh, sc, 0, 0, st, metric=metric, mode=1, tol=1e-11, k_cap=300, lin_iters=32)
        assert np.abs(st.q - sc.q0[0]).max() < 1e-12
        top = (st.cobs == oracle.OVT_SLOT) & (st.ctri == 7)   # triangle 0, obstacle 0, corner 7 = (+,+,+)
        assert top.sum() == 1
        W = sc.mass.sum() * 9.81
        assert abs(st.gamma[top, 0][0] / sc.h - W * sc.h) <= 1e-9 * W * sc.h
        assert np.abs(st.gamma[~top]).max(initial=0.0) <= 1e-15 and np.abs(st.gamma[top, 1:]).max() <= 1e-15


def test_edge_support_closed_form():
    """A square (diagonal 0-3) resting one thickness above a knife edge under
    its middle line: the edge crosses the square's edges 0-2, 0-3 and 1-3 at
    their midpoints, so each row's force goes half to each end.  Vertex
    equilibrium then fixes the rows uniquely: 2 m g on the side edges 0-2
    and 1-3, none on the diagonal; the square stays at rest."""
    sc = scenes.edge_support()
    mesh = oracle.Mesh.from_scene(sc, 0)
    st = oracle.EnvState(sc.q0[0], sc.v0[0])
    oracle.step(mesh, sc, 0, 0, st, metric=1, mode=1, tol=1e-11, k_cap=300)
    assert np.abs(st.q - sc.q0[0]).max() < 1e-10
    edges = mesh.edges
    ned = len(edges)
    assert ned == 5
    got = {}
    for v, o, f, g in zip(st.cvert, st.cobs, st.ctri, st.gamma):
        assert o == oracle.OEE_SLOT
        e, rest = divmod(int(f), 12 * oracle.MAX_OBS)
        assert rest == 3          # obstacle 0, box edge 3 = along x at (+y, +z): the top after the turn
        got[tuple(int(x) for x in edges[e])] = g[0] / sc.h
    mg = 1e-3 * 9.81
    assert set(got) == {(0, 2), (0, 3), (1, 3)}
    # r_ncp <= 1e-11 m bounds the multipliers' error near m x 1e-11 m (impulse ~1e-12 N s)
    assert abs(got[(0, 2)] - 2 * mg * sc.h) <= 1e-7 * mg * sc.h
    assert abs(got[(1, 3)] - 2 * mg * sc.h) <= 1e-7 * mg * sc.h
    assert abs(got[(0, 3)]) <= 1e-7 * mg * sc.h


def _box_world(sc, e, o, pts):
    """Body-frame points of obstacle o of environment e at t+h of step 0, by
    scipy's rotation (quaternion given scalar-last)."""
    from scipy.spatial.transform import Rotation
    p = sc.poses[e, 1, o]
    return Rotation.from_quat([p[4], p[5], p[6], p[3]]).apply(pts) + p[:3]


def _corners(d):
    return np.array([[d[i] if (k >> i) & 1 else -d[i] for i in range(3)] for k in range(8)])


def _box_edges(d):
    """The 12 edges: j // 4 = the axis they run along, bit 0 / bit 1 of j % 4
    = the + side of the other two axes in increasing order."""
    out = []
    for j in range(12):
        a, m = divmod(j, 4)
        b, c = [x for x in range(3) if x != a]
        p0, p1 = np.zeros(3), np.zeros(3)
        p0[a], p1[a] = -d[a], d[a]
        p0[b] = p1[b] = d[b] if m & 1 else -d[b]
        p0[c] = p1[c] = d[c] if m & 2 else -d[c]
        out.append((p0, p1))
    return out


def _feature_candidates_numpy(sc, e, q0, q1, reach):
    """Independent box-feature detection: corners and edges of each box by
    scipy rotations, each triangle's plane by SVD and barycentric weights by
    pseudo-inverse, closest points of two lines by least squares, both
    configurations, the first OFEAT_MAX rows of each kind per owner vertex
    in feature order."""
    tris = sc.elems
    E = np.unique(np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]]), axis=1), axis=0)
    boxes = [o for o in range(sc.n_obs) if sc.obs_type[e, o] == scenes.BOX]
    corners = {o: _box_world(sc, e, o, _corners(sc.obs_dims[e, o])) for o in boxes}
    bedges = {o: [_box_world(sc, e, o, np.array(pq)) for pq in _box_edges(sc.obs_dims[e, o])] for o in boxes}
    ovt, oee = set(), set()
    for i in range(sc.n_verts):
        found = []
        for f in np.nonzero(tris[:, 0] == i)[0]:
            for o in boxes:
                for k, C in enumerate(corners[o]):
                    hit = False
                    for x in (q0, q1):
                        P = x[tris[f]]
                        nrm = np.linalg.svd(P - P.mean(0))[2][2]
                        d = nrm @ (C - P[0])
                        w12 = np.linalg.pinv(np.c_[P[1] - P[0], P[2] - P[0]]) @ (C - d * nrm - P[0])
                        w = np.r_[1 - w12.sum(), w12]
                        hit = hit or (abs(d) < reach and w.min() >= -0.1)
                    if hit:
                        found.append((int(f) * oracle.MAX_OBS + o) * 8 + k)
        ovt.update((i, f) for f in found[:oracle.OFEAT_MAX])
        found = []
        for en in np.nonzero(E[:, 0] == i)[0]:
            a, b = E[en]
            for o in boxes:
                for j, (C, D) in enumerate(bedges[o]):
                    hit = False
                    for x in (q0, q1):
                        M = np.c_[x[b] - x[a], -(D - C)]
                        if np.linalg.matrix_rank(M, tol=1e-9) < 2:
                            continue
                        s, t = np.linalg.lstsq(M, C - x[a], rcond=None)[0]
                        if 0 < s < 1 and 0 < t < 1:
                            hit = hit or np.linalg.norm(x[a] + s * (x[b] - x[a]) - C - t * (D - C)) < reach
                    if hit:
                        found.append((int(en) * oracle.MAX_OBS + o) * 12 + j)
        oee.update((i, f) for f in found[:oracle.OFEAT_MAX])
    return ovt, oee


def test_box_feature_detection_matches_brute_force():
    """Box-corner and box-edge rows of the bar-and-post scene (a turned bar,
    after the cloth has landed) equal an independent brute force over every
    triangle, cloth edge, box corner and box edge."""
    sc = scenes.cloth_bar_drop(n_envs=2, steps=10)
    e = 1
    mesh = oracle.Mesh.from_scene(sc, e)
    st = oracle.EnvState(sc.q0[e], sc.v0[e])
    for s in range(4):
        oracle.step(mesh, sc, e, s, st, metric=2)
    sc.poses[e, 1] = sc.poses[e, 5]    # the obstacles are static: step 4's poses are step 0's
    dp = oracle.params(sc, e)[0]
    cv, co, ct = oracle.detect(mesh, sc, e, 4, st.q, st.v, dp)
    got_vt = {(int(v), int(t)) for v, o, t in zip(cv, co, ct) if o == oracle.OVT_SLOT}
    got_ee = {(int(v), int(t)) for v, o, t in zip(cv, co, ct) if o == oracle.OEE_SLOT}
    qp = st.q + sc.h * st.v + sc.h ** 2 * np.asarray(sc.gravity)
    ref_vt, ref_ee = _feature_candidates_numpy(sc, e, st.q, qp, sc.thickness + sc.margin)
    assert len(got_vt) >= 4 and len(got_ee) > 30
    assert got_vt == ref_vt and got_ee == ref_ee


def test_bar_and_post_hold_the_cloth_between_its_vertices():
    """The cloth dropped onto a bar and a post narrower than its cells: with
    box-feature rows it comes to rest one thickness above their tops (the
    rows, not the vertices, hold it: no vertex row is active), and every
    converged box-feature row satisfies gap >= -1e-8 m, lambda_n >= 0,
    complementarity and the friction cone (gaps recomputed here from the
    geometry); without them it falls past both to the ground."""
    for on in (True, False):
        sc = scenes.cloth_bar_drop(n_envs=1, steps=20)
        if not on:
            sc.meta = {}
        mesh = oracle.Mesh.from_scene(sc, 0)
        st = oracle.EnvState(sc.q0[0], sc.v0[0])
        for s in range(12):
            oracle.step(mesh, sc, 0, s, st, metric=2, mode=1, tol=1e-9, k_cap=400, lin_iters=32)
        z_top = 0.05
        if not on:
            assert st.q[:, 2].max() < 2 * sc.thickness
            continue
        assert st.rncp <= 1e-9
        assert st.q[:, 2].min() > z_top + 0.9 * sc.thickness
        feat = (st.cobs == oracle.OVT_SLOT) | (st.cobs == oracle.OEE_SLOT)
        assert (st.gamma[feat, 0] > 1e-9).sum() >= 4
        assert np.abs(st.gamma[~feat, 0]).max() == 0.0
        corners = {o: _box_world(sc, 0, o, _corners(sc.obs_dims[0, o])) for o in (1, 2)}
        bedges = {o: [_box_world(sc, 0, o, np.array(pq)) for pq in _box_edges(sc.obs_dims[0, o])] for o in (1, 2)}
        E = mesh.edges
        for i in np.nonzero(feat)[0]:
            f = int(st.ctri[i])
            if st.cobs[i] == oracle.OVT_SLOT:
                tri, o, k = f // (8 * oracle.MAX_OBS), f // 8 % oracle.MAX_OBS, f % 8
                P = st.q[sc.elems[tri]]
                nrm = np.linalg.svd(P - P.mean(0))[2][2]
                gap = abs(nrm @ (corners[o][k] - P[0])) - sc.thickness
            else:
                en, o, j = f // (12 * oracle.MAX_OBS), f // 12 % oracle.MAX_OBS, f % 12
                a, b = E[en]
                C, D = bedges[o][j]
                nn = np.cross(st.q[b] - st.q[a], D - C)
                gap = abs(nn @ (st.q[a] - C)) / np.linalg.norm(nn) - sc.thickness
            g = st.gamma[i]
            assert gap >= -1e-8 and g[0] >= -1e-15 and abs(g[0] * gap) <= 1e-14
            assert np.linalg.norm(g[1:]) <= sc.mu[0] * max(g[0], 0) + 1e-13


@pytest.mark.parametrize("u", [0.01, 0.2])
def test_box_feature_friction_closed_form(u):
    """Coulomb friction through box-edge rows: the knife edge under the
    square translates along its own axis x at speed u.
    The body's weight rests on those rows, so friction can change its
    velocity by at most mu g h per step: for u <= mu g h it sticks and rides
    along (x_n = u h n); for u > mu g h it slides, x_n = mu g h^2 n (n + 1) / 2
    until it reaches the support's speed, then rides along.  Heights stay at
    rest.  This pins the kinematic motion in the rows' slip and the cone."""
    mu, h, g = 0.5, 0.01, 9.81
    sc = scenes.edge_support(steps=6, mu=mu)
    sc.poses[0, :, 0, 0] = u * h * np.arange(sc.poses.shape[1])
    mesh = oracle.Mesh.from_scene(sc, 0)
    st = oracle.EnvState(sc.q0[0], sc.v0[0])
    x, v = 0.0, 0.0
    for n in range(1, 6):
        oracle.step(mesh, sc, 0, n - 1, st, metric=1, mode=1, tol=1e-12, k_cap=400)
        v = min(v + mu * g * h, u)          # the velocity friction can reach, capped at the support's
        x += v * h
        assert np.abs(st.q[:, 0] - sc.q0[0][:, 0] - x).max() < 1e-9, (n, st.q[:, 0] - sc.q0[0][:, 0], x)
        assert np.abs(st.q[:, 2] - sc.q0[0][:, 2]).max() < 1e-9


# ------------------------------------------------------------ sphere, compliance, tet stiffness
_SPHERE_C = np.array([0.1, -0.2, 0.3])
_SPHERE_R = 0.15


def _sphere_particle(theta, mu, steps, phi=0.7, tau=1e-3, mass=0.01):
    """A particle released at rest one thickness outside a sphere (off the
    origin), at polar angle theta from its top and azimuth phi."""
    d = np.array([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)])
    x0 = _SPHERE_C + (_SPHERE_R + tau) * d
    poses = np.array([[[*_SPHERE_C, 1, 0, 0, 0]] for _ in range(steps + 1)])
    sc = _particle_scene([(scenes.SPHERE, (_SPHERE_R, 0, 0))], poses, mu, steps, x0, mass=mass)
    return sc, d


def test_particle_resting_on_top_of_sphere():
    """Sphere SDF (Sec. III-A contact; obstacle geometry): a particle at the
    top of a sphere whose centre is not the origin carries its weight through
    one normal contact, gamma_n = m g h^2, with zero gap, and does not move;
    the contact frame's normal is the radial direction (+z there)."""
    sc, _ = _sphere_particle(0.0, 0.3, 6)
    st = oracle.rollout(sc, 0, 6, mode=1, tol=1e-13, k_cap=100)
    m, g, h = sc.mass[0], 9.81, sc.h
    assert len(st.cvert) == 1
    assert abs(st.gamma[0, 0] - m * g * h * h) < 1e-12
    assert np.abs(st.q[0] - sc.q0[0, 0]).max() < 1e-12
    sd, nrm = oracle.sdf(scenes.SPHERE, (_SPHERE_R, 0, 0), sc.poses[0, 0, 0], st.q[0])
    assert abs(sd - sc.thickness) < 1e-12 and np.abs(nrm - [0, 0, 1]).max() < 1e-12


@pytest.mark.parametrize("theta", [0.25, 0.5])
def test_particle_on_sphere_sticks_iff_tan_theta_le_mu(theta):
    """On a sphere the supporting tangent plane at polar angle theta is an
    incline of angle theta: Coulomb friction holds the particle iff
    tan(theta) <= mu (mu swept in steps of 0.001 around tan theta).  A sliding
    particle keeps its gap zero (it stays on the sphere, one thickness out)
    and moves downhill along the sphere's meridian."""
    t = np.tan(theta)
    for dmu in (-0.002, -0.001, 0.001, 0.002):
        mu = t + dmu
        sc, d = _sphere_particle(theta, mu, 8)
        st = oracle.rollout(sc, 0, 8, mode=1, tol=1e-13, k_cap=200)
        disp = st.q[0] - sc.q0[0, 0]
        if mu >= t:
            assert np.linalg.norm(disp) < 1e-12, (mu, disp)
        else:
            assert np.linalg.norm(disp) > 1e-7, (mu, disp)
            assert abs(np.linalg.norm(st.q[0] - _SPHERE_C) - (_SPHERE_R + sc.thickness)) < 1e-10
            # downhill: the polar angle grows, the azimuth is kept
            r = st.q[0] - _SPHERE_C
            assert np.arccos(r[2] / np.linalg.norm(r)) > theta
            assert abs(np.arctan2(r[1], r[0]) - 0.7) < 1e-9


@pytest.mark.parametrize("comp", [5e-4, 2e-3])
def test_compliant_plane_gap_closed_form(comp):
    """Normal compliance c (m/N) of an obstacle: the normal law is
    FB(a + alpha y_n, y_n) with y_n = gamma_n / m and alpha = c m / h^2.  A
    particle resting on the plane carries y_n = g h^2, and FB = 0 with
    y_n > 0 needs a + alpha y_n = 0: it sinks to the gap -c m g, while the
    multiplier stays m g h^2.  m = 0.03 kg and h = 1/50 s, so a misplaced mass
    or h^2 factor changes the gap."""
    m, h = 0.03, 0.02
    steps = 30
    poses = np.array([[[0, 0, 0, 1, 0, 0, 0]] for _ in range(steps + 1)])
    sc = _particle_scene([(scenes.PLANE, (0, 0, 0))], poses, 0.4, steps, (0, 0, 1e-3), h=h, mass=m)
    sc.obs_comp[:] = comp
    st = oracle.rollout(sc, 0, steps, mode=1, tol=1e-13, k_cap=200)
    g = 9.81
    gap = st.q[0, 2] - sc.thickness
    assert abs(gap - (-comp * m * g)) < 1e-9 * max(1.0, comp * m * g / 1e-6)
    assert abs(st.gamma[0, 0] - m * g * h * h) < 1e-10
    assert abs(st.v[0, 2]) < 1e-6


def test_tet_uniform_stretch_energy_with_stiffness_scale():
    """Corotational tets (Eq. internal): w_i = w_stretch * k_e * rest volume.
    Stretching the whole block by (1 + eps) along x gives F = diag(1 + eps,
    1, 1) in every tet, closest rotation I, so the energy is
    w_stretch * k_e * V * eps^2 / 2 with V the block's volume."""
    sc = scenes.tet_squeeze(n_envs=2, steps=1)
    sc.stiff[1] = 37.0
    vol = 0.08 * 0.08 * 0.04
    eps = 0.021
    for env in (0, 1):
        m = oracle.Mesh.from_scene(sc, env)
        q = sc.rest.copy()
        q[:, 0] *= 1 + eps
        p = m.project(q)
        E = m.energy(q, q, p)
        ref = 0.5 * sc.w_stretch * sc.stiff[env] * vol * eps ** 2
        assert abs(E - ref) < 1e-9 * ref, (env, E, ref)


def test_tet_energy_hessian_equals_system_matrix():
    """The tet block's PD energy Hessian (central differences, fixed
    projections) equals A / h^2 with A = M + h^2 sum w_i G_i^T G_i, at a
    stiffness scale k_e != 1: this pins the scale of A's stiffness block."""
    sc = scenes.tet_squeeze(n_envs=1, steps=1)
    sc.stiff[0] = 13.0
    m = oracle.Mesh.from_scene(sc, 0)
    A = m.matrix()
    rng = np.random.default_rng(8)
    q0 = sc.rest + 1e-3 * rng.normal(size=sc.rest.shape)
    p0 = m.project(q0)
    for _ in range(3):
        d = rng.normal(size=q0.shape)
        t = 1e-4
        e_p, e_0, e_m = (m.energy(q0 + t * d, q0, p0), m.energy(q0, q0, p0), m.energy(q0 - t * d, q0, p0))
        fd = (e_p - 2 * e_0 + e_m) / t ** 2
        exact = np.sum(d * (A @ d)) / sc.h ** 2
        assert abs(fd - exact) < 1e-6 * abs(exact)
