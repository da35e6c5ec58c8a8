"""Seeded synthetic scenes for the batched deformable + contact time step.

This module is INPUT DATA ONLY: rest geometry, element connectivity, lumped
masses, material weights, per-environment parameters and kinematic obstacle
trajectories.  It contains none of the solver's arithmetic (no deformation
gradients, no system matrix, no projections, no contact law), so both the FP64
oracle and the CUDA path can consume the same arrays without sharing method
code.

Every random draw comes from a counter-based Philox stream keyed by
``(seed << 32) | env``, so scene ``e`` of a batch is identical whether the
batch holds 1 or 4096 environments and on x86 and Arm hosts alike.

Conventions (shared by oracle and library):
  * z is up, gravity (0, 0, -9.81) m/s^2.
  * obstacle pose = (px, py, pz, qw, qx, qy, qz): body -> world.
  * obstacle types: PLANE (normal = body +z through the pose origin),
    SPHERE (dims[0] = radius), BOX (dims = half extents).
  * positions are [n][3] (vertex-major, xyz), float64 here.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

NONE, PLANE, SPHERE, BOX = 0, 1, 2, 3
TRI, TET = 0, 1
MODE_FIXED, MODE_TOL = 0, 1
IDENTITY_POSE = (0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0)


def env_rng(seed: int, env: int) -> np.random.Generator:
    """Counter-based stream for environment ``env`` of scene seed ``seed``."""
    return np.random.Generator(np.random.Philox(key=(int(seed) << 32) | int(env)))


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------
def cloth_grid(nx: int, ny: int, side_x: float, side_y: float | None = None):
    """Square/rectangular cloth in the z=0 plane, centred at the origin.

    Cells are split along alternating diagonals, so a 16x16 grid has 450
    triangles and a 32x32 grid 1922.  Returns (rest [n][3], tris [T][3]).
    """
    side_y = side_x if side_y is None else side_y
    xs = np.linspace(-side_x / 2, side_x / 2, nx)
    ys = np.linspace(-side_y / 2, side_y / 2, ny)
    rest = np.zeros((nx * ny, 3))
    for j in range(ny):
        for i in range(nx):
            rest[j * nx + i] = (xs[i], ys[j], 0.0)
    tris = []
    for j in range(ny - 1):
        for i in range(nx - 1):
            a, b = j * nx + i, j * nx + i + 1
            c, d = (j + 1) * nx + i, (j + 1) * nx + i + 1
            if (i + j) % 2 == 0:
                tris += [(a, b, d), (a, d, c)]
            else:
                tris += [(a, b, c), (b, d, c)]
    return rest, np.asarray(tris, dtype=np.int32)


_EVEN = ((1, 2, 4, 7), (0, 1, 2, 4), (3, 2, 1, 7), (5, 4, 7, 1), (6, 7, 4, 2))
_ODD = ((0, 3, 5, 6), (1, 0, 3, 5), (2, 3, 0, 6), (4, 5, 6, 0), (7, 6, 5, 3))


def tet_block(cx: int, cy: int, cz: int, sx: float, sy: float, sz: float):
    """Box of cx*cy*cz cubes, 5 tets per cube with alternating parity.

    The block spans [-sx/2, sx/2] x [-sy/2, sy/2] x [0, sz].  Every tet is
    ordered with positive orientation.  Returns (rest [n][3], tets [E][4]).
    """
    nx, ny, nz = cx + 1, cy + 1, cz + 1
    rest = np.zeros((nx * ny * nz, 3))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                rest[(k * ny + j) * nx + i] = (-sx / 2 + sx * i / cx, -sy / 2 + sy * j / cy, sz * k / cz)
    tets = []
    for k in range(cz):
        for j in range(cy):
            for i in range(cx):
                corner = [((k + (c >> 2)) * ny + (j + ((c >> 1) & 1))) * nx + i + (c & 1) for c in range(8)]
                for t in (_EVEN if (i + j + k) % 2 == 0 else _ODD):
                    v = [corner[c] for c in t]
                    e1, e2, e3 = (rest[v[1]] - rest[v[0]], rest[v[2]] - rest[v[0]], rest[v[3]] - rest[v[0]])
                    if np.dot(np.cross(e1, e2), e3) < 0:
                        v[2], v[3] = v[3], v[2]
                    tets.append(v)
    return rest, np.asarray(tets, dtype=np.int32)


def lumped_tet_mass(rest, tets, density):
    """Per-vertex mass: a quarter of rho*volume of every incident tet."""
    m = np.zeros(len(rest))
    for t in tets:
        e1, e2, e3 = rest[t[1]] - rest[t[0]], rest[t[2]] - rest[t[0]], rest[t[3]] - rest[t[0]]
        vol = abs(np.dot(np.cross(e1, e2), e3)) / 6.0
        m[t] += density * vol / 4.0
    return m


# --------------------------------------------------------------------------
# scene container
# --------------------------------------------------------------------------
@dataclass
class Scene:
    """One mesh template shared by ``n_envs`` environments.

    Arrays (float64 unless noted):
      rest [n][3], elems int32 [E][3|4], mass [n]
      q0, v0 [N][n][3]
      mu [N], stiff [N] (multiplies w_stretch per environment)
      obs_type int32 [N][K], obs_dims [N][K][3], obs_comp [N][K] (m/N)
      poses [N][S+1][K][7]: obstacle pose at the start of step s (s = 0..S)
    """
    name: str
    elem_type: int
    rest: np.ndarray
    elems: np.ndarray
    mass: np.ndarray
    w_stretch: float
    w_bend: float
    q0: np.ndarray
    v0: np.ndarray
    mu: np.ndarray
    stiff: np.ndarray
    obs_type: np.ndarray
    obs_dims: np.ndarray
    obs_comp: np.ndarray
    poses: np.ndarray
    h: float = 0.01
    gravity: tuple = (0.0, 0.0, -9.81)
    k_max: int = 10
    k_min: int = 1
    k_cap: int = 200
    mode: int = MODE_FIXED
    tol_ncp: float = 1e-5
    maxforce: float = 1e10
    thickness: float = 1e-3
    margin: float = 1e-2
    steps: int = 1
    meta: dict = field(default_factory=dict)

    @property
    def n_envs(self) -> int:
        return self.q0.shape[0]

    @property
    def n_verts(self) -> int:
        return self.rest.shape[0]

    @property
    def n_obs(self) -> int:
        return self.obs_type.shape[1]

    def subset(self, envs) -> "Scene":
        """The same scene restricted to the listed environments."""
        envs = np.asarray(envs)
        kw = {k: getattr(self, k) for k in self.__dataclass_fields__}
        for k in ("q0", "v0", "mu", "stiff", "obs_type", "obs_dims", "obs_comp", "poses"):
            kw[k] = getattr(self, k)[envs].copy()
        return Scene(**kw)


def _pose(p, q=(1.0, 0.0, 0.0, 0.0)):
    return np.array([p[0], p[1], p[2], q[0], q[1], q[2], q[3]], dtype=np.float64)


def _static_poses(n_envs, steps, poses_k):
    """[N][S+1][K][7] array holding a fixed pose per obstacle."""
    out = np.zeros((n_envs, steps + 1, len(poses_k), 7))
    for k, p in enumerate(poses_k):
        out[:, :, k, :] = p
    return out


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
def cloth_drop(seed: int = 0, n_side: int = 16, side: float = 0.5, steps: int = 200,
               n_envs: int = 1, mu: float = 0.3, k_max: int = 10) -> Scene:
    """Square cloth dropped 0.3 m onto a static sphere (r = 0.15 m) and the ground.

    16x16 vertices, 0.5 m side, 0.1 kg spread evenly over the vertices, stretch
    weight 1e4 and bending weight 10, z-perturbation N(0, 1e-3 m) per vertex,
    h = 1/100 s, Coulomb mu = 0.3, 10 local-global iterations per step.
    """
    rest, tris = cloth_grid(n_side, n_side, side)
    n = len(rest)
    mass = np.full(n, 0.1 / n)
    q0 = np.zeros((n_envs, n, 3))
    for e in range(n_envs):
        g = env_rng(seed, e)
        q0[e] = rest
        q0[e, :, 2] = 0.6 + g.normal(0.0, 1e-3, n)
    obs_type = np.tile(np.array([PLANE, SPHERE], np.int32), (n_envs, 1))
    obs_dims = np.zeros((n_envs, 2, 3))
    obs_dims[:, 1, 0] = 0.15
    poses = _static_poses(n_envs, steps, [_pose((0, 0, 0)), _pose((0, 0, 0.15))])
    return Scene("cloth_drop", TRI, rest, tris, mass, 1e4, 10.0, q0, np.zeros_like(q0),
                 np.full(n_envs, mu), np.ones(n_envs), obs_type, obs_dims,
                 np.zeros((n_envs, 2)), poses, h=0.01, k_max=k_max, steps=steps)


def _waypoint_path(g, start, n_seg, speed, bound, steps, h, t_hold):
    """Piecewise-linear xy path: hold for t_hold, then n_seg straight segments
    at constant speed towards random waypoints inside [-bound, bound]^2.
    Returns positions [steps+1][2]."""
    pts = [np.asarray(start, float)]
    for _ in range(n_seg):
        pts.append(g.uniform(-bound, bound, 2))
    out = np.zeros((steps + 1, 2))
    seg, pos, t = 0, pts[0].copy(), 0.0
    for s in range(steps + 1):
        out[s] = pos
        t += h
        if t <= t_hold:
            continue
        move = speed * h
        while move > 0 and seg < n_seg:
            tgt = pts[seg + 1]
            d = tgt - pos
            L = np.linalg.norm(d)
            if L <= move:
                pos, move, seg = tgt.copy(), move - L, seg + 1
            else:
                pos, move = pos + d / L * move, 0.0
    return out


def cloth_gripper(seed: int = 1, n_envs: int = 1024, n_side: int = 32, side: float = 0.5,
                  steps: int = 500, k_max: int = 10, squeeze: float = 5e-4,
                  finger_comp: float = 5e-4) -> Scene:
    """Cloth lying on the ground, pinched against it by a kinematic two-finger box
    gripper and dragged along a seeded piecewise-linear path.

    Fingers are 2x2x4 cm boxes 3 cm apart along x, lowered in the first 0.1 s
    until their bottom faces sit ``squeeze`` below the cloth's upper surface
    (thickness 1 mm), then moved in xy through 4-8 random waypoints at a speed
    drawn from U[0.05, 0.3] m/s.  mu ~ U[0.2, 0.8] per environment (ground and
    fingers); the finger contacts carry a normal compliance (m/N) so that the
    pinch force is determined.  h = 1/100 s.
    """
    rest, tris = cloth_grid(n_side, n_side, side)
    n = len(rest)
    mass = np.full(n, 0.1 * side * side / 0.25 / n)
    tau = 1e-3
    q0 = np.repeat(rest[None], n_envs, 0).copy()
    q0[:, :, 2] = tau
    K = 3
    obs_type = np.tile(np.array([PLANE, BOX, BOX], np.int32), (n_envs, 1))
    obs_dims = np.zeros((n_envs, K, 3))
    obs_dims[:, 1:, :] = (0.01, 0.01, 0.02)
    obs_comp = np.zeros((n_envs, K))
    obs_comp[:, 1:] = finger_comp
    mu = np.zeros(n_envs)
    poses = np.zeros((n_envs, steps + 1, K, 7))
    h = 0.01
    z_press = 2 * tau - squeeze + 0.02      # box centre when pressing
    z_start = z_press + 0.01
    for e in range(n_envs):
        g = env_rng(seed, e)
        mu[e] = g.uniform(0.2, 0.8)
        speed = g.uniform(0.05, 0.3)
        n_seg = int(g.integers(4, 9))
        start = g.uniform(-0.12, 0.12, 2)
        path = _waypoint_path(g, start, n_seg, speed, 0.12, steps, h, t_hold=0.15)
        poses[e, :, 0] = _pose((0, 0, 0))
        for s in range(steps + 1):
            t = s * h
            z = z_press + (z_start - z_press) * max(0.0, 1.0 - t / 0.1)
            poses[e, s, 1] = _pose((path[s, 0] - 0.015, path[s, 1], z))
            poses[e, s, 2] = _pose((path[s, 0] + 0.015, path[s, 1], z))
    return Scene("cloth_gripper", TRI, rest, tris, mass, 1e4, 10.0, q0, np.zeros_like(q0),
                 mu, np.ones(n_envs), obs_type, obs_dims, obs_comp, poses, h=h,
                 k_max=k_max, thickness=tau, steps=steps)


def cloth_grasp(seed: int = 2, n_envs: int = 64, n_side: int = 16, side: float = 0.25, steps: int = 120,
                k_max: int = 10, grasp_step: int = 2, release_step: int = 90, lift=(0.08, 0.15),
                inward=(0.03, 0.08), rise_time: float = 0.5) -> Scene:
    """Cloth lying on the ground, grasped at one corner by a point gripper
    (appendix, Bilateral Constraint for Cloth Control), lifted, carried and
    released.

    The gripper is a kinematic pose carrier (obstacle type NONE: no contact of
    its own) starting on a random corner vertex; at step ``grasp_step`` every
    vertex within 0.3 grid spacings of its anchor is attached (the corner
    vertex), the corner is lifted by U[lift] m over ``rise_time`` s while
    moving U[inward] m towards the centre, held, and released at
    ``release_step``.
    mu ~ U[0.2, 0.8]; h = 1/100 s.  The grasp schedule is in meta["grasp"].
    """
    rest, tris = cloth_grid(n_side, n_side, side)
    n = len(rest)
    mass = np.full(n, 0.1 * side * side / 0.25 / n)
    tau = 1e-3
    q0 = np.repeat(rest[None], n_envs, 0).copy()
    q0[:, :, 2] = tau
    K = 2
    obs_type = np.tile(np.array([PLANE, NONE], np.int32), (n_envs, 1))
    obs_dims = np.zeros((n_envs, K, 3))
    mu = np.zeros(n_envs)
    poses = np.zeros((n_envs, steps + 1, K, 7))
    h = 0.01
    corners = [0, n_side - 1, n - n_side, n - 1]
    for e in range(n_envs):
        g = env_rng(seed, e)
        mu[e] = g.uniform(0.2, 0.8)
        c = corners[int(g.integers(0, 4))]
        up = g.uniform(*lift)
        shift = g.uniform(*inward)
        p0 = np.array([rest[c, 0], rest[c, 1], tau])
        d = -np.sign(p0[:2])
        poses[e, :, 0] = _pose((0, 0, 0))
        for s_ in range(steps + 1):
            u = min(1.0, max(0.0, (s_ - grasp_step) * h / rise_time))
            p = p0 + np.array([d[0] * shift * u / np.sqrt(2), d[1] * shift * u / np.sqrt(2), up * u])
            poses[e, s_, 1] = _pose(p)
    spacing = side / (n_side - 1)
    meta = {"grasp": {"obstacle": 1, "anchor": (0.0, 0.0, 0.0), "radius": 0.3 * spacing,
                      "schedule": {grasp_step: 1, release_step: 0}}}
    return Scene("cloth_grasp", TRI, rest, tris, mass, 1e4, 10.0, q0, np.zeros_like(q0),
                 mu, np.ones(n_envs), obs_type, obs_dims, np.zeros((n_envs, K)), poses, h=h,
                 k_max=k_max, thickness=tau, steps=steps, meta=meta)


def tet_squeeze(seed: int = 1, n_envs: int = 4096, cubes=(8, 8, 4), size=(0.08, 0.08, 0.04),
                steps: int = 100, k_max: int = 10, mu: float = 0.5) -> Scene:
    """Soft tet block on the ground squeezed by a kinematic parallel gripper.

    8x8x4 cubes x 5 tets = 1280 tets, 405 vertices, 8x8x4 cm, density 1000
    kg/m^3, per-environment stiffness log-uniform in [1e3, 1e5] (weight per
    unit rest volume), closing depth U[0.5, 2] cm reached after 0.1 s and then
    held, h = 1/200 s.  Plates are 1 x 6 x 6 cm boxes closing along x.
    """
    rest, tets = tet_block(*cubes, *size)
    n = len(rest)
    mass = lumped_tet_mass(rest, tets, 1000.0)
    q0 = np.repeat(rest[None], n_envs, 0).copy()
    K = 3
    obs_type = np.tile(np.array([PLANE, BOX, BOX], np.int32), (n_envs, 1))
    obs_dims = np.zeros((n_envs, K, 3))
    obs_dims[:, 1:, :] = (0.005, 0.03, 0.03)
    stiff = np.zeros(n_envs)
    poses = np.zeros((n_envs, steps + 1, K, 7))
    h = 1.0 / 200
    half = size[0] / 2 + 0.005
    for e in range(n_envs):
        g = env_rng(seed, e)
        stiff[e] = 10.0 ** g.uniform(3.0, 5.0)
        depth = g.uniform(0.005, 0.02)
        poses[e, :, 0] = _pose((0, 0, 0))
        for s in range(steps + 1):
            c = 0.5 * depth * min(1.0, s * h / 0.1)
            poses[e, s, 1] = _pose((-half + c, 0, size[2] / 2))
            poses[e, s, 2] = _pose((half - c, 0, size[2] / 2))
    return Scene("tet_squeeze", TET, rest, tets, mass, 1.0, 0.0, q0, np.zeros_like(q0),
                 np.full(n_envs, mu), stiff, obs_type, obs_dims, np.zeros((n_envs, K)), poses,
                 h=h, k_max=k_max, thickness=0.0, steps=steps)


def incline_particle(theta: float, mu: float, steps: int = 20, h: float = 0.01, mass: float = 0.01):
    """A single free particle resting on a plane tilted by ``theta`` about y.

    Used for the Coulomb stick/slide pin: the particle sticks iff
    tan(theta) <= mu.  The mesh is one vertex with no elements.
    """
    rest = np.zeros((1, 3))
    nrm = np.array([-np.sin(theta), 0.0, np.cos(theta)])
    tau = 1e-3
    q0 = (rest + tau * nrm)[None].copy()
    half = theta / 2
    poses = _static_poses(1, steps, [_pose((0, 0, 0), (np.cos(half), 0.0, -np.sin(half), 0.0))])
    return Scene("incline", TRI, rest, np.zeros((0, 3), np.int32), np.array([mass]), 0.0, 0.0,
                 q0, np.zeros_like(q0), np.array([mu]), np.ones(1), np.array([[PLANE]], np.int32),
                 np.zeros((1, 1, 3)), np.zeros((1, 1)), poses, h=h, thickness=tau, steps=steps)


def _tet_dims_for(n_target):
    """Cube counts (cx, cy, cz) of a block whose vertex count (cx+1)(cy+1)(cz+1)
    is closest to n_target, with cx = cy = 2 cz rounded (flat blocks)."""
    best = None
    for cz in range(1, 12):
        for cx in range(cz, 4 * cz + 1):
            n = (cx + 1) * (cx + 1) * (cz + 1)
            d = abs(n - n_target)
            if best is None or d < best[0]:
                best = (d, (cx, cx, cz))
    return best[1]


def mixed_batch(seed: int = 3, n_envs: int = 2048, steps: int = 1000, side_choices=None, tet_targets=None,
                max_obs: int = 4):
    """Uneven batch: half cloths with side U{16..64} vertices, half tet blocks
    with 200-3000 vertices, each dropped onto 1-4 random boxes/spheres and the
    ground; mu ~ U[0.1, 0.9]; h = 1/100 s.

    Environments of equal mesh share one template (one Scene per template,
    returned as a list).  ``side_choices`` / ``tet_targets`` restrict the
    drawn sizes (for small test batches)."""
    side_choices = list(range(16, 65)) if side_choices is None else list(side_choices)
    tet_targets = (200, 3000) if tet_targets is None else tet_targets
    groups = {}
    for e in range(n_envs):
        g = env_rng(seed, e)
        if e % 2 == 0:
            key = ("cloth", int(side_choices[int(g.integers(0, len(side_choices)))]))
        else:
            if isinstance(tet_targets, tuple):
                key = ("tet", _tet_dims_for(int(g.integers(tet_targets[0], tet_targets[1] + 1))))
            else:
                key = ("tet", _tet_dims_for(int(tet_targets[int(g.integers(0, len(tet_targets)))])))
        groups.setdefault(key, []).append(e)
    out = []
    for key, envs in sorted(groups.items(), key=lambda kv: kv[1][0]):
        if key[0] == "cloth":
            ns = key[1]
            side = 0.5 * ns / 32
            rest, elems = cloth_grid(ns, ns, side)
            mass = np.full(len(rest), 0.1 * side * side / 0.25 / len(rest))
            etype, ws, wb, tau, z0 = TRI, 1e4, 10.0, 1e-3, 0.25
        else:
            cx, cy, cz = key[1]
            sx, sy, sz = 0.01 * cx, 0.01 * cy, 0.01 * cz
            rest, elems = tet_block(cx, cy, cz, sx, sy, sz)
            mass = lumped_tet_mass(rest, elems, 1000.0)
            etype, ws, wb, tau, z0 = TET, 3e4, 0.0, 0.0, 0.12
        n = len(rest)
        N = len(envs)
        K = 1 + max_obs
        q0 = np.zeros((N, n, 3))
        mu = np.zeros(N)
        obs_type = np.zeros((N, K), np.int32)
        obs_dims = np.zeros((N, K, 3))
        poses = np.zeros((N, steps + 1, K, 7))
        poses[:, :, :, 3] = 1.0
        for i, e in enumerate(envs):
            g = env_rng(seed, e)
            g.integers(0, 2)  # the draw that picked the size
            mu[i] = g.uniform(0.1, 0.9)
            q0[i] = rest + (0.0, 0.0, z0)
            obs_type[i, 0] = PLANE
            k_obs = int(g.integers(1, max_obs + 1))
            for o in range(1, 1 + k_obs):
                if g.uniform() < 0.5:
                    obs_type[i, o] = SPHERE
                    r = g.uniform(0.03, 0.1)
                    obs_dims[i, o, 0] = r
                    c = (g.uniform(-0.15, 0.15), g.uniform(-0.15, 0.15), r)
                else:
                    obs_type[i, o] = BOX
                    hx = g.uniform(0.02, 0.08, 3)
                    obs_dims[i, o] = hx
                    c = (g.uniform(-0.15, 0.15), g.uniform(-0.15, 0.15), hx[2])
                poses[i, :, o, :3] = c
        out.append(Scene(f"mixed_{key[0]}_{key[1]}", etype, rest, elems, mass, ws, wb, q0, np.zeros_like(q0), mu,
                         np.ones(N), obs_type, obs_dims, np.zeros((N, K)), poses, h=0.01, thickness=tau, steps=steps,
                         meta={"envs": envs}))
    return out


# --------------------------------------------------------------------------
# ray-casting inputs
# --------------------------------------------------------------------------
def _quat_axis_angle(axis, ang):
    a = np.asarray(axis, np.float64) / np.linalg.norm(axis)
    return np.array([np.cos(ang / 2), *(np.sin(ang / 2) * a)])


def _quat_mul(a, b):
    """Hamilton product of quaternions (w, x, y, z)."""
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


@dataclass
class RayScene:
    """Batched ray-casting input: N environments sharing one triangle mesh.

    verts [N][n][3], tris int32 [T][3]; obstacles obs_type int32 [N][K],
    obs_dims [N][K][3], obs_poses [N][K][7]; cam_poses [N][7]
    (camera-to-world, camera x right, y down, z along the view); cam =
    (width, height, fx, fy, cx, cy, z_near, z_far).
    """
    name: str
    verts: np.ndarray
    tris: np.ndarray
    obs_type: np.ndarray
    obs_dims: np.ndarray
    obs_poses: np.ndarray
    cam_poses: np.ndarray
    cam: tuple

    @property
    def n_envs(self) -> int:
        return self.verts.shape[0]


def towel_views(seed: int = 4, n_envs: int = 128, n_side: int = 181, side: float = 0.6, width: int = 640,
                height: int = 480, hfov_deg: float = 56.0, cam_height=(0.8, 1.0), tilt_deg: float = 15.0) -> RayScene:
    """Towel-folding views for depth rendering (appendix, depth rendering
    overhead: a towel on a table seen by an overhead depth camera).

    The towel is an n_side x n_side grid (181: 32,761 vertices, 64,800
    triangles) of side ``side`` lying on the ground 1 mm up, with wrinkles
    (four plane waves, wavelength U[3, 15] cm, amplitude U[0, 4] mm) and one
    fold: the part beyond a random line near the centre wraps around a
    cylinder of radius U[5, 15] mm by U[144, 180] degrees and continues
    straight, so the folded layer lies over the towel.  Obstacles: the ground plane, two
    gripper finger boxes (2 x 2 x 4 cm) 5-15 cm above the towel, and one
    invisible pose carrier.  The camera looks down at the towel (its centre
    within 2 cm) from U[cam_height] m with
    up to ``tilt_deg`` of tilt and a random yaw; pinhole with horizontal field
    of view ``hfov_deg``, depth range [0.05, 5] m.
    """
    rest, tris = cloth_grid(n_side, n_side, side)
    n = len(rest)
    verts = np.zeros((n_envs, n, 3))
    K = 4
    obs_type = np.tile(np.array([PLANE, BOX, BOX, NONE], np.int32), (n_envs, 1))
    obs_dims = np.zeros((n_envs, K, 3))
    obs_dims[:, 1:3] = (0.01, 0.01, 0.02)
    obs_poses = np.zeros((n_envs, K, 7))
    cam_poses = np.zeros((n_envs, 7))
    fx = width / 2 / np.tan(np.radians(hfov_deg) / 2)
    cam = (width, height, fx, fx, width / 2, height / 2, 0.05, 5.0)
    tau = 1e-3
    for e in range(n_envs):
        g = env_rng(seed, e)
        xy = rest[:, :2].copy()
        z = np.full(n, tau)
        for _ in range(4):
            ang, lam = g.uniform(0, 2 * np.pi), g.uniform(0.03, 0.15)
            amp, ph = g.uniform(0, 0.004), g.uniform(0, 2 * np.pi)
            k = 2 * np.pi / lam * np.array([np.cos(ang), np.sin(ang)])
            z += amp * 0.5 * (1 + np.sin(xy @ k + ph))
        c = g.uniform(-0.25 * side, 0.25 * side, 2)
        beta = g.uniform(0, 2 * np.pi)
        m = np.array([np.cos(beta), np.sin(beta)])
        alpha, rf = g.uniform(0.8 * np.pi, np.pi), g.uniform(0.005, 0.015)
        s = (xy - c) @ m
        th = np.minimum(s / rf, alpha)
        sp = np.where(s < rf * alpha, rf * np.sin(th), rf * np.sin(alpha) + (s - rf * alpha) * np.cos(alpha))
        zp = np.where(s < rf * alpha, rf * (1 - np.cos(th)), rf * (1 - np.cos(alpha)) + (s - rf * alpha) * np.sin(alpha))
        fold = s > 0
        xy[fold] += ((sp - s)[fold])[:, None] * m
        z[fold] += zp[fold]
        verts[e] = np.c_[xy, z]
        obs_poses[e, 0] = _pose((0, 0, 0))
        for k in (1, 2):
            p = g.uniform(-0.3 * side, 0.3 * side, 2)
            obs_poses[e, k] = _pose((p[0], p[1], g.uniform(0.05, 0.15)),
                                    _quat_axis_angle((0, 0, 1), g.uniform(0, 2 * np.pi)))
        obs_poses[e, 3] = _pose((0, 0, 0.3))
        q = _quat_mul(_quat_axis_angle((0, 0, 1), g.uniform(0, 2 * np.pi)),
                      _quat_axis_angle((1, 0, 0), np.pi + np.radians(g.uniform(-tilt_deg, tilt_deg))))
        ctr = verts[e, :, :2].mean(0)
        pc = (ctr[0] + g.uniform(-0.02, 0.02), ctr[1] + g.uniform(-0.02, 0.02), g.uniform(*cam_height))
        cam_poses[e] = _pose(pc, q)
    return RayScene("towel_views", verts, tris, obs_type, obs_dims, obs_poses, cam_poses, cam)


def cloth_stack_drop(seed: int = 5, n_envs: int = 8, n_side: int = 16, side: float = 0.25, steps: int = 60,
                     k_max: int = 10, drop=(0.004, 0.012)) -> Scene:
    """A small cloth dropped onto a larger one lying on the ground: both are
    components of one mesh, so they meet through cloth self-collision.

    Base: n_side x n_side grid of side ``side`` on the ground 1 mm up.  Top:
    a (n_side/2) x (n_side/2) grid of side side/2, turned by U[0, 90] degrees
    about z, its centre U[-side/8, side/8] off the base's, released flat at
    U[drop] m above the base (at rest).  Self-collision on
    (meta["self_collision"]), ground plane only, mu ~ U[0.2, 0.6],
    h = 1/100; the same areal mass and stiffness as the other cloths.
    """
    rb, tb = cloth_grid(n_side, n_side, side)
    m_side = max(n_side // 2, 2)
    rt, tt = cloth_grid(m_side, m_side, side / 2)
    nb = len(rb)
    rest = np.concatenate([rb, rt + [0.0, 0.0, 0.05]])   # rest shapes are flat; the offset only separates them
    tris = np.concatenate([tb, tt + nb]).astype(np.int32)
    n = len(rest)
    mass = np.concatenate([np.full(nb, 0.1 * side * side / 0.25 / nb),
                           np.full(len(rt), 0.1 * (side / 2) ** 2 / 0.25 / len(rt))])
    tau = 1e-3
    q0 = np.zeros((n_envs, n, 3))
    K = 1
    obs_type = np.full((n_envs, K), PLANE, np.int32)
    obs_dims = np.zeros((n_envs, K, 3))
    mu = np.zeros(n_envs)
    poses = np.zeros((n_envs, steps + 1, K, 7))
    poses[:, :, 0] = _pose((0, 0, 0))
    for e in range(n_envs):
        g = env_rng(seed, e)
        mu[e] = g.uniform(0.2, 0.6)
        ang = g.uniform(0, 0.5 * np.pi)
        ca, sa = np.cos(ang), np.sin(ang)
        off = g.uniform(-side / 8, side / 8, 2)
        top = rt[:, :2] @ np.array([[ca, sa], [-sa, ca]]) + off
        z_top = 2 * tau + g.uniform(*drop)
        q0[e, :nb] = np.c_[rb[:, :2], np.full(nb, tau)]
        q0[e, nb:] = np.c_[top, np.full(len(rt), z_top)]
    return Scene("cloth_stack_drop", TRI, rest, tris, mass, 1e4, 10.0, q0, np.zeros_like(q0), mu, np.ones(n_envs),
                 obs_type, obs_dims, np.zeros((n_envs, K)), poses, h=0.01, k_max=k_max, thickness=tau, steps=steps,
                 meta={"self_collision": True})


def strips_cross_drop(seed: int = 6, n_envs: int = 4, steps: int = 40, k_max: int = 10) -> Scene:
    """Two narrow cloth strips crossing at right angles: the top one is
    released U[2, 6] mm above the bottom one (on the ground).  Each strip is
    2 x 4 vertices, 1 cm wide and 20 cm long (cells 6.7 cm long), placed so
    that no vertex of one strip lies over the other: they can meet only edge
    against edge (cloth self-collision, meta["self_collision"]).  Ground
    plane, mu ~ U[0.2, 0.6], h = 1/100."""
    m, L, wdt = 4, 0.2, 0.01
    xs = np.linspace(-L / 2, L / 2, m)
    bottom = np.array([(x, y, 0.0) for y in (-wdt / 2, wdt / 2) for x in xs])
    top = np.array([(x, y, 0.0) for x in (-wdt / 2, wdt / 2) for y in xs])
    tris = []
    for k in range(m - 1):
        a, b, c, d = k, k + 1, m + k, m + k + 1
        tris += [(a, b, d), (a, d, c)]
    tris = np.array(tris + [tuple(v + 2 * m for v in t) for t in tris], np.int32)
    rest = np.concatenate([bottom, top + [0.0, 0.0, 0.05]])
    n = len(rest)
    mass = np.full(n, 1e-3)
    tau = 1e-3
    q0 = np.zeros((n_envs, n, 3))
    K = 1
    obs_type = np.full((n_envs, K), PLANE, np.int32)
    mu = np.zeros(n_envs)
    poses = np.zeros((n_envs, steps + 1, K, 7))
    poses[:, :, 0] = _pose((0, 0, 0))
    for e in range(n_envs):
        g = env_rng(seed, e)
        mu[e] = g.uniform(0.2, 0.6)
        q0[e, :2 * m] = bottom + [0.0, 0.0, tau]
        q0[e, 2 * m:] = top + [0.0, 0.0, 2 * tau + g.uniform(0.002, 0.006)]
    return Scene("strips_cross_drop", TRI, rest, tris, mass, 1e4, 10.0, q0, np.zeros_like(q0), mu, np.ones(n_envs),
                 obs_type, np.zeros((n_envs, K, 3)), np.zeros((n_envs, K)), poses, h=0.01, k_max=k_max,
                 thickness=tau, steps=steps, meta={"self_collision": True})


def cloth_bar_drop(seed: int = 7, n_envs: int = 4, n_side: int = 16, side: float = 0.25, steps: int = 40,
                   k_max: int = 10) -> Scene:
    """A cloth released flat a few millimetres above a thin horizontal bar
    and a thin vertical post, both box obstacles narrower than the cloth's
    cells, over the ground.  The bar (5 x 5 mm section, 40 cm long) runs
    along x midway between vertex rows n_side/4 and n_side/4 + 1; the post
    (6 x 6 mm section, 6 cm tall) stands under the incentre of a triangle
    (the cell at column n_side/2, row 3 n_side/4 - 1), its top inside that
    triangle.  Both tops are at z = 5 cm.  The cloth meets them between its
    vertices, through box edges against cloth edges and box corners against
    cloth triangles (meta["obstacle_features"]); without those rows it falls
    past both.  Per environment: the bar turned by U[-4, 4] degrees about z
    (environment 0: not turned), release height U[2, 6] mm above the tops,
    mu ~ U[0.2, 0.6]; h = 1/100; the areal mass and stiffness of the other
    cloths."""
    rest, tris = cloth_grid(n_side, n_side, side)
    n = len(rest)
    sp = side / (n_side - 1)
    mass = np.full(n, 0.1 * side * side / 0.25 / n)
    tau, z_top = 1e-3, 0.05
    K = 3
    obs_type = np.tile(np.array([PLANE, BOX, BOX], np.int32), (n_envs, 1))
    obs_dims = np.zeros((n_envs, K, 3))
    obs_dims[:, 1] = (0.2, 0.0025, 0.0025)
    obs_dims[:, 2] = (0.003, 0.003, 0.03)
    jb = n_side // 4
    y_bar = -side / 2 + (jb + 0.5) * sp
    ip, jp = n_side // 2, 3 * n_side // 4 - 1
    r_in = sp * (2 - np.sqrt(2)) / 2     # incentre of the right-angled triangle at the cell's corner (ip, jp)
    post = (-side / 2 + ip * sp + r_in, -side / 2 + jp * sp + r_in, z_top - 0.03)
    mu = np.zeros(n_envs)
    q0 = np.zeros((n_envs, n, 3))
    poses = np.zeros((n_envs, steps + 1, K, 7))
    for e in range(n_envs):
        g = env_rng(seed, e)
        mu[e] = g.uniform(0.2, 0.6)
        yaw = 0.0 if e == 0 else np.deg2rad(g.uniform(-4.0, 4.0))
        drop = g.uniform(0.002, 0.006)
        poses[e, :, 0] = _pose((0, 0, 0))
        poses[e, :, 1] = _pose((0.0, y_bar, z_top - 0.0025), _quat_axis_angle((0, 0, 1), yaw))
        poses[e, :, 2] = _pose(post)
        q0[e] = rest + [0.0, 0.0, z_top + tau + drop]
    return Scene("cloth_bar_drop", TRI, rest, tris, mass, 1e4, 10.0, q0, np.zeros_like(q0), mu, np.ones(n_envs),
                 obs_type, obs_dims, np.zeros((n_envs, K)), poses, h=0.01, k_max=k_max, thickness=tau, steps=steps,
                 meta={"obstacle_features": True})


def corner_support(steps: int = 4, mu: float = 0.5) -> Scene:
    """One equilateral triangle (4 cm sides, 1 g per vertex) lying flat with
    its centroid one thickness above the top corner of a cube (2 cm side)
    standing on a vertex: the cube's (1, 1, 1) diagonal is turned onto +z, so
    corner 7 = (+,+,+) is the top, the three next corners are 1.15 cm lower
    (out of reach).  No other obstacle; box-feature rows on."""
    tau, d, zc = 1e-3, 0.01, 0.1
    L = 0.04
    rest = np.array([(L / np.sqrt(3) * np.cos(a), L / np.sqrt(3) * np.sin(a), 0.0)
                     for a in (np.pi / 2, np.pi / 2 + 2 * np.pi / 3, np.pi / 2 + 4 * np.pi / 3)])
    tris = np.array([(0, 1, 2)], np.int32)
    u = np.array([1.0, 1.0, 1.0]) / np.sqrt(3)
    axis = np.cross(u, [0.0, 0.0, 1.0])
    quat = _quat_axis_angle(axis, np.arccos(u[2]))
    z_corner = zc + d * np.sqrt(3)
    q0 = (rest + [0.0, 0.0, z_corner + tau])[None]
    K = 1
    poses = np.zeros((1, steps + 1, K, 7))
    poses[0, :, 0] = _pose((0.0, 0.0, zc), quat)
    return Scene("corner_support", TRI, rest, tris, np.full(3, 1e-3), 1e4, 10.0, q0, np.zeros_like(q0),
                 np.array([mu]), np.ones(1), np.full((1, K), BOX, np.int32), np.full((1, K, 3), d),
                 np.zeros((1, K)), poses, h=0.01, thickness=tau, steps=steps, meta={"obstacle_features": True})


def edge_support(steps: int = 4, mu: float = 0.5) -> Scene:
    """A square of two triangles (4 cm sides, 1 g per vertex, diagonal from
    vertex 0 to vertex 3) lying flat one thickness above the top edge of a
    bar (10 x 2 x 2 cm) turned by 45 degrees about its long axis x, so that
    one of its long edges is the top, under the square's middle line y = 0;
    the bar's other edges are out of reach.  That edge crosses the square's
    edges 0-2, 0-3 and 1-3 at their midpoints.  No other obstacle;
    box-feature rows on."""
    tau, d, zc = 1e-3, 0.01, 0.1
    rest, tris = cloth_grid(2, 2, 0.04)
    z_edge = zc + d * np.sqrt(2)
    q0 = (rest + [0.0, 0.0, z_edge + tau])[None]
    K = 1
    poses = np.zeros((1, steps + 1, K, 7))
    poses[0, :, 0] = _pose((0.0, 0.0, zc), _quat_axis_angle((1, 0, 0), np.pi / 4))
    dims = np.array([[[0.05, d, d]]])
    return Scene("edge_support", TRI, rest, tris, np.full(4, 1e-3), 1e4, 10.0, q0, np.zeros_like(q0),
                 np.array([mu]), np.ones(1), np.full((1, K), BOX, np.int32), dims, np.zeros((1, K)), poses,
                 h=0.01, thickness=tau, steps=steps, meta={"obstacle_features": True})
