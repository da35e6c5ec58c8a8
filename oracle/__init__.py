"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline arm of
``bench.py`` may import this package.  It compiles ``oracle.c`` with the host C
compiler into ``oracle/_build/`` on first use and shares nothing with the CUDA
library except the seeded scene arrays it is given.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, f) for f in ("oracle.c", "mlp.c", "raycast.c")]
_lib = None

DP_H, DP_GX, DP_GY, DP_GZ, DP_TOL, DP_MAXFORCE, DP_TAU, DP_MARGIN, DP_MU, DP_GRASP_OBS = range(10)
DP_ANCHOR, DP_SELF, DP_OFEAT, DP_SIZE = 10, 13, 14, 15
GRASP_SLOT = 8   # contact-list slot of grasp constraints (after every obstacle)
SELF_SLOT = 9    # contact-list slot of cloth vertex-triangle self contacts (after the grasp row)
SELF_MAX = 4     # vertex-triangle self contacts per vertex at most
EE_SLOT = 10     # contact-list slot of cloth edge-edge self contacts
EE_MAX = 4       # edge-edge self contacts per vertex (owning the first edge) at most
OVT_SLOT = 11    # contact-list slot of box corners against cloth triangles (under the triangle's first vertex)
OEE_SLOT = 12    # contact-list slot of box edges against cloth edges (under the edge's first vertex)
OFEAT_MAX = 4    # rows of each box-feature kind per vertex at most
MAX_OBS = 8      # obstacle slots per environment (box-feature indices count in them)
IP_KMAX, IP_KMIN, IP_KCAP, IP_MODE, IP_METRIC, IP_LINIT = range(6)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no vector extensions)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRC + [os.path.join(_HERE, "oracle.h")])
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, *_SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        d, i = C.c_double, C.c_int
        pd, pi = P(d), P(i)
        _lib.or_mesh_new.restype = C.c_void_p
        _lib.or_mesh_new.argtypes = [i, i, pd, i, pi, pd, d, d, d]
        _lib.or_mesh_free.argtypes = [C.c_void_p]
        _lib.or_mesh_hinges.argtypes = [C.c_void_p]
        _lib.or_mesh_edges.argtypes = [C.c_void_p, pi]
        _lib.or_mesh_edges.restype = i
        _lib.or_mesh_matrix.argtypes = [C.c_void_p, pd]
        _lib.or_solve.argtypes = [C.c_void_p, pd, pd]
        _lib.or_project.argtypes = [C.c_void_p, pd, pd]
        _lib.or_assemble_b.argtypes = [C.c_void_p, pd, pd, pd]
        _lib.or_pd_energy.restype = d
        _lib.or_pd_energy.argtypes = [C.c_void_p, pd, pd, pd]
        _lib.or_closest_rotation.argtypes = [i, pd, pd]
        _lib.or_sdf.restype = d
        _lib.or_sdf.argtypes = [i, pd, pd, pd, pd]
        _lib.or_fb.restype = d
        _lib.or_fb.argtypes = [d, d]
        _lib.or_detect.restype = i
        _lib.or_detect.argtypes = [C.c_void_p, pd, i, pi, pd, pd, pd, pd, C.POINTER(C.c_ubyte), i, pi, pi, pi]
        _lib.or_solve_step.restype = i
        _lib.or_solve_step.argtypes = [C.c_void_p, pd, pi, i, pi, pd, pd, pd, pd, pd, pd, pd, i,
                                       pi, pi, pi, pd, pi, pd, pd]
        _lib.or_residual.restype = d
        _lib.or_residual.argtypes = [C.c_void_p, pd, i, pi, pd, pd, pd, pd, pd, pd, i, pi, pi, pi, pd]
        _lib.or_raycast.argtypes = [i, pd, i, pi, i, pi, pd, pd, pd, pd, i, i, d, pd, pi, pd]
        _lib.or_raycast.restype = None
        _lib.or_raycast_pixels.argtypes = [i, pd, i, pi, i, pi, pd, pd, pd, pd, i, pi, d, pd, pi, pd]
        _lib.or_raycast_pixels.restype = None
        _lib.or_mlp_forward.argtypes = [i, pd, pd, pd]
        _lib.or_mlp_loss_grad.restype = d
        _lib.or_mlp_loss_grad.argtypes = [i, pd, pd, pd, pd]
    return _lib


def _pd(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _pi(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class Mesh:
    """System matrix and element data of one mesh (one stiffness scale)."""

    def __init__(self, elem_type, rest, elems, mass, w_stretch, w_bend, h):
        self.rest, self.elems, self.mass = _f64(rest), _i32(elems).reshape(-1, 3 if elem_type == 0 else 4), _f64(mass)
        self.n, self.ne, self.type = len(self.rest), len(self.elems), elem_type
        self.h = h
        self._p = lib().or_mesh_new(elem_type, self.n, _pd(self.rest), self.ne, _pi(self.elems),
                                    _pd(self.mass), w_stretch, w_bend, h)
        if not self._p:
            raise ValueError("system matrix is not positive definite")

    @classmethod
    def from_scene(cls, sc, env: int = 0):
        return cls(sc.elem_type, sc.rest, sc.elems, sc.mass, sc.w_stretch * sc.stiff[env], sc.w_bend, sc.h)

    def __del__(self):
        if getattr(self, "_p", None):
            lib().or_mesh_free(self._p)
            self._p = None

    @property
    def hinges(self) -> int:
        return lib().or_mesh_hinges(self._p)

    @property
    def edges(self):
        """Unique edges (a < b) of a triangle mesh, sorted: [n_edges][2]."""
        ne = lib().or_mesh_edges(self._p, None)
        out = np.zeros((max(ne, 1), 2), np.int32)
        lib().or_mesh_edges(self._p, _pi(out))
        return out[:ne]

    def matrix(self):
        A = np.zeros((self.n, self.n))
        lib().or_mesh_matrix(self._p, _pd(A))
        return A

    def solve(self, rhs):
        rhs = _f64(rhs).reshape(self.n, 3)
        out = np.zeros_like(rhs)
        lib().or_solve(self._p, _pd(rhs), _pd(out))
        return out

    def project(self, q):
        q = _f64(q)
        p = np.zeros((max(self.ne, 1), 9))
        lib().or_project(self._p, _pd(q), _pd(p))
        return p[: self.ne]

    def assemble_b(self, qt, p):
        b = np.zeros((self.n, 3))
        pp = _f64(p) if len(p) else np.zeros((1, 9))
        lib().or_assemble_b(self._p, _pd(_f64(qt)), _pd(pp), _pd(b))
        return b

    def energy(self, q, qt, p):
        pp = _f64(p) if len(p) else np.zeros((1, 9))
        return lib().or_pd_energy(self._p, _pd(_f64(q)), _pd(_f64(qt)), _pd(pp))


def closest_rotation(F):
    F = _f64(F)
    cols = F.shape[1]
    R = np.zeros_like(F)
    lib().or_closest_rotation(cols, _pd(F), _pd(R))
    return R


def sdf(otype, dims, pose, x):
    n = np.zeros(3)
    sd = lib().or_sdf(int(otype), _pd(_f64(dims)), _pd(_f64(pose)), _pd(_f64(x)), _pd(n))
    return sd, n


def fb(a, b):
    return lib().or_fb(float(a), float(b))


def params(sc, env: int = 0, mode=None, metric: int = 0, k_max=None, k_min=None, k_cap=None, tol=None,
           lin_iters: int = 10):
    dp = np.zeros(DP_SIZE)
    dp[DP_H] = sc.h
    dp[DP_GX:DP_GZ + 1] = sc.gravity
    dp[DP_TOL] = sc.tol_ncp if tol is None else tol
    dp[DP_MAXFORCE] = sc.maxforce
    dp[DP_TAU] = sc.thickness
    dp[DP_MARGIN] = sc.margin
    dp[DP_MU] = sc.mu[env]
    g = sc.meta.get("grasp") if sc.meta else None
    dp[DP_GRASP_OBS] = g["obstacle"] if g else -1
    if g:
        dp[DP_ANCHOR:DP_ANCHOR + 3] = g["anchor"]
    dp[DP_SELF] = 1.0 if (sc.meta and sc.meta.get("self_collision")) else 0.0
    dp[DP_OFEAT] = 1.0 if (sc.meta and sc.meta.get("obstacle_features")) else 0.0
    ip = np.zeros(6, np.int32)
    ip[IP_KMAX] = sc.k_max if k_max is None else k_max
    ip[IP_KMIN] = sc.k_min if k_min is None else k_min
    ip[IP_KCAP] = sc.k_cap if k_cap is None else k_cap
    ip[IP_MODE] = sc.mode if mode is None else mode
    ip[IP_METRIC] = metric
    ip[IP_LINIT] = lin_iters
    return dp, ip


class EnvState:
    """q, v and the last contact list of one environment."""

    def __init__(self, q, v):
        self.q, self.v = _f64(q).copy(), _f64(v).copy()
        self.cvert = np.zeros(0, np.int32)
        self.cobs = np.zeros(0, np.int32)
        self.ctri = np.zeros(0, np.int32)     # triangle of each self contact, -1 otherwise
        self.gamma = np.zeros((0, 4))
        self.iters, self.rncp = 0, 0.0
        self.trace = None
        self.attached = np.zeros(len(self.q), np.uint8)   # grasped vertices


def _to_world(pose, p):
    """pose = (x, y, z, qw, qx, qy, qz) applied to a body-frame point."""
    w, x, y, z = pose[3:7]
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    return R @ np.asarray(p, float) + pose[:3]


def apply_grasp(sc, env, s, st):
    """Grasp schedule of the scene (appendix, Bilateral Constraint for Cloth
    Control) at the start of step s: a request 1 attaches every vertex within
    the radius of the anchor (gripper pose at the start of the step); 0
    releases all.  Scenes keep vertices away from the radius boundary, so the
    FP32 test of the CUDA path takes the same decision."""
    g = sc.meta.get("grasp") if sc.meta else None
    if not g:
        return
    req = g["schedule"].get(s)
    if req == 1:
        p = _to_world(sc.poses[env, s, g["obstacle"]], g["anchor"])
        st.attached = (np.linalg.norm(st.q - p, axis=1) <= g["radius"]).astype(np.uint8)
    elif req == 0:
        st.attached = np.zeros(len(st.q), np.uint8)


def detect(mesh: Mesh, sc, env, step, q, v, dp=None, attached=None):
    dp = params(sc, env)[0] if dp is None else dp
    K = sc.n_obs
    ot, od = _i32(sc.obs_type[env]), _f64(sc.obs_dims[env])
    pth = _f64(sc.poses[env, step + 1])
    cap = mesh.n * (K + 1 + SELF_MAX + EE_MAX + 2 * OFEAT_MAX)
    cv, co, ct = np.zeros(cap, np.int32), np.zeros(cap, np.int32), np.zeros(cap, np.int32)
    att = None if attached is None else np.ascontiguousarray(attached, np.uint8)
    cnt = lib().or_detect(mesh._p, _pd(dp), K, _pi(ot), _pd(od), _pd(pth), _pd(_f64(q)), _pd(_f64(v)),
                          None if att is None else att.ctypes.data_as(C.POINTER(C.c_ubyte)),
                          cap, _pi(cv), _pi(co), _pi(ct))
    return cv[:cnt].copy(), co[:cnt].copy(), ct[:cnt].copy()


def warm_from_previous(cvert, cobs, ctri, prev: EnvState):
    """gamma^0 of the new list: the previous step's gamma of the same (vertex, slot, triangle)."""
    g = np.zeros((len(cvert), 4))
    if len(prev.cvert):
        pos = {(int(v), int(o), int(t)): i for i, (v, o, t) in enumerate(zip(prev.cvert, prev.cobs, prev.ctri))}
        for i, key in enumerate(zip(cvert, cobs, ctri)):
            j = pos.get(tuple(int(x) for x in key))
            if j is not None:
                g[i] = prev.gamma[j]
    return g


def step(mesh: Mesh, sc, env, s, st: EnvState, mode=None, metric=0, warm="cold", gamma0=None,
         q_init=None, k_max=None, k_min=None, k_cap=None, tol=None, trace=False, lin_iters=10):
    """Advance one environment by one step (Algorithm 1 body).  Mutates ``st``.
    metric 0: lite Z = J M^-1 J^T + E; 1: full Z = J A^-1 J^T + E solved
    exactly; 2: full Z solved by ``lin_iters`` steps of preconditioned GMRES."""
    dp, ip = params(sc, env, mode, metric, k_max, k_min, k_cap, tol, lin_iters)
    apply_grasp(sc, env, s, st)
    cvert, cobs, ctri = detect(mesh, sc, env, s, st.q, st.v, dp, st.attached)
    if gamma0 is not None:
        gam = _f64(gamma0).reshape(len(cvert), 4).copy()
    elif warm == "prev":
        gam = warm_from_previous(cvert, cobs, ctri, st)
    else:
        gam = np.zeros((len(cvert), 4))
    K = sc.n_obs
    it, rn = C.c_int(0), C.c_double(0.0)
    tr = np.zeros(int(ip[IP_KCAP]) + int(ip[IP_KMAX]) + 2)
    gbuf = gam if len(gam) else np.zeros((1, 4))
    lib().or_solve_step(mesh._p, _pd(dp), _pi(ip), K, _pi(_i32(sc.obs_type[env])), _pd(_f64(sc.obs_dims[env])),
                        _pd(_f64(sc.obs_comp[env])), _pd(_f64(sc.poses[env, s])), _pd(_f64(sc.poses[env, s + 1])),
                        _pd(st.q), _pd(st.v), None if q_init is None else _pd(_f64(q_init)), len(cvert),
                        _pi(cvert if len(cvert) else np.zeros(1, np.int32)),
                        _pi(cobs if len(cobs) else np.zeros(1, np.int32)),
                        _pi(ctri if len(ctri) else np.zeros(1, np.int32)), _pd(gbuf), C.byref(it), C.byref(rn),
                        _pd(tr))
    st.cvert, st.cobs, st.ctri, st.gamma = cvert, cobs, ctri, gbuf[: len(cvert)].copy()
    st.iters, st.rncp = it.value, rn.value
    st.trace = tr[: it.value + 1].copy() if trace else None
    return st


def residual(mesh: Mesh, sc, env, s, q_t, q, cvert, cobs, gamma, ctri=None):
    dp = params(sc, env)[0]
    ctri = np.full(len(cvert), -1, np.int32) if ctri is None else _i32(ctri)
    g = _f64(gamma).reshape(-1, 4) if len(cvert) else np.zeros((1, 4))
    return lib().or_residual(mesh._p, _pd(dp), sc.n_obs, _pi(_i32(sc.obs_type[env])), _pd(_f64(sc.obs_dims[env])),
                             _pd(_f64(sc.obs_comp[env])), _pd(_f64(sc.poses[env, s])), _pd(_f64(sc.poses[env, s + 1])),
                             _pd(_f64(q_t)), _pd(_f64(q)), len(cvert),
                             _pi(_i32(cvert) if len(cvert) else np.zeros(1, np.int32)),
                             _pi(_i32(cobs) if len(cobs) else np.zeros(1, np.int32)),
                             _pi(ctri if len(ctri) else np.zeros(1, np.int32)), _pd(g))


def rollout(sc, env=0, steps=None, mode=None, warm="cold", metric=0, k_max=None, k_min=None, k_cap=None, tol=None,
            mesh=None, record=False, lin_iters=10):
    """Run ``steps`` steps of one environment; returns the final EnvState (and the
    per-step positions when ``record``)."""
    mesh = Mesh.from_scene(sc, env) if mesh is None else mesh
    st = EnvState(sc.q0[env], sc.v0[env])
    steps = sc.steps if steps is None else steps
    traj = []
    for s in range(steps):
        step(mesh, sc, env, s, st, mode=mode, metric=metric, warm=warm, k_max=k_max, k_min=k_min, k_cap=k_cap, tol=tol,
             lin_iters=lin_iters)
        if record:
            traj.append((st.q.copy(), st.iters, st.rncp))
    return (st, traj) if record else st


# ------------------------------------------------------------------ MLP
def mlp_forward(params_flat, x):
    """FP64 forward of the 10-128-128-6 warm-start MLP; x [B][10] -> [B][6]."""
    x = _f64(x)
    y = np.zeros((len(x), 6))
    lib().or_mlp_forward(len(x), _pd(_f64(params_flat)), _pd(x), _pd(y))
    return y


def mlp_loss_grad(params_flat, x, t):
    """Mean-squared loss 0.5*mean_b |y_b - t_b|^2 and its gradient w.r.t. the parameters."""
    x, t = _f64(x), _f64(t)
    p = _f64(params_flat)
    g = np.zeros_like(p)
    loss = lib().or_mlp_loss_grad(len(x), _pd(p), _pd(x), _pd(t), _pd(g))
    return loss, g


def _rc_args(x, tris, otype, odims, opose):
    x = _f64(x).reshape(-1, 3)
    tris = _i32(tris).reshape(-1, 3)
    otype = _i32(otype).reshape(-1)
    K = len(otype)
    odims = _f64(odims).reshape(K, 3) if K else np.zeros((1, 3))
    opose = _f64(opose).reshape(K, 7) if K else np.zeros((1, 7))
    return (len(x), _pd(x if len(x) else np.zeros((1, 3))), len(tris),
            _pi(tris if len(tris) else np.zeros((1, 3), np.int32)), K,
            _pi(otype if K else np.zeros(1, np.int32)), _pd(odims), _pd(opose)), (x, tris, otype, odims, opose)


def raycast(x, tris, otype, odims, opose, cam_pose, intr, W, H, dil=0.0):
    """Depth ray casting of one environment (appendix, depth rendering), by
    brute force in FP64.  x [n][3], tris [T][3]; obstacles otype [K], odims
    [K][3], opose [K][7]; cam_pose [7] camera-to-world; intr = (fx, fy, cx,
    cy, z_near, z_far).  Returns depth [H][W] (0: no hit), seg [H][W] (0 none,
    1 mesh, 2 + k obstacle k), points [H][W][3] (NaN: no hit).  ``dil`` grows
    (> 0) or shrinks (< 0) every primitive (see oracle.h)."""
    args, keep = _rc_args(x, tris, otype, odims, opose)
    depth = np.zeros((H, W))
    seg = np.zeros((H, W), np.int32)
    pts = np.zeros((H, W, 3))
    cam, it = _f64(cam_pose), _f64(intr)
    lib().or_raycast(*args, _pd(cam), _pd(it), W, H, float(dil), _pd(depth), _pi(seg), _pd(pts))
    return depth, seg, pts


def raycast_pixels(x, tris, otype, odims, opose, cam_pose, intr, uv, dil=0.0):
    """``raycast`` for the pixels uv [m][2] = (u, v) only; outputs [m]."""
    args, keep = _rc_args(x, tris, otype, odims, opose)
    uv = _i32(uv).reshape(-1, 2)
    m = len(uv)
    depth = np.zeros(m)
    seg = np.zeros(m, np.int32)
    pts = np.zeros((m, 3))
    cam, it = _f64(cam_pose), _f64(intr)
    lib().or_raycast_pixels(*args, _pd(cam), _pd(it), m, _pi(uv), float(dil), _pd(depth), _pi(seg), _pd(pts))
    return depth, seg, pts
