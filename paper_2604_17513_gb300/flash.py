"""Thin Python binding of ``libflash.so`` (argument marshalling only).

Every step of the simulation runs in the library's CUDA kernels; this module
only fills the C descriptors, passes device pointers of torch tensors and the
current torch stream, and raises on error codes.  If the shared library is
missing the import fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import scenes as _sc

_HERE = os.path.dirname(os.path.abspath(__file__))
# FLASH_CHECKED_BUILD=1 loads the checked variant (every index a step kernel
# reads is range-checked; an out-of-range one is reported as FLASH_EINDEX)
LIB_PATH = os.path.join(_HERE, "libflash_check.so" if os.environ.get("FLASH_CHECKED_BUILD") == "1" else "libflash.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTIMPL, ESTATE, ENUMERIC, EINDEX = 0, -1, -2, -3, -4, -5, -6, -7, -8
WOVERFLOW = 1
MAX_OBS = 8
GRASP_SLOT = MAX_OBS   # contact-list obstacle slot of grasp rows
SELF_SLOT = MAX_OBS + 1   # contact-list slot of cloth vertex-triangle self contacts
SELF_MAX = 4           # vertex-triangle self contacts per vertex at most
EE_SLOT = MAX_OBS + 2  # contact-list slot of cloth edge-edge contacts
EE_MAX = 4             # edge-edge contacts per vertex at most
OVT_SLOT = MAX_OBS + 3  # contact-list slot of box corners against cloth triangles
OEE_SLOT = MAX_OBS + 4  # contact-list slot of box edges against cloth edges
OFEAT_MAX = 4           # rows of each box-feature kind per vertex at most
MODE_FIXED, MODE_TOL = 0, 1
METRIC_LITE, METRIC_FULL = 0, 1
SOLVE_F32, SOLVE_F16X3, SOLVE_BF16R = 0, 1, 2
WARM_COLD, WARM_PREV, WARM_LEARNED = 0, 1, 2
GROUPED_AUTO, GROUPED_OFF, GROUPED_ON = 0, 1, 2
THREADS_TUNE = -1   # local_threads / ncp_threads: time the candidates on the first step
SPLITK_AUTO, SPLITK_OFF, SPLITK_ON = 0, 1, 2


class FlashError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"flash error {code}: {msg}")
        self.code = code


class Camera(C.Structure):
    """Pinhole camera of the ray caster (flash_camera): image size in pixels,
    intrinsics fx, fy, cx, cy in pixels, depth range [z_near, z_far] in m."""
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("z_near", C.c_float), ("z_far", C.c_float)]


class SceneDesc(C.Structure):
    _fields_ = [("h", C.c_double), ("gravity", C.c_double * 3), ("tol_ncp", C.c_double), ("maxforce", C.c_double),
                ("thickness", C.c_double), ("margin", C.c_double), ("k_max", C.c_int32), ("k_min", C.c_int32),
                ("k_cap", C.c_int32), ("mode", C.c_int32), ("contact_cap", C.c_int32), ("solve", C.c_int32),
                ("warm", C.c_int32), ("lanes", C.c_int32), ("eager", C.c_int32), ("metric", C.c_int32),
                ("lin_iters", C.c_int32), ("self_collide", C.c_int32), ("obstacle_features", C.c_int32),
                ("grouped_solve", C.c_int32), ("refine_steps", C.c_int32), ("local_threads", C.c_int32),
                ("ncp_threads", C.c_int32), ("split_k", C.c_int32)]


class MeshDesc(C.Structure):
    _fields_ = [("type", C.c_int32), ("n_verts", C.c_int32), ("n_elems", C.c_int32),
                ("rest", C.POINTER(C.c_double)), ("elems", C.POINTER(C.c_int32)), ("mass", C.POINTER(C.c_double)),
                ("w_stretch", C.c_double), ("w_bend", C.c_double), ("thickness", C.c_double)]


class EnvDesc(C.Structure):
    _fields_ = [("mu", C.c_float), ("stiffness", C.c_float), ("n_obs", C.c_int32),
                ("obs_type", C.c_int32 * MAX_OBS), ("obs_dims", (C.c_float * 3) * MAX_OBS),
                ("obs_compliance", C.c_float * MAX_OBS)]


_lib = None


def lib():
    """Load libflash.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2604_17513_gb300.build` "
                              "(the simulator has no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.flash_last_error.restype = C.c_char_p
        L.flash_scene_create.argtypes = [C.POINTER(SceneDesc), C.POINTER(vp)]
        L.flash_mesh_add.argtypes = [vp, C.POINTER(MeshDesc), C.POINTER(i32)]
        L.flash_envs_add.argtypes = [vp, i32, i32, C.POINTER(EnvDesc), C.POINTER(i32)]
        L.flash_scene_finalize.argtypes = [vp, vp]
        L.flash_scene_destroy.argtypes = [vp]
        L.flash_scene_destroy.restype = None
        L.flash_num_envs.argtypes = [vp]
        L.flash_num_verts.argtypes = [vp]
        L.flash_num_verts.restype = i64
        L.flash_env_offsets.argtypes = [vp, C.POINTER(i64)]
        L.flash_set_state.argtypes = [vp, vp, vp, vp]
        L.flash_get_state.argtypes = [vp, vp, vp, vp]
        L.flash_set_obstacle_poses.argtypes = [vp, vp, i32, vp]
        L.flash_step.argtypes = [vp, i32, vp]
        L.flash_grasp.argtypes = [vp, i32, i32, C.POINTER(i32), i32, C.POINTER(C.c_float), C.c_float, vp]
        L.flash_render.argtypes = [vp, C.POINTER(Camera), vp, vp, vp, vp, vp]
        L.flash_get_contact_tris.argtypes = [vp, vp, vp]
        L.flash_raycaster_create.argtypes = [C.POINTER(Camera), i32, i32, i32, C.POINTER(i32), C.POINTER(vp)]
        L.flash_raycast.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.flash_raycaster_destroy.argtypes = [vp]
        L.flash_raycaster_destroy.restype = None
        L.flash_raycaster_profile.argtypes = [vp, i32]
        L.flash_raycaster_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(i64)]
        L.flash_get_contacts.argtypes = [vp, vp, vp, vp, vp, vp]
        L.flash_contact_cap.argtypes = [vp]
        L.flash_get_stats.argtypes = [vp, vp, vp, vp]
        L.flash_status_word.argtypes = [vp, vp]
        L.flash_global_apply.argtypes = [vp, i32, i32, vp, vp, vp]
        L.flash_profile_enable.argtypes = [vp, i32]
        L.flash_profile_read.argtypes = [vp, i32, C.POINTER(C.c_double), C.POINTER(i64)]
        L.flash_launch_count.argtypes = [vp]
        L.flash_launch_count.restype = i64
        L.flash_lane_count.argtypes = [vp]
        L.flash_lane_count.restype = i32
        L.flash_tile_widths.argtypes = [vp, C.POINTER(i32), i32]
        L.flash_tile_widths.restype = i32
        L.flash_tile_splits.argtypes = [vp, C.POINTER(i32), i32]
        L.flash_tile_splits.restype = i32
        L.flash_grouped_solve.argtypes = [vp]
        L.flash_grouped_solve.restype = i32
        L.flash_scene_threads.argtypes = [vp, i32, C.POINTER(i32), i32]
        L.flash_scene_threads.restype = i32
        L.flash_test_bounded_wait.argtypes = [vp, i64, vp]
        L.flash_checked_build.argtypes = []
        L.flash_checked_build.restype = i32
        L.flash_check_poke_element.argtypes = [vp, i32, i32, i32, i32, C.POINTER(i32)]
        L.flash_warmstart_set.argtypes = [vp, vp, i32, i32]
        L.flash_warmstart_bounds.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_float)]
        L.flash_record_contacts.argtypes = [vp, i32]
        L.flash_get_recorded.argtypes = [vp, vp, vp, i64, C.POINTER(i64), vp]
        L.flash_mlp_num_params.restype = i32
        L.flash_mlp_forward.argtypes = [vp, vp, vp, i64, vp]
        L.flash_mlp_loss_grad.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp]
        L.flash_mlp_work_floats.argtypes = [i32]
        L.flash_mlp_work_floats.restype = i64
        L.flash_mlp_adam.argtypes = [vp, vp, vp, vp, i32, C.c_float, vp]
        L.flash_dense_apply_noalloc.argtypes = [vp, i32, i32, vp, vp, vp]
        for name in ("flash_scene_create", "flash_mesh_add", "flash_envs_add", "flash_scene_finalize",
                     "flash_env_offsets", "flash_set_state", "flash_get_state", "flash_set_obstacle_poses",
                     "flash_step", "flash_grasp", "flash_render", "flash_raycaster_create", "flash_raycast", "flash_get_contact_tris",
                     "flash_raycaster_profile", "flash_raycaster_profile_read", "flash_get_contacts", "flash_get_stats", "flash_status_word",
                     "flash_global_apply", "flash_profile_enable", "flash_profile_read", "flash_warmstart_set",
                     "flash_warmstart_bounds",
                     "flash_record_contacts", "flash_get_recorded", "flash_mlp_forward", "flash_mlp_loss_grad",
                     "flash_mlp_adam", "flash_dense_apply_noalloc"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def _check(code):
    if code < 0:
        raise FlashError(code, lib().flash_last_error().decode())
    return code


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Sim:
    """A batch of environments behind one C scene.

    ``scenes`` is one :class:`scenes.Scene` or a list of them (one mesh
    template each); environments are numbered in list order.
    """

    def __init__(self, scenes, solve=SOLVE_F32, mode=None, k_max=None, k_min=None, k_cap=None, tol=None,
                 warm=WARM_COLD, contact_cap=None, lanes=0, eager=False, metric=0, lin_iters=10,
                 self_collision=None, obstacle_features=None, grouped=GROUPED_AUTO, refine_steps=1,
                 local_threads=0, ncp_threads=0, split_k=SPLITK_AUTO):
        if isinstance(scenes, _sc.Scene):
            scenes = [scenes]
        self.scenes = scenes
        s0 = scenes[0]
        d = SceneDesc()
        d.h = s0.h
        d.gravity[:] = list(s0.gravity)
        d.tol_ncp = s0.tol_ncp if tol is None else tol
        d.maxforce = s0.maxforce
        d.thickness = s0.thickness
        d.margin = s0.margin
        d.k_max = s0.k_max if k_max is None else k_max
        d.k_min = s0.k_min if k_min is None else k_min
        d.k_cap = s0.k_cap if k_cap is None else k_cap
        d.mode = s0.mode if mode is None else mode
        if self_collision is None:   # on when a scene asks for it
            self_collision = any(sc.meta.get("self_collision") for sc in scenes)
        if obstacle_features is None:
            obstacle_features = any(sc.meta.get("obstacle_features") for sc in scenes)
        # one row per (vertex, obstacle), plus one grasp row per vertex where grasps are
        # scheduled, plus up to SELF_MAX + EE_MAX self rows per vertex with self-collision
        # and 2 OFEAT_MAX box-feature rows with those on
        d.contact_cap = contact_cap or max(sc.n_verts * (sc.n_obs + (1 if sc.meta.get("grasp") else 0) +
                                                         (SELF_MAX + EE_MAX if self_collision else 0) +
                                                         (2 * OFEAT_MAX if obstacle_features else 0))
                                           for sc in scenes)
        d.self_collide = 1 if self_collision else 0
        d.obstacle_features = 1 if obstacle_features else 0
        d.solve = solve
        d.warm = warm
        d.lanes = lanes
        d.eager = 1 if eager else 0
        d.metric = metric
        d.lin_iters = lin_iters
        d.grouped_solve = grouped
        d.refine_steps = refine_steps
        d.local_threads = local_threads
        d.ncp_threads = ncp_threads
        d.split_k = split_k
        self.desc = d
        self._h = C.c_void_p()
        _check(lib().flash_scene_create(C.byref(d), C.byref(self._h)))
        self._keep = []
        for sc in scenes:
            rest = np.ascontiguousarray(sc.rest, np.float64)
            el = np.ascontiguousarray(sc.elems, np.int32)
            if el.size == 0:
                el = np.zeros((1, 3 if sc.elem_type == 0 else 4), np.int32)
            mass = np.ascontiguousarray(sc.mass, np.float64)
            self._keep += [rest, el, mass]
            m = MeshDesc(sc.elem_type, sc.n_verts, len(sc.elems), rest.ctypes.data_as(C.POINTER(C.c_double)),
                         el.ctypes.data_as(C.POINTER(C.c_int32)), mass.ctypes.data_as(C.POINTER(C.c_double)),
                         sc.w_stretch, sc.w_bend, sc.thickness)
            mid = C.c_int32()
            _check(lib().flash_mesh_add(self._h, C.byref(m), C.byref(mid)))
            envs = (EnvDesc * sc.n_envs)()
            for e in range(sc.n_envs):
                ed = envs[e]
                ed.mu = float(sc.mu[e])
                ed.stiffness = float(sc.stiff[e])
                ed.n_obs = sc.n_obs
                for o in range(sc.n_obs):
                    ed.obs_type[o] = int(sc.obs_type[e, o])
                    ed.obs_compliance[o] = float(sc.obs_comp[e, o])
                    for c in range(3):
                        ed.obs_dims[o][c] = float(sc.obs_dims[e, o, c])
            first = C.c_int32()
            _check(lib().flash_envs_add(self._h, mid, sc.n_envs, envs, C.byref(first)))
        _check(lib().flash_scene_finalize(self._h, _stream()))
        self.n_envs = lib().flash_num_envs(self._h)
        self.n_verts = lib().flash_num_verts(self._h)
        off = (C.c_int64 * (self.n_envs + 1))()
        _check(lib().flash_env_offsets(self._h, off))
        self.offsets = np.array(off[:], np.int64)
        self.cap = lib().flash_contact_cap(self._h)
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.step_index = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().flash_scene_destroy(h)
            self._h = None

    # ------------------------------------------------------------ state
    def set_state(self, q=None, v=None):
        """q, v: float32 tensors [n_verts, 3] on the device (either may be None)."""
        for t in (q, v):
            if t is not None:
                assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.shape == (self.n_verts, 3)
        _check(lib().flash_set_state(self._h, _ptr(q), _ptr(v), _stream()))

    def get_state(self):
        q = torch.empty((self.n_verts, 3), dtype=torch.float32, device=self.dev)
        v = torch.empty_like(q)
        _check(lib().flash_get_state(self._h, _ptr(q), _ptr(v), _stream()))
        return q, v

    def set_poses(self, poses, which=1):
        """poses: float32 [n_envs, 8, 7] device tensor (target pose of the next step)."""
        assert poses.is_cuda and poses.dtype == torch.float32 and poses.shape == (self.n_envs, MAX_OBS, 7)
        poses = poses.contiguous()
        _check(lib().flash_set_obstacle_poses(self._h, _ptr(poses), which, _stream()))

    def step(self, n=1):
        _check(lib().flash_step(self._h, n, _stream()))
        self.step_index += n

    def grasp(self, request, obstacle, anchor=(0.0, 0.0, 0.0), radius=0.0, first_env=0):
        """Grasp requests for environments [first_env, first_env + len(request)):
        1 activates (vertices within ``radius`` of ``anchor`` on obstacle
        ``obstacle`` at the start of the next step), 0 releases, -1 keeps."""
        req = np.ascontiguousarray(np.atleast_1d(request), np.int32)
        an = np.ascontiguousarray(anchor, np.float32)
        _check(lib().flash_grasp(self._h, first_env, len(req), req.ctypes.data_as(C.POINTER(C.c_int32)), obstacle,
                                 an.ctypes.data_as(C.POINTER(C.c_float)), float(radius), _stream()))

    def apply_grasp_schedule(self, step):
        """Issue the grasp requests that the scenes' schedules (meta["grasp"])
        hold for the start of step ``step``."""
        first = 0
        for sc in self.scenes:
            g = sc.meta.get("grasp")
            if g and step in g["schedule"]:
                self.grasp(np.full(sc.n_envs, g["schedule"][step], np.int32), g["obstacle"], g["anchor"],
                           g["radius"], first)
            first += sc.n_envs

    def render(self, cam, cam_poses, seg=True, points=True):
        """Ray cast every environment from its current state (flash_render):
        cam a Camera, cam_poses CUDA float32 [N][7] camera-to-world.  Returns
        depth [N][H][W] (0: no hit), seg uint8 [N][H][W] (0 none, 1 mesh, 2 + k
        obstacle k) and world points [N][H][W][3] (NaN: no hit), or None for
        the outputs not asked for."""
        assert cam_poses.is_cuda and cam_poses.dtype == torch.float32 and cam_poses.shape == (self.n_envs, 7)
        cam_poses = cam_poses.contiguous()
        H, W = cam.height, cam.width
        depth = torch.empty((self.n_envs, H, W), dtype=torch.float32, device=self.dev)
        sg = torch.empty((self.n_envs, H, W), dtype=torch.uint8, device=self.dev) if seg else None
        pt = torch.empty((self.n_envs, H, W, 3), dtype=torch.float32, device=self.dev) if points else None
        _check(lib().flash_render(self._h, C.byref(cam), _ptr(cam_poses), _ptr(depth), _ptr(sg), _ptr(pt),
                                  _stream()))
        return depth, sg, pt

    def contacts(self):
        cnt = torch.empty(self.n_envs, dtype=torch.int32, device=self.dev)
        vert = torch.empty((self.n_envs, self.cap), dtype=torch.int32, device=self.dev)
        obs = torch.empty_like(vert)
        gam = torch.empty((self.n_envs, self.cap, 4), dtype=torch.float32, device=self.dev)
        _check(lib().flash_get_contacts(self._h, _ptr(cnt), _ptr(vert), _ptr(obs), _ptr(gam), _stream()))
        return cnt, vert, obs, gam

    def contact_tris(self):
        """Feature of each row of the last step's contact lists, [N][cap]:
        the triangle of a vertex-triangle row, e1 * n_edges + e2 of an
        edge-edge row (unique edges (a < b) in (a, b) order), -1 otherwise."""
        tri = torch.empty((self.n_envs, self.cap), dtype=torch.int32, device=self.dev)
        _check(lib().flash_get_contact_tris(self._h, _ptr(tri), _stream()))
        return tri

    def stats(self):
        it = torch.empty(self.n_envs, dtype=torch.int32, device=self.dev)
        r = torch.empty(self.n_envs, dtype=torch.float32, device=self.dev)
        _check(lib().flash_get_stats(self._h, _ptr(it), _ptr(r), _stream()))
        return it, r

    def status(self):
        return _check(lib().flash_status_word(self._h, _stream()))

    KINDS = ("begin", "local", "solve", "ncp", "end", "warm")

    def profile(self, enable=True):
        """Bracket every launch with CUDA events on the launching stream."""
        _check(lib().flash_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self):
        """{kind: (total device ms, launches)} since the last profile() call."""
        out = {}
        for k, name in enumerate(self.KINDS):
            ms, n = C.c_double(), C.c_int64()
            _check(lib().flash_profile_read(self._h, k, C.byref(ms), C.byref(n)))
            out[name] = (ms.value, n.value)
        return out

    def launch_count(self):
        return lib().flash_launch_count(self._h)

    def lane_count(self):
        return lib().flash_lane_count(self._h)

    def grouped_solve(self):
        """True if the lanes apply their dense inverses in one grouped launch."""
        return bool(lib().flash_grouped_solve(self._h))

    def threads(self):
        """Threads per environment in use: (local pass, one per batch lane by
        lane; lite NCP pass, one per lane)."""
        out = []
        for kind in (0, 1):
            n = lib().flash_scene_threads(self._h, kind, None, 0)
            buf = (C.c_int32 * max(n, 1))()
            lib().flash_scene_threads(self._h, kind, buf, n)
            out.append(list(buf[:n]))
        return tuple(out)

    def tile_widths(self):
        """Autotuned tensor-core tile width of each lane's column range."""
        n = lib().flash_tile_widths(self._h, None, 0)
        out = (C.c_int32 * max(n, 1))()
        lib().flash_tile_widths(self._h, out, n)
        return list(out[:n])

    def tile_splits(self):
        """Per lane column range: 2 where each tile's K halves run on two CTAs."""
        n = lib().flash_tile_splits(self._h, None, 0)
        out = (C.c_int32 * max(n, 1))()
        lib().flash_tile_splits(self._h, out, n)
        return list(out[:n])

    def warmstart(self, params=None, mode=WARM_LEARNED, use_dq=False, normal_only=False, bounds=None):
        """Select the warm start; ``params`` (device float32, flat) is copied.
        ``bounds`` = (lo[10], hi[10]): the trained input range; contacts
        outside it start cold."""
        flags = (1 if use_dq else 0) | (2 if normal_only else 0)
        _check(lib().flash_warmstart_set(self._h, _ptr(params), mode, flags))
        if bounds is not None:
            lo = np.ascontiguousarray(np.asarray(bounds[0], np.float32).reshape(10))
            hi = np.ascontiguousarray(np.asarray(bounds[1], np.float32).reshape(10))
            fp = C.POINTER(C.c_float)
            _check(lib().flash_warmstart_bounds(self._h, lo.ctypes.data_as(fp), hi.ctypes.data_as(fp)))

    def record(self, enable=True):
        _check(lib().flash_record_contacts(self._h, 1 if enable else 0))

    def recorded(self):
        """(features [rows][10], targets [rows][6]) of the last step."""
        rows = C.c_int64()
        _check(lib().flash_get_recorded(self._h, None, None, 0, C.byref(rows), _stream()))
        X = torch.empty((rows.value, 10), dtype=torch.float32, device=self.dev)
        T = torch.empty((rows.value, 6), dtype=torch.float32, device=self.dev)
        if rows.value:
            _check(lib().flash_get_recorded(self._h, _ptr(X), _ptr(T), rows.value, C.byref(rows), _stream()))
        return X, T

    def global_apply(self, first_env, n, rhs):
        out = torch.empty_like(rhs)
        _check(lib().flash_global_apply(self._h, first_env, n, _ptr(rhs), _ptr(out), _stream()))
        return out


def poses_tensor(scenes, step, device):
    """[N, 8, 7] float32 device tensor of the obstacle poses at the start of ``step``."""
    if isinstance(scenes, _sc.Scene):
        scenes = [scenes]
    parts = []
    for sc in scenes:
        p = np.zeros((sc.n_envs, MAX_OBS, 7), np.float32)
        p[:, :, 3] = 1.0
        p[:, : sc.n_obs] = sc.poses[:, min(step, sc.poses.shape[1] - 1)]
        parts.append(p)
    return torch.from_numpy(np.concatenate(parts)).to(device)


def state_tensors(scenes, device):
    if isinstance(scenes, _sc.Scene):
        scenes = [scenes]
    q = np.concatenate([sc.q0.reshape(-1, 3) for sc in scenes]).astype(np.float32)
    v = np.concatenate([sc.v0.reshape(-1, 3) for sc in scenes]).astype(np.float32)
    return torch.from_numpy(q).to(device), torch.from_numpy(v).to(device)


# ------------------------------------------------------------------ network
def mlp_num_params():
    return lib().flash_mlp_num_params()


def mlp_forward(params, x):
    y = torch.empty((x.shape[0], 6), dtype=torch.float32, device=x.device)
    _check(lib().flash_mlp_forward(_ptr(params), _ptr(x), _ptr(y), x.shape[0], _stream()))
    return y


def mlp_loss_grad(params, x, t, work=None):
    """(sum of squared errors [device scalar], gradient of the mean 0.5-loss)."""
    rows = x.shape[0]
    if work is None or work.numel() < lib().flash_mlp_work_floats(rows):
        work = torch.empty(lib().flash_mlp_work_floats(rows), dtype=torch.float32, device=x.device)
    grad = torch.empty_like(params)
    sse = torch.empty(1, dtype=torch.float32, device=x.device)
    _check(lib().flash_mlp_loss_grad(_ptr(params), _ptr(x), _ptr(t), rows, _ptr(grad), _ptr(sse), _ptr(work),
                                     _stream()))
    return sse, grad


def mlp_adam(params, grad, m, v, step, lr):
    _check(lib().flash_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), step, lr, _stream()))


class Raycaster:
    """Standalone batched ray caster (flash_raycaster_*): N environments that
    share one triangle mesh ``tris`` [T][3] over ``n_verts`` vertices."""

    def __init__(self, cam, n_envs, n_verts, tris):
        tris = np.ascontiguousarray(np.asarray(tris, np.int32).reshape(-1, 3))
        self.cam, self.n_envs, self.n_verts = cam, n_envs, n_verts
        self._h = C.c_void_p()
        _check(lib().flash_raycaster_create(C.byref(cam), n_envs, n_verts, len(tris),
                                            tris.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(self._h)))
        self.dev = torch.device("cuda", torch.cuda.current_device())

    def __del__(self):
        if getattr(self, "_h", None):
            lib().flash_raycaster_destroy(self._h)
            self._h = None

    def cast(self, verts, obs_type, obs_dims, obs_poses, cam_poses, seg=True, points=True, out=None):
        """verts CUDA float32 [N][n][3]; obs_type int32 [N][K], obs_dims [N][K][3],
        obs_poses [N][K][7] (K may be 0); cam_poses [N][7].  Returns (depth,
        seg, points) like Sim.render; ``out`` reuses a previous result's
        tensors."""
        N, H, W = self.n_envs, self.cam.height, self.cam.width
        K = 0 if obs_type is None else obs_type.shape[1]
        if out is None:
            depth = torch.empty((N, H, W), dtype=torch.float32, device=self.dev)
            sg = torch.empty((N, H, W), dtype=torch.uint8, device=self.dev) if seg else None
            pt = torch.empty((N, H, W, 3), dtype=torch.float32, device=self.dev) if points else None
        else:
            depth, sg, pt = out
        _check(lib().flash_raycast(self._h, _ptr(verts), K, _ptr(obs_type) if K else None,
                                   _ptr(obs_dims) if K else None, _ptr(obs_poses) if K else None, _ptr(cam_poses),
                                   _ptr(depth), _ptr(sg), _ptr(pt), _stream()))
        return depth, sg, pt

    def profile(self, enable=True):
        """Bracket the two kernels of every later cast with CUDA events."""
        _check(lib().flash_raycaster_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """{"tri": (ms, launches), "resolve": (ms, launches)} since profile()."""
        ms, n = (C.c_double * 2)(), (C.c_int64 * 2)()
        _check(lib().flash_raycaster_profile_read(self._h, ms, n))
        return {"tri": (ms[0], n[0]), "resolve": (ms[1], n[1])}
