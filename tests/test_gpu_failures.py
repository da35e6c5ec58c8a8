"""Failure paths of the step, injected on the host (no GPU fault, no trap).

The kernels never trap: a device-side problem sets a bit of the scene's
status word, and flash_status_word turns it into the documented code (with
flash_last_error naming the cause).  Here the problem is put into the
inputs by the host: a NaN in one environment's state through
flash_set_state, a contact capacity smaller than the scene needs, a vertex
with more contacts than the lite metric's per-vertex block.  The resume test
checks that flash_get_state / flash_set_state / flash_set_obstacle_poses
carry everything a cold-started step depends on: a rollout interrupted and
resumed from its checkpoint is bit-identical to the uninterrupted one.  The
checked build (libflash_check.so, every index a step kernel reads
range-checked) is loaded in a child process: it steps like the regular
build, and an element index corrupted on the host through its test hook is
reported as FLASH_EINDEX instead of being dereferenced.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2604_17513_gb300 import scenes

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _state(sim, sc, q, v, s):
    import torch
    from paper_2604_17513_gb300 import flash
    sim.set_state(torch.from_numpy(np.asarray(q, np.float32).reshape(-1, 3)).to(sim.dev),
                  torch.from_numpy(np.asarray(v, np.float32).reshape(-1, 3)).to(sim.dev))
    sim.set_poses(flash.poses_tensor(sc, s, sim.dev), which=0)


def _steps(sim, sc, s0, n):
    from paper_2604_17513_gb300 import flash
    for s in range(s0, s0 + n):
        sim.set_poses(flash.poses_tensor(sc, s + 1, sim.dev), which=1)
        sim.step(1)


@pytest.mark.parametrize("solve", [0, 1])
def test_nan_state_reports_enumeric_and_spares_other_envs(cuda, solve):
    """A NaN position in environment 1 (of 3): the status word reports
    FLASH_ENUMERIC, and environments 0 and 2 end bit-identical to a run
    without the NaN (environments share no data)."""
    import torch
    from paper_2604_17513_gb300 import flash
    sc = scenes.cloth_drop(n_envs=3, steps=40)
    s = 26
    outs = []
    for poison in (False, True):
        sim = flash.Sim(sc, solve=solve)
        q = sc.q0.copy() + np.array([0.0, 0.0, -0.3])
        if poison:
            q[1, 17, 2] = np.nan
        _state(sim, sc, q, sc.v0, s)
        assert sim.status() == flash.OK
        _steps(sim, sc, s, 2)
        qg, _ = sim.get_state()
        torch.cuda.synchronize()
        if poison:
            with pytest.raises(flash.FlashError) as ei:
                sim.status()
            assert ei.value.code == flash.ENUMERIC and "non-finite" in str(ei.value)
            # a clean state clears the word
            _state(sim, sc, sc.q0, sc.v0, s)
            assert sim.status() == flash.OK
        else:
            assert sim.status() == flash.OK
        outs.append(qg.cpu().numpy().reshape(3, sc.n_verts, 3))
    clean, poisoned = outs
    assert np.isfinite(clean).all() and not np.isfinite(poisoned[1]).all()
    assert np.array_equal(clean[0], poisoned[0]) and np.array_equal(clean[2], poisoned[2])


def test_contact_capacity_overflow_warns(cuda):
    """A contact capacity of 2 rows for a cloth touching the sphere with 4
    vertices: the rows past 2 are dropped and the status word reports
    FLASH_WOVERFLOW (a warning, > 0), naming the capacity; the same scene with
    the default capacity reports FLASH_OK."""
    import oracle
    from paper_2604_17513_gb300 import flash
    sc = scenes.cloth_drop(n_envs=1, steps=60)
    mesh = oracle.Mesh.from_scene(sc)
    st = oracle.EnvState(sc.q0[0], sc.v0[0])
    s = 40
    for k in range(s):
        oracle.step(mesh, sc, 0, k, st)
    nxt = oracle.EnvState(st.q, st.v)
    oracle.step(mesh, sc, 0, s, nxt)
    assert len(nxt.cvert) > 2
    for cap, want in ((2, flash.WOVERFLOW), (None, flash.OK)):
        sim = flash.Sim(sc, contact_cap=cap)
        _state(sim, sc, st.q[None], st.v[None], s)
        _steps(sim, sc, s, 1)
        assert sim.status() == want, cap
        cnt = sim.contacts()[0].cpu().numpy()
        if cap:
            assert cnt[0] == 2
            assert b"capacity" in flash.lib().flash_last_error()
        else:
            assert cnt[0] == len(nxt.cvert)


def _five_planes_particle(steps=3):
    """One particle 1 mm above the ground and four more planes through the
    origin, tilted by 0.1 rad about four horizontal axes: five obstacle rows
    on one vertex, one more than the lite metric's per-vertex block."""
    ang = 0.1
    poses = [scenes._pose((0, 0, 0))]
    for ax in ((1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0)):
        c, sn = np.cos(ang / 2), np.sin(ang / 2)
        poses.append(scenes._pose((0, 0, 0), (c, sn * ax[0], sn * ax[1], sn * ax[2])))
    P = np.array([[poses for _ in range(steps + 1)]], float)
    q0 = np.array([[[0.0, 0.0, 1e-3]]])
    return scenes.Scene("five_planes", scenes.TRI, np.zeros((1, 3)), np.zeros((0, 3), np.int32), np.array([0.01]),
                        0.0, 0.0, q0, np.zeros_like(q0), np.array([0.5]), np.ones(1),
                        np.full((1, 5), scenes.PLANE, np.int32), np.zeros((1, 5, 3)), np.zeros((1, 5)), P,
                        thickness=1e-3, steps=steps)


def test_too_many_contacts_on_one_vertex_warns(cuda):
    """Five rows on one vertex with the lite metric (blocks of at most four):
    FLASH_WOVERFLOW naming the per-vertex block; the full metric solves all
    rows jointly and reports FLASH_OK."""
    from paper_2604_17513_gb300 import flash
    sc = _five_planes_particle()
    for metric, want in ((flash.METRIC_LITE, flash.WOVERFLOW), (flash.METRIC_FULL, flash.OK)):
        sim = flash.Sim(sc, metric=metric)
        _state(sim, sc, sc.q0, sc.v0, 0)
        _steps(sim, sc, 0, 1)
        cnt = sim.contacts()[0].cpu().numpy()
        assert cnt[0] == 5
        assert sim.status() == want, metric
        if want == flash.WOVERFLOW:
            assert b"per-vertex" in flash.lib().flash_last_error()


@pytest.mark.parametrize("mode", ["fixed", "tol"])
def test_checkpoint_resume_is_bit_exact(cuda, mode):
    """Checkpoint (flash_get_state) after 3 steps of the gripper scene, 4 more
    steps; then restore the checkpoint (flash_set_state, obstacle poses of
    the checkpoint's step) in the same scene and in a new scene, and take the
    same 4 steps: positions and velocities are bit-identical (cold start: a
    step depends only on q, v and the obstacle poses)."""
    import torch
    from paper_2604_17513_gb300 import flash
    sc = scenes.cloth_gripper(n_envs=8, steps=20)
    kw = dict(mode=flash.MODE_TOL, k_cap=20) if mode == "tol" else dict(mode=flash.MODE_FIXED)
    sim = flash.Sim(sc, solve=flash.SOLVE_F16X3, **kw)
    _state(sim, sc, sc.q0, sc.v0, 0)
    _steps(sim, sc, 0, 3)
    q_ck, v_ck = (t.clone() for t in sim.get_state())
    _steps(sim, sc, 3, 4)
    q_ref, v_ref = (t.cpu().numpy() for t in sim.get_state())
    it_ref = sim.stats()[0].cpu().numpy()
    for target in (sim, flash.Sim(sc, solve=flash.SOLVE_F16X3, **kw)):
        target.set_state(q_ck, v_ck)
        target.set_poses(flash.poses_tensor(sc, 3, target.dev), which=0)
        _steps(target, sc, 3, 4)
        q, v = (t.cpu().numpy() for t in target.get_state())
        torch.cuda.synchronize()
        assert np.array_equal(q, q_ref) and np.array_equal(v, v_ref)
        assert np.array_equal(target.stats()[0].cpu().numpy(), it_ref)
        assert target.status() == flash.OK


_CHECKED_CHILD = r"""
import ctypes as C, json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
from paper_2604_17513_gb300 import flash, scenes
L = flash.lib()
assert L.flash_checked_build() == 1
dev = torch.device("cuda", 0)
out = {}
for name in ("tri", "tet"):
    sc = scenes.cloth_drop(n_envs=3, steps=12) if name == "tri" else scenes.tet_squeeze(n_envs=4, steps=12)
    sim = flash.Sim(sc, solve=flash.SOLVE_F16X3)
    q0, v0 = flash.state_tensors(sc, dev)
    sim.set_state(q0, v0)
    sim.set_poses(flash.poses_tensor(sc, 0, dev), which=0)
    for s in range(6):
        sim.set_poses(flash.poses_tensor(sc, s + 1, dev))
        sim.step(1)
    clean = L.flash_status_word(sim._h, None)
    q, v = (t.clone() for t in sim.get_state())
    old = C.c_int32(-1)
    poke = L.flash_check_poke_element(sim._h, 0, 5, 1, sc.n_verts + 7, C.byref(old))
    sim.set_poses(flash.poses_tensor(sc, 7, dev))
    sim.step(1)
    bad = L.flash_status_word(sim._h, None)
    msg = L.flash_last_error().decode()
    finite = bool(torch.isfinite(sim.get_state()[0]).all().item())
    back = L.flash_check_poke_element(sim._h, 0, 5, 1, old.value, None)
    sim.set_state(q, v)
    sim.set_poses(flash.poses_tensor(sc, 6, dev), which=0)
    sim.set_poses(flash.poses_tensor(sc, 7, dev))
    sim.step(1)
    again = L.flash_status_word(sim._h, None)
    out[name] = dict(clean=clean, poke=poke, old=old.value, bad=bad, msg=msg, finite=finite, back=back,
                     again=again, q=q.cpu().numpy().ravel().tolist())
print("RESULT" + json.dumps(out))
"""


def test_checked_build_steps_alike_and_reports_corrupted_index(cuda):
    """The checked build (child process, FLASH_CHECKED_BUILD=1): 6 steps of
    a cloth and of a tet scene report FLASH_OK and end within 1e-6 m of the
    regular build's; an element corner set to an index past the mesh
    through flash_check_poke_element makes the next step report
    FLASH_EINDEX (named in flash_last_error) with finite positions, and
    after the index is restored and the state reset the step is clean
    again.  The regular build refuses the hook (FLASH_ENOTIMPL)."""
    import ctypes as C
    import torch
    from paper_2604_17513_gb300 import flash
    lib = flash.lib()
    assert lib.flash_checked_build() == 0
    env = dict(os.environ, FLASH_CHECKED_BUILD="1")
    res = subprocess.run([sys.executable, "-c", _CHECKED_CHILD.replace("ROOT", repr(ROOT))], env=env,
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-3000:]
    line = [x for x in res.stdout.splitlines() if x.startswith("RESULT")][-1]
    out = json.loads(line[len("RESULT"):])
    for name in ("tri", "tet"):
        r = out[name]
        assert r["clean"] == flash.OK and r["poke"] == flash.OK and r["back"] == flash.OK, r
        assert 0 <= r["old"] and r["bad"] == flash.EINDEX and "index" in r["msg"] and r["finite"], r
        assert r["again"] == flash.OK, r
        sc = scenes.cloth_drop(n_envs=3, steps=12) if name == "tri" else scenes.tet_squeeze(n_envs=4, steps=12)
        sim = flash.Sim(sc, solve=flash.SOLVE_F16X3)
        q0, v0 = flash.state_tensors(sc, cuda)
        sim.set_state(q0, v0)
        sim.set_poses(flash.poses_tensor(sc, 0, cuda), which=0)
        for s in range(6):
            sim.set_poses(flash.poses_tensor(sc, s + 1, cuda))
            sim.step(1)
        q = sim.get_state()[0].cpu().numpy().ravel()
        assert np.abs(q - np.asarray(r["q"])).max() <= 1e-6, name
        old = C.c_int32(0)
        assert lib.flash_check_poke_element(sim._h, 0, 5, 1, 0, C.byref(old)) == flash.ENOTIMPL
        torch.cuda.synchronize()


def test_bounded_wait_runs_out_and_reports_timeout(cuda):
    """A bounded mbarrier wait that nothing completes (the solve's own wait
    routine, a 2e6-cycle limit, about 1 ms): the waiting thread gives up and
    sets the timeout bit, flash_status_word reports FLASH_ETIMEOUT naming
    the wait, flash_set_state clears it, and the context stays usable: the
    next steps are clean and equal a scene that never timed out."""
    import torch
    from paper_2604_17513_gb300 import flash
    sc = scenes.cloth_drop(n_envs=2, steps=12)
    qs = []
    for probe in (True, False):
        sim = flash.Sim(sc, solve=flash.SOLVE_F16X3)
        _state(sim, sc, sc.q0, sc.v0, 0)
        if probe:
            assert flash.lib().flash_test_bounded_wait(sim._h, 2_000_000, None) == flash.OK
            with pytest.raises(flash.FlashError) as ei:
                sim.status()
            assert ei.value.code == flash.ETIMEOUT and "bounded wait" in str(ei.value)
            assert flash.lib().flash_test_bounded_wait(sim._h, 0, None) == flash.EINVAL
            _state(sim, sc, sc.q0, sc.v0, 0)
            assert sim.status() == flash.OK
        _steps(sim, sc, 0, 3)
        assert sim.status() == flash.OK
        qs.append(sim.get_state()[0].cpu().numpy())
        torch.cuda.synchronize()
    assert np.array_equal(qs[0], qs[1])
