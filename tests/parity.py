"""Shared checks of the GPU parity tests: contact lists and contact impulses.

A contact row stores gamma = (gamma_n, gamma_t as a world vector), gamma =
h^2 lambda (kg m); its impulse is gamma / h.  The GPU and the oracle store
the same four numbers per row and sort a list by (vertex, obstacle slot),
with the feature order inside a slot, so matching lists are the same
sequence of (vertex, slot, feature) keys: the lists must be identical.

Impulses.  The tolerance is 1e-4 relative to the environment's largest
impulse, |d gamma| <= 1e-4 |gamma|_inf, with two additions that come from
what FP32 states can resolve, and with what is not unique compared as a
total:

  * Compliant rows (normal compliance c > 0): the compliance law fixes
    lambda_n = -gap / c, so a position error dq allows
    |d gamma_n| <= h^2 dq / c (and mu times that on the friction that the
    normal force bounds).  dq is the step's measured max vertex error.
  * FP32 force resolution: a resting cloth vertex's friction (and the
    elastic part of its normal force) balances stretch forces computed from
    FP32 deformation gradients, |dF| ~ 2^-23, which carry about
    h^2 sum_tri w A |D| 2^-23 ~ 1e-2 m_v g h^2 for these cloths (measured up
    to 4e-2 m_v g h^2 on a 64x64 cloth); 0.1 m_v g h^2 per row is added.
  * Several obstacle rows on one vertex (a point squeezed between a finger
    and the ground, a particle in a corner) can trade load along directions
    in which they cancel (a squeeze pair, two sticking rows sharing one
    tangential load): the positions do not see the trade, and FP32 and FP64
    iterates settle at different members of that family.  The unique
    quantity is the vertex's total contact force sum_rows (n gamma_n +
    gamma_t), compared with the sum of its rows' allowances.  n is the
    oracle's normal at the oracle's end state on both sides, so only the
    multipliers are compared.
Rows alone on their vertex, grasp, self and box-feature rows are compared
row by row (all four stored numbers).

Ill-conditioned steps.  Where a step amplifies the rounding of its input
(intermediate iterates of the full metric's inexact GMRES Newton steps,
strips balanced on a crossing), the oracle itself moves when its input is
rounded differently.  ``oracle_spread`` measures that: it reruns the
oracle's step from the same state with every coordinate moved by one FP32
ulp (random sign) and returns the largest position move and, per row, the
largest multiplier move.  Tests of such steps add twice the measured spread
to the allowances: the GPU may differ from the oracle by no more than the
oracle differs from itself under FP32 rounding of its input.
"""
import numpy as np

import oracle

IMPULSE_REL_TOL = 1e-4
FP32_FORCE_FLOOR = 0.1   # in units of the row vertex's weight impulse m_v g h^2
MAX_OBS = 8


def gpu_contacts(sim):
    """Host copies of the last step's lists: count [N], vert, obs, feature
    [N][cap], gamma [N][cap][4]."""
    import torch
    cnt, vert, obs, gam = sim.contacts()
    feat = sim.contact_tris()
    torch.cuda.synchronize()
    return cnt.cpu().numpy(), vert.cpu().numpy(), obs.cpu().numpy(), feat.cpu().numpy(), gam.cpu().numpy()


def env_rows(contacts, e):
    cnt, vert, obs, feat, gam = contacts
    c = int(cnt[e])
    return vert[e, :c], obs[e, :c], feat[e, :c], gam[e, :c].astype(np.float64)


def ulp_perturbed(x, rng, ulps=1):
    """x rounded to FP32, then every entry moved by ``ulps`` ulps up or down."""
    x32 = np.asarray(x, np.float32)
    up = rng.integers(0, 2, size=x32.shape).astype(bool)
    to = np.where(up, np.inf, -np.inf).astype(np.float32)
    for _ in range(ulps):
        x32 = np.nextafter(x32, to)
    return x32.astype(np.float64)


def oracle_spread(step_fn, q0, v0, ref, trials=3, seed=0, ulps=1):
    """(max position move, per-row max multiplier move [rows][4]) of the
    oracle's step ``step_fn(q, v) -> EnvState`` under FP32 noise of ``ulps``
    ulps on (q0, v0), against its unperturbed result ``ref``; trials whose
    contact list differs from ref's are skipped.  A GPU step of k iterations
    rounds its state in FP32 k times; as a random walk that is about sqrt(k)
    ulps, the ``ulps`` a test of a k-iteration step passes."""
    rng = np.random.default_rng(seed)
    dq, dg = 0.0, np.zeros_like(ref.gamma)
    for _ in range(trials):
        b = step_fn(ulp_perturbed(q0, rng, ulps), ulp_perturbed(v0, rng, ulps))
        dq = max(dq, float(np.abs(b.q - ref.q).max()))
        if np.array_equal(b.cvert, ref.cvert) and np.array_equal(b.cobs, ref.cobs):
            dg = np.maximum(dg, np.abs(b.gamma - ref.gamma))
    return dq, dg


def impulse_check(contacts, e, ref, sc, le, s, dq, spread=None):
    """Environment e of the GPU lists against the oracle's EnvState ``ref``
    of environment le of scene ``sc`` after the step that started at step
    index s, with the step's max vertex error dq (m).  Returns (lists equal,
    worst ratio error / allowance over the compared quantities; <= 1
    passes)."""
    v, o, f, g = env_rows(contacts, e)
    rf = ref.ctri if len(ref.ctri) == len(ref.cvert) else np.full(len(ref.cvert), -1)
    same = (len(v) == len(ref.cvert) and np.array_equal(v, ref.cvert) and np.array_equal(o, ref.cobs)
            and np.array_equal(f, rf))
    if not same:
        return False, np.inf
    if len(v) == 0:
        return True, 0.0
    G = ref.gamma
    h2, grav = sc.h ** 2, float(np.linalg.norm(sc.gravity))
    base = IMPULSE_REL_TOL * np.abs(G).max()
    obs_row = o < MAX_OBS
    nrows = {}
    for vv in v[obs_row]:
        nrows[int(vv)] = nrows.get(int(vv), 0) + 1
    worst = 0.0
    tot_o, tot_g, tot_tol = {}, {}, {}
    for j in range(len(v)):
        vv = int(v[j])
        floor = FP32_FORCE_FLOOR * sc.mass[vv] * grav * h2
        comp = float(sc.obs_comp[le, o[j]]) if obs_row[j] else 0.0
        allow_n = base + floor + (h2 * dq / comp if comp > 0 else 0.0)
        allow_t = base + floor + (sc.mu[le] * h2 * dq / comp if comp > 0 else 0.0)
        if spread is not None:
            allow_n += 2.0 * spread[j, 0]
            allow_t += 2.0 * spread[j, 1:].max()
        if not obs_row[j] or nrows[vv] == 1:
            worst = max(worst, abs(g[j, 0] - G[j, 0]) / allow_n, np.abs(g[j, 1:] - G[j, 1:]).max() / allow_t)
            continue
        _, n = oracle.sdf(sc.obs_type[le, o[j]], sc.obs_dims[le, o[j]], sc.poses[le, s + 1, o[j]], ref.q[vv])
        tot_o[vv] = tot_o.get(vv, 0.0) + n * G[j, 0] + G[j, 1:]
        tot_g[vv] = tot_g.get(vv, 0.0) + n * g[j, 0] + g[j, 1:]
        tot_tol[vv] = tot_tol.get(vv, 0.0) + allow_n + allow_t
    for vv in tot_o:
        worst = max(worst, np.abs(tot_o[vv] - tot_g[vv]).max() / tot_tol[vv])
    return True, float(worst)


def assert_impulses(contacts, e, ref, sc, le, s, dq, what="", spread=None):
    same, worst = impulse_check(contacts, e, ref, sc, le, s, dq, spread)
    assert same, f"{what} env {e}: contact lists differ"
    assert worst <= 1.0, f"{what} env {e}: impulse error {worst:.3g} x its allowance"
    return worst
