"""Shared checks of the GPU parity tests: contact lists and contact impulses.

The contact impulse of a row is gamma / h (N s), gamma = (gamma_n, gamma_t
world x, y, z); the GPU and the oracle store the same four numbers per row.
Rows are matched by (vertex, obstacle slot, feature): the lists of both sides
are sorted by (vertex, slot) with the feature order inside a slot, so a
matching list is the same sequence of keys.

Impulse error of an environment: the normwise relative error
    max_j |gamma_gpu,j - gamma_oracle,j|_inf / max_j |gamma_oracle,j|_inf,
the usual relative error of a vector quantity (an environment's impulses are
one vector; rows that carry no load have no relative error of their own).
"""
import numpy as np

IMPULSE_REL_TOL = 1e-4   # the contact-impulse tolerance the parity tests state


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


def impulse_error(contacts, e, ref):
    """(lists equal, normwise relative impulse error) of environment e of the
    GPU lists against the oracle's EnvState ``ref``."""
    v, o, f, g = env_rows(contacts, e)
    rf = ref.ctri if len(ref.ctri) == len(ref.cvert) else np.full(len(ref.cvert), -1)
    same = (len(v) == len(ref.cvert) and np.array_equal(v, ref.cvert) and np.array_equal(o, ref.cobs)
            and np.array_equal(f, rf))
    if not same:
        return False, np.inf
    if len(v) == 0:
        return True, 0.0
    scale = np.abs(ref.gamma).max()
    if scale == 0.0:
        return True, float(np.abs(g).max())
    return True, float(np.abs(g - ref.gamma).max() / scale)


def assert_impulses(contacts, e, ref, tol=IMPULSE_REL_TOL, what=""):
    same, err = impulse_error(contacts, e, ref)
    assert same, f"{what} env {e}: contact lists differ"
    assert err <= tol, f"{what} env {e}: impulse relative error {err:.3g} > {tol:g}"
    return err
