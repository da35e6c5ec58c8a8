"""Warm-start network kernels against the FP64 oracle, through the C ABI.

The GPU rounds weights to bf16 and accumulates in FP32, so the oracle is
evaluated on the same bf16-rounded weights (biases stay FP32); what remains
is FP32 vs FP64 accumulation."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def bf16_round(x):
    a = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def _params(seed):
    from paper_2604_17513_gb300 import warmstart
    return warmstart.init_params(seed).cpu().numpy()


def _oracle_params(p):
    q = bf16_round(p)
    nh, ni, no = 128, 10, 6
    o_b1 = nh * ni
    o_b2 = o_b1 + nh + nh * nh
    o_b3 = o_b2 + nh + no * nh
    for lo, hi in ((o_b1, o_b1 + nh), (o_b2, o_b2 + nh), (o_b3, o_b3 + no)):
        q[lo:hi] = p[lo:hi]
    return q


def test_mlp_forward_matches_oracle(cuda):
    import torch
    from paper_2604_17513_gb300 import flash
    p = _params(3)
    p[1280:1408] = np.random.default_rng(1).normal(size=128) * 0.1   # nonzero biases
    x = np.random.default_rng(2).normal(size=(1000, 10)).astype(np.float32)
    y = flash.mlp_forward(torch.from_numpy(p).to(cuda), torch.from_numpy(x).to(cuda)).cpu().numpy()
    ref = oracle.mlp_forward(_oracle_params(p), x.astype(np.float64))
    assert np.abs(y - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())


def test_mlp_gradient_matches_oracle(cuda):
    import torch
    from paper_2604_17513_gb300 import flash
    p = _params(4)
    rng = np.random.default_rng(5)
    x = rng.normal(size=(777, 10)).astype(np.float32)
    t = rng.normal(size=(777, 6)).astype(np.float32)
    sse, g = flash.mlp_loss_grad(torch.from_numpy(p).to(cuda), torch.from_numpy(x).to(cuda),
                                 torch.from_numpy(t).to(cuda))
    loss_ref, g_ref = oracle.mlp_loss_grad(_oracle_params(p), x.astype(np.float64), t.astype(np.float64))
    assert abs(0.5 * sse.item() / 777 - loss_ref) <= 1e-5 * loss_ref
    g = g.cpu().numpy()
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()


def test_adam_decreases_loss(cuda):
    """A few hundred Adam steps of the GPU training loop fit a smooth target."""
    import torch
    from paper_2604_17513_gb300 import warmstart
    rng = np.random.default_rng(7)
    x = rng.normal(size=(8192, 10)).astype(np.float32)
    t = np.stack([np.sin(x[:, 0]), x[:, 1] * x[:, 2], np.tanh(x[:, 3]), x[:, 4], 0.5 * x[:, 5], np.cos(x[:, 6])], 1)
    X, T = torch.from_numpy(x).to(cuda), torch.from_numpy(t.astype(np.float32)).to(cuda)
    _, hist, held = warmstart.train(X, T, epochs=30, batch=512, lr=2e-3)
    assert hist[-1] < 0.2 * hist[0] and held < 2 * hist[-1]


def test_learned_warm_start_gain(cuda):
    """Train on the simulator's own converged steps (tolerance mode), then on
    held-out rows inside the trained input range (the rows the library's gate
    lets through) compare the initial multipliers with the converged ones:
    the network's prediction must beat the cold start (zero) and the previous
    step's multipliers.  With the learned start the plain iteration still runs
    to the same residual."""
    import torch
    from paper_2604_17513_gb300 import flash, scenes, warmstart
    sc = scenes.cloth_gripper(n_envs=64, n_side=16, side=0.25, steps=80)
    sim = flash.Sim(sc, solve=flash.SOLVE_F16X3, mode=flash.MODE_TOL, k_cap=60, tol=1e-5)
    q, v = flash.state_tensors(sc, cuda)
    sim.set_state(q, v)
    sim.set_poses(flash.poses_tensor(sc, 0, cuda), which=0)
    for s in range(5):
        sim.set_poses(flash.poses_tensor(sc, s + 1, cuda))
        sim.step(1)
    X, T = warmstart.collect(sim, sc, 5, 45, cuda)
    p, hist, _ = warmstart.train(X, T, epochs=6, batch=2048, lr=1e-3)
    lo, hi = warmstart.input_range(X, T)
    assert hist[-1] < hist[0]
    Xh, Th = warmstart.collect(sim, sc, 50, 10, cuda)       # later steps: held out
    Xh, Th = warmstart.usable(Xh, Th)
    keep = warmstart.in_range(Xh, lo, hi)
    assert keep.float().mean().item() > 0.9
    Xh, Th = Xh[keep].contiguous(), Th[keep].contiguous()
    pred = flash.mlp_forward(p, Xh)
    err = lambda y: ((y[:, :3] - Th[:, :3]) ** 2).sum(1).mean().item()
    e_learned = err(pred)
    e_cold = err(torch.zeros_like(pred))
    e_prev = err(torch.cat([Xh[:, 7:10], Xh[:, 7:10]], 1))
    assert e_learned < e_cold and e_learned < e_prev, (e_learned, e_cold, e_prev)
    # same residual target with the learned start (the plain iteration decides)
    sim.warmstart(p, flash.WARM_LEARNED, bounds=(lo, hi))
    conv = []
    for s in range(60, 70):
        sim.set_poses(flash.poses_tensor(sc, s + 1, cuda))
        sim.step(1)
        it, r = sim.stats()
        conv.append(((r <= 1e-5) | (it >= 60)).all().item())
    assert all(conv) and sim.status() == 0


def test_learned_and_recording_steps_replay_from_the_graph(cuda):
    """With the learned warm start (a fixed random network, default input
    range) and contact recording on, steps replayed from the captured graph
    (tolerance mode, loop on the device, two lanes) give bit-identical
    states, multipliers, iteration counts and recorded rows to steps
    launched kernel by kernel."""
    import torch
    from paper_2604_17513_gb300 import flash, scenes, warmstart
    sc = scenes.cloth_gripper(n_envs=130, n_side=16, side=0.25, steps=30)
    p = (warmstart.init_params(3) * 0.01).to(cuda)   # small predictions: the iteration stays well inside its range
    out = []
    for eager in (True, False):
        sim = flash.Sim(sc, solve=flash.SOLVE_F16X3, mode=flash.MODE_TOL, k_cap=20, tol=1e-5, lanes=2, eager=eager)
        q, v = flash.state_tensors(sc, cuda)
        sim.set_state(q, v)
        sim.set_poses(flash.poses_tensor(sc, 0, cuda), which=0)
        sim.warmstart(p, flash.WARM_LEARNED)
        sim.record(True)
        rec = []
        for s in range(12):
            sim.set_poses(flash.poses_tensor(sc, s + 1, cuda))
            sim.step(1)
            X, T = sim.recorded()
            rec.append((X.cpu().numpy(), T.cpu().numpy()))
        it, r = sim.stats()
        cnt, vert, obs, gam = sim.contacts()
        out.append((sim.get_state()[0].cpu().numpy(), gam.cpu().numpy(), it.cpu().numpy(), rec, sim.status()))
    (qe, ge, ie, re, se), (qg, gg, ig, rg, sg) = out
    assert se == 0 and sg == 0
    assert np.array_equal(qe, qg) and np.array_equal(ge, gg) and np.array_equal(ie, ig)
    # targets of environments that did not converge are NaN rows in both (no target)
    assert all(np.array_equal(a[0], b[0], equal_nan=True) and np.array_equal(a[1], b[1], equal_nan=True)
               for a, b in zip(re, rg))
    assert sum(len(a[0]) for a in re) > 1000
