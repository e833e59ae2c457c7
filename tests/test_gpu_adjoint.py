"""GPU adjoint: collision VJP, per-channel |g|^2 gradients and RK4 trajectory
gradients, against the FP64 oracle's reverse mode and against central finite differences
of the GPU forward map (h = 1e-6, random directions)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2511_03683_gb300 as pb
    import torch

    assert torch.cuda.is_available()
    return pb


def T(x):
    import torch

    return torch.tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def nrel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("model", [synth.make_tiny(4), synth.make_window4(12), synth.make_config("tiny")],
                         ids=["tiny4", "win12", "tiny8"])
def test_collision_vjp_matches_oracle(pb, model):
    import torch

    ch = pb.Channels.from_model(model)
    dev = pb.Device(ch)
    o = oracle.Oracle(model)
    rng = np.random.default_rng(3)
    f = rng.uniform(0, 1, o.nstate)
    lam = rng.normal(size=o.nstate)
    gg2 = torch.zeros(dev.nchannels, dtype=torch.float64, device="cuda")
    g = dev.collision_vjp(T(f), T(lam), grad_g2=gg2).cpu().numpy()
    assert nrel(g, o.collision_vjp(f, lam)) <= 1e-11
    e = ch.export()
    rows = np.repeat(np.arange(ch.nstate), np.diff(e["row_ptr"]))
    pick = rng.choice(ch.nchannels, size=min(300, ch.nchannels), replace=False)
    ref = o.g2_grad(f, lam, rows[pick], e["col"][pick], e["nu"][pick])
    got = gg2.cpu().numpy()[pick]
    assert nrel(got, ref) <= 1e-11


def test_rk4_step_adjoint_matches_oracle(pb):
    m = synth.make_config("tiny")
    dev = pb.Device(pb.Channels.from_model(m))
    o = oracle.Oracle(m)
    f0 = o.window_values(m.f_hot())
    eps = o.window_values(m.eps)
    lam = T(eps)
    dev.rk4_vjp(T(f0), lam, 1.0)
    assert nrel(lam.cpu().numpy(), o.rk4_vjp(f0, 1.0, 1, eps)) <= 1e-11


def _oracle_rk4_g2_grad(o, f, lam, dt, s, p, nu):
    """dL/dg2 of one classic RK4 step from the oracle's collision, VJP and per-call |g|^2
    gradient: stage states u_j, stage cotangents g_j by the chain rule, then the sum over the
    four stages of g2_grad(u_j, g_j)."""
    k1 = o.collision(f)
    u2 = f + 0.5 * dt * k1
    u3 = f + 0.5 * dt * o.collision(u2)
    u4 = f + dt * o.collision(u3)
    g4 = dt / 6.0 * lam
    m4 = o.collision_vjp(u4, g4)
    g3 = dt / 3.0 * lam + dt * m4
    m3 = o.collision_vjp(u3, g3)
    g2 = dt / 3.0 * lam + 0.5 * dt * m3
    m2 = o.collision_vjp(u2, g2)
    g1 = dt / 6.0 * lam + 0.5 * dt * m2
    return sum(o.g2_grad(u, g, s, p, nu) for u, g in ((f, g1), (u2, g2), (u3, g3), (u4, g4)))


@pytest.mark.parametrize("opts,tol", [({}, 1e-11), ({"dense_rows": 2}, 1e-11), ({"merge_branches": 2}, 1e-11),
                                      ({"variant": "g32"}, 1e-5)],
                         ids=["merged-tiles", "merged-indexed", "per-channel", "g32"])
@pytest.mark.parametrize("model", [synth.make_window4(12), synth.make_tiny(4)], ids=["win12", "tiny4"])
def test_rk4_step_g2_gradient_matches_oracle(pb, model, opts, tol):
    """One RK4 step with grad_g2: the four stages' |g|^2 gradients accumulated in one pass over
    the channels, against the oracle's stage-by-stage sum; dL/df against the oracle adjoint."""
    import torch

    ch = pb.Channels.from_model(model)
    dev = pb.Device(ch, **opts)
    o = oracle.Oracle(model)
    rng = np.random.default_rng(7)
    f = rng.uniform(0, 1, o.nstate)
    lam0 = rng.normal(size=o.nstate)
    dt = 2.0
    gg2 = torch.zeros(dev.nchannels, dtype=torch.float64, device="cuda")
    lam = T(lam0)
    dev.rk4_vjp(T(f), lam, dt, grad_g2=gg2)
    assert nrel(lam.cpu().numpy(), o.rk4_vjp(f, dt, 1, lam0)) <= tol
    e = ch.export()
    rows = np.repeat(np.arange(ch.nstate), np.diff(e["row_ptr"]))
    pick = rng.choice(ch.nchannels, size=min(400, ch.nchannels), replace=False)
    ref = _oracle_rk4_g2_grad(o, f, lam0, dt, rows[pick], e["col"][pick], e["nu"][pick])
    err = nrel(gg2.cpu().numpy()[pick], ref)
    print(f"{opts} rk4 g2-gradient normwise error {err:.2e}")
    assert err <= tol


def _carrier_energy_grad(pb, model, nsteps, every):
    import torch
    from paper_2511_03683_gb300 import autograd as pa

    ch = pb.Channels.from_model(model)
    dev = pb.Device(ch)
    ids = ch.state_ids()
    f0 = torch.tensor(model.f_hot().reshape(-1)[ids], device="cuda", requires_grad=True)
    eps = torch.tensor(model.eps.reshape(-1)[ids], device="cuda")
    g2 = pa.g2_tensor(ch).requires_grad_(True)
    L = (eps * pa.trajectory(dev, f0, g2, 1.0, nsteps, every)).sum()
    L.backward()
    return ch, dev, f0, eps, g2, L


def test_trajectory_gradient_matches_oracle_adjoint(pb):
    """Short trajectory on the 8^3 workload: autograd gradient w.r.t. f0 == oracle adjoint."""
    m = synth.make_config("tiny")
    ch, dev, f0, eps, g2, L = _carrier_energy_grad(pb, m, nsteps=6, every=4)
    o = oracle.Oracle(m)
    ref = o.rk4_vjp(o.window_values(m.f_hot()), 1.0, 6, o.window_values(m.eps))
    assert nrel(f0.grad.cpu().numpy(), ref) <= 1e-10


def test_trajectory_at_given_couplings(pb):
    """trajectory() takes the couplings it is given: with every |g|^2 doubled (not yet on the
    device) the f0 gradient is the oracle adjoint of the model whose couplings are doubled
    (log-normal mean raised by ln 2), and the device then holds the doubled values."""
    import torch
    from paper_2511_03683_gb300 import autograd as pa

    m = synth.make_config("tiny")
    ch = pb.Channels.from_model(m)
    dev = pb.Device(ch)
    ids = ch.state_ids()
    f0 = torch.tensor(m.f_hot().reshape(-1)[ids], device="cuda", requires_grad=True)
    eps = torch.tensor(m.eps.reshape(-1)[ids], device="cuda")
    g2 = (2.0 * pa.g2_tensor(ch)).requires_grad_(True)
    (eps * pa.trajectory(dev, f0, g2, 1.0, 6, 4)).sum().backward()
    m2 = m.with_(g2_mu=m.g2_mu + np.log(2.0))
    o2 = oracle.Oracle(m2)
    ref = o2.rk4_vjp(o2.window_values(m2.f_hot()), 1.0, 6, o2.window_values(m2.eps))
    assert nrel(f0.grad.cpu().numpy(), ref) <= 1e-10
    assert torch.equal(dev.g2_values(), g2.detach())
    with pytest.raises(ValueError):
        pa.trajectory(dev, f0, g2[:-1], 1.0, 1, 1)


def test_trajectory_gradient_finite_differences_24cubed(pb):
    """The adjoint workload: 24^3 grids, 4 bands, 6 modes, loss = carrier energy after
    200 RK4 steps of 1 fs, checkpoints every 20 steps; 50 random directions in f0 and 5 in
    |g|^2, central differences with h = 1e-6."""
    import torch

    m = synth.make_config("window24")
    ch, dev, f0, eps, g2, L = _carrier_energy_grad(pb, m, nsteps=200, every=20)
    gf = f0.grad.detach()
    gg = g2.grad.detach()
    rng = np.random.default_rng(24)
    h = 1e-6

    fbuf = torch.empty_like(f0.detach())

    def loss(f_init):
        fbuf.copy_(f_init)  # one buffer: the RK4 graph is captured once
        dev.rk4(fbuf, 1.0, 200)
        return float((eps * fbuf).sum())

    base = f0.detach()
    worst = 0.0
    for _ in range(50):
        d = torch.tensor(rng.normal(size=dev.nstate), device="cuda") * base.abs().max()
        fd = (loss(base + h * d) - loss(base - h * d)) / (2 * h)
        an = float((gf * d).sum())
        worst = max(worst, abs(an - fd) / max(abs(fd), 1e-30))
    assert worst <= 1e-6, worst
    g2v = g2.detach().clone()
    worst = 0.0
    for _ in range(5):
        d = torch.tensor(rng.normal(size=dev.nchannels), device="cuda") * g2v
        vals = []
        for sgn in (1.0, -1.0):
            dev.set_g2(g2v + sgn * h * d)
            vals.append(loss(base))
        dev.set_g2(g2v)
        fd = (vals[0] - vals[1]) / (2 * h)
        an = float((gg * d).sum())
        worst = max(worst, abs(an - fd) / max(abs(fd), 1e-30))
    assert worst <= 1e-6, worst


# ------------------------------------------------------------------ FP32 adjoint (G32 variant)

@pytest.mark.parametrize("variant,vjp_tol", [("g32", 1e-5), ("h16", 1e-3)])
def test_fp32_collision_vjp_against_fp64_oracle(pb, variant, vjp_tol):
    """FP32 adjoint against the FP64 oracle; with FP16 |g|^2 (h16) the VJP carries the 2^-11
    rounding of |g|^2 while the |g|^2 gradient (whose bracket has no |g|^2) keeps FP32 accuracy."""
    import torch

    m = synth.make_window4(16)
    ch = pb.Channels.from_model(m)
    dev = pb.Device(ch, variant=variant)
    o = oracle.Oracle(m)
    rng = np.random.default_rng(31)
    f = rng.uniform(0, 1, o.nstate)
    lam = rng.normal(size=o.nstate)
    gg2 = torch.zeros(dev.nchannels, dtype=torch.float64, device="cuda")
    g = dev.collision_vjp(T(f), T(lam), grad_g2=gg2).cpu().numpy()
    err = nrel(g, o.collision_vjp(f, lam))
    print(f"{variant} vjp normwise error {err:.2e}")
    assert err <= vjp_tol
    e = ch.export()
    rows = np.repeat(np.arange(ch.nstate), np.diff(e["row_ptr"]))
    pick = rng.choice(ch.nchannels, size=500, replace=False)
    ref = o.g2_grad(f, lam, rows[pick], e["col"][pick], e["nu"][pick])
    err2 = nrel(gg2.cpu().numpy()[pick], ref)
    print(f"{variant} g2-gradient normwise error {err2:.2e}")
    assert err2 <= 1e-5


def test_fp32_trajectory_gradient_against_fp64(pb):
    """The adjoint workload in FP32 (G32): gradient of the carrier energy after 200 RK4 steps
    against the FP64-accurate (FF) gradient."""
    import torch
    from paper_2511_03683_gb300 import autograd as pa

    m = synth.make_config("window24")
    ch = pb.Channels.from_model(m)
    ids = ch.state_ids()
    eps = torch.tensor(m.eps.reshape(-1)[ids], device="cuda")
    grads = {}
    for v in ("ff", "g32"):
        dev = pb.Device(ch, variant=v)
        f0 = torch.tensor(m.f_hot().reshape(-1)[ids], device="cuda", requires_grad=True)
        g2 = pa.g2_tensor(ch).requires_grad_(True)
        (eps * pa.trajectory(dev, f0, g2, 1.0, 200, 20)).sum().backward()
        grads[v] = (f0.grad.cpu().numpy(), g2.grad.cpu().numpy())
        dev.close()
    ef = nrel(grads["g32"][0], grads["ff"][0])
    eg = nrel(grads["g32"][1], grads["ff"][1])
    print(f"fp32 trajectory gradient errors: f0 {ef:.2e}, g2 {eg:.2e}")
    assert ef <= 1e-4 and eg <= 1e-4


@pytest.mark.parametrize("opts,tol", [({}, 1e-12), ({"dense_rows": 2}, 1e-12), ({"variant": "g32"}, 1e-6),
                                      ({"variant": "g32", "channel_per_lane": 4}, 1e-6)],
                         ids=["merged-tiles", "merged-indexed", "g32-dense", "g32-lanes"])
def test_deferred_g2_gradient_matches_per_step(pb, opts, tol):
    """Three RK4 adjoint steps with the |g|^2 gradient deferred to per-pair accumulators and
    flushed once, against the same steps applying it to every channel per step: dL/df is the
    same arithmetic (bit-equal); dL/dg2 differs only in where the stage sums are rounded (FP32:
    the per-step form rounds each step's bracket to FP32, the deferred one forms it once in
    FP64).  A second flush adds nothing (the accumulators are cleared)."""
    import torch

    m = synth.make_window4(12)
    ch = pb.Channels.from_model(m)
    dev = pb.Device(ch, adjoint=True, **opts)
    assert dev.deferred
    rng = np.random.default_rng(11)
    fs = [T(rng.uniform(0, 1, dev.nstate)) for _ in range(3)]
    lam0 = rng.normal(size=dev.nstate)
    ref = torch.zeros(dev.nchannels, dtype=torch.float64, device="cuda")
    lam_ref = T(lam0)
    for f in fs:
        dev.rk4_vjp(f, lam_ref, 1.5, grad_g2=ref)
    got = torch.zeros_like(ref)
    lam = T(lam0)
    for f in fs:
        dev.rk4_vjp_defer(f, lam, 1.5)
    dev.g2grad_flush(got)
    assert torch.equal(lam, lam_ref)
    err = nrel(got.cpu().numpy(), ref.cpu().numpy())
    print(f"{opts} deferred g2-gradient normwise difference {err:.2e}")
    assert err <= tol
    again = got.clone()
    dev.g2grad_flush(again)
    assert torch.equal(again, got)


def test_deferred_trajectory_gradient_matches(pb):
    """autograd.trajectory on adjoint=True devices (deferred |g|^2 gradient) on the 8^3
    workload, 10 steps: dL/df0 bit-equal to the per-step form of the same variant; dL/dg2
    against the FF per-step gradient at the FP64 (1e-11) and FP32 (1e-4) trajectory bounds.
    This gradient is ill-conditioned (its terms cancel: the two FF forms differ by ~1e-12 here
    against ~5e-15 for three random steps), so the forms are compared with the FP64-accurate
    one rather than with each other."""
    import torch
    from paper_2511_03683_gb300 import autograd as pa

    m = synth.make_config("tiny")
    ch = pb.Channels.from_model(m)
    ids = ch.state_ids()
    eps = torch.tensor(m.eps.reshape(-1)[ids], device="cuda")
    out = {}
    for variant in ("ff", "g32"):
        for adj in (False, True):
            dev = pb.Device(ch, variant=variant, adjoint=adj)
            assert dev.deferred == adj
            f0 = torch.tensor(m.f_hot().reshape(-1)[ids], device="cuda", requires_grad=True)
            g2 = pa.g2_tensor(ch).requires_grad_(True)
            (eps * pa.trajectory(dev, f0, g2, 1.0, 10, 4)).sum().backward()
            out[variant, adj] = (f0.grad.cpu().numpy(), g2.grad.cpu().numpy())
            dev.close()
    ref = out["ff", False][1]
    for variant, tol in (("ff", 1e-11), ("g32", 1e-4)):
        assert np.array_equal(out[variant, False][0], out[variant, True][0])
        e_step, e_def = nrel(out[variant, False][1], ref), nrel(out[variant, True][1], ref)
        print(f"{variant} trajectory g2-gradient vs FF per-step: per-step {e_step:.2e}, deferred {e_def:.2e}")
        assert e_def <= tol


def test_deferred_entry_points_need_accumulators(pb):
    import torch

    ch = pb.Channels.from_model(synth.make_window4(12))
    dev = pb.Device(ch)
    z = torch.zeros(dev.nstate, dtype=torch.float64, device="cuda")
    with pytest.raises(pb.PBError):
        dev.rk4_vjp_defer(z, z.clone(), 1.0)
    with pytest.raises(pb.PBError):
        dev.g2grad_flush(torch.zeros(dev.nchannels, dtype=torch.float64, device="cuda"))
