"""GPU parity: the sm_103a library (through its C ABI) against the FP64 CPU oracle.

Error measures for the FP64-accurate variants (per-element relative error is
undefined where the collision integral vanishes):
  * e_abs = max_s |I_gpu - I_ref| / max_s S_s <= 1e-13 always, where S_s is the row's
    gross scattering (the magnitudes of the in- and out-scattering products that F_abs
    and F_em difference): the error scale of any floating-point evaluation of Eq. 2,
    whatever the cancellation;
  * e = max_s |I_gpu - I_ref| / max_s |I_ref| <= 1e-12 whenever the integral is not
    dominated by cancellation (max|I_ref| >= 1e-2 max_s S_s).
Rates, RK4 states and transport iterates have no such cancellation: e <= 1e-12.
Conservation: |sum_s I_s| <= 1e-13 * sum_s S_s.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12
MUTUAL = 3e-14  # agreement of two FP64-accurate layouts, relative to the gross scattering


@pytest.fixture(scope="module")
def pb():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2511_03683_gb300 as pb
    import torch

    assert torch.cuda.is_available()
    return pb


def nrel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def check_I(I, ref, absum, tol=TOL, abs_tol=1e-13):
    """Collision-integral parity with the conditioning-aware measures above."""
    d = np.abs(np.asarray(I) - ref).max()
    scale = np.abs(absum).max()
    assert d <= abs_tol * scale, f"e_abs = {d / scale:.3e}"
    if np.abs(ref).max() >= 1e-2 * scale:
        assert d <= tol * np.abs(ref).max(), f"e = {d / np.abs(ref).max():.3e}"


def T(x):
    import torch

    return torch.tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def _three_band_window():
    w = np.array([[e - 1.0, e + 0.3] for e in (0.0, 0.2, 1.1, 1.3)])
    w[3] = [-10.0, -9.0]
    return w


SMALL = {
    "tiny4": lambda: synth.make_tiny(4),
    "tiny5": lambda: synth.make_tiny(5),
    "win12": lambda: synth.make_window4(12),
    "win16": lambda: synth.make_window4(16),
    "tiny8": lambda: synth.make_config("tiny"),
    # three bands (the fourth band's window is empty): 81 and 99 states, so the last
    # 64-state block is ragged with an odd number of states (17, 35)
    "odd81": lambda: synth.make_window4(11, win=_three_band_window()),
    "odd99": lambda: synth.make_window4(13, win=_three_band_window()),
}
VARIANTS = ["ff", "f64", "literal"]

_cache = {}


def setup_case(pb, name, variant, **kw):
    key = (name, variant, tuple(sorted(kw.items())))
    if key not in _cache:
        m = SMALL[name]()
        ch = pb.Channels.from_model(m)
        dev = pb.Device(ch, variant=variant, transport=True, **kw)
        _cache[key] = (m, oracle.Oracle(m), dev)
    return _cache[key]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("name", list(SMALL))
def test_collision_and_rates(pb, name, variant):
    m, o, dev = setup_case(pb, name, variant)
    assert dev.nstate == o.nstate and dev.nchannels == o.count_channels()
    for f in (np.random.default_rng(7).uniform(0, 1, o.nstate), o.window_values(m.f_hot())):
        ref, ab = o.collision(f, with_abs=True)
        check_I(dev.collision(T(f)).cpu().numpy(), ref, ab)
        assert nrel(dev.rates(T(f)).cpu().numpy(), o.rates(f)) <= TOL


@pytest.mark.parametrize("variant", VARIANTS)
def test_conservation(pb, variant):
    m, o, dev = setup_case(pb, "tiny8", variant)
    f = o.window_values(m.f_hot())
    _, ab = o.collision(f, with_abs=True)
    obs = dev.observables(T(f)).cpu().numpy()
    assert abs(obs[2]) <= 1e-13 * ab.sum()
    assert abs(obs[0] - f.sum()) <= 1e-14 * f.sum()
    assert abs(obs[1] - (o.model.eps.reshape(-1)[o.ids] * f).sum()) <= 1e-13 * abs((o.model.eps.reshape(-1)[o.ids] * f).sum())


@pytest.mark.parametrize("variant", VARIANTS)
def test_rk4_tiny_workload(pb, variant):
    """The 8^3 workload's dynamics: 10 RK4 steps of 1 fs from the hot population."""
    m, o, dev = setup_case(pb, "tiny8", variant)
    f0 = o.window_values(m.f_hot())
    ft = T(f0)
    dev.rk4(ft, 1.0, 10)
    ref = o.rk4(f0, 1.0, 10)
    assert nrel(ft.cpu().numpy(), ref) <= TOL
    # the host-buffer entry point gives the same trajectory
    out = dev.rk4_host(f0, 1.0, 10)
    assert np.array_equal(out, ft.cpu().numpy())


@pytest.mark.parametrize("name", ["tiny5", "win12", "win16", "tiny8"])
def test_paper_layout_collision_and_rk4(pb, name):
    """The paper's own layout (half list + sc_col + signed target gather) reaches the oracle."""
    m, o, dev = setup_case(pb, name, "paper")
    for f in (np.random.default_rng(7).uniform(0, 1, o.nstate), o.window_values(m.f_hot())):
        ref, ab = o.collision(f, with_abs=True)
        check_I(dev.collision(T(f)).cpu().numpy(), ref, ab)
    if name == "tiny8":
        f0 = o.window_values(m.f_hot())
        ft = T(f0)
        dev.rk4(ft, 1.0, 10)
        assert nrel(ft.cpu().numpy(), o.rk4(f0, 1.0, 10)) <= TOL


@pytest.mark.parametrize("variant", ["ff", "paper", "literal"])
def test_cutoffs_on(pb, variant):
    """The paper's |g| and delta cutoffs switched on: the pruned list, every layout, the
    identically pruned oracle."""
    m = synth.make_window4(16)
    ch = pb.Channels.from_model(m, g2_min=5e-4, delta_nsigma=4.0)
    o = oracle.Oracle(m, g2_min=5e-4, delta_nsigma=4.0)
    dev = pb.Device(ch, variant=variant)
    assert dev.nchannels == o.count_channels()
    f = np.random.default_rng(12).uniform(0, 1, o.nstate)
    ref, ab = o.collision(f, with_abs=True)
    check_I(dev.collision(T(f)).cpu().numpy(), ref, ab)


@pytest.mark.parametrize("name", ["tiny5", "win16", "tiny8"])
def test_bulk_copy_sweep(pb, name):
    """The collision sweep staged by TMA bulk copies reaches the oracle; no bounded wait gave up."""
    m, o, dev = setup_case(pb, name, "ff", stream_mode=2)
    for f in (np.random.default_rng(7).uniform(0, 1, o.nstate), o.window_values(m.f_hot())):
        ref, ab = o.collision(f, with_abs=True)
        check_I(dev.collision(T(f)).cpu().numpy(), ref, ab)
    if name == "tiny8":
        f0 = o.window_values(m.f_hot())
        ft = T(f0)
        dev.rk4(ft, 1.0, 10)
        assert nrel(ft.cpu().numpy(), o.rk4(f0, 1.0, 10)) <= TOL
    dev.check()


def test_bounded_wait_gives_up_and_the_device_stays_usable(pb):
    """The bounded-wait machinery of the bulk-copy sweeps, exercised without a fault: a wait on
    an mbarrier that nothing completes gives up after its limit (20 ms here), the error word
    reaches the host as PB_ETIMEOUT once, and the handle keeps computing the same integral."""
    import time

    m = SMALL["win16"]()
    dev = pb.Device(pb.Channels.from_model(m))
    f = np.random.default_rng(5).uniform(0, 1, dev.nstate)
    I0 = dev.collision(T(f)).cpu().numpy()
    dev.check()
    t0 = time.perf_counter()
    dev.selftest_wait(20000)
    with pytest.raises(pb.PBError) as ei:
        dev.check()
    dt = time.perf_counter() - t0
    assert ei.value.code == pb.PB_ETIMEOUT
    assert 0.015 <= dt < 2.0, dt
    dev.check()  # reported once
    assert np.array_equal(dev.collision(T(f)).cpu().numpy(), I0)
    dev.check()


@pytest.mark.parametrize("item_channels", [64, 256, 4096])
def test_item_split_is_invisible(pb, item_channels):
    """Rows split into many small items (ragged tails, several tiles per row) or few large
    ones give the same integral."""
    m, o, dev = setup_case(pb, "win16", "ff", item_channels=item_channels)
    f = np.random.default_rng(3).uniform(0, 1, o.nstate)
    ref, ab = o.collision(f, with_abs=True)
    check_I(dev.collision(T(f)).cpu().numpy(), ref, ab)


@pytest.mark.parametrize("variant", ["ff", "f64"])
@pytest.mark.parametrize("merge,dense", [(1, 0), (1, 1), (1, 2), (2, 0)],
                         ids=["merged-tiles", "merged-positional", "merged-indexed", "per-channel"])
@pytest.mark.parametrize("name", ["tiny5", "win16"])
def test_branch_merged_and_per_channel_sweeps(pb, name, variant, merge, dense):
    """The coefficient sweeps with one entry per state pair (branches summed at setup; on
    these complete rows the FF collision sweep streams symmetric tiles of the pair matrix by
    default, the row stream with positional partners with dense=1, with partner indices with
    dense=2) and with one entry per channel: collision, rates, RK4 and the transport map all
    meet the oracle; the layouts agree with each other to rounding."""
    m = SMALL[name]()
    o = oracle.Oracle(m)
    ch = pb.Channels.from_model(m)
    dev = pb.Device(ch, variant=variant, merge_branches=merge, dense_rows=dense, transport=True, item_channels=256)
    rng = np.random.default_rng(21)
    f = rng.uniform(0, 1, o.nstate)
    ref, ab = o.collision(f, with_abs=True)
    I = dev.collision(T(f)).cpu().numpy()
    check_I(I, ref, ab)
    assert nrel(dev.rates(T(f)).cpu().numpy(), o.rates(f)) <= TOL
    f0 = o.window_values(m.f_hot())
    ft = T(f0)
    dev.rk4(ft, 1.0, 3)
    assert nrel(ft.cpu().numpy(), o.rk4(f0, 1.0, 3)) <= TOL
    v = o.window_values(m.vel)
    Fin = rng.normal(size=(o.nstate, 3))
    fe = o.window_values(m.f_fermi(m.emin() - 0.2))
    Fr, _ = o.transport_map(fe, v, Fin)
    assert nrel(dev.transport_map(T(fe), T(v), T(Fin)).cpu().numpy(), Fr) <= TOL
    # two float-float evaluations that round the coefficients and order the sums differently:
    # each carries about 16 roundings of 2^-48 relative to the gross scattering on the way to a
    # partial, so they may differ by a few 1e-14 of it (the oracle bound is 1e-13)
    other = pb.Device(ch, variant=variant, merge_branches=3 - merge)
    assert np.abs(other.collision(T(f)).cpu().numpy() - I).max() <= MUTUAL * ab.max()
    if merge == 1:
        assert dev.bytes_per_channel < other.bytes_per_channel
    if merge == 1 and variant == "ff":
        other_rows = pb.Device(ch, variant="ff", dense_rows=0 if dense == 2 else 2)
        assert np.abs(other_rows.collision(T(f)).cpu().numpy() - I).max() <= MUTUAL * ab.max()
        if dense != 2:  # tiles and positional partners stream fewer bytes than the index form
            assert dev.bytes_per_channel < other_rows.bytes_per_channel


@pytest.mark.parametrize("tile_sweep", [1, 2, 3], ids=["global-loads", "bulk-copies", "half-tiles"])
@pytest.mark.parametrize("name", ["odd81", "odd99", "win16", "tiny8"])
def test_tile_sweep_shapes(pb, name, tile_sweep):
    """The symmetric tile sweep with per-thread global loads, with the TMA bulk-copy ring of
    whole tiles and with the ring of half-tiles (two CTAs per SM): collision, rates and RK4
    against the oracle on complete rows whose last 64-state block is ragged (odd for odd81 /
    odd99; for odd81 the second half of the last block holds no state); the shapes agree to
    rounding."""
    m = SMALL[name]()
    o = oracle.Oracle(m)
    ch = pb.Channels.from_model(m)
    dev = pb.Device(ch, tile_sweep=tile_sweep)
    rng = np.random.default_rng(33)
    f = rng.uniform(0, 1, o.nstate)
    ref, ab = o.collision(f, with_abs=True)
    I = dev.collision(T(f)).cpu().numpy()
    check_I(I, ref, ab)
    assert nrel(dev.rates(T(f)).cpu().numpy(), o.rates(f)) <= TOL
    f0 = o.window_values(m.f_hot())
    ft = T(f0)
    dev.rk4(ft, 1.0, 3)
    assert nrel(ft.cpu().numpy(), o.rk4(f0, 1.0, 3)) <= TOL
    dev.check()
    other = pb.Device(ch, tile_sweep=1 if tile_sweep != 1 else 2)
    assert np.abs(other.collision(T(f)).cpu().numpy() - I).max() <= MUTUAL * ab.max()


@pytest.mark.parametrize("tile_sweep", [2, 3])
@pytest.mark.parametrize("name", ["odd81", "win16"])
def test_tile_sweep_signed_inputs(pb, name, tile_sweep):
    """The bulk-copy tile sweeps with occupations of both signs (outside the physical [0, 1]:
    products and partial sums of either sign in the float-float tile sums) and with their
    absolute values, against the oracle."""
    m = SMALL[name]()
    o = oracle.Oracle(m)
    ch = pb.Channels.from_model(m)
    dev = pb.Device(ch, tile_sweep=tile_sweep)
    rng = np.random.default_rng(35)
    f = rng.uniform(0, 1, o.nstate)
    f[rng.choice(o.nstate, size=o.nstate // 10, replace=False)] *= -0.5
    ref, ab = o.collision(f, with_abs=True)
    I = dev.collision(T(f)).cpu().numpy()
    check_I(I, ref, ab)
    fp = np.abs(f)
    refp, abp = o.collision(fp, with_abs=True)
    Ip = dev.collision(T(fp)).cpu().numpy()
    check_I(Ip, refp, abp)
    dev.check()


def test_time_sweep_measures_without_changing_results(pb):
    m = SMALL["win12"]()
    o = oracle.Oracle(m)
    dev = pb.Device(pb.Channels.from_model(m))
    f = np.random.default_rng(8).uniform(0, 1, o.nstate)
    before = dev.collision(T(f)).cpu().numpy()
    ms = dev.time_sweep(T(f), 5)
    assert 0.0 < ms < 100.0
    assert np.array_equal(dev.collision(T(f)).cpu().numpy(), before)
    assert 0.0 < dev.time_sweep(T(f), 6, order=1) < 100.0  # alternating tile order, as in RK4
    assert np.array_equal(dev.collision(T(f)).cpu().numpy(), before)
    with pytest.raises(pb.PBError):
        dev.time_sweep(T(f), 0)
    with pytest.raises(pb.PBError):
        dev.time_sweep(T(f), 2, order=2)


@pytest.mark.parametrize("gather", [1, 2, 3, 4, 5, 6, 7])
def test_transport_sweep_shapes(pb, gather):
    """Every transport sweep shape (shared-memory or L1 gathers, 256- or 1024-thread CTAs,
    eager or lazily renormalised float-float sums) on a ragged case: rows of many lengths
    split into 256-channel items, so full trips and tails both occur."""
    m = synth.make_window4(16)
    o = oracle.Oracle(m)
    dev = pb.Device(pb.Channels.from_model(m), transport=True, transport_gather=gather, item_channels=256)
    f0 = o.window_values(m.f_fermi(m.emin() - 0.2))
    v = o.window_values(m.vel)
    Fin = np.random.default_rng(6).normal(size=(o.nstate, 3))
    ref, _ = o.transport_map(f0, v, Fin)
    assert nrel(dev.transport_map(T(f0), T(v), T(Fin)).cpu().numpy(), ref) <= TOL


@pytest.mark.parametrize("name", ["tiny4", "odd81", "odd99", "win16", "tiny8"])
def test_transport_row_blocks(pb, name):
    """The row-block transport sweep (transport_gather 7): four rows per warp item, a ragged last
    block where nstate is not a multiple of four (81, 99), one segment of partners per item or
    several (324 states: two, the second shorter; 1024: four), against the oracle's transport
    map and against the one-row-per-item shape 4 (the automatic one)."""
    m = SMALL[name]()
    o = oracle.Oracle(m)
    ch = pb.Channels.from_model(m)
    f0 = o.window_values(m.f_fermi(m.emin() - 0.2))
    v = o.window_values(m.vel)
    Fin = np.random.default_rng(16).normal(size=(o.nstate, 3))
    ref, _ = o.transport_map(f0, v, Fin)
    got = {}
    for gather in (0, 7, 4):
        dev = pb.Device(ch, transport=True, transport_gather=gather)
        got[gather] = dev.transport_map(T(f0), T(v), T(Fin)).cpu().numpy()
        assert nrel(got[gather], ref) <= TOL
    assert np.array_equal(got[0], got[4])  # the automatic shape
    assert nrel(got[7], got[4]) <= 1e-14


def test_transport_row_blocks_need_complete_rows(pb):
    """transport_gather 7 on a list whose rows miss partners (|g|^2 cutoff) is PB_EINVAL at creation."""
    m = synth.make_window4(12)
    ch = pb.Channels.from_model(m, g2_min=1e-3)
    with pytest.raises(pb.PBError):
        pb.Device(ch, transport=True, transport_gather=7)
    pb.Device(ch, transport=True)  # the automatic shape takes any list


def test_transport_map_and_solve(pb):
    m = synth.make_tiny(4).with_(sigma=0.01)
    o = oracle.Oracle(m)
    dev = pb.Device(pb.Channels.from_model(m), transport=True)
    f0 = o.window_values(m.f_fermi(0.0))
    v = o.window_values(m.vel)
    Fin = np.random.default_rng(5).normal(size=(o.nstate, 3))
    ref, _ = o.transport_map(f0, v, Fin)
    assert nrel(dev.transport_map(T(f0), T(v), T(Fin)).cpu().numpy(), ref) <= TOL
    # the host-buffer pass with the same weights gives the same iterate bit for bit, and its
    # residual numbers are those of the device pass
    dev_out = dev.transport_iterate(T(v), T(Fin))
    res_host = np.zeros(3)
    host_out = dev.transport_iterate_host(T(v), Fin, resid=res_host)
    assert np.array_equal(host_out, dev_out.cpu().numpy())
    d = np.abs(host_out - Fin).max()
    assert res_host[1] == d and res_host[2] == np.abs(host_out).max() and res_host[0] == d / res_host[2]
    F, iters, res, ok = dev.transport(T(f0), T(v), tol=1e-12, maxit=3000)
    Fr, iters_r, res_r, ok_r = o.transport(f0, v, tol=1e-12, maxit=3000)
    assert ok and ok_r and abs(iters - iters_r) <= 1
    F = F.cpu().numpy()
    wgt = (f0 * (1 - f0))[:, None]
    s_gpu, s_ref = (wgt * v * F).sum(0), (wgt * v * Fr).sum(0)
    assert np.abs(s_gpu - s_ref).max() <= 1e-10 * np.abs(s_ref).max()
    assert nrel(F, Fr) <= 1e-9


def test_transport_solve_counts_its_passes(pb):
    """pb_iter_transport queues each pass before it checks the previous one's residual: with
    maxit 0 it returns F^0 = tau v, with tol 0 it stops after exactly maxit passes and returns
    the iterate of that many device passes (bit for bit) with its residual, and a tolerance met
    by the first pass stops after one pass."""
    import torch

    m = synth.make_window4(12)
    o = oracle.Oracle(m)
    dev = pb.Device(pb.Channels.from_model(m), transport=True)
    fe = T(o.window_values(m.f_fermi(m.emin() - 0.2)))
    v = T(o.window_values(m.vel))
    F0, it0, _, ok0 = dev.transport(fe, v, tol=0.0, maxit=0)
    assert it0 == 0 and not ok0
    F0 = F0.clone()
    res = T(np.zeros(3))
    for k in (1, 2, 3, 6):
        Fk, itk, rk, okk = dev.transport(fe, v, tol=0.0, maxit=k)
        assert itk == k and not okk
        G = F0.clone()
        for _ in range(k):
            G = dev.transport_iterate(v, G.clone(), resid=res)
        assert torch.equal(Fk, G)
        assert rk == res.cpu().numpy()[0]
    F1, it1, r1, ok1 = dev.transport(fe, v, tol=1e30, maxit=10)
    assert it1 == 1 and ok1
    assert torch.equal(F1, dev.transport_iterate(v, F0.clone()))


def test_call_graph_cache_evicts_and_recaptures(pb):
    """More argument sets than the handle keeps graphs for (twelve): collision calls into 15
    output buffers, twice round, so that every graph is evicted and captured again, all give the
    first call's integral bit for bit."""
    import torch

    m = synth.make_window4(12)
    o = oracle.Oracle(m)
    dev = pb.Device(pb.Channels.from_model(m))
    f = T(np.random.default_rng(71).uniform(0, 1, o.nstate))
    ref = dev.collision(f).cpu().numpy()
    outs = [torch.empty(o.nstate, dtype=torch.float64, device="cuda") for _ in range(15)]
    for _ in range(2):
        for out in outs:
            out.zero_()
            dev.collision(f, out=out)
            assert np.array_equal(out.cpu().numpy(), ref)


def test_transport_iterate_replays_graphs(pb):
    """pb_transport_iterate replays one captured graph per argument set: an iteration that
    alternates between two buffers (with and without the residual output), interleaved with
    host-buffer passes (another argument set), gives the same iterates and residuals bit for bit
    on both paths."""
    import torch

    m = synth.make_window4(12)
    o = oracle.Oracle(m)
    dev = pb.Device(pb.Channels.from_model(m), transport=True)
    f0 = o.window_values(m.f_fermi(m.emin() - 0.2))
    v = T(o.window_values(m.vel))
    dev.transport_setup(T(f0))
    F = np.random.default_rng(3).normal(size=(o.nstate, 3))
    a, b, res = T(F), T(np.zeros_like(F)), T(np.zeros(3))
    Fh = F.copy()
    for it in range(6):
        src, dst = (a, b) if it % 2 == 0 else (b, a)
        dev.transport_iterate(v, src, out=dst, resid=res if it < 4 else None)
        rh = np.zeros(3)
        Fh = dev.transport_iterate_host(v, Fh, resid=rh)
        assert np.array_equal(dst.cpu().numpy(), Fh)
        if it < 4:
            assert np.array_equal(res.cpu().numpy(), rh)


@pytest.mark.parametrize("variant", ["ff", "c32"])
def test_host_buffer_calls_from_pinned_memory(pb, variant):
    """From page-locked host buffers the host-buffer calls replay one graph holding both copies
    and the launches: one RK4 step per call (in place on one pinned buffer, then with another dt,
    then from pageable memory) and transport passes with the residual, bit for bit the device
    calls' results."""
    import torch

    m = synth.make_window4(12)
    o = oracle.Oracle(m)
    dev = pb.Device(pb.Channels.from_model(m), variant=variant, transport=True)
    f0 = o.window_values(m.f_hot())
    fd = T(f0)
    fh = torch.tensor(f0).pin_memory()
    for dt in (1.0, 1.0, 1.0, 0.5, 0.5, 1.0):
        dev.rk4(fd, dt, 1)
        dev.rk4_host(fh, dt, 1, out=fh)
        assert np.array_equal(fh.numpy(), fd.cpu().numpy())
    out = dev.rk4_host(fh.numpy().copy(), 1.0, 1)  # pageable: the copies outside the graph
    dev.rk4(fd, 1.0, 1)
    assert np.array_equal(out, fd.cpu().numpy())
    fe = o.window_values(m.f_fermi(m.emin() - 0.2))
    v = T(o.window_values(m.vel))
    dev.transport_setup(T(fe))
    F = np.random.default_rng(4).normal(size=(o.nstate, 3))
    Fd, Fo, res = T(F), T(np.zeros_like(F)), T(np.zeros(3))
    Fh = torch.tensor(F).pin_memory()
    rh = torch.zeros(3, dtype=torch.float64).pin_memory()
    for it in range(4):
        src, dst = (Fd, Fo) if it % 2 == 0 else (Fo, Fd)
        dev.transport_iterate(v, src, out=dst, resid=res)
        dev.transport_iterate_host(v, Fh, out=Fh, resid=rh)
        assert np.array_equal(Fh.numpy(), dst.cpu().numpy())
        assert np.array_equal(rh.numpy(), res.cpu().numpy())


def test_no_channels(pb):
    """Acoustic-only modes on a 1x1x1 grid: no channel survives, every output is zero."""
    eps = np.array([[0.0, 0.1]])
    ch = pb.Channels.build((1, 1, 1), 2, 1, eps, np.zeros((1, 1)), 300.0, 0.01, lambda s, p, nu: np.ones(len(s)))
    dev = pb.Device(ch, transport=True)
    f = T([0.3, 0.6])
    assert np.all(dev.collision(f).cpu().numpy() == 0.0)
    assert np.all(dev.rates(f).cpu().numpy() == 0.0)
    dev.rk4(f, 1.0, 3)
    assert np.array_equal(f.cpu().numpy(), [0.3, 0.6])


def test_single_state(pb):
    """One state, one Einstein mode: only the self channel, which contributes nothing to I."""
    ch = pb.Channels.build((1, 1, 1), 1, 1, np.array([[0.0]]), np.array([[0.03]]), 300.0, 0.01,
                           lambda s, p, nu: np.full(len(s), 2e-3))
    dev = pb.Device(ch)
    assert dev.nchannels == 1
    # 1/tau of the self channel: c g2 G(w) (2N+1)
    N = 1 / np.expm1(0.03 / (8.617333262e-5 * 300))
    G = np.exp(-0.03 ** 2 / (2 * 0.01 ** 2)) / (np.sqrt(2 * np.pi) * 0.01)
    ref = 2 * np.pi / 0.6582119569 * 2e-3 * G * (2 * N + 1)
    assert abs(dev.rates(T([0.4])).cpu().numpy()[0] - ref) <= 1e-13 * ref
    # the self channel's in- and out-scattering cancel
    assert abs(dev.collision(T([0.4])).cpu().numpy()[0]) <= 1e-13 * 0.4 * ref
    # the FP32 coefficient tiles: one diagonal tile with one state; the self pair's two FP32
    # coefficients are equal, so its net term vanishes exactly and its two first-order terms
    # cancel up to the rounding of one FMA (about 2^-48 of the term)
    d32 = pb.Device(ch, variant="c32")
    assert abs(d32.rates(T([0.4])).cpu().numpy()[0] - ref) <= 1e-6 * ref
    assert abs(d32.collision(T([0.4])).cpu().numpy()[0]) <= 1e-13 * 0.4 * ref
    d32.check()


# ------------------------------------------------------------------ mixed precision
# |g|^2 stored FP32 / BF16 / FP16 (times a power of two), per-channel arithmetic in FP32, Kahan
# lane sums, FP64 state.  Bounds on df/dt (normwise) on the small grids below: 1e-6 for FP32.
# BF16 rounds each |g|^2 by up to 2^-9 relative; on these coarse grids one channel can dominate a
# row, so the bound here is 2.5e-3.  The 40^3 workload (the mixed-precision configuration) is
# held to the 1e-3 target itself (FULL_TOL below): met at the hot start, missed along the
# 1000-step trajectory (2.08e-3, an expected failure there).  FP16 rounds by up to 2^-11: the
# error is at most 2^-11 of the gross scattering plus the FP32 terms' 1e-6, so 5e-4 holds even
# where one channel dominates.
MIXED_TOL = {"g32": 1e-6, "g16": 2.5e-3, "h16": 5e-4}


@pytest.mark.parametrize("variant", ["g32", "g16", "h16"])
@pytest.mark.parametrize("name", ["tiny5", "win12", "win16", "tiny8"])
def test_mixed_precision_collision_and_rates(pb, name, variant):
    m, o, dev = setup_case(pb, name, variant)
    tol = MIXED_TOL[variant]
    for f in (np.random.default_rng(7).uniform(0, 1, o.nstate), o.window_values(m.f_hot())):
        ref, ab = o.collision(f, with_abs=True)
        check_I(dev.collision(T(f)).cpu().numpy(), ref, ab, tol=tol, abs_tol=tol)
        assert nrel(dev.rates(T(f)).cpu().numpy(), o.rates(f)) <= tol


@pytest.mark.parametrize("shape", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("variant", ["g32", "g16", "h16"])
def test_mixed_precision_sweep_shapes(pb, variant, shape):
    """Every launch shape of the FP32/BF16 sweep on a ragged case (rows of many lengths,
    items split inside rows; 5: the dense pair-major form) meets the same bound against the
    oracle."""
    m = synth.make_window4(16)
    o = oracle.Oracle(m)
    dev = pb.Device(pb.Channels.from_model(m), variant=variant, channel_per_lane=shape, item_channels=256)
    f = np.random.default_rng(11).uniform(0, 1, o.nstate)
    ref, ab = o.collision(f, with_abs=True)
    check_I(dev.collision(T(f)).cpu().numpy(), ref, ab, tol=MIXED_TOL[variant], abs_tol=MIXED_TOL[variant])
    assert nrel(dev.rates(T(f)).cpu().numpy(), o.rates(f)) <= MIXED_TOL[variant]


@pytest.mark.parametrize("variant", ["g32", "g16", "h16"])
def test_mixed_precision_set_g2_refreshes_dense_slots(pb, variant):
    """pb_dev_set_g2 on a dense pair-major device rewrites the (state, partner, branch) slots:
    Eq. 2 is linear in |g|^2, so doubling every |g|^2 doubles the integral (a factor of two
    commutes with rounding to FP32, BF16 and scaled FP16, so only the summation order
    differs)."""
    import torch

    m = SMALL["win16"]()
    ch = pb.Channels.from_model(m)
    dev = pb.Device(ch, variant=variant)
    f = T(np.random.default_rng(4).uniform(0, 1, dev.nstate))
    I0 = dev.collision(f).cpu().numpy()
    g2 = torch.tensor(ch.export()["g2"], dtype=torch.float64, device="cuda")
    dev.set_g2(2.0 * g2)
    I1 = dev.collision(f).cpu().numpy()
    assert np.abs(I1 - 2.0 * I0).max() <= 1e-6 * np.abs(I0).max()
    dev.set_g2(g2)
    assert np.abs(dev.collision(f).cpu().numpy() - I0).max() <= 1e-7 * np.abs(I0).max()


@pytest.mark.parametrize("shape", [0, 5])
def test_mixed_precision_with_cutoffs(pb, shape):
    """With the |g| and delta cutoffs on, the channel list fills few (row, branch, partner)
    slots: the automatic shape keeps the per-channel sweep, and the dense pair-major form
    (forced) still meets the oracle with zeros in the missing slots."""
    m = synth.make_window4(16)
    ch = pb.Channels.from_model(m, g2_min=5e-4, delta_nsigma=4.0)
    o = oracle.Oracle(m, g2_min=5e-4, delta_nsigma=4.0)
    dev = pb.Device(ch, variant="g32", channel_per_lane=shape)
    f = np.random.default_rng(12).uniform(0, 1, o.nstate)
    ref, ab = o.collision(f, with_abs=True)
    check_I(dev.collision(T(f)).cpu().numpy(), ref, ab, tol=MIXED_TOL["g32"], abs_tol=MIXED_TOL["g32"])
    assert nrel(dev.rates(T(f)).cpu().numpy(), o.rates(f)) <= MIXED_TOL["g32"]


def test_fp16_storage_overflow_is_reported(pb):
    """Scaled FP16 |g|^2: the storage factor maps the largest value at creation into
    [2^9, 2^10), so pb_dev_set_g2 with values 100 times larger overflows; the conversion
    flags it and pb_dev_check returns PB_EINVAL.  Restoring the values clears it."""
    import torch

    m = SMALL["win16"]()
    ch = pb.Channels.from_model(m)
    dev = pb.Device(ch, variant="h16")
    f = T(np.random.default_rng(5).uniform(0, 1, dev.nstate))
    I0 = dev.collision(f).cpu().numpy()
    dev.check()
    g2 = torch.tensor(ch.export()["g2"], dtype=torch.float64, device="cuda")
    dev.set_g2(32.0 * g2)  # inside the range: exact factor
    assert np.abs(dev.collision(f).cpu().numpy() - 32.0 * I0).max() <= 1e-6 * 32.0 * np.abs(I0).max()
    dev.check()
    dev.set_g2(100.0 * g2)
    with pytest.raises(pb.PBError) as e:
        dev.check()
    assert e.value.code == pb.PB_EINVAL
    dev.set_g2(g2)
    dev.check()
    assert np.abs(dev.collision(f).cpu().numpy() - I0).max() <= 1e-7 * np.abs(I0).max()


def test_fp16_storage_underflow_is_reported(pb):
    """Scaled FP16 |g|^2 keeps 11 significand bits only down to 2^-23 of the largest value at
    creation: values set 2^30 times smaller fall below FP16's smallest normal number, the
    conversion flags it and pb_dev_check returns PB_EINVAL; a factor of 2^-8 stays inside the
    range and is exact."""
    import torch

    m = SMALL["win16"]()
    ch = pb.Channels.from_model(m)
    dev = pb.Device(ch, variant="h16")
    f = T(np.random.default_rng(8).uniform(0, 1, dev.nstate))
    I0 = dev.collision(f).cpu().numpy()
    g2 = torch.tensor(ch.export()["g2"], dtype=torch.float64, device="cuda")
    dev.set_g2(2.0 ** -8 * g2)
    assert np.abs(dev.collision(f).cpu().numpy() - 2.0 ** -8 * I0).max() <= 1e-6 * 2.0 ** -8 * np.abs(I0).max()
    dev.check()
    dev.set_g2(2.0 ** -30 * g2)
    with pytest.raises(pb.PBError) as e:
        dev.check()
    assert e.value.code == pb.PB_EINVAL and "too small" in str(e.value)
    dev.set_g2(g2)
    dev.check()


def test_bf16_storage_takes_large_values(pb):
    """The FP16 range check is the H16 variant's alone: BF16 storage (FP32 range) takes |g|^2
    a million times larger without a report, and the integral scales with it."""
    import torch

    m = SMALL["win16"]()
    ch = pb.Channels.from_model(m)
    dev = pb.Device(ch, variant="g16")
    f = T(np.random.default_rng(6).uniform(0, 1, dev.nstate))
    I0 = dev.collision(f).cpu().numpy()
    g2 = torch.tensor(ch.export()["g2"], dtype=torch.float64, device="cuda")
    dev.set_g2(2.0 ** 20 * g2)
    I1 = dev.collision(f).cpu().numpy()
    dev.check()
    assert np.abs(I1 - 2.0 ** 20 * I0).max() <= 1e-6 * 2.0 ** 20 * np.abs(I0).max()


@pytest.mark.parametrize("variant", ["g32", "g16", "h16"])
def test_mixed_precision_rk4(pb, variant):
    m, o, dev = setup_case(pb, "tiny8", variant)
    f0 = o.window_values(m.f_hot())
    ft = T(f0)
    dev.rk4(ft, 1.0, 10)
    assert nrel(ft.cpu().numpy(), o.rk4(f0, 1.0, 10)) <= MIXED_TOL[variant]


# ------------------------------------------------------------------ FP32 coefficient tiles (C32)
# The branch-merged coefficients in FP32 symmetric tiles with the ratio P_out / P_in kept, each
# entry's net term formed in FP32 with an exact leading product, first-order terms in the low
# part of f, FP64 per-state combination: df/dt within 1e-6 normwise (the FP32 target of Eq. 2's
# reduced-precision forms), rates within 1e-6, particle number conserved to 1e-6 of the gross
# scattering.
C32_TOL = 1e-6


@pytest.mark.parametrize("name", list(SMALL))
def test_c32_collision_rates_conservation(pb, name):
    m, o, dev = setup_case(pb, name, "c32")
    assert dev.bytes_per_channel > 0
    for f in (np.random.default_rng(7).uniform(0, 1, o.nstate), o.window_values(m.f_hot())):
        ref, ab = o.collision(f, with_abs=True)
        I = dev.collision(T(f)).cpu().numpy()
        check_I(I, ref, ab, tol=C32_TOL, abs_tol=C32_TOL)
        assert abs(I.sum()) <= C32_TOL * ab.sum()
        assert nrel(dev.rates(T(f)).cpu().numpy(), o.rates(f)) <= C32_TOL
    dev.check()


@pytest.mark.parametrize("shape", [3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("name", ["odd81", "odd99", "tiny8"])
def test_c32_launch_shapes(pb, name, shape):
    """Every launch shape of the FP32 tile sweep (stages x CTAs per SM; 7, 8: half-tiles) on
    ragged complete rows (odd81: the last block's second half holds no state): collision and rates
    against the oracle at the C32 bound, RK4 steps, and the same integral as the default shape to
    FP32 rounding."""
    m = SMALL[name]()
    o = oracle.Oracle(m)
    ch = pb.Channels.from_model(m)
    dev = pb.Device(ch, variant="c32", tile_sweep=shape)
    f = np.random.default_rng(41).uniform(0, 1, o.nstate)
    ref, ab = o.collision(f, with_abs=True)
    I = dev.collision(T(f)).cpu().numpy()
    check_I(I, ref, ab, tol=C32_TOL, abs_tol=C32_TOL)
    assert nrel(dev.rates(T(f)).cpu().numpy(), o.rates(f)) <= C32_TOL
    f0 = o.window_values(m.f_hot())
    ft = T(f0)
    dev.rk4(ft, 1.0, 3)
    assert nrel(ft.cpu().numpy(), o.rk4(f0, 1.0, 3)) <= C32_TOL
    dev.check()
    default = pb.Device(ch, variant="c32")
    assert np.abs(default.collision(T(f)).cpu().numpy() - I).max() <= 1e-7 * ab.max()


def test_c32_signed_inputs(pb):
    """The net-term arithmetic holds for occupations of either sign (as the adjoint and
    finite-difference probes use them): random f in [-1, 1] on the ragged 99-state case."""
    m, o, dev = setup_case(pb, "odd99", "c32")
    f = np.random.default_rng(21).uniform(-1, 1, o.nstate)
    ref, ab = o.collision(f, with_abs=True)
    check_I(dev.collision(T(f)).cpu().numpy(), ref, ab, tol=C32_TOL, abs_tol=C32_TOL)


def test_c32_rk4(pb):
    m, o, dev = setup_case(pb, "tiny8", "c32")
    f0 = o.window_values(m.f_hot())
    ft = T(f0)
    dev.rk4(ft, 1.0, 10)
    assert nrel(ft.cpu().numpy(), o.rk4(f0, 1.0, 10)) <= C32_TOL
    dev.check()


def _acoustic_tiny(n):
    t = synth.make_tiny(n)
    s = synth.acoustic_shape(t.nk).reshape(-1)
    return t.with_(omega=np.stack([15e-3 * s, 20e-3 * s, 25e-3 * s], axis=1))


@pytest.mark.parametrize("variant", ["ff", "c32"])
@pytest.mark.parametrize("case", ["acoustic", "cutoffs"])
def test_tiles_on_rows_that_miss_partners(pb, variant, case):
    """Symmetric tiles filled by scattering rows that miss partners (zero where a pair has no
    channel): an acoustic-only model (no channel between the bands at one k point; tiles taken
    automatically) and the 16^3 window with the |g| and delta cutoffs (tiles forced with
    dense_rows 3): collision, rates and 3 RK4 steps against the identically built oracle, and the
    float-float tiles against the rows of the same list."""
    if case == "acoustic":
        m, kw, dev_kw = _acoustic_tiny(6), {}, {}
    else:
        m, kw, dev_kw = synth.make_window4(16), dict(g2_min=5e-4, delta_nsigma=4.0), dict(dense_rows=3)
    o = oracle.Oracle(m, **kw)
    ch = pb.Channels.from_model(m, **kw)
    dev = pb.Device(ch, variant=variant, **dev_kw)
    rows = pb.Device(ch, dense_rows=2)
    assert dev.bytes_per_channel != rows.bytes_per_channel  # the tiles, not the rows
    tol = TOL if variant == "ff" else C32_TOL
    f = np.random.default_rng(61).uniform(0, 1, o.nstate)
    ref, ab = o.collision(f, with_abs=True)
    I = dev.collision(T(f)).cpu().numpy()
    if variant == "ff":
        check_I(I, ref, ab)
        assert np.abs(I - rows.collision(T(f)).cpu().numpy()).max() <= MUTUAL * ab.max()
    else:
        assert np.abs(I - ref).max() <= tol * ab.max()
    assert nrel(dev.rates(T(f)).cpu().numpy(), o.rates(f)) <= tol
    f0 = o.window_values(m.f_hot())
    ft = T(f0)
    dev.rk4(ft, 1.0, 3)
    assert nrel(ft.cpu().numpy(), o.rk4(f0, 1.0, 3)) <= tol
    dev.check()


def test_symmetric_tiles_need_a_closure_checked_list(pb):
    """The tiles serve each pair (s, p) and its reverse from one entry, which holds only when the
    reverse channels exist with equal |g|^2: a list built without the closure check streams the
    rows and meets the oracle all the same; C32, which needs the tiles, refuses it."""
    m = synth.make_window4(12)
    o = oracle.Oracle(m)
    checked_ch = pb.Channels.from_model(m)
    checked = pb.Device(checked_ch)
    unchecked_ch = pb.Channels.from_model(m, check_closure=False)
    unchecked = pb.Device(unchecked_ch)
    # the streamed bytes of the positional rows (dense_rows 1), not of the tiles
    rows = pb.Device(checked_ch, dense_rows=1)
    assert unchecked.bytes_per_channel == rows.bytes_per_channel != checked.bytes_per_channel
    f = np.random.default_rng(57).uniform(0, 1, o.nstate)
    ref, ab = o.collision(f, with_abs=True)
    check_I(unchecked.collision(T(f)).cpu().numpy(), ref, ab)
    check_I(checked.collision(T(f)).cpu().numpy(), ref, ab)
    with pytest.raises(pb.PBError) as e:
        pb.Device(unchecked_ch, variant="c32")
    assert e.value.code == pb.PB_EINVAL


def test_c32_needs_complete_rows_and_the_tile_sweep(pb):
    m = synth.make_window4(16)
    ch = pb.Channels.from_model(m, g2_min=5e-4, delta_nsigma=4.0)
    with pytest.raises(pb.PBError) as e:
        pb.Device(ch, variant="c32")
    assert e.value.code == pb.PB_EINVAL
    full = pb.Channels.from_model(m)
    for kw in ({"tile_sweep": 1}, {"merge_branches": 2}, {"stream_mode": 2}, {"dense_rows": 2}):
        with pytest.raises(pb.PBError) as e:
            pb.Device(full, variant="c32", **kw)
        assert e.value.code == pb.PB_EINVAL


def test_c32_adjoint_is_refused_and_set_g2_streams_rows(pb):
    """A C32 device has no FP32 adjoint (PB_EINVAL); after pb_dev_set_g2 it streams the
    float-float rows, so doubling |g|^2 doubles the integral to FP64 accuracy."""
    import torch

    m, o, dev0 = setup_case(pb, "win12", "c32")
    ch = pb.Channels.from_model(m)
    dev = pb.Device(ch, variant="c32")
    f = np.random.default_rng(9).uniform(0, 1, dev.nstate)
    with pytest.raises(pb.PBError) as e:
        dev.collision_vjp(T(f), T(f))
    assert e.value.code == pb.PB_EINVAL
    g2 = torch.tensor(ch.export()["g2"], dtype=torch.float64, device="cuda")
    dev.set_g2(2.0 * g2)
    ref, ab = o.collision(f, with_abs=True)
    check_I(dev.collision(T(f)).cpu().numpy(), 2.0 * ref, 2.0 * ab)


# ------------------------------------------------------------------ full size (40^3)

@pytest.fixture(scope="module")
def big(pb):
    m = synth.make_config("window40")
    ch = pb.Channels.from_model(m)
    dev = pb.Device(ch, variant="ff", transport=True)
    return m, oracle.Oracle(m), dev


def test_full_size_counts(big):
    m, o, dev = big
    assert dev.nstate == o.nstate == 4756
    assert dev.nchannels == o.count_channels()


def test_full_size_collision_sampled_and_conserved(big):
    m, o, dev = big
    f = o.window_values(m.f_hot())
    I = dev.collision(T(f)).cpu().numpy()
    rows = np.unique(np.concatenate([np.arange(0, o.nstate, 97), [o.nstate - 1]]))
    ref, ab = o.collision(f, rows=rows, with_abs=True)
    check_I(I[rows], ref, ab)
    Ifull, abfull = o.collision(f, with_abs=True)
    check_I(I, Ifull, abfull)
    assert np.abs(Ifull).max() >= 1e-2 * abfull.max()  # the hot population is well conditioned
    assert abs(I.sum()) <= 1e-13 * abfull.sum()
    r = dev.rates(T(f)).cpu().numpy()
    assert nrel(r[rows], o.rates(f, rows=rows)) <= TOL


def test_full_size_rk4_two_steps(big):
    m, o, dev = big
    f0 = o.window_values(m.f_hot())
    ft = T(f0)
    dev.rk4(ft, 1.0, 2)
    assert nrel(ft.cpu().numpy(), o.rk4(f0, 1.0, 2)) <= TOL


# the 40^3 workload (the mixed-precision configuration): the targets themselves
FULL_TOL = {"g32": 1e-6, "g16": 1e-3, "h16": 5e-4, "c32": C32_TOL}


@pytest.mark.parametrize("variant", ["g32", "g16", "h16", "c32"])
def test_full_size_mixed_precision(pb, big, variant):
    m, o, _ = big
    dev = pb.Device(big[2].channels, variant=variant)
    f = o.window_values(m.f_hot())
    ref, ab = o.collision(f, with_abs=True)
    I = dev.collision(T(f)).cpu().numpy()
    check_I(I, ref, ab, tol=FULL_TOL[variant], abs_tol=FULL_TOL[variant])
    print(f"{variant}: normwise df/dt error {np.abs(I - ref).max() / np.abs(ref).max():.3e}")
    rows = np.arange(3, o.nstate, 151)
    assert nrel(dev.rates(T(f)).cpu().numpy()[rows], o.rates(f, rows=rows)) <= FULL_TOL[variant]
    dev.check()
    dev.close()


@pytest.mark.parametrize("variant,bound", [
    ("g32", 1e-6), ("h16", 1e-3), ("c32", C32_TOL),
    pytest.param("g16", 1e-3, marks=pytest.mark.xfail(
        strict=True, reason="BF16 rounds each |g|^2 by up to 2^-9: measured 2.08e-3 at the worst of the 1000 "
                            "steps; the 16-bit form that meets 1e-3 is h16 (FP16 x 2^k)"))])
def test_full_size_mixed_error_along_trajectory(pb, big, variant, bound):
    """Reduced-precision forms along 1000 RK4 steps of the 40^3 hot start (FP32 |g|^2, FP16 and
    BF16 |g|^2 with FP32 per-channel terms; the FP32 coefficient tiles): the df/dt error against
    the FP64-accurate sweep (itself held to the oracle at 1e-12) at every 100th step, normwise,
    against the 1e-6 (FP32) and 1e-3 (16-bit) targets, while max|df/dt| shrinks as f relaxes."""
    m, o, dev = big
    mixed = pb.Device(dev.channels, variant=variant)
    f = T(o.window_values(m.f_hot()))
    worst = 0.0
    for k in range(11):
        a = dev.collision(f).cpu().numpy()
        b = mixed.collision(f).cpu().numpy()
        worst = max(worst, np.abs(b - a).max() / np.abs(a).max())
        if k < 10:
            dev.rk4(f, 1.0, 100)
    print(f"{variant} worst normwise df/dt error over 1000 steps: {worst:.3e}")
    mixed.close()
    assert worst <= bound


def test_full_size_bulk_copy_sweep(pb, big):
    m, o, dev = big
    bulk = pb.Device(dev.channels, variant="ff", stream_mode=2)
    f = o.window_values(m.f_hot())
    rows = np.unique(np.concatenate([np.arange(0, o.nstate, 53), [o.nstate - 1]]))
    ref, ab = o.collision(f, rows=rows, with_abs=True)
    check_I(bulk.collision(T(f)).cpu().numpy()[rows], ref, ab)
    bulk.check()


@pytest.mark.parametrize("tile_sweep", [1, 2, 3])
def test_full_size_tile_sweep_shapes(pb, big, tile_sweep):
    """Every tile sweep at 40^3 against the full oracle and the default (2850 tiles, about 19
    per CTA of the persistent rings, so every stage is refilled many times); no bounded wait
    gave up."""
    m, o, dev = big
    alt = pb.Device(dev.channels, variant="ff", tile_sweep=tile_sweep)
    f = o.window_values(m.f_hot())
    ref, ab = o.collision(f, with_abs=True)
    I = alt.collision(T(f)).cpu().numpy()
    check_I(I, ref, ab)
    alt.check()
    dev.check()
    assert np.abs(dev.collision(T(f)).cpu().numpy() - I).max() <= MUTUAL * ab.max()


def test_full_size_transport_map_sampled(big):
    m, o, dev = big
    f0 = o.window_values(m.f_fermi(o.model.emin() - 0.2))
    v = o.window_values(m.vel)
    Fin = np.random.default_rng(11).normal(size=(o.nstate, 3))
    out = dev.transport_map(T(f0), T(v), T(Fin)).cpu().numpy()
    rows = np.arange(5, o.nstate, 211)
    ref, _ = o.transport_map(f0, v, Fin, rows=rows)
    assert np.abs(out[rows] - ref).max() <= TOL * np.abs(ref).max()


def test_full_size_transport_row_blocks_sampled(pb, big):
    """The row-block transport sweep (transport_gather 7) at 40^3: 1189 blocks of four rows, three
    segments of 1600 partners (the last 1556), 3567 items in one wave of 24-warp CTAs, each CTA
    staging F over its one or two segments; sampled rows against the oracle and all rows against
    the automatic shape."""
    m, o, dev = big
    rb = pb.Device(dev.channels, variant="ff", transport=True, transport_gather=7)
    f0 = o.window_values(m.f_fermi(o.model.emin() - 0.2))
    v = o.window_values(m.vel)
    Fin = np.random.default_rng(17).normal(size=(o.nstate, 3))
    out = rb.transport_map(T(f0), T(v), T(Fin)).cpu().numpy()
    rows = np.unique(np.concatenate([np.arange(3, o.nstate, 197), [o.nstate - 1]]))
    ref, _ = o.transport_map(f0, v, Fin, rows=rows)
    assert np.abs(out[rows] - ref).max() <= TOL * np.abs(ref).max()
    assert nrel(out, dev.transport_map(T(f0), T(v), T(Fin)).cpu().numpy()) <= 1e-14


def test_full_size_paper_layout_sampled(pb, big):
    """The paper's own layout (half list, sc_col, signed target gather) at 40^3 on sampled rows."""
    m, o, dev = big
    pap = pb.Device(dev.channels, variant="paper")
    f = o.window_values(m.f_hot())
    rows = np.unique(np.concatenate([np.arange(0, o.nstate, 61), [o.nstate - 1]]))
    ref, ab = o.collision(f, rows=rows, with_abs=True)
    check_I(pap.collision(T(f)).cpu().numpy()[rows], ref, ab)


def test_full_size_1000_steps_two_arithmetics(pb, big):
    """The 40^3 workload's dynamics: 1000 RK4 steps of 1 fs with the float-float default and
    with native FP64 FMAs (independent arithmetic) agree, and the particle number sum_s f_s is
    conserved to rounding (sum_s I_s = 0 for the closed channel list)."""
    m, o, dev = big
    f0 = o.window_values(m.f_hot())
    a = T(f0)
    dev.rk4(a, 1.0, 1000)
    d64 = pb.Device(dev.channels, variant="f64")
    b = T(f0)
    d64.rk4(b, 1.0, 1000)
    fa, fb = a.cpu().numpy(), b.cpu().numpy()
    assert nrel(fa, fb) <= 1e-11
    assert abs(fa.sum() - f0.sum()) <= 1e-12 * f0.sum()
    assert fa.min() >= -1e-12 and fa.max() <= 1.0
    # the hot carriers cool towards the lattice: carrier energy decreases
    e = o.window_values(m.eps)
    assert (e * fa).sum() < (e * f0).sum()


def _trajectory_fixture(name):
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", f"trajectory_{name}.txt")
    return np.loadtxt(path, ndmin=2)


@pytest.mark.parametrize("variant,tol", [("ff", TOL), ("c32", C32_TOL)])
def test_1000_step_trajectory_against_the_oracle(pb, variant, tol):
    """The rt-BTE workload on the 24^3 grids (1028 states, 6.3e6 channels): 1000 classic RK4
    steps of 1 fs from the hot population, against the oracle's own trajectory
    (tests/golden/trajectory_window24.txt, written by the oracle alone) after 250, 500, 750 and
    1000 steps: normwise 1e-12 for the FP64-accurate default, 1e-6 for the FP32 coefficient
    tiles."""
    m = synth.make_config("window24")
    ch = pb.Channels.from_model(m)
    dev = pb.Device(ch, variant=variant)
    ref = _trajectory_fixture("window24")
    f = T(m.f_hot().reshape(-1)[ch.state_ids()])
    for k in range(ref.shape[1]):
        dev.rk4(f, 1.0, 250)
        err = nrel(f.cpu().numpy(), ref[:, k])
        print(f"{variant}: step {250 * (k + 1)}: normwise error {err:.2e}")
        assert err <= tol
    dev.check()


def test_full_size_50_steps_against_the_oracle(big):
    """The 40^3 workload: 50 RK4 steps of 1 fs against the oracle's trajectory
    (tests/golden/trajectory_window40.txt) at 1e-12 normwise."""
    m, o, dev = big
    ref = _trajectory_fixture("window40")[:, 0]
    f = T(o.window_values(m.f_hot()))
    dev.rk4(f, 1.0, 50)
    assert nrel(f.cpu().numpy(), ref) <= TOL


def test_full_size_transport_solve_matches_oracle(pb, big):
    """pb_iter_transport on the 40^3 workload for x, y, z to 1e-10 against the oracle's own
    iteration: same iteration count (+-1), conductivity-like tensor and isotropy."""
    m, o, dev = big
    f0 = o.window_values(m.f_fermi(m.emin() - 0.2))
    v = o.window_values(m.vel)
    F, it, res, ok = dev.transport(T(f0), T(v), tol=1e-10, maxit=1000)
    Fr, itr, resr, okr = o.transport(f0, v, tol=1e-10, maxit=1000)
    assert ok and okr and abs(it - itr) <= 1
    F = F.cpu().numpy()
    w = (f0 * (1 - f0))[:, None, None]
    S = (w * v[:, :, None] * F[:, None, :]).sum(0)
    Sr = (w * v[:, :, None] * Fr[:, None, :]).sum(0)
    assert np.abs(S - Sr).max() <= 1e-9 * np.abs(np.diag(Sr)).max()
    assert nrel(F, Fr) <= 1e-8
    d = np.diag(S)
    assert np.abs(d - d.mean()).max() <= 1e-9 * abs(d.mean())
