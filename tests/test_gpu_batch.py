"""Batched rt-BTE: many instances of the batched workload in one launch per stage,
against the unbatched FP32 device and the FP64 oracle of each instance."""
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


def small_instances(k=10):
    """The k smallest-grid instances among the first 40 of the batched workload (fast oracle)."""
    inst = [synth.make_batch_instance(i) for i in range(40)]
    inst.sort(key=lambda t: np.prod(t[0].nk) * t[0].nbands)
    return inst[:k]


@pytest.fixture(scope="module")
def batch(pb):
    import torch

    inst = small_instances()
    chs = [pb.Channels.from_model(m) for m, _ in inst]
    b = pb.Batch(chs)
    f = np.concatenate([m.f_hot(e_exc=e).reshape(-1)[c.state_ids()] for (m, e), c in zip(inst, chs)])
    return inst, chs, b, f


def test_batch_collision_matches_unbatched_and_oracle(pb, batch):
    import torch

    inst, chs, b, f = batch
    assert b.nstate == sum(c.nstate for c in chs) and b.nchannels == sum(c.nchannels for c in chs)
    rng = np.random.default_rng(9)
    fr = rng.uniform(0, 1, b.nstate)
    I = b.collision(torch.tensor(fr, device="cuda")).cpu().numpy()
    for i, ((m, _), ch) in enumerate(zip(inst, chs)):
        a, e = b.offsets[i], b.offsets[i + 1]
        dev = pb.Device(ch, variant="g32")
        ref32 = dev.collision(torch.tensor(fr[a:e], device="cuda")).cpu().numpy()
        assert np.abs(I[a:e] - ref32).max() <= 1e-6 * np.abs(ref32).max()
        o = oracle.Oracle(m)
        ref, ab = o.collision(fr[a:e], with_abs=True)
        d = np.abs(I[a:e] - ref).max()
        assert d <= 1e-6 * ab.max()
        if np.abs(ref).max() >= 1e-2 * ab.max():
            assert d <= 1e-6 * np.abs(ref).max()


def test_batch_layouts_agree(pb, batch):
    """The dense pair-major FP32 batch (the default on these complete rows) and the form with
    one entry per channel (layout 1) give the same integral to FP32 rounding."""
    import torch

    inst, chs, b, f = batch
    per_channel = pb.Batch(chs, layout=1)
    ft = torch.tensor(f, device="cuda")
    a = b.collision(ft).cpu().numpy()
    c = per_channel.collision(ft).cpu().numpy()
    assert np.abs(a - c).max() <= 1e-6 * np.abs(c).max()


def test_batch_rk4_matches_oracle(pb, batch):
    import torch

    inst, chs, b, f = batch
    ft = torch.tensor(f, device="cuda")
    b.rk4(ft, 1.0, 5)
    got = ft.cpu().numpy()
    for i, ((m, _), ch) in enumerate(zip(inst[:4], chs[:4])):
        a, e = b.offsets[i], b.offsets[i + 1]
        ref = oracle.Oracle(m).rk4(f[a:e], 1.0, 5)
        assert np.abs(got[a:e] - ref).max() <= 1e-6 * np.abs(ref).max()


def test_batch_autotune_keeps_results(pb, batch):
    import torch

    inst, chs, b, f = batch
    ft = torch.tensor(f, device="cuda")
    before = b.collision(ft).cpu().numpy()
    item, ctas, ms = b.autotune(ft)
    assert item in (1024, 2048, 4096) and ctas in (2, 3, 4) and ms > 0
    after = b.collision(ft).cpu().numpy()
    assert np.abs(after - before).max() <= 1e-6 * np.abs(before).max()


# ------------------------------------------------------------------ FP64-accurate batch (precision "ff")

# layout 0: the symmetric tiles (these instances' rows are complete and the tiles stream fewer
# bytes); layout 1: one row entry per directed state pair
@pytest.fixture(scope="module", params=[0, 1], ids=["tiles", "rows"])
def batch_ff(pb, batch, request):
    inst, chs, _, f = batch
    b = pb.Batch(chs, precision="ff", layout=request.param)
    assert b.tiled == (request.param == 0)
    return b


def test_ff_batch_collision_matches_oracle_and_unbatched(pb, batch, batch_ff):
    """The branch-merged float-float batch: every instance's df/dt meets its FP64 oracle at
    the FF bound and agrees with the same instance on its own device to rounding."""
    import torch

    inst, chs, _, _ = batch
    b = batch_ff
    rng = np.random.default_rng(19)
    fr = rng.uniform(0, 1, b.nstate)
    I = b.collision(torch.tensor(fr, device="cuda")).cpu().numpy()
    for i, ((m, _), ch) in enumerate(zip(inst, chs)):
        a, e = b.offsets[i], b.offsets[i + 1]
        ref, ab = oracle.Oracle(m).collision(fr[a:e], with_abs=True)
        d = np.abs(I[a:e] - ref).max()
        assert d <= 1e-13 * ab.max()
        if np.abs(ref).max() >= 1e-2 * ab.max():
            assert d <= 1e-12 * np.abs(ref).max()
        own = pb.Device(ch).collision(torch.tensor(fr[a:e], device="cuda")).cpu().numpy()
        assert np.abs(I[a:e] - own).max() <= 1e-14 * ab.max()


def test_ff_batch_rk4_matches_oracle(pb, batch, batch_ff):
    import torch

    inst, chs, _, f = batch
    ft = torch.tensor(f, device="cuda")
    batch_ff.rk4(ft, 1.0, 5)
    got = ft.cpu().numpy()
    for i, ((m, _), ch) in enumerate(zip(inst[:4], chs[:4])):
        a, e = batch_ff.offsets[i], batch_ff.offsets[i + 1]
        ref = oracle.Oracle(m).rk4(f[a:e], 1.0, 5)
        assert np.abs(got[a:e] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_ff_batch_autotune_keeps_results(pb, batch, batch_ff):
    import torch

    _, _, _, f = batch
    ft = torch.tensor(f, device="cuda")
    before = batch_ff.collision(ft).cpu().numpy()
    item, ctas, ms = batch_ff.autotune(ft)
    assert (item == 0 if batch_ff.tiled else item in (1024, 2048, 4096)) and ctas in (2, 3, 4) and ms > 0
    after = batch_ff.collision(ft).cpu().numpy()
    assert np.abs(after - before).max() <= 1e-12 * np.abs(before).max()
    batch_ff.check()


# ------------------------------------------------------------------ FP32 pair coefficients (precision "c32")

@pytest.fixture(scope="module", params=[0, 1], ids=["tiles", "rows"])
def batch_c32(pb, batch, request):
    inst, chs, _, f = batch
    b = pb.Batch(chs, precision="c32", layout=request.param)
    assert b.tiled == (request.param == 0)
    return b


def test_c32_batch_collision_matches_oracle(pb, batch, batch_c32):
    """The branch-merged coefficients as FP32 pairs, net terms per entry: every instance's
    df/dt within 1e-6 of its FP64 oracle (normwise; relative to the gross scattering where the
    integral itself is dominated by cancellation)."""
    import torch

    inst, chs, _, _ = batch
    b = batch_c32
    fr = np.random.default_rng(23).uniform(0, 1, b.nstate)
    I = b.collision(torch.tensor(fr, device="cuda")).cpu().numpy()
    for i, ((m, _), ch) in enumerate(zip(inst, chs)):
        a, e = b.offsets[i], b.offsets[i + 1]
        ref, ab = oracle.Oracle(m).collision(fr[a:e], with_abs=True)
        d = np.abs(I[a:e] - ref).max()
        assert d <= 1e-6 * ab.max()
        if np.abs(ref).max() >= 1e-2 * ab.max():
            assert d <= 1e-6 * np.abs(ref).max()


def test_c32_batch_rk4_matches_oracle(pb, batch, batch_c32):
    import torch

    inst, chs, _, f = batch
    ft = torch.tensor(f, device="cuda")
    batch_c32.rk4(ft, 1.0, 5)
    got = ft.cpu().numpy()
    for i, ((m, _), ch) in enumerate(zip(inst[:4], chs[:4])):
        a, e = batch_c32.offsets[i], batch_c32.offsets[i + 1]
        ref = oracle.Oracle(m).rk4(f[a:e], 1.0, 5)
        assert np.abs(got[a:e] - ref).max() <= 1e-6 * np.abs(ref).max()


_largest = {}


def _largest_reference(m, e, fr, f, rows):
    """Oracle df/dt on sampled rows and the 3-step trajectory of one instance (computed once)."""
    key = m.name
    if key not in _largest:
        o = oracle.Oracle(m)
        _largest[key] = (o.collision(fr, rows=rows, with_abs=True), o.rk4(f, 1.0, 3))
    return _largest[key]


@pytest.mark.parametrize("precision,layout,tol,tol_gross", [("fp32", 0, 1e-6, 1e-6), ("ff", 0, 1e-12, 1e-13),
                                                             ("ff", 1, 1e-12, 1e-13), ("c32", 0, 1e-6, 1e-6),
                                                             ("c32", 1, 1e-6, 1e-6)])
def test_batch_largest_instances_sampled(pb, precision, layout, tol, tol_gross):
    """The 36^3 instances of the batched workload (the largest rows: 4 bands, 5 modes, and 2
    bands, 6 modes), batched with a small one, against the oracle at the bounds of each
    precision and layout: df/dt at a random population on sampled rows (relative to the gross
    scattering) and f after 3 RK4 steps from the hot population (normwise)."""
    import torch

    inst = [synth.make_batch_instance(i) for i in (38, 16, 0)]
    chs = [pb.Channels.from_model(m) for m, _ in inst]
    b = pb.Batch(chs, precision=precision, layout=layout)
    assert b.tiled == (precision != "fp32" and layout == 0)
    fr = np.random.default_rng(29).uniform(0, 1, b.nstate)
    I = b.collision(torch.tensor(fr, device="cuda")).cpu().numpy()
    f = np.concatenate([m.f_hot(e_exc=e).reshape(-1)[c.state_ids()] for (m, e), c in zip(inst, chs)])
    ft = torch.tensor(f, device="cuda")
    b.rk4(ft, 1.0, 3)
    got = ft.cpu().numpy()
    for i, ((m, e), ch) in enumerate(zip(inst, chs)):
        a, z = b.offsets[i], b.offsets[i + 1]
        rows = np.unique(np.concatenate([np.arange(0, ch.nstate, 41), [ch.nstate - 1]]))
        (ref, ab), fref = _largest_reference(m, e, fr[a:z], f[a:z], rows)
        d = np.abs(I[a:z][rows] - ref).max()
        assert d <= tol_gross * ab.max(), f"instance {i}: {d / ab.max():.2e} of the gross scattering"
        assert np.abs(got[a:z] - fref).max() <= tol * np.abs(fref).max()


# ------------------------------------------------------------------ symmetric tiles: ragged blocks, fallback

def _three_band_window():
    # the fourth band's window empty: 81 / 99 states on 11^3 / 13^3, odd ragged last blocks
    w = np.array([[e - 1.0, e + 0.3] for e in (0.0, 0.2, 1.1, 1.3)])
    w[3] = [-10.0, -9.0]
    return w


@pytest.mark.parametrize("precision,tol,tol_gross", [("ff", 1e-12, 1e-13), ("c32", 1e-6, 1e-6)])
def test_tile_batch_ragged_blocks(pb, precision, tol, tol_gross):
    """Instances whose states fill their last 64-state block partly (81 = 64 + 17, 99 = 64 + 35,
    and one with fewer than 64 states), batched in the symmetric-tile form (layout 2): each instance's
    df/dt and 3 RK4 steps against its oracle, and the partials of one instance never reach
    another (each is checked on its own)."""
    import torch

    win = _three_band_window()
    models = [synth.make_window4(11, win=win), synth.make_tiny(3), synth.make_window4(13, win=win)]
    chs = [pb.Channels.from_model(m) for m in models]
    b = pb.Batch(chs, precision=precision, layout=2)  # tiles (they stream more bytes than rows here)
    assert b.tiled
    ns = [c.nstate for c in chs]
    assert ns[0] == 81 and ns[2] == 99 and ns[1] < 64
    rng = np.random.default_rng(41)
    fr = rng.uniform(0, 1, b.nstate)
    I = b.collision(torch.tensor(fr, device="cuda")).cpu().numpy()
    f0 = np.concatenate([oracle.Oracle(m).window_values(m.f_hot()) for m in models])
    ft = torch.tensor(f0, device="cuda")
    b.rk4(ft, 1.0, 3)
    got = ft.cpu().numpy()
    b.check()
    for i, m in enumerate(models):
        a, z = b.offsets[i], b.offsets[i + 1]
        o = oracle.Oracle(m)
        ref, ab = o.collision(fr[a:z], with_abs=True)
        assert np.abs(I[a:z] - ref).max() <= tol_gross * ab.max()
        fref = o.rk4(f0[a:z], 1.0, 3)
        assert np.abs(got[a:z] - fref).max() <= tol * np.abs(fref).max()


def test_tiles_and_rows_agree(pb, batch):
    """The two layouts of each precision on the same instances: float-float to a few 1e-14 of
    the gross scattering (different rounding of the merged coefficients and summation orders),
    the FP32 pairs to their 1e-6 bound."""
    import torch

    inst, chs, _, _ = batch
    fr = torch.tensor(np.random.default_rng(43).uniform(0, 1, sum(c.nstate for c in chs)), device="cuda")
    for precision, tol in (("ff", 1e-13), ("c32", 2e-6)):
        a = pb.Batch(chs, precision=precision).collision(fr).cpu().numpy()
        r = pb.Batch(chs, precision=precision, layout=1).collision(fr).cpu().numpy()
        assert np.abs(a - r).max() <= tol * np.abs(r).max(), precision


@pytest.mark.parametrize("precision,tol_gross", [("ff", 1e-13), ("c32", 1e-6)])
def test_tile_batch_sparse_rows(pb, precision, tol_gross):
    """Rows that are far from complete (the |g| and delta cutoffs on, and acoustic-only
    instances with no channel between states of one k point), in tiles (layout 2; the automatic
    choice keeps such sparse rows): the tiles hold zeros where a pair has no channel, and each
    instance meets its identically pruned oracle."""
    import torch

    m1 = synth.make_window4(12)
    m2 = synth.make_window4(16)
    m3, _ = small_instances(1)[0]  # 17^3, 3 acoustic modes: rows of 160 of 162 states
    cut = dict(g2_min=5e-4, delta_nsigma=4.0)
    chs = [pb.Channels.from_model(m1), pb.Channels.from_model(m2, **cut), pb.Channels.from_model(m3)]
    assert not pb.Batch(chs, precision=precision).tiled  # the tiles would stream more bytes here
    b = pb.Batch(chs, precision=precision, layout=2)
    assert b.tiled
    fr = np.random.default_rng(47).uniform(0, 1, b.nstate)
    I = b.collision(torch.tensor(fr, device="cuda")).cpu().numpy()
    for i, o in enumerate([oracle.Oracle(m1), oracle.Oracle(m2, **cut), oracle.Oracle(m3)]):
        a, z = b.offsets[i], b.offsets[i + 1]
        ref, ab = o.collision(fr[a:z], with_abs=True)
        assert np.abs(I[a:z] - ref).max() <= tol_gross * ab.max(), i
    b.check()


def test_tile_batch_needs_a_closure_checked_list(pb):
    """A list built without the closure check may lack reverse channels, which the tiles would
    supply: such a batch streams rows, as the single-system device does."""
    import torch

    m = synth.make_window4(12)
    chs = [pb.Channels.from_model(m, check_closure=False)]
    b = pb.Batch(chs, precision="ff")
    assert not b.tiled
    with pytest.raises(pb.PBError) as e:
        pb.Batch(chs, precision="ff", layout=2)
    assert e.value.code == pb.PB_EINVAL
    fr = np.random.default_rng(53).uniform(0, 1, b.nstate)
    ref, ab = oracle.Oracle(m).collision(fr, with_abs=True)
    assert np.abs(b.collision(torch.tensor(fr, device="cuda")).cpu().numpy() - ref).max() <= 1e-13 * ab.max()


_traj = {}


@pytest.mark.parametrize("precision,tol,tol_n", [("ff", 1e-12, 1e-12), ("c32", 1e-6, 1e-5)])
def test_tile_batch_200_step_trajectory(pb, precision, tol, tol_n):
    """200 RK4 steps of 1 fs of three small instances in one tile batch (the stages alternate
    the tile order) against each instance's oracle trajectory, normwise, and the carrier number
    of every instance conserved (sum_s I_s = 0 on a closed list: to rounding in float-float; the
    FP32 net terms enter a state's row sum and its partner's column sum grouped differently, so
    there it drifts by the FP32 rounding of the sums)."""
    import torch

    inst = small_instances(3)
    chs = [pb.Channels.from_model(m) for m, _ in inst]
    b = pb.Batch(chs, precision=precision, layout=2)  # tiles (these small rows would stay rows)
    assert b.tiled
    f = np.concatenate([m.f_hot(e_exc=e).reshape(-1)[c.state_ids()] for (m, e), c in zip(inst, chs)])
    ft = torch.tensor(f, device="cuda")
    b.rk4(ft, 1.0, 200)
    got = ft.cpu().numpy()
    b.check()
    for i, ((m, e), ch) in enumerate(zip(inst, chs)):
        a, z = b.offsets[i], b.offsets[i + 1]
        if m.name not in _traj:
            _traj[m.name] = oracle.Oracle(m).rk4(f[a:z], 1.0, 200)
        ref = _traj[m.name]
        assert np.abs(got[a:z] - ref).max() <= tol * np.abs(ref).max(), i
        assert abs(got[a:z].sum() - f[a:z].sum()) <= tol_n * f[a:z].sum()
