"""Host-side tests of the C ABI (no GPU): the library loads, exports every symbol the
header declares, and the channel builder (host C++) produces the CSR the paper's
problem statement defines, checked against the oracle's own enumeration."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pb():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2511_03683_gb300 as pb

    return pb


def test_every_declared_symbol_is_exported(pb):
    hdr = open(os.path.join(ROOT, "include", "pb.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(pb_[a-z0-9_]+)\s*\(", hdr))
    names -= {"pb_g2_fn"}
    assert len(names) >= 15
    L = ctypes.CDLL(pb.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    assert pb.lib().pb_version().decode().startswith("pb ")


def test_no_global_atomics_in_device_code():
    src = open(os.path.join(ROOT, "paper_2511_03683_gb300", "csrc", "kernels.cuh")).read()
    src += open(os.path.join(ROOT, "paper_2511_03683_gb300", "csrc", "device.cu")).read()
    code = re.sub(r"//[^\n]*", "", re.sub(r"/\*.*?\*/", "", src, flags=re.S))
    assert not re.search(r"\batomic[A-Za-z_]*\s*\(|\bred\.|\batom\.", code)


@pytest.mark.parametrize("model", [synth.make_tiny(4), synth.make_window4(12), synth.make_window4(16)],
                         ids=["tiny4", "win12", "win16"])
def test_builder_csr_matches_oracle_enumeration(pb, model):
    ch = pb.Channels.from_model(model)
    o = oracle.Oracle(model)
    assert ch.nstate == o.nstate
    assert ch.nchannels == o.count_channels()
    e = ch.export()
    assert np.array_equal(e["state_ids"], o.ids)
    rp = e["row_ptr"]
    assert rp[0] == 0 and rp[-1] == ch.nchannels and np.all(np.diff(rp) >= 0)
    nk = model.nk
    nb = model.nbands
    ik = o.ids // nb
    j = np.stack([ik // (nk[1] * nk[2]), (ik // nk[2]) % nk[1], ik % nk[2]], axis=1)
    for r in [0, 1, ch.nstate // 2, ch.nstate - 1]:
        cols = e["col"][rp[r]:rp[r + 1]]
        nus = e["nu"][rp[r]:rp[r + 1]]
        # sorted by (partner, nu), every partner in range
        key = cols.astype(np.int64) * 256 + nus
        assert np.all(np.diff(key) > 0)
        q = (j[cols] - j[r]) % np.array(nk)
        iq = (q[:, 0] * nk[1] + q[:, 1]) * nk[2] + q[:, 2]
        assert np.all(model.omega[iq, nus] > 0)
        # |g|^2 comes from the callback with full-grid ids
        g = [model.g2(int(o.ids[r]), int(o.ids[p]), int(v)) for p, v in zip(cols[:20], nus[:20])]
        assert np.array_equal(np.array(g), e["g2"][rp[r]:rp[r] + 20])


def test_python_callback_and_closure_check(pb):
    m = synth.make_tiny(3)
    sym = pb.Channels.build(m.nk, m.nbands, m.nmodes, m.eps, m.omega, m.T, m.sigma,
                            lambda s, p, nu: 1e-3 * (1.0 + 0.1 * ((s + p) % 7) + 0.01 * nu))
    assert sym.nchannels == (27 * 2) ** 2 * 3
    with pytest.raises(pb.PBError) as ei:
        pb.Channels.build(m.nk, m.nbands, m.nmodes, m.eps, m.omega, m.T, m.sigma,
                          lambda s, p, nu: 1e-3 * (1.0 + 0.1 * (s % 5)))
    assert ei.value.code == pb.PB_ENOTCLOSED
    with pytest.raises(pb.PBError) as ei:
        pb.Channels.build(m.nk, m.nbands, m.nmodes, m.eps, m.omega, m.T, m.sigma, lambda s, p, nu: -np.ones(len(s)))
    assert ei.value.code == pb.PB_ECALLBACK


def test_builder_rejects_bad_input(pb):
    m = synth.make_tiny(3)
    with pytest.raises(pb.PBError) as ei:
        pb.Channels.build(m.nk, m.nbands, m.nmodes, m.eps, m.omega, -1.0, m.sigma, m.g2_batch_ptr(), m.g2_user_ptr())
    assert ei.value.code == pb.PB_EINVAL
    win = np.array([[10.0, 11.0], [10.0, 11.0]])
    with pytest.raises(pb.PBError) as ei:
        pb.Channels.build(m.nk, m.nbands, m.nmodes, m.eps, m.omega, m.T, m.sigma, m.g2_batch_ptr(), m.g2_user_ptr(),
                          win=win)
    assert ei.value.code == pb.PB_EINVAL
    bad = m.eps.copy()
    bad[3, 1] = np.nan
    with pytest.raises(pb.PBError):
        pb.Channels.build(m.nk, m.nbands, m.nmodes, bad, m.omega, m.T, m.sigma, m.g2_batch_ptr(), m.g2_user_ptr())


def test_g2_cutoff_drops_channels_symmetrically(pb):
    m = synth.make_tiny(4)
    full = pb.Channels.from_model(m)
    cut = pb.Channels.from_model(m, g2_min=1e-3)
    g = full.export()["g2"]
    assert cut.nchannels == int((g >= 1e-3).sum()) < full.nchannels


def test_acoustic_only_gamma_has_no_channels(pb):
    """A 1x1x1 grid with only acoustic modes: hbar*w(Gamma) = 0 removes every channel."""
    eps = np.array([[0.0, 0.1]])
    ch = pb.Channels.build((1, 1, 1), 2, 1, eps, np.zeros((1, 1)), 300.0, 0.01, lambda s, p, nu: np.ones(len(s)))
    assert ch.nstate == 2 and ch.nchannels == 0


@pytest.mark.parametrize("g2_min,nsig", [(1e-3, 0.0), (0.0, 3.0), (5e-4, 4.0)])
def test_builder_cutoffs_match_oracle_count(pb, g2_min, nsig):
    m = synth.make_window4(16)
    ch = pb.Channels.from_model(m, g2_min=g2_min, delta_nsigma=nsig)
    assert ch.nchannels == oracle.Oracle(m, g2_min=g2_min, delta_nsigma=nsig).count_channels()


@pytest.mark.parametrize("field,bad", [("variant", 9), ("merge_branches", 3), ("dense_rows", 4), ("tile_sweep", 9),
                                       ("tile_sweep", -1), ("stream_mode", 3), ("channel_per_lane", 6),
                                       ("transport_gather", 8), ("ctas_per_sm", 9), ("item_channels", 100),
                                       ("adjoint", 2)])
def test_device_options_are_checked_on_the_host(pb, field, bad):
    """pb_dev_arena_bytes resolves and checks pb_dev_opts without touching a GPU: every field
    out of its documented range is PB_EINVAL, and the defaults size an arena."""
    import ctypes

    ch = pb.Channels.from_model(synth.make_window4(12))
    L = pb.lib()
    nbytes = ctypes.c_size_t(0)
    ok = pb._DevOpts()
    assert L.pb_dev_arena_bytes(ch._h, ctypes.byref(ok), ctypes.byref(nbytes)) == pb.PB_OK
    assert nbytes.value > 0
    o = pb._DevOpts()
    setattr(o, field, bad)
    assert L.pb_dev_arena_bytes(ch._h, ctypes.byref(o), ctypes.byref(nbytes)) == pb.PB_EINVAL


def test_adjoint_accumulators_are_sized_per_state_pair(pb):
    """adjoint = 1 reserves one float-float (u, v) accumulator of 16 bytes per sweep entry on a
    branch-merged FF device, three doubles per (state, partner) pair on G32, and nothing on
    the per-channel FF form."""
    import ctypes

    ch = pb.Channels.from_model(synth.make_window4(12))
    L = pb.lib()

    def arena(**kw):
        o = pb._DevOpts()
        for k, v in kw.items():
            setattr(o, k, v)
        n = ctypes.c_size_t(0)
        assert L.pb_dev_arena_bytes(ch._h, ctypes.byref(o), ctypes.byref(n)) == pb.PB_OK
        return n.value

    grow = arena(adjoint=1) - arena()
    assert 16 * ch.nchannels // 8 <= grow <= 16 * ch.nchannels + 4096
    assert arena(adjoint=1, merge_branches=2) == arena(merge_branches=2)
    g32 = pb.VARIANTS["g32"]
    grow = arena(adjoint=1, variant=g32) - arena(variant=g32)
    assert abs(grow - 24 * ch.nstate ** 2) <= 4096  # up to the alignment of the arena regions


def test_row_block_transport_partials_are_sized_per_row_and_segment(pb):
    """transport_gather 7 reserves one FP64 (x, y, z) partial of 32 bytes per (row, segment) and
    a row index of nstate + 1 int32 on complete rows with transport, and nothing otherwise: not
    without transport, not on the automatic shape, not on a list whose rows miss partners."""
    import ctypes

    L = pb.lib()

    def arena(ch, **kw):
        o = pb._DevOpts()
        for k, v in kw.items():
            setattr(o, k, v)
        n = ctypes.c_size_t(0)
        assert L.pb_dev_arena_bytes(ch._h, ctypes.byref(o), ctypes.byref(n)) == pb.PB_OK
        return n.value

    ch = pb.Channels.from_model(synth.make_window4(16))  # complete rows, 324 states
    ns = ch.nstate
    grow = arena(ch, transport=1, transport_gather=7) - arena(ch, transport=1)
    nseg = round(grow / (32 * ns))  # the segments (two at 324 states on any SM count of 3 or more)
    assert nseg >= 1 and abs(grow - (32 * ns * nseg + 4 * (ns + 1))) <= 2048  # up to the regions' alignment
    assert arena(ch, transport_gather=7) == arena(ch)
    cut = pb.Channels.from_model(synth.make_window4(12), g2_min=1e-3)
    assert arena(cut, transport=1, transport_gather=7) == arena(cut, transport=1)


def test_fp16_variant_sizes_like_bf16(pb):
    """The FP16 |g|^2 variant (h16) keeps 2 bytes per value like BF16 (g16): the same arena."""
    import ctypes

    ch = pb.Channels.from_model(synth.make_window4(12))
    L = pb.lib()
    sizes = []
    for v in ("g16", "h16"):
        o = pb._DevOpts()
        o.variant = pb.VARIANTS[v]
        n = ctypes.c_size_t(0)
        assert L.pb_dev_arena_bytes(ch._h, ctypes.byref(o), ctypes.byref(n)) == pb.PB_OK
        sizes.append(n.value)
    assert sizes[0] == sizes[1]
    o = pb._DevOpts()
    o.variant = 8
    assert L.pb_dev_arena_bytes(ch._h, ctypes.byref(o), ctypes.byref(ctypes.c_size_t(0))) == pb.PB_EINVAL


def test_c32_arena_and_options(pb):
    """The FP32 coefficient tiles (c32) hold 8 bytes per state pair of the upper block triangle
    instead of 16: the arena is the FF arena less 8 * tiles * 64^2 bytes (up to region
    alignment).  They need the symmetric tiles (automatic on complete rows, forced by
    dense_rows 3 on sparse ones) and the bulk-copy tile sweep: PB_EINVAL otherwise."""
    import ctypes

    m = synth.make_window4(12)
    ch = pb.Channels.from_model(m)
    L = pb.lib()

    def arena(chs, **kw):
        o = pb._DevOpts()
        for k, v in kw.items():
            setattr(o, k, v)
        n = ctypes.c_size_t(0)
        rc = L.pb_dev_arena_bytes(chs._h, ctypes.byref(o), ctypes.byref(n))
        return rc, n.value

    nb = (ch.nstate + 63) // 64
    nt = nb * (nb + 1) // 2
    rc_ff, ff = arena(ch)
    rc_32, c32 = arena(ch, variant=pb.VARIANTS["c32"])
    assert rc_ff == rc_32 == pb.PB_OK
    assert abs((ff - c32) - 8 * nt * 64 * 64) <= 256
    for kw in ({"tile_sweep": 1}, {"merge_branches": 2}, {"stream_mode": 2}, {"dense_rows": 2}):
        assert arena(ch, variant=pb.VARIANTS["c32"], **kw)[0] == pb.PB_EINVAL
    cut = pb.Channels.from_model(m, g2_min=5e-4, delta_nsigma=4.0)
    assert arena(cut, variant=pb.VARIANTS["c32"])[0] == pb.PB_EINVAL
    assert "symmetric tiles" in L.pb_last_error().decode()
    assert arena(cut, variant=pb.VARIANTS["c32"], dense_rows=3)[0] == pb.PB_OK


def acoustic_tiny(n):
    """The n^3 two-band model with three acoustic modes only (zero at Gamma: no channel joins
    the two states of one k point)."""
    t = synth.make_tiny(n)
    s = synth.acoustic_shape(t.nk).reshape(-1)
    return t.with_(omega=np.stack([15e-3 * s, 20e-3 * s, 25e-3 * s], axis=1))


def test_tiles_on_rows_that_miss_partners(pb):
    """The FF device takes the symmetric tiles (zero where a pair has no channel) on rows that
    miss few partners, when the tiles stream at most 0.7 of the rows' bytes: an acoustic-only
    model (no channel between the bands at one k point) gets them automatically, a list with the
    cutoffs on (a fifth of its pairs stored) keeps the rows unless dense_rows 3 forces the tiles;
    a list built without the closure check never gets them."""
    import ctypes

    L = pb.lib()

    def arena(chs, **kw):
        o = pb._DevOpts()
        for k, v in kw.items():
            setattr(o, k, v)
        n = ctypes.c_size_t(0)
        assert L.pb_dev_arena_bytes(chs._h, ctypes.byref(o), ctypes.byref(n)) == pb.PB_OK
        return n.value

    def tile_bytes(chs):
        nb = (chs.nstate + 63) // 64
        return 16 * nb * (nb + 1) // 2 * 64 * 64

    acoustic = pb.Channels.from_model(acoustic_tiny(5))
    assert acoustic.nchannels < acoustic.nstate ** 2 * 3  # no channel between the bands at one k
    assert arena(acoustic) - arena(acoustic, dense_rows=2) >= tile_bytes(acoustic)
    m = synth.make_window4(16)
    cut = pb.Channels.from_model(m, g2_min=5e-4, delta_nsigma=4.0)
    assert arena(cut, dense_rows=3) - arena(cut) >= tile_bytes(cut)
    unchecked = pb.Channels.from_model(m, g2_min=5e-4, delta_nsigma=4.0, check_closure=False)
    assert arena(unchecked, dense_rows=3) == arena(unchecked)


def test_batch_arena_and_layouts_on_the_host(pb):
    """pb_batch_arena_bytes sizes a batch arena without a GPU. The symmetric-tile form of a
    precision-1 batch (layout 2; layout 0 takes it when it streams fewer bytes) adds each
    instance's upper block triangle as 64 x 64 tiles of 16 B entries, one tile partial per padded
    state and partner block of the largest instance, and the padded maps to the rows' arena.
    Layouts out of range, and layout 2 on a list built without the closure check, are
    PB_EINVAL; such a list still sizes a row batch."""
    import ctypes

    m = synth.make_window4(12)
    chs = [pb.Channels.from_model(m), pb.Channels.from_model(synth.make_tiny(3))]
    unchecked = [pb.Channels.from_model(m, check_closure=False)]

    def arena(prec, layout, lists=chs):
        arr = (ctypes.c_void_p * len(lists))(*[c._h.value for c in lists])
        o = pb._BatchOpts(0, 0, prec, layout)
        n = ctypes.c_size_t(0)
        rc = pb.lib().pb_batch_arena_bytes(arr, len(lists), ctypes.byref(o), ctypes.byref(n))
        return rc, n.value

    blocks = [(c.nstate + 63) // 64 for c in chs]
    nt = sum(b * (b + 1) // 2 for b in blocks)
    nsp = 64 * sum(blocks)
    rc_rows, rows = arena(1, 1)
    rc_tiles, tiles = arena(1, 2)
    assert rc_rows == rc_tiles == pb.PB_OK
    assert 16 * nt * 4096 + 16 * nsp * max(blocks) <= tiles - rows <= 16 * nt * 4096 + 16 * nsp * max(blocks) + 65536
    rc_c32, c32 = arena(2, 2)
    assert rc_c32 == pb.PB_OK and 0 < c32
    for prec, layout in ((0, 2), (1, 3), (2, -1), (0, -1)):
        assert arena(prec, layout)[0] == pb.PB_EINVAL
    assert arena(1, 2, unchecked)[0] == pb.PB_EINVAL
    assert arena(1, 0, unchecked)[0] == pb.PB_OK
