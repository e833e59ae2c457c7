"""The seeded input generator: determinism and the exact symmetries the inputs carry."""
import itertools

import numpy as np

import synth


def _ik(j, n):
    return (j[..., 0] * n + j[..., 1]) * n + j[..., 2]


def test_g2_swap_and_cubic_invariance():
    m = synth.make_window4(10)
    n, nb = 10, m.nbands
    rng = np.random.default_rng(0)
    for _ in range(200):
        j, jp = rng.integers(0, n, 3), rng.integers(0, n, 3)
        a, b, nu = int(rng.integers(0, nb)), int(rng.integers(0, nb)), int(rng.integers(0, m.nmodes))
        s, p = int(_ik(j, n)) * nb + a, int(_ik(jp, n)) * nb + b
        g = m.g2(s, p, nu)
        assert g == m.g2(p, s, nu)
        perm = rng.permutation(3)
        sign = rng.choice([-1, 1], 3)
        tj, tjp = (sign * j[perm]) % n, (sign * jp[perm]) % n
        assert g == m.g2(int(_ik(tj, n)) * nb + a, int(_ik(tjp, n)) * nb + b, nu)
        assert 0.0 < g < 1.0


def test_g2_lognormal_statistics():
    m = synth.make_tiny(8)
    ids = np.arange(0, 1024, 7, dtype=np.int32)
    g = m.g2_dense(ids, ids)
    iu = np.triu_indices(len(ids), 1)
    lg = np.log(g[iu[0], iu[1], :]).ravel()
    assert abs(lg.mean() - m.g2_mu) < 0.05 and abs(lg.std() - m.g2_sigma_ln) < 0.05


def test_bands_phonons_velocities_symmetric():
    n = 12
    m = synth.make_window4(n)
    j = m.kcoords()
    for perm, sign in itertools.product(itertools.permutations(range(3)), itertools.product([-1, 1], repeat=3)):
        tj = (np.array(sign) * j[:, list(perm)]) % n
        ik2 = _ik(tj, n)
        assert np.array_equal(m.eps[ik2], m.eps)
        assert np.array_equal(m.omega[ik2], m.omega)
        # v transforms as a vector: v'(Rk) = R v(k)
        assert np.array_equal(m.vel[ik2][:, :, :], (np.array(sign)[None, None, :] * m.vel[:, :, list(perm)]))


def test_named_configs():
    m = synth.make_config("tiny")
    assert m.nk == (8, 8, 8) and m.nbands == 2 and m.nmodes == 3 and m.win is None
    assert m.sigma == 0.005 and m.T == 300.0
    m1 = synth.make_config("window40")
    assert m1.nk == (40, 40, 40) and m1.nbands == 4 and m1.nmodes == 6 and m1.sigma == 0.008
    assert np.allclose(m1.omega[:, 3:].max(axis=0), [0.035, 0.0475, 0.06])
    assert abs(m1.omega[:, :3].max() - 0.025) < 1e-12 and m1.omega[0, :3].max() == 0.0


def test_fp16_storage_range_covers_the_lognormal_couplings():
    """The FP16 |g|^2 storage (one power-of-two factor that maps the largest value into
    [2^9, 2^10)) keeps every coupling of the 24^3 workload a normal FP16 number, so each is
    rounded by at most 2^-11 relative: the premise of the 16-bit variant's error bound.  numpy's
    float16 conversion stands in for the device's round-to-nearest."""
    import paper_2511_03683_gb300 as pb

    g2 = pb.Channels.from_model(synth.make_config("window24")).export()["g2"]
    scale = 2.0 ** (9 - np.floor(np.log2(g2.max())))
    assert 2.0 ** 9 <= g2.max() * scale < 2.0 ** 10
    h = (g2 * scale).astype(np.float16)
    assert np.all(np.isfinite(h)) and h.min() >= np.float16(2.0 ** -14)
    rel = np.abs(h.astype(np.float64) / scale - g2) / g2
    assert rel.max() <= 2.0 ** -11
    print(f"span max/min = 2^{np.log2(g2.max() / g2.min()):.1f}, max relative rounding {rel.max():.2e}")
