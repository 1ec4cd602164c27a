"""Device random-number layer against the oracle: Philox words bit-exact,
proposal normals within the FP32 (or FP64) error of Box-Muller."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _counters(n, seed=0):
    rng = np.random.default_rng(seed)
    t = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    v = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    c = rng.integers(0, 2 ** 24, n, dtype=np.uint64).astype(np.uint32)
    t[:4] = [0, 1, 0xFFFFFFFF, 5000]
    v[:4] = [0, 999_999, 0xFFFFFFFF, 7]
    c[:4] = [0, 3, 0xFFFFFF, 1]
    return t, v, c


@pytest.mark.parametrize("seed", [0, 1002, 0xFFFFFFFFFFFFFFFF, 0x0123456789ABCDEF])
def test_philox_words_bit_exact(gac, orc, seed):
    n, nw = 1_000_000, 11
    t, v, c = _counters(n, seed & 0xFFFF)
    out = np.zeros((n, nw), np.uint32)
    gac.gac_philox_words(seed, t, v, c, n, nw, out)
    np.testing.assert_array_equal(out, orc.words_many(seed, t, v, c, nw))


@pytest.mark.parametrize("n_par", [2, 4, 9])
def test_normals_against_oracle(gac, orc, n_par):
    n = 200_000
    t, v, c = _counters(n, n_par)
    seed = 1234567
    nw = orc.n_words(n_par)
    w_ref = orc.words_many(seed, t, v, c, nw)
    z_ref = orc.normals_many(w_ref, n_par)
    # FP32: hardware sin/cos (~4e-7 absolute) times a radius <= 6.7; u1 rounded
    # to float makes the radius 0 instead of <= 2.4e-4 when u1 > 1 - 2^-25.
    for prec, tol, tail in ((gac.PREC_MIXED, 4e-6, 2.5e-4), (gac.PREC_FP64, 1e-13, 1e-13)):
        z = np.zeros((n, n_par))
        wa = np.zeros(n, np.uint32)
        gac.gac_normals(seed, t, v, c, n, n_par, prec, z, wa)
        np.testing.assert_array_equal(wa, w_ref[:, nw - 1])
        err = np.abs(z - z_ref)
        assert np.quantile(err, 1 - 1e-5) <= tol, (prec, np.quantile(err, 1 - 1e-5))
        assert err.max() <= tail, (prec, err.max())
