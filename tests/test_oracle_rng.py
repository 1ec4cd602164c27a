"""Pins of the oracle's random-number layer against things other than itself.

- Philox4x32-10 known-answer vectors of the Random123 distribution (Salmon et
  al., SC'11) -- they cover all four counter words and both key words;
- cuRAND's *host* Philox4x32-10 generator (a library routine run on the CPU):
  its output block j is Philox(ctr = (j>>16, j>>48, j & 0xffff, 0),
  key = (seed lo, seed hi)), so it pins counter words 0-2 and the key;
- Box-Muller invariants (radius and angle identities) and the distribution of
  the normals (moments and a Kolmogorov-Smirnov test against scipy).
"""
import ctypes as ct
import ctypes.util
import glob
import os

import numpy as np
import pytest
from scipy import stats

KAT = [  # (ctr, key, expected) -- Random123 kat_vectors, philox4x32 10 rounds
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,expected", KAT)
def test_philox_known_answers(orc, ctr, key, expected):
    assert tuple(int(x) for x in orc.philox(ctr, key)) == expected


def _curand_host():
    cands = []
    for d in (os.environ.get("CUDA_HOME", "/usr/local/cuda"), "/usr/local/cuda"):
        cands += sorted(glob.glob(os.path.join(d, "lib64", "libcurand.so*")))
        cands += sorted(glob.glob(os.path.join(d, "targets", "*", "lib", "libcurand.so*")))
    found = ctypes.util.find_library("curand")
    if found:
        cands.append(found)
    for c in cands:
        try:
            return ct.CDLL(c)
        except OSError:
            continue
    return None


def _curand_block(lib, seed, offset_words, n_words=4):
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    gen = ct.c_void_p()
    assert lib.curandCreateGeneratorHost(ct.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ct.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ct.c_ulonglong(offset_words)) == 0
        buf = (ct.c_uint * n_words)()
        assert lib.curandGenerate(gen, buf, ct.c_size_t(n_words)) == 0
        return [int(x) for x in buf]
    finally:
        lib.curandDestroyGenerator(gen)


@pytest.mark.parametrize("seed", [0, 1, 77, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(orc, seed):
    lib = _curand_host()
    if lib is None:
        pytest.skip("libcurand not found")
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for j in [0, 1, 2, 3, 65535, 65536, 65537, 3 * 65536 + 2, (1 << 48) + 5 * 65536 + 3,
              (1 << 48) * 3 + (0xFFFFFFFF << 16) + 0xFFFC]:
        got = _curand_block(lib, seed, 4 * j)
        ctr = (j >> 16) & 0xFFFFFFFF, j >> 48, j & 0xFFFF, 0
        assert got == [int(x) for x in orc.philox(ctr, key)], (seed, j)


def test_word_layout(orc):
    """Call k of iteration t, voxel v, chain c uses ctr (t, v, c<<8 | k, 0) and
    key (seed lo, seed hi); its four words are words 4k..4k+3."""
    seed = 0x0123456789ABCDEF
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for t, v, c in [(1, 0, 0), (4999, 999_999, 3), (0xFFFFFFFF, 7, 2)]:
        w = orc.words(seed, t, v, c, 11)
        ref = np.concatenate([orc.philox((t, v, (c << 8) | k, 0), key) for k in range(3)])[:11]
        np.testing.assert_array_equal(w, ref)


def test_u01_open_interval_and_exact(orc):
    assert orc.u01(0) == 0.5 * 2.0 ** -32
    assert orc.u01(0xFFFFFFFF) == 1.0 - 0.5 * 2.0 ** -32
    assert 0.0 < orc.u01(0) < orc.u01(0xFFFFFFFF) < 1.0
    assert orc.u01(1 << 31) == 0.5 + 0.5 * 2.0 ** -32


def test_n_words(orc):
    # two words per Box-Muller pair, then one acceptance word
    assert [orc.n_words(p) for p in (1, 2, 3, 4, 9)] == [3, 3, 5, 5, 11]


def test_box_muller_radius_and_angle(orc):
    rng = np.random.default_rng(5)
    for _ in range(200):
        w = rng.integers(0, 2 ** 32, size=10, dtype=np.uint64).astype(np.uint32)
        z = orc.normals_from_words(w, 10)
        for j in range(5):
            u1, u2 = orc.u01(int(w[2 * j])), orc.u01(int(w[2 * j + 1]))
            # z_{2j}^2 + z_{2j+1}^2 = -2 ln u1 ; atan2(z_{2j+1}, z_{2j}) = 2 pi u2 (mod 2 pi)
            assert np.isclose(z[2 * j] ** 2 + z[2 * j + 1] ** 2, -2 * np.log(u1), rtol=1e-13)
            ang = np.arctan2(z[2 * j + 1], z[2 * j]) % (2 * np.pi)
            assert np.isclose(ang, (2 * np.pi * u2) % (2 * np.pi), atol=1e-11) or \
                abs(ang - (2 * np.pi * u2) % (2 * np.pi)) > 2 * np.pi - 1e-11
    # odd P drops the sine of the last pair
    w = rng.integers(0, 2 ** 32, size=10, dtype=np.uint64).astype(np.uint32)
    np.testing.assert_array_equal(orc.normals_from_words(w, 9), orc.normals_from_words(w, 10)[:9])


def test_normals_distribution(orc):
    """Normals of many (t, voxel, chain) draws are N(0,1): moments and KS."""
    zs = []
    for v in range(2000):
        for t in range(1, 51):
            zs.append(orc.normals_from_words(orc.words(99, t, v, 1, 11), 9))
    z = np.concatenate(zs)
    assert z.size == 900_000
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
    assert abs(stats.skew(z)) < 5 * np.sqrt(6.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the acceptance words are uniform
    u = np.array([orc.u01(int(orc.words(99, t, v, 1, 11)[10])) for v in range(200) for t in range(1, 51)])
    assert stats.kstest(u, "uniform").pvalue > 1e-3
