"""Pins of the oracle's counter-based random numbers (heatbath of Sec. I and
the Metropolis test).

* the Philox4x64-10 block equals the published known-answer vector for a zero
  counter and key (Salmon et al., SC'11, Random123 distribution) and numpy's
  independent Philox bit generator for arbitrary counters and keys;
* uniforms lie in (0, 1) and pass a Kolmogorov-Smirnov test;
* normals (Box-Muller) pass a KS test against N(0, 1), with mean, variance and
  the correlation of the two members of a pair within 5 sigma; a wrong factor
  in the transform (a dropped -2 or 2 pi) fails the KS test;
* sources have E|eta_k|^2 = 1 (density exp(-|eta|^2)), real and imaginary
  parts independent N(0, 1/2);
* different counters and streams give different numbers, the same ones the
  same numbers.
"""
import numpy as np
import pytest

stats = pytest.importorskip("scipy.stats")


def test_philox_known_answer(orc):
    got = orc.philox([0, 0, 0, 0], [0, 0])
    want = [0x16554D9ECA36314C, 0xDB20FE9D672D0FDC, 0xD7E772CEE186176B, 0x7E68B68AEC7BA23B]
    assert [int(x) for x in got] == want


def _inc(c):
    c = list(c)
    for i in range(4):
        c[i] = (c[i] + 1) % (1 << 64)
        if c[i]:
            break
    return c


@pytest.mark.parametrize("ctr,key", [([5, 7, 0, 0], [123, 456]),
                                     ([2**64 - 1, 3, 9, 2**63], [2**64 - 1, 1]),
                                     ([0x243F6A8885A308D3, 0x13198A2E03707344, 1, 2],
                                      [0xA4093822299F31D0, 0x082EFA98EC4E6C89])])
def test_philox_matches_numpy(orc, ctr, key):
    # numpy's generator advances its counter before each block
    bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64),
                          key=np.array(key, dtype=np.uint64))
    raw = [int(x) for x in bg.random_raw(12)]
    c = list(ctr)
    for b in range(3):
        c = _inc(c)
        assert [int(x) for x in orc.philox(c, key)] == raw[4 * b: 4 * b + 4]


def test_uniforms(orc):
    u = orc.random_uniforms(5, orc.STREAM_METROPOLIS, 0, 200000)
    assert u.min() > 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    assert orc.metropolis_uniform(5, 0) == u[0]


def test_normals(orc):
    n = 400000
    z = orc.random_normals(11, orc.STREAM_MOMENTA, 4, n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    pairs = z.reshape(-1, 2)
    assert abs(np.mean(pairs[:, 0] * pairs[:, 1])) < 5 / np.sqrt(n / 2)


def test_momenta_and_sources(orc):
    L = (8, 8, 8, 8)
    P = orc.random_momenta(L, 3, 9)
    assert P.shape == (4096, 4, 8)
    assert stats.kstest(P.ravel(), "norm").pvalue > 1e-4
    eta = orc.random_sources(L, 2, 3, 9)
    assert eta.shape == (2, 2048, 4, 3)
    m = np.abs(eta) ** 2
    assert abs(m.mean() - 1.0) < 5 / np.sqrt(m.size)
    assert stats.kstest(np.sqrt(2.0) * eta.real.ravel(), "norm").pvalue > 1e-4
    assert stats.kstest(np.sqrt(2.0) * eta.imag.ravel(), "norm").pvalue > 1e-4
    assert abs(np.mean(eta.real * eta.imag)) < 5 * 0.5 / np.sqrt(m.size)


def test_counters_and_streams_separate(orc):
    a = orc.random_normals(1, 0, 0, 64)
    assert np.array_equal(a, orc.random_normals(1, 0, 0, 64))
    for other in (orc.random_normals(1, 0, 1, 64), orc.random_normals(1, 1, 0, 64),
                  orc.random_normals(2, 0, 0, 64)):
        assert not np.any(a == other)
