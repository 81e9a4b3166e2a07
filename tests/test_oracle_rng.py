"""Pins of the oracle's random numbers: Philox4x32-10 against published known
answers and statistical properties, Box-Muller against closed forms."""
import math

import numpy as np
import pytest

from conftest import golden


def _kat():
    rows = []
    with open(golden("philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = orc.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want


def test_philox_bits_balanced(orc):
    # 20 000 blocks = 80 000 words: each of the 32 bit positions is set with
    # probability 1/2 (5 standard errors).
    words = []
    for k in range(20000):
        words.extend(orc.philox4x32_10([k, 7, 3, 0], [11, 13]))
    w = np.array(words, dtype=np.uint64)
    n = w.size
    for b in range(32):
        frac = ((w >> b) & 1).mean()
        assert abs(frac - 0.5) < 5 * 0.5 / math.sqrt(n)


def test_philox_counter_sensitivity(orc):
    # changing any counter or key word changes every output word (avalanche)
    base = orc.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        o = orc.philox4x32_10(c, [5, 6])
        assert all(int(a) != int(b) for a, b in zip(base, o))
    o = orc.philox4x32_10([1, 2, 3, 4], [5, 7])
    assert all(int(a) != int(b) for a, b in zip(base, o))


def test_box_muller_closed_forms(orc):
    # x = 0xffffffff: u1 = 1 -> radius 0 -> both normals 0
    z0, z1 = orc.box_muller(0xFFFFFFFF, 0x12345678)
    assert z0 == 0.0 and abs(z1) == 0.0
    # x = 0: u1 = 2^-24 -> radius sqrt(48 ln 2); y = 0: angle 0
    r = math.sqrt(48.0 * math.log(2.0))
    z0, z1 = orc.box_muller(0, 0)
    assert z0 == pytest.approx(r, rel=1e-15) and z1 == 0.0
    # y = 2^30: u2 = 1/4 -> angle pi/2
    z0, z1 = orc.box_muller(0, 1 << 30)
    assert abs(z0) < 1e-15 and z1 == pytest.approx(r, rel=1e-15)
    # y = 2^31: u2 = 1/2 -> angle pi
    z0, z1 = orc.box_muller(0, 1 << 31)
    assert z0 == pytest.approx(-r, rel=1e-15) and abs(z1) < 1e-14
    # the low 8 bits are ignored
    assert orc.box_muller(0x00000100, 0x100) == orc.box_muller(0x000001FF, 0x1FF)


def test_normal_moments(orc):
    # 200 000 normals of the force layout: mean 0, variance 1, kurtosis 3
    z = np.array([orc.normal(3, 1, k, n, 5) for k in range(5000) for n in range(40)])
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    kurt = np.mean(z ** 4)
    assert abs(kurt - 3.0) < 5 * math.sqrt(96.0 / n)
    # uncorrelated neighbours in the layout (cos/sin pair and across words)
    zz = z.reshape(5000, 40)
    for a, b in ((0, 1), (1, 2), (3, 4)):
        c = np.corrcoef(zz[:, a], zz[:, b])[0, 1]
        assert abs(c) < 5 / math.sqrt(5000)


def test_normal_counter_layout(orc):
    # normal n uses draw 1 + n // 4; slots 0,1 are words (0,1), slots 2,3 words (2,3)
    seed, ctrl, k, it = 9, 4, 17, (1 << 33) + 5
    w = orc.philox4x32_10([k, 1 + 2, it & 0xFFFFFFFF, it >> 32], [seed, ctrl])
    a0, a1 = orc.box_muller(int(w[0]), int(w[1]))
    b0, b1 = orc.box_muller(int(w[2]), int(w[3]))
    got = [orc.normal(seed, ctrl, k, n, it) for n in (8, 9, 10, 11)]
    assert got == [a0, a1, b0, b1]
    w0 = orc.philox4x32_10([k, 0, it & 0xFFFFFFFF, it >> 32], [seed, ctrl])
    assert orc.freq_normal(seed, ctrl, k, it) == orc.box_muller(int(w0[0]), int(w0[1]))[0]


def test_quantise_freq(orc):
    # q = round(1000 clip(mu + sigma z)) in mHz; clipping at both ends
    q, m = orc.quantise_freq(2.0, 0.3, 0.0, 1.0, 4.0)
    assert q == 2000 and m == pytest.approx(0.5)
    q, _ = orc.quantise_freq(2.0, 0.3, -100.0, 1.0, 4.0)
    assert q == 1000
    q, _ = orc.quantise_freq(2.0, 0.3, 100.0, 1.0, 4.0)
    assert q == 4000
    rng = np.random.default_rng(0)
    for z in rng.normal(size=2000):
        q, margin = orc.quantise_freq(2.0, 0.3, float(z), 1.0, 4.0)
        exact = 1000.0 * min(4.0, max(1.0, 2.0 + 0.3 * z))
        if margin > 1e-3:
            assert q == math.floor(exact + 0.5)
        else:
            assert q in (math.floor(exact), math.floor(exact) + 1)
