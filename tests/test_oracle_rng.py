"""Pins of the oracle's random numbers: Philox4x32-10 against published known
answers and statistical properties, Box-Muller against closed forms."""
import math
from fractions import Fraction

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


def test_box_muller21_closed_forms(orc):
    # a = 2^21 - 1: u1 = 1 -> radius 0; a = 0: u1 = 2^-21 -> radius sqrt(42 ln 2)
    z0, z1 = orc.box_muller21((1 << 21) - 1, 12345)
    assert z0 == 0.0 and abs(z1) == 0.0
    r = math.sqrt(42.0 * math.log(2.0))
    z0, z1 = orc.box_muller21(0, 0)
    assert z0 == pytest.approx(r, rel=1e-15) and z1 == 0.0
    z0, z1 = orc.box_muller21(0, 1 << 19)  # u2 = 1/4: angle pi/2
    assert abs(z0) < 1e-15 and z1 == pytest.approx(r, rel=1e-15)
    z0, z1 = orc.box_muller21(0, 1 << 20)  # u2 = 1/2: angle pi
    assert z0 == pytest.approx(-r, rel=1e-15) and abs(z1) < 1e-14


def test_uniforms21_partition_the_block(orc):
    # the six 21-bit integers take 126 distinct bits of the block: each used input
    # bit sets exactly one output bit, no two input bits the same one (so the map
    # is a bijection onto the integers); bits 10 of words 1 and 3 are unused
    images = set()
    for word in range(4):
        for bit in range(32):
            w = np.zeros(4, dtype=np.uint32)
            w[word] = np.uint32(1) << np.uint32(bit)
            u = orc.uniforms21(w)
            nz = np.nonzero(u)[0]
            if (word, bit) in ((1, 10), (3, 10)):
                assert nz.size == 0
                continue
            v = int(u[nz[0]])
            assert nz.size == 1 and v & (v - 1) == 0 and v < (1 << 21)
            images.add((int(nz[0]), v.bit_length() - 1))
    assert len(images) == 126


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
    # force normal n uses draw 1 + n // 6; slots 2p, 2p+1 are the pair (u_2p, u_2p+1)
    seed, ctrl, k, it = 9, 4, 17, (1 << 33) + 5
    w = orc.philox4x32_10([k, 1 + 2, it & 0xFFFFFFFF, it >> 32], [seed, ctrl])
    u = orc.uniforms21(w)
    want = []
    for p in range(3):
        want += list(orc.box_muller21(int(u[2 * p]), int(u[2 * p + 1])))
    got = [orc.normal(seed, ctrl, k, n, it) for n in range(12, 18)]
    assert got == want
    w0 = orc.philox4x32_10([k, 0, it & 0xFFFFFFFF, it >> 32], [seed, ctrl])
    assert orc.freq_normal(seed, ctrl, k, it) == orc.box_muller(int(w0[0]), int(w0[1]))[0]


def test_quantise_freq(orc):
    # q = round(1000 clip(mu + sigma z)) in mHz (Sec. IV-C, FP64); clipping at both ends
    q, m = orc.quantise_freq(2.0, 0.3, 0.0, 1.0, 4.0)
    assert q == 2000 and m == pytest.approx(0.5)
    q, _ = orc.quantise_freq(2.0, 0.3, -100.0, 1.0, 4.0)
    assert q == 1000
    q, _ = orc.quantise_freq(2.0, 0.3, 100.0, 1.0, 4.0)
    assert q == 4000
    # against exact rational arithmetic on the same double inputs: the FP64 value
    # rounds the same way except within ~1e-9 mHz of a half-integer, and the
    # margin is the distance to that boundary
    rng = np.random.default_rng(0)
    for mu, sig in ((2.0, 0.3), (1.7351, 0.0731), (3.9, 0.5)):
        for z in rng.normal(size=700):
            q, margin = orc.quantise_freq(mu, sig, float(z), 1.0, 4.0)
            f = Fraction(mu) + Fraction(sig) * Fraction(float(z))
            f = min(Fraction(4), max(Fraction(1), f))
            t = 1000 * f
            exact_q = math.floor(t + Fraction(1, 2))
            exact_m = abs((t - math.floor(t)) - Fraction(1, 2))
            assert margin == pytest.approx(float(exact_m), abs=1e-9)
            if exact_m > 1e-9:
                assert q == exact_q
            else:
                assert q in (exact_q - 1, exact_q)

def test_normals6_equals_per_entry_normals(orc):
    # one Philox block and its three Box-Muller pairs give the six normals of a draw
    for seed, ctrl, k, d, it in ((0, 0, 0, 1, 0), (7, 3, 12345, 9, 2 ** 33 + 5), (1, 255, 99, 50, 17)):
        got = orc.normals6(seed, ctrl, k, d, it)
        want = [orc.normal(seed, ctrl, k, 6 * (d - 1) + s, it) for s in range(6)]
        assert list(got) == want
