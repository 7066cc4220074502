"""Pins of the oracle's random-number layer against its published definition."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert oracle.philox(ctr, key) == out


def test_normals_are_standard():
    # Box-Muller output (Section 3 noise, Algorithm 5 momenta): moments and a KS distance
    z = np.concatenate([oracle.normals(123, 0, 0, oracle.P_NOISE, s, t, 64) for s in range(40) for t in range(8)])
    assert abs(z.mean()) < 4 / math.sqrt(len(z))
    assert abs(z.var() - 1.0) < 6 * math.sqrt(2.0 / len(z))
    zs = np.sort(z)
    cdf = 0.5 * (1 + np.vectorize(math.erf)(zs / math.sqrt(2)))
    ks = np.max(np.abs(cdf - (np.arange(1, len(zs) + 1) / len(zs))))
    assert ks < 1.63 / math.sqrt(len(zs))  # 1% critical value


def test_counter_streams_are_distinct():
    a = oracle.normals(1, 0, 0, oracle.P_NOISE, 0, 1, 8)
    b = oracle.normals(1, 0, 0, oracle.P_NOISE, 0, 2, 8)
    c = oracle.normals(1, 0, 0, oracle.P_PRUNE, 0, 1, 8)
    d = oracle.normals(1, 1, 0, oracle.P_NOISE, 0, 1, 8)
    for u, v in [(a, b), (a, c), (a, d)]:
        assert not np.allclose(u, v)


def test_normals_follow_the_counter_layout():
    # block b of (key=(seed_lo, seed_hi ^ run), ctr=(b, step, slot, iter<<4 | purpose)) feeds components 4b..4b+3
    seed, run, it, purpose, slot, step = 0x1234567887654321, 5, 9, oracle.P_MOM, 17, 3
    z = oracle.normals(seed, run, it, purpose, slot, step, 8)
    key = [seed & 0xFFFFFFFF, (seed >> 32) ^ run]
    for b in range(2):
        w = oracle.philox([b, step, slot, (it << 4) | purpose], key)
        u = [((x >> 9) + 0.5) / 8388608.0 for x in w]
        r0, r1 = math.sqrt(-2 * math.log(u[0])), math.sqrt(-2 * math.log(u[2]))
        ref = [r0 * math.cos(2 * math.pi * u[1]), r0 * math.sin(2 * math.pi * u[1]),
               r1 * math.cos(2 * math.pi * u[3]), r1 * math.sin(2 * math.pi * u[3])]
        np.testing.assert_allclose(z[4 * b:4 * b + 4], ref, rtol=1e-13, atol=1e-13)
