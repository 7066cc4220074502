"""Pins of the oracle's torus reward (Section 4, eq. torus) and periodic prior against the
closed-form normaliser of Appendix F and the invariance a wrapping walk must have."""
import itertools
import math

import numpy as np
import pytest

import oracle


def _z_recursion(n, c):
    """Appendix F: Z_1 = 2 pi c^3 + 3 pi c, Z_n = 2 pi Z_{n-1} + 3 pi c (2 pi)^(n-1)."""
    z = 2 * math.pi * c**3 + 3 * math.pi * c
    for m in range(2, n + 1):
        z = 2 * math.pi * z + 3 * math.pi * c * (2 * math.pi) ** (m - 1)
    return z


def _torus(n, alpha, beta, c):
    return oracle.Likelihood(oracle.LIK_TORUS, n, torus=(alpha, beta, c))


@pytest.mark.parametrize("n,alpha,beta,c", [(1, 1, 1, 2.5), (2, 2, 3, 3.5), (3, 1, 2, 4.0), (4, 3, 1, 5.0)])
def test_normaliser_recursion_matches_exact_grid_quadrature(n, alpha, beta, c):
    """R is a trigonometric polynomial of degree at most 3 max(alpha, beta) in each coordinate
    (integer alpha, beta), so the mean over M equispaced points per coordinate with
    M > 3 max(alpha, beta) is its exact average: (2 pi)^n times it is Z_n, which must equal the
    recursion.  R comes from the oracle's log-likelihood, which this pins as well."""
    lik = _torus(n, alpha, beta, c)
    M = 3 * max(alpha, beta) + 2
    g = 2 * math.pi * np.arange(M) / M
    tot = 0.0
    for x in itertools.product(g, repeat=n):
        tot += math.exp(lik.loglik(np.array(x)))
    z_grid = (2 * math.pi) ** n * tot / M**n
    assert z_grid == pytest.approx(_z_recursion(n, c), rel=1e-12)


def test_recursion_needs_whole_periods():
    """The recursion rests on the sine integrals vanishing over [0, 2 pi), which holds for an
    integer sine frequency alpha only (the appendix says rational): with alpha = 1/2 the
    sine factor of eq. z1 no longer integrates to 2 pi c^3 + 3 pi c."""
    c = 2.5
    x = (np.arange(200000) + 0.5) * (2 * math.pi / 200000)
    z_half = np.sum((np.sin(0.5 * x) + c) ** 3) * (2 * math.pi / 200000)
    assert abs(z_half - _z_recursion(1, c)) > 1.0
    z_one = np.sum((np.sin(x) + c) ** 3) * (2 * math.pi / 200000)
    assert z_one == pytest.approx(_z_recursion(1, c), rel=1e-10)


def test_score_matches_central_differences():
    rng = np.random.default_rng(7)
    lik = _torus(5, 2, 3, 6.0)
    for _ in range(20):
        x = rng.uniform(0, 2 * math.pi, 5)
        v, g = lik.loglik(x, grad=True)
        h = 1e-6
        fd = np.array([(lik.loglik(x + h * e) - lik.loglik(x - h * e)) / (2 * h) for e in np.eye(5)])
        np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-8)


def test_coordinate_parity_follows_the_paper():
    """Paper indices are 1-based: x_1, x_3, ... take the cosine (beta), x_2, x_4, ... the sine
    (alpha)."""
    lik = _torus(2, 2.0, 3.0, 4.0)
    x = np.array([0.3, 1.1])
    s = math.cos(3.0 * 0.3) + math.sin(2.0 * 1.1) + 4.0
    assert lik.loglik(x) == pytest.approx(3 * math.log(s), rel=1e-14)


def test_periodic_walk_keeps_the_torus_uniform():
    """With the slice covering the whole torus (L* below the minimum of L), no step is
    outside, the walk is free motion with momentum refresh and wrapping, and uniform start
    points must leave uniform; every output lies in [0, 2 pi)."""
    n = 3
    lik = _torus(n, 1, 2, 4.0)
    lo, hi = np.zeros(n), np.full(n, 2 * math.pi)
    rng = np.random.default_rng(5)
    outs = []
    for b in range(4):
        x0 = rng.uniform(0, 2 * math.pi, (400, n))
        cfg = oracle.make_cfg(seed=300 + b, noise_mode=1, delta_p=0.2, min_ref=0, max_ref=1, n_steps=40,
                              prune_after=0, periodic=1)
        o = oracle.hss_batch(lik, lo, hi, cfg, 0, x0, [lik.loglik(q) for q in x0], -1e300, 0.7)
        assert o["n_out"] == 0 and o["n_fallback"] == 0
        outs.append(o["x"])
    x = np.concatenate(outs)
    assert np.all(x >= 0.0) and np.all(x < 2 * math.pi)
    # the walk moved far enough to wrap
    u = x / (2 * math.pi)
    for i in range(n):
        us = np.sort(u[:, i])
        ks = np.max(np.abs(us - (np.arange(1, len(us) + 1) - 0.5) / len(us)))
        assert ks < 1.63 / math.sqrt(len(us)) + 0.5 / len(us)  # 1 % level


def test_torus_evidence_matches_the_normaliser():
    """Full runs (Algorithm 3) on the periodic prior U[0, 2 pi)^2: log Z = log Z_2 - 2 log 2 pi."""
    n, alpha, beta, c = 2, 1, 1, 2.5
    truth = math.log(_z_recursion(n, c)) - n * math.log(2 * math.pi)
    lik = _torus(n, alpha, beta, c)
    lo, hi = np.zeros(n), np.full(n, 2 * math.pi)
    zs, errs = [], []
    for r in range(6):
        cfg = oracle.make_cfg(n_live=200, n_steps=400, dt_init=0.1, delta_p=0.2, noise_mode=1, tol=1e-3,
                              termination=1, min_ref=1, max_ref=3, clustering=0, seed=21, run_id=r,
                              periodic=1)
        out = oracle.run(lik, lo, hi, cfg)
        assert out["status"] == 0 and out["terminated"] == 1
        zs.append(out["logz"])
        errs.append(out["logz_err"])
    mean, err = float(np.mean(zs)), float(np.mean(errs)) / math.sqrt(len(zs))
    assert abs(mean - truth) < 4 * err + 0.02
