"""Pins of the oracle's likelihood families and the reflection equation (Section 2.3)."""
import math

import numpy as np
import pytest

import oracle
from paper_2312_03911_gb300 import workloads as W


def _fd_grad(lik, x, h=1e-6):
    g = np.zeros_like(x)
    for i in range(len(x)):
        e = np.zeros_like(x)
        e[i] = h
        g[i] = (lik.loglik(x + e) - lik.loglik(x - e)) / (2 * h)
    return g


@pytest.mark.parametrize("kind,d", [("iso", 5), ("mix", 6), ("dense", 7), ("dense_mix", 5), ("rosen", 6)])
def test_gradient_matches_central_differences(kind, d):
    w = W.small_workload(kind, d, 20, seed=3)
    lik = oracle.Likelihood.from_spec(w["spec"])
    rng = np.random.default_rng(0)
    for _ in range(5):
        x = rng.uniform(-0.6, 0.6, d)
        v, g = lik.loglik(x, grad=True)
        assert np.isfinite(v)
        fd = _fd_grad(lik, x)
        assert np.linalg.norm(g - fd) <= 1e-6 * max(1.0, np.linalg.norm(fd))


def test_iso_gaussian_is_the_normalised_density():
    d, s = 3, 0.3
    mu = np.array([0.1, -0.2, 0.05])
    lik = oracle.Likelihood(W.LIK_ISO, d, means=mu, sigma=[s])
    x = np.array([0.4, 0.1, -0.3])
    ref = -0.5 * np.sum((x - mu) ** 2) / s**2 - 0.5 * d * math.log(2 * math.pi * s**2)
    assert lik.loglik(x) == pytest.approx(ref, rel=1e-14)


def test_dense_reduces_to_iso_and_logdet():
    d, s = 4, 0.2
    mu = np.array([0.1, -0.2, 0.05, 0.3])
    iso = oracle.Likelihood(W.LIK_ISO, d, means=mu, sigma=[s])
    den = oracle.Likelihood(W.LIK_DENSE, d, means=mu, precision=np.eye(d) / s**2)
    x = np.array([0.4, 0.1, -0.3, 0.0])
    assert den.loglik(x) == pytest.approx(iso.loglik(x), rel=1e-12)
    rng = np.random.default_rng(1)
    prec, _, _, _ = W.dense_precision(rng, 9)
    lik = oracle.Likelihood(W.LIK_DENSE, 9, means=np.zeros(9), precision=prec)
    assert lik.logdet() == pytest.approx(np.linalg.slogdet(prec)[1], rel=1e-10)


def test_mixture_is_a_log_sum_exp_of_components():
    w = W.small_workload("mix", 5, 10, seed=4)
    sp = w["spec"]
    mix = oracle.Likelihood.from_spec(sp)
    x = np.full(5, 0.05)
    comps = [oracle.Likelihood(W.LIK_ISO, 5, means=sp["means"][k], sigma=[sp["sigma"][k]]).loglik(x)
             for k in range(4)]
    ref = math.log(sum(math.exp(c) for c in comps) / 4)
    assert mix.loglik(x) == pytest.approx(ref, rel=1e-12)


def test_rosenbrock_minimum_and_value():
    lik = oracle.Likelihood(W.LIK_ROSEN, 4, rosen_scale=0.05)
    v, g = lik.loglik(np.ones(4), grad=True)
    assert v == 0.0 and np.all(g == 0.0)
    x = np.array([0.0, 1.0, -1.0, 0.5])
    ref = -0.05 * sum(100 * (x[i + 1] - x[i] ** 2) ** 2 + (1 - x[i]) ** 2 for i in range(3))
    assert lik.loglik(x) == pytest.approx(ref, rel=1e-14)


def test_reflection_invariants():
    rng = np.random.default_rng(5)
    for _ in range(20):
        d = int(rng.integers(2, 40))
        p = rng.standard_normal(d)
        n = rng.standard_normal(d)
        n /= np.linalg.norm(n)
        q = oracle.reflect(p, n)
        assert np.linalg.norm(q) == pytest.approx(np.linalg.norm(p), rel=1e-13)   # |p'| = |p|
        assert np.dot(q, n) == pytest.approx(-np.dot(p, n), rel=1e-12, abs=1e-12)  # p'.n = -p.n
        np.testing.assert_allclose(oracle.reflect(q, n), p, rtol=1e-12, atol=1e-12)  # involution
        t = q - np.dot(q, n) * n
        np.testing.assert_allclose(t, p - np.dot(p, n) * n, atol=1e-12)  # tangential part kept


def test_posterior_parameter_gradient_formula():
    # d log L / d mu for the dense mixture: resp_k P (x - mu_k); checked by central differences in mu
    w = W.small_workload("dense_mix", 4, 10, seed=6)
    sp = w["spec"]
    lik = oracle.Likelihood.from_spec(sp)
    x = np.array([0.1, -0.2, 0.3, 0.05])
    g = lik.dmeans(x)
    h = 1e-6
    for k in range(sp["means"].shape[0]):
        for i in range(4):
            mp = sp["means"].copy(); mp[k, i] += h
            mm = sp["means"].copy(); mm[k, i] -= h
            lp = oracle.Likelihood.from_spec(dict(sp, means=mp)).loglik(x)
            lm = oracle.Likelihood.from_spec(dict(sp, means=mm)).loglik(x)
            assert g[k, i] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-7)
