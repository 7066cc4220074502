"""Pins of the oracle's HSS sampler (Algorithm 5) and full runs (Algorithm 3) against
closed forms, quadrature and the invariance the sampler must have."""
import math

import numpy as np
import pytest

import oracle
from paper_2312_03911_gb300 import workloads as W


def _ball_case(d, R=0.3, sig=0.1):
    lik = oracle.Likelihood(W.LIK_ISO, d, means=np.zeros(d), sigma=[sig])
    lstar = -0.5 * R * R / sig**2 - 0.5 * d * math.log(2 * math.pi * sig**2)
    return lik, lstar


def test_hss_keeps_the_slice_uniform():
    """Walkers started uniformly in the slice {L > L*} (a ball) must leave uniformly: the
    prior-volume rank u = (r/R)^d of the returned points is U(0,1)."""
    d, R = 12, 0.3
    lik, lstar = _ball_case(d, R)
    rng = np.random.default_rng(11)
    us = []
    for b in range(6):
        v = rng.standard_normal((300, d))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        x0 = v * R * rng.uniform(size=(300, 1)) ** (1.0 / d)
        cfg = oracle.make_cfg(seed=100 + b, noise_mode=1, delta_p=0.2)
        o = oracle.hss_batch(lik, -np.ones(d), np.ones(d), cfg, 0, x0, [lik.loglik(q) for q in x0], lstar, 0.01)
        assert np.all(o["logl"] > lstar)
        us.append(((o["x"] ** 2).sum(1) / R**2) ** (d / 2))
    u = np.concatenate(us)
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / len(u))


def test_trajectory_speed_is_conserved_without_noise():
    d = 6
    lik, lstar = _ball_case(d)
    x0 = np.full((4, d), 0.01)
    cfg = oracle.make_cfg(seed=3, delta_p=0.0, noise_mode=0, n_steps=60, min_steps=60, max_ref=10**6, prune_after=0)
    o = oracle.hss_batch(lik, -np.ones(d), np.ones(d), cfg, 0, x0, [lik.loglik(q) for q in x0], lstar, 0.02,
                         trace=True)
    tr = o["trace"]
    speed = np.linalg.norm(tr[:, :, d:2 * d], axis=2)
    np.testing.assert_allclose(speed, np.broadcast_to(speed[0], speed.shape), rtol=1e-12)
    assert tr[:, :, 2 * d + 1].sum() > 0  # reflections happened


def test_c1_evidence_matches_closed_form():
    w = W.workload("c1")
    truth = 2 * math.log(math.erf(1 / (0.1 * math.sqrt(2))) / 2)
    assert W.truth_logz(w) == pytest.approx(truth, rel=1e-13)
    assert truth == pytest.approx(-1.3862943611198906, rel=1e-12)
    lik = oracle.Likelihood.from_spec(w["spec"])
    zs, errs = [], []
    for r in range(12):
        out = oracle.run(lik, w["lo"], w["hi"], oracle.make_cfg(**dict(w["cfg"], run_id=r)))
        assert out["status"] == 0 and out["terminated"] == 1
        zs.append(out["logz"]); errs.append(out["logz_err"])
        assert abs(out["logz"] - truth) < 4 * out["logz_err"]
    zs = np.array(zs)
    assert abs(zs.mean() - truth) < 3.5 * np.mean(errs) / math.sqrt(len(zs))


def _gauss_legendre_2d(f, lo, hi, n=400):
    xg, wg = np.polynomial.legendre.leggauss(n)
    xs = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
    ws = 0.5 * (hi - lo) * wg
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    return np.sum(ws[:, None] * ws[None, :] * f(X, Y))


def test_rosenbrock_d2_against_grid_quadrature():
    scale = 1.0 / 20.0
    f = lambda x, y: np.exp(-scale * (100 * (y - x * x) ** 2 + (1 - x) ** 2))
    # piecewise quadrature on a grid fine enough for the banana ridge; prior density 1/16
    edges = np.linspace(-2, 2, 17)
    Z = 0.0
    for i in range(16):
        for j in range(16):
            xg, wg = np.polynomial.legendre.leggauss(48)
            xs = 0.5 * (edges[i + 1] - edges[i]) * xg + 0.5 * (edges[i + 1] + edges[i])
            ys = 0.5 * (edges[j + 1] - edges[j]) * xg + 0.5 * (edges[j + 1] + edges[j])
            wx = 0.5 * (edges[i + 1] - edges[i]) * wg
            wy = 0.5 * (edges[j + 1] - edges[j]) * wg
            X, Y = np.meshgrid(xs, ys, indexing="ij")
            Z += np.sum(wx[:, None] * wy[None, :] * f(X, Y))
    truth = math.log(Z / 16.0)
    w = W.small_workload("rosen", 2, 200, seed=5)
    lik = oracle.Likelihood.from_spec(w["spec"])
    zs, errs = [], []
    for r in range(10):
        out = oracle.run(lik, w["lo"], w["hi"], oracle.make_cfg(**dict(w["cfg"], run_id=r)))
        zs.append(out["logz"]); errs.append(out["logz_err"])
    assert abs(np.mean(zs) - truth) < 3.5 * np.mean(errs) / math.sqrt(len(zs)) + 0.02


def _posterior(out):
    lw = out["dead_logw"] + out["dead_logl"] - out["logz"]
    return np.exp(lw)


def test_posterior_weights_and_moments():
    w = W.workload("c1")
    lik = oracle.Likelihood.from_spec(w["spec"])
    means, ses = [], []
    for r in range(4):
        out = oracle.run(lik, w["lo"], w["hi"], oracle.make_cfg(**dict(w["cfg"], run_id=r)))
        p = _posterior(out)
        assert p.sum() == pytest.approx(1.0, abs=1e-12)
        ess = p.sum() ** 2 / np.sum(p**2)
        m = (p[:, None] * out["dead_x"]).sum(0)
        v = (p[:, None] * (out["dead_x"] - m) ** 2).sum(0)
        # the truncation at +-1 is 10 sigma away: posterior mean 0, variance 0.01
        assert np.all(np.abs(m) < 4 * math.sqrt(0.01 / ess))
        assert np.all(np.abs(v - 0.01) < 4 * 0.01 * math.sqrt(2 / ess))


def test_grad_logz_is_the_derivative_of_the_frozen_sample_estimate():
    w = W.small_workload("mix", 3, 100, seed=9)
    sp = w["spec"]
    lik = oracle.Likelihood.from_spec(sp)
    out = oracle.run(lik, w["lo"], w["hi"], oracle.make_cfg(**w["cfg"]))
    g = oracle.grad_logz_means(lik, out["dead_x"], out["dead_logl"], out["dead_logw"], out["logz"])

    def frozen_logz(means):
        l2 = oracle.Likelihood.from_spec(dict(sp, means=means))
        ll = np.array([l2.loglik(x) for x in out["dead_x"]])
        a = out["dead_logw"] + ll
        return a.max() + math.log(np.exp(a - a.max()).sum())

    h = 1e-5
    for k in range(sp["means"].shape[0]):
        for i in range(3):
            mp = sp["means"].copy(); mp[k, i] += h
            mm = sp["means"].copy(); mm[k, i] -= h
            fd = (frozen_logz(mp) - frozen_logz(mm)) / (2 * h)
            assert g[k, i] == pytest.approx(fd, rel=1e-4, abs=1e-6)


def test_grad_logz_statistically_matches_the_truncation_effect():
    mu, sig = 0.9, 0.1
    a, b = (-1 - mu) / sig, (1 - mu) / sig
    phi = lambda t: math.exp(-0.5 * t * t) / math.sqrt(2 * math.pi)
    Phi = lambda t: 0.5 * (1 + math.erf(t / math.sqrt(2)))
    truth = (phi(a) - phi(b)) / (sig * (Phi(b) - Phi(a)))
    lik = oracle.Likelihood(W.LIK_ISO, 2, means=[mu, mu], sigma=[sig])
    gs = []
    for r in range(8):
        cfg = oracle.make_cfg(**dict(W.DEFAULT_CFG, n_live=200, seed=31, run_id=r, clustering=0))
        out = oracle.run(lik, -np.ones(2), np.ones(2), cfg)
        gs.append(oracle.grad_logz_means(lik, out["dead_x"], out["dead_logl"], out["dead_logw"], out["logz"])[0])
    gs = np.array(gs)
    se = gs.std(0) / math.sqrt(len(gs)) + 1e-3
    assert np.all(np.abs(gs.mean(0) - truth) < 4 * se), (gs.mean(0), truth, se)


def test_keep_last_returns_the_last_inside_state():
    """The App. G ablation: a fixed number of steps (min_steps = n_steps, saving from the first
    step) and the last inside state kept, instead of a uniform pick over the saved states."""
    d = 4
    lik, lstar = _ball_case(d, R=0.3)
    rng = np.random.default_rng(2)
    v = rng.standard_normal((32, d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    x0 = v * 0.3 * rng.uniform(size=(32, 1)) ** (1.0 / d)
    cfg = oracle.make_cfg(seed=9, noise_mode=1, delta_p=0.2, min_ref=0, max_ref=10**6, n_steps=20, min_steps=20,
                          prune_after=0, keep_last=1)
    o = oracle.hss_batch(lik, -np.ones(d), np.ones(d), cfg, 0, x0, [lik.loglik(q) for q in x0], lstar, 0.05,
                         trace=True)
    tr = o["trace"]
    assert tr.shape[0] == 20
    for j in range(len(x0)):
        inside = np.nonzero(tr[:, j, 2 * d + 1] == 0)[0]
        if len(inside):
            np.testing.assert_array_equal(o["x"][j], tr[inside[-1], j, :d])
        else:
            np.testing.assert_array_equal(o["x"][j], x0[j])
