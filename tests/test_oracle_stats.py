"""Pins of the Appendix H summary statistics against the stochastic model they average.

Killing the lowest of n_p live points of cluster p shrinks its volume by t ~ Beta(n_p, 1)
(the largest of n_p uniforms) and adds (1 - t) X_p L to the evidence; splitting a cluster of
n points into parts of n_i points shares its volume and evidence by D ~ Dirichlet(n_i).
The recursions update0-update9 and new0-new6 are the exact first and second moments of this
model, so a Monte Carlo of the model pins them independently of their algebra.
"""
import math

import numpy as np
import pytest

import oracle


def _mc(n0, ops, cap, n_mc=400000, seed=0):
    rng = np.random.default_rng(seed)
    X = np.zeros((cap, n_mc)); X[0] = 1.0
    Zp = np.zeros((cap, n_mc))
    Z = np.zeros(n_mc)
    n = np.zeros(cap, dtype=int); n[0] = n0
    alive = np.zeros(cap, bool); alive[0] = True
    for kind, p, v in ops:
        if kind == "kill":
            t = rng.uniform(size=n_mc) ** (1.0 / n[p])
            inc = (1 - t) * X[p] * math.exp(v)
            Z += inc; Zp[p] += inc; X[p] *= t; n[p] -= 1
        else:
            q = 0
            while alive[q] or q == p:
                q += 1
            a, b = int(v), n[p] - int(v)
            g1, g2 = rng.gamma(a, size=n_mc), rng.gamma(b, size=n_mc)
            D = g1 / (g1 + g2)
            X[q] = (1 - D) * X[p]; X[p] = D * X[p]
            Zp[q] = (1 - D) * Zp[p]; Zp[p] = D * Zp[p]
            n[q], n[p] = b, a; alive[q] = True
    return X, Z, Zp, n


def _check(mc_vals, logv, tol_sd=5.0):
    m = mc_vals.mean()
    se = mc_vals.std() / math.sqrt(len(mc_vals))
    assert abs(math.exp(logv) - m) <= tol_sd * se + 1e-12 * abs(m), (math.exp(logv), m, se)


def test_single_cluster_telescoping_closed_form():
    n, k = 9, 6
    L = np.linspace(-3.0, 1.0, k)
    out = oracle.stats_program(1, n, [("kill", 0, l) for l in L])
    # X after k kills = (n + 1 - k) / (n + 1); every kill takes mass 1/(n+1) of the initial volume
    assert out["logx"][0] == pytest.approx(math.log((n + 1 - k) / (n + 1)), rel=1e-13)
    assert out["logz"] == pytest.approx(math.log(np.sum(np.exp(L)) / (n + 1)), rel=1e-13)
    r = oracle.stats_sequence([n], [0.0], np.zeros(k, dtype=np.int32), L)
    np.testing.assert_allclose(r["logw"], np.full(k, -math.log(n + 1)), rtol=1e-13)


def test_kill_moments_single_cluster():
    n = 5
    ops = [("kill", 0, l) for l in (-1.0, -0.5, 0.0, 0.3)]
    out = oracle.stats_program(1, n, ops)
    X, Z, Zp, _ = _mc(n, ops, 1)
    _check(Z, out["logz"]); _check(Z ** 2, out["logz2"]); _check(X[0], out["logx"][0])
    _check(X[0] ** 2, out["logx2"][0]); _check(Z * X[0], out["logzx"][0])


def test_kill_and_split_moments_two_clusters():
    ops = [("kill", 0, -2.0), ("kill", 0, -1.5), ("split", 0, 3), ("kill", 1, -0.7), ("kill", 0, -0.4),
           ("kill", 1, 0.1), ("kill", 0, 0.2)]
    n0 = 9
    out = oracle.stats_program(3, n0, ops)
    X, Z, Zp, n = _mc(n0, ops, 3)
    assert list(out["n"][:2]) == list(n[:2])
    _check(Z, out["logz"]); _check(Z ** 2, out["logz2"])
    for p in (0, 1):
        _check(X[p], out["logx"][p]); _check(X[p] ** 2, out["logx2"][p]); _check(Z * X[p], out["logzx"][p])
        _check(Zp[p], out["logzp"][p]); _check(Zp[p] ** 2, out["logzp2"][p]); _check(Zp[p] * X[p], out["logzpxp"][p])
    _check(X[0] * X[1], out["logxx"][0, 1])
    assert out["logxx"][0, 1] == out["logxx"][1, 0]


def test_cluster_removed_when_empty():
    out = oracle.stats_program(2, 2, [("kill", 0, -1.0), ("kill", 0, 0.0)])
    assert out["n"][0] == 0 and out["logx"][0] == -math.inf
    # the whole volume was handed out: Z = (1/3) e^-1 + (2/3)(1/2) e^0
    assert out["logz"] == pytest.approx(math.log(math.exp(-1) / 3 + 1.0 / 3), rel=1e-13)
