"""Pins of the oracle's readings of Algorithm 5 and of the cluster bookkeeping:
the noise taken on inside steps only, the pick over every step of the saving window
with rejection to the start point, the printed multiplicative noise, the region
rule for new points, and the prior box as an exact reflection whose folds count for
the step-size control.  Each is checked against its definition on traces, against a
brute-force statement, or against the invariance the sampler must have."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2312_03911_gb300 import workloads as W


def _ball(d, R=0.3, sig=0.1):
    lik = oracle.Likelihood(W.LIK_ISO, d, means=np.zeros(d), sigma=[sig])
    lstar = -0.5 * R * R / sig**2 - 0.5 * d * math.log(2 * math.pi * sig**2)
    return lik, lstar


def _uniform_ball(rng, n, d, R):
    v = rng.standard_normal((n, d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v * R * rng.uniform(size=(n, 1)) ** (1.0 / d)


def _ball_rank_z(over, d=16, R=0.3, dt=0.01, n=4000, reps=12):
    """z-score of the mean prior-volume rank u = (r/R)^d of the HSS outputs from uniform
    starts in the ball slice (u ~ U(0,1) for a sampler that keeps the slice uniform)."""
    lik, lstar = _ball(d, R)
    rng = np.random.default_rng(11)
    us = []
    for b in range(reps):
        x0 = _uniform_ball(rng, n, d, R)
        cfg = oracle.make_cfg(**dict(dict(seed=100 + b), **over))
        o = oracle.hss_batch(lik, -np.ones(d), np.ones(d), cfg, 0, x0, [lik.loglik(q) for q in x0], lstar, dt)
        assert np.all(o["logl"] > lstar)
        us.append(((o["x"] ** 2).sum(1) / R**2) ** (d / 2))
    u = np.concatenate(us)
    return (u.mean() - 0.5) / math.sqrt(1 / 12 / len(u))


def test_window_pick_with_rejection_keeps_the_slice_uniform():
    """The library's reading (noise on inside steps, pick over every window step, an outside
    pick returning the start point) leaves a uniform slice uniform; the pick among inside states
    alone, with the same trajectories, drifts outward: walkers that spend steps outside give
    each of their inside states more weight."""
    reading = dict(noise_mode=1, delta_p=0.5, noise_inside=1)
    assert abs(_ball_rank_z(dict(reading, pick_all=1))) < 4
    assert _ball_rank_z(dict(reading, pick_all=0)) > 4


def _trace_case(over, d=6, n=16, steps=40):
    lik, lstar = _ball(d)
    rng = np.random.default_rng(5)
    x0 = _uniform_ball(rng, n, d, 0.3)
    cfg = oracle.make_cfg(**dict(dict(seed=21, n_steps=steps, min_steps=steps, max_ref=10**6, prune_after=0), **over))
    o = oracle.hss_batch(lik, -np.ones(d), np.ones(d), cfg, 3, x0, [lik.loglik(q) for q in x0], lstar, 0.03,
                         trace=True)
    return lik, cfg, o["trace"], d, n


def test_noise_perturbs_inside_steps_only():
    """noise_inside: an outside step applies the reflection p - 2 (p.n) n alone; an inside step
    applies the refresh p <- sqrt(1 - dp^2) p + dp eps with eps the step's Philox normals."""
    dp = 0.5
    lik, cfg, tr, d, n = _trace_case(dict(noise_mode=1, delta_p=dp, noise_inside=1))
    keep = math.sqrt(1 - dp * dp)
    n_out = 0
    for j in range(n):
        p = oracle.normals(cfg.seed, 0, 3, oracle.P_MOM, j, 0, d)
        for t in range(1, tr.shape[0] + 1):
            x, p_new, out = tr[t - 1, j, :d], tr[t - 1, j, d:2 * d], tr[t - 1, j, 2 * d + 1]
            if out:
                n_out += 1
                _, g = lik.loglik(x, grad=True)
                nrm = g / np.linalg.norm(g)
                np.testing.assert_allclose(p_new, p - 2 * np.dot(p, nrm) * nrm, rtol=1e-12, atol=1e-14)
                assert np.linalg.norm(p_new) == pytest.approx(np.linalg.norm(p), rel=1e-12)
            else:
                eps = oracle.normals(cfg.seed, 0, 3, oracle.P_NOISE, j, t, d)
                np.testing.assert_allclose(p_new, keep * p + dp * eps, rtol=1e-12, atol=1e-14)
            p = p_new
    assert n_out > 20


def test_printed_noise_is_the_componentwise_product():
    """noise_mode 0 (Algorithm 5 as printed): p_i <- p_i (1 + dp eps_i) with a fresh eps_i per
    component and step, so E |p'|^2 = (1 + dp^2) |p|^2 and the factors of different components
    are uncorrelated (Monte Carlo over the inside steps of many walkers)."""
    dp = 0.05
    lik, cfg, tr, d, n = _trace_case(dict(noise_mode=0, delta_p=dp, noise_inside=1), d=8, n=400, steps=30)
    ratios, facs = [], []
    for j in range(n):
        p = oracle.normals(cfg.seed, 0, 3, oracle.P_MOM, j, 0, d)
        for t in range(1, tr.shape[0] + 1):
            p_new, out = tr[t - 1, j, d:2 * d], tr[t - 1, j, 2 * d + 1]
            if not out:
                eps = oracle.normals(cfg.seed, 0, 3, oracle.P_NOISE, j, t, d)
                np.testing.assert_allclose(p_new, p * (1 + dp * eps), rtol=1e-12, atol=1e-14)
                ratios.append(((p_new / p) ** 2).mean())
                facs.append(p_new / p - 1.0)
            p = p_new
    ratios, facs = np.array(ratios), np.array(facs)
    # per-component (1 + dp eps)^2 has mean 1 + dp^2 and standard deviation ~ 2 dp
    se = 2 * dp / math.sqrt(d * len(ratios))
    assert abs(ratios.mean() - (1 + dp * dp)) < 4 * se
    c = np.corrcoef(facs.T)
    off = c[~np.eye(d, dtype=bool)]
    assert np.all(np.abs(off) < 4 / math.sqrt(len(facs)))


def test_region_rule_matches_brute_force():
    """orc_territory keeps a new point when its nearest survivor (FP32 distances) carries the
    label it was spawned with; checked against an FP64 brute-force nearest neighbour on random
    points (no near ties), and on a planted case."""
    rng = np.random.default_rng(8)
    d, m, k = 7, 300, 200
    surv = rng.uniform(-1, 1, size=(m, d)).astype(np.float32)
    lab = rng.integers(0, 4, size=m).astype(np.int32)
    xn = rng.uniform(-1, 1, size=(k, d)).astype(np.float32)
    want = rng.integers(0, 4, size=k).astype(np.int32)
    keep = oracle.territory(surv, lab, xn, want)
    d2 = ((xn[:, None, :].astype(np.float64) - surv[None].astype(np.float64)) ** 2).sum(-1)
    nn = d2.argmin(1)
    srt = np.sort(d2, axis=1)
    assert np.all(srt[:, 1] - srt[:, 0] > 1e-5 * srt[:, 0])  # no near ties in this draw
    np.testing.assert_array_equal(keep, (lab[nn] == want).astype(np.int32))
    # planted: two tight groups; a point spawned in group 0 that landed in group 1 is rejected
    a = np.zeros((5, 3), np.float32); b = np.full((5, 3), 1.0, np.float32)
    s2 = np.concatenate([a, b]); l2 = np.array([0] * 5 + [1] * 5, np.int32)
    keep2 = oracle.territory(s2, l2, np.array([[0.9, 0.9, 0.9], [0.1, 0, 0]], np.float32), np.array([0, 0], np.int32))
    assert list(keep2) == [0, 1]
    # exact tie: the lower survivor row wins
    keep3 = oracle.territory(np.array([[1, 0], [-1, 0]], np.float32), np.array([5, 6], np.int32),
                             np.zeros((1, 2), np.float32), np.array([5], np.int32))
    assert list(keep3) == [1]


def test_mixture_evidence_with_clustering_is_unbiased():
    """Full runs of the library's reading on a 4-mode isotropic mixture (d = 8, sigma 0.05,
    clustering on): the mean of 16 seeded runs matches the erf closed form within 3.5 standard
    errors, every run lies within 4 of its own error estimates, and the region rule fired."""
    rng = np.random.default_rng(5)
    d, K = 8, 4
    spec = dict(kind=W.LIK_MIX_ISO, d=d, means=rng.uniform(-0.5, 0.5, size=(K, d)), sigma=np.full(K, 0.05),
                log_weights=np.full(K, -math.log(K)))
    lo, hi = -np.ones(d), np.ones(d)
    truth = W.truth_logz_iso_mixture(spec["means"], spec["sigma"], spec["log_weights"], lo, hi)
    lik = oracle.Likelihood.from_spec(spec)
    zs, errs, rej = [], [], 0
    for r in range(16):
        cfg = oracle.make_cfg(**dict(W.DEFAULT_CFG, n_live=500, seed=777, run_id=r, clustering=1))
        out = oracle.run(lik, lo, hi, cfg, dead_cap=500 * 200)
        assert out["status"] == 0 and out["terminated"] == 1
        zs.append(out["logz"]); errs.append(out["logz_err"]); rej += out["n_region_rejected"]
        assert abs(out["logz"] - truth) < 4 * out["logz_err"]
    zs = np.array(zs)
    se = zs.std(ddof=1) / math.sqrt(len(zs))
    assert abs(zs.mean() - truth) < 3.5 * se, (zs.mean() - truth, se)
    assert rej > 0


def test_fold_count_is_the_inside_steps_whose_move_left_the_box():
    """box_fold: n_fold counts the inside steps on which the straight move x + p dt left the box
    (re-derived from the trace: the position before the step, the momentum the step moved with);
    outside steps are not counted; the folded positions lie in the box."""
    d, n = 6, 24
    lik = oracle.Likelihood(W.LIK_ISO, d, means=np.full(d, 0.9), sigma=[0.6])
    rng = np.random.default_rng(3)
    x0 = np.clip(0.8 + 0.1 * rng.standard_normal((n, d)), -0.99, 0.99)
    l0 = np.array([lik.loglik(q) for q in x0])
    lstar = float(np.min(l0) - 2.0)
    lo, hi = -np.ones(d), np.ones(d)
    dt = 0.05
    cfg = oracle.make_cfg(**dict(W.DEFAULT_CFG, n_steps=30, min_steps=30, max_ref=10**6, prune_after=0, seed=9,
                                 **W.BOX_FOLD_COUNTED))
    o = oracle.hss_batch(lik, lo, hi, cfg, 2, x0, l0, lstar, dt, trace=True)
    tr = o["trace"]
    x_prev = x0.copy()
    p_prev = np.array([oracle.normals(cfg.seed, 0, 2, oracle.P_MOM, j, 0, d) for j in range(n)])
    n_fold = 0
    for t in range(tr.shape[0]):
        x, p, out = tr[t, :, :d], tr[t, :, d:2 * d], tr[t, :, 2 * d + 1]
        moved = x_prev + p_prev * dt
        left = np.any((moved < lo) | (moved > hi), axis=1)
        n_fold += int(np.sum(left & (out == 0)))
        assert np.all((x >= lo) & (x <= hi))
        x_prev, p_prev = x, p
    assert o["n_fold"] == n_fold and n_fold > 20
    o0 = oracle.hss_batch(lik, lo, hi, oracle.make_cfg(**dict(cfg_dict(cfg), box_fold=0)), 2, x0, l0, lstar, dt)
    assert o0["n_fold"] == 0 and o0["n_out"] > o["n_out"]


def cfg_dict(cfg):
    return {name: getattr(cfg, name) for name, _ in cfg._fields_}


def _iso_run(args):
    d, rid = args
    import oracle as orc
    from paper_2312_03911_gb300 import workloads as WW
    lik = orc.Likelihood(WW.LIK_ISO, d, means=np.zeros(d), sigma=[0.1])
    cfg = orc.make_cfg(**dict(WW.DEFAULT_CFG, n_live=200, clustering=0, seed=777, run_id=rid, **WW.BOX_FOLD_COUNTED))
    r = orc.run(lik, -np.ones(d), np.ones(d), cfg, dead_cap=200 * 600)
    return r["logz"], r["status"]


def test_box_reflection_counted_for_dt_keeps_high_dimensional_evidence_unbiased():
    """The isotropic N(0, 0.1^2 I) on [-1, 1]^64, n_live 200 (the d-sweep of Section 4.1), ten
    seeded runs with the exact box reflection whose folds count for the step size: the mean log Z
    lies within 3.5 standard errors of the closed form (the box as an outside region, the default,
    is -1.3 nats off here)."""
    import multiprocessing as mp
    d = 64
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        res = pool.map(_iso_run, [(d, r) for r in range(10)])
    assert all(st == 0 for _, st in res)
    z = np.array([v for v, _ in res])
    truth = W.truth_logz_iso_mixture(np.zeros((1, d)), [0.1], None, -np.ones(d), np.ones(d))
    se = z.std(ddof=1) / math.sqrt(len(z))
    assert abs(z.mean() - truth) < 3.5 * se + 0.1, (z.mean() - truth, se)


def test_symmetric_step_is_time_reversible_and_the_printed_step_is_not():
    """The step of Algorithm 5 (move, then reflect with the normal at the new point) and its
    symmetric splitting (half move, reflect at the half step, half move) near the contour of a
    correlated Gaussian: from (x', -p') the symmetric step returns to (x, -p) whenever it
    reflected; the printed step does not come back to x.  This is why the printed walk's evidence
    offset grows with the trajectory length at d = 128 (oracle/trajectory_length.py)."""
    d = 12
    rng = np.random.default_rng(21)
    prec, _, _, _ = W.dense_precision(rng, d, 1e-2, 1e-1)
    lik = oracle.Likelihood(W.LIK_DENSE, d, means=np.zeros(d), precision=prec)
    lstar = lik.loglik(np.zeros(d)) - 3.0
    dt = 0.05
    n_refl = {0: 0, 1: 0}
    back_err = {0: [], 1: []}
    for _ in range(400):
        x = rng.standard_normal(d)
        # a point close to the contour log L = L*, inside
        lo_, hi_ = 0.0, 5.0
        for _ in range(60):
            mid = 0.5 * (lo_ + hi_)
            (lo_, hi_) = (mid, hi_) if lik.loglik(mid * x) > lstar else (lo_, mid)
        x = lo_ * x * 0.999
        p = rng.standard_normal(d)
        for mode in (0, 1):
            x1, p1, r1 = oracle.walk_step(lik, mode, lstar, dt, x, p)
            if not r1:
                continue
            n_refl[mode] += 1
            x2, p2, _ = oracle.walk_step(lik, mode, lstar, dt, x1, -p1)
            back_err[mode].append(max(np.abs(x2 - x).max(), np.abs(p2 + p).max()))
    assert n_refl[0] > 50 and n_refl[1] > 50, n_refl
    assert max(back_err[1]) < 1e-12, max(back_err[1])
    assert np.median(back_err[0]) > 1e-3, np.median(back_err[0])


def test_symmetric_walk_keeps_the_slice_uniform():
    """The option midpoint (the time-reversible step, refresh noise on every state, the drawn
    state tested against L* at the end) leaves a uniform ball slice uniform."""
    assert abs(_ball_rank_z(dict(noise_mode=1, delta_p=0.5, pick_all=1, midpoint=1))) < 4


def test_fixed_length_symmetric_walk_keeps_the_slice_uniform():
    """The reversible step with keep_last over a fixed number of steps (min_ref 0, max_ref out
    of reach, no pruning): the end point of a fixed-length reversible trajectory, accepted when
    inside and otherwise replaced by the start point, leaves a uniform ball slice uniform, and
    the walker's output is its state after exactly that many steps."""
    fixed = dict(noise_mode=1, delta_p=0.5, pick_all=1, midpoint=1, keep_last=1, min_ref=0,
                 max_ref=10**6, n_steps=30, min_steps=30, prune_after=0)
    assert abs(_ball_rank_z(fixed)) < 4
    lik, lstar = _ball(6)
    rng = np.random.default_rng(9)
    x0 = _uniform_ball(rng, 32, 6, 0.3)
    cfg = oracle.make_cfg(**dict(fixed, seed=3, n_steps=12, min_steps=12))
    o = oracle.hss_batch(lik, -np.ones(6), np.ones(6), cfg, 0, x0, [lik.loglik(q) for q in x0], lstar, 0.03,
                         trace=True)
    last = o["trace"][11, :, :6]
    inside = np.array([lik.loglik(q) > lstar for q in last])
    assert o["t_stop"] == 12 and 0 < inside.sum() < 32
    np.testing.assert_array_equal(o["x"][inside], last[inside])
    np.testing.assert_array_equal(o["x"][~inside], x0[~inside])
