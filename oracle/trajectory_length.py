"""Trajectory length against the evidence offset, on the oracle (test infrastructure, CPU only).

Correlated Gaussians of the c3 family (Sigma = Q diag(lambda) Q^T, lambda log-uniform in
[1e-3, 1e-1], mean U[-0.3, 0.3]) in d dimensions on [-1, 1]^d, n_live 500, the prior box
as an exact reflection, 8 (--seeds) seeded runs with max_ref 3 and with max_ref 9: the mean log Z
minus the closed form, its standard error, the spread, the stated error and the
likelihood evaluations.  With --midpoint the walk takes the time-reversible step (the
oracle's midpoint option) instead of the printed one; --first N starts the run ids at N (new
replicas beside earlier ones), --max-ref M runs that one trajectory length only, and --fixed K
runs trajectories of exactly K steps that keep their last state (keep_last, min_ref 0, max_ref
out of reach, no pruning) in place of the window; --delta-p X sets the refresh strength and
--out-band LO HI the band of outside fractions the step-size control aims for.  Beside the offset each line gives the
fraction of walkers that returned their start point (the oracle's fallback count: with the
reversible step every start-point return, with the printed step only the walkers whose window
saved nothing) and the mean steps per walker.

    python oracle/trajectory_length.py 128 [--midpoint] [--seeds 8] [--first 0] [--max-ref 9 | --fixed 60] [--delta-p 0.5] [--out-band 0.05 0.15]
"""
import math, multiprocessing as mp, os, sys, time
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import numpy as np

def one(args):
    d, n_live, mode, val, rid, mid, dp, band = args
    import oracle
    from paper_2312_03911_gb300 import workloads as W
    rng = np.random.default_rng(W.SEED_BASE + 3)
    prec, _, _, _ = W.dense_precision(rng, d)
    spec = dict(kind=W.LIK_DENSE, d=d, means=rng.uniform(-0.3, 0.3, size=(1, d)), precision=prec)
    lik = oracle.Likelihood.from_spec(spec)
    if mode == "max_ref":
        walk = dict(max_ref=val)
    else:
        walk = dict(keep_last=1, min_ref=0, max_ref=10**9, n_steps=val, min_steps=val, prune_after=0)
    cfg = oracle.make_cfg(**dict(W.DEFAULT_CFG, n_live=n_live, clustering=0, seed=4242, run_id=rid, midpoint=mid, delta_p=dp,
                                 out_lo=band[0], out_hi=band[1],
                                 **dict(W.BOX_FOLD, **walk)))
    r = oracle.run(lik, -np.ones(d), np.ones(d), cfg)
    truth = W.truth_logz(dict(name="x", spec=spec, lo=-np.ones(d), hi=np.ones(d), cfg={}))
    walkers = max(r["n_dead"] - n_live, 1)
    return ((mode, val), r["logz"] - truth, r["logz_err"], r["n_like"], r["status"],
            r["n_fallback"] / walkers, r["n_steps_total"] / walkers)

def _arg(name, default):
    return int(sys.argv[sys.argv.index(name) + 1]) if name in sys.argv else default

if __name__ == "__main__":
    import oracle; oracle.build()
    from paper_2312_03911_gb300 import workloads as W
    d = int(sys.argv[1]) if len(sys.argv) > 1 else 32
    mid = int("--midpoint" in sys.argv)
    seeds, first = _arg("--seeds", 8), _arg("--first", 0)
    if "--fixed" in sys.argv:
        groups = [("fixed", _arg("--fixed", 0))]
    elif "--max-ref" in sys.argv:
        groups = [("max_ref", _arg("--max-ref", 0))]
    else:
        groups = [("max_ref", 3), ("max_ref", 9)]
    dp = float(sys.argv[sys.argv.index("--delta-p") + 1]) if "--delta-p" in sys.argv else W.DEFAULT_CFG["delta_p"]
    band = (W.DEFAULT_CFG["out_lo"], W.DEFAULT_CFG["out_hi"])
    if "--out-band" in sys.argv:
        i = sys.argv.index("--out-band")
        band = (float(sys.argv[i + 1]), float(sys.argv[i + 2]))
    jobs = [(d, 500, m, v, r, mid, dp, band) for m, v in groups for r in range(first, first + seeds)]
    t0 = time.time()
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        res = pool.map(one, jobs, chunksize=1)
    for g in groups:
        rows = [x for x in res if x[0] == g]
        z = np.array([x[1] for x in rows])
        print(f"d {d} {g[0]} {g[1]} delta_p {dp} out band {band}: offset {z.mean():+.3f} +- {z.std(ddof=1)/math.sqrt(len(z)):.3f} "
              f"sd {z.std(ddof=1):.3f} stated {np.mean([x[2] for x in rows]):.3f} "
              f"n_like {np.mean([x[3] for x in rows]):.3g} fallback {np.mean([x[5] for x in rows]):.3f} "
              f"steps/walker {np.mean([x[6] for x in rows]):.1f} status {[x[4] for x in rows]}", flush=True)
        print("  per run:", " ".join(f"{v:+.3f}" for v in z), flush=True)
    print("took", time.time() - t0)
