"""Trajectory length against the evidence offset, on the oracle (test infrastructure, CPU only).

Correlated Gaussians of the c3 family (Sigma = Q diag(lambda) Q^T, lambda log-uniform in
[1e-3, 1e-1], mean U[-0.3, 0.3]) in d dimensions on [-1, 1]^d, n_live 500, the prior box
as an exact reflection, 8 (--seeds) seeded runs with max_ref 3 and with max_ref 9: the mean log Z
minus the closed form, its standard error, the spread, the stated error and the
likelihood evaluations.  With --midpoint the walk takes the time-reversible step (the
oracle's midpoint option) instead of the printed one.

    python oracle/trajectory_length.py 128 [--midpoint] [--seeds 8]
"""
import math, multiprocessing as mp, os, sys, time
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import numpy as np

def one(args):
    d, n_live, max_ref, rid, fold, mid = args
    import oracle
    from paper_2312_03911_gb300 import workloads as W
    rng = np.random.default_rng(W.SEED_BASE + 3)
    prec, _, _, _ = W.dense_precision(rng, d)
    spec = dict(kind=W.LIK_DENSE, d=d, means=rng.uniform(-0.3, 0.3, size=(1, d)), precision=prec)
    lik = oracle.Likelihood.from_spec(spec)
    over = dict(W.BOX_FOLD) if fold else {}
    cfg = oracle.make_cfg(**dict(W.DEFAULT_CFG, n_live=n_live, clustering=0, seed=4242, run_id=rid, max_ref=max_ref, midpoint=mid, **over))
    r = oracle.run(lik, -np.ones(d), np.ones(d), cfg)
    truth = W.truth_logz(dict(name="x", spec=spec, lo=-np.ones(d), hi=np.ones(d), cfg={}))
    return d, max_ref, fold, r["logz"] - truth, r["logz_err"], r["n_like"], r["status"]

if __name__ == "__main__":
    import oracle; oracle.build()
    d = int(sys.argv[1]) if len(sys.argv) > 1 else 32
    mid = int("--midpoint" in sys.argv)
    seeds = int(sys.argv[sys.argv.index("--seeds") + 1]) if "--seeds" in sys.argv else 8
    jobs = [(d, 500, mr, r, fold, mid) for mr in (3, 9) for fold in (1,) for r in range(seeds)]
    t0 = time.time()
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        res = pool.map(one, jobs, chunksize=1)
    for mr in (3, 9):
        z = np.array([x[3] for x in res if x[1] == mr]); e = np.mean([x[4] for x in res if x[1] == mr]); nl = np.mean([x[5] for x in res if x[1] == mr])
        print(f"d {d} max_ref {mr}: offset {z.mean():+.3f} +- {z.std(ddof=1)/math.sqrt(len(z)):.3f} sd {z.std(ddof=1):.3f} stated {e:.3f} n_like {nl:.3g} status {[x[6] for x in res if x[1]==mr]}", flush=True)
    print("took", time.time() - t0)
