"""Ablation of the readings of Algorithm 5 on the oracle (test infrastructure, CPU only).

The c2 workload (d = 32, four isotropic Gaussians, n_live 1000, clustering on) with one
reading changed at a time, 16 seeded runs each; prints the mean log Z minus the closed
form with its standard error, the run-to-run spread, the mean stated error and the
likelihood evaluations per run.

    python oracle/ablate_readings.py
"""
import math, multiprocessing as mp, os, sys, time
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import numpy as np

VARIANTS = {
    "default": {},
    "noise on every step (noise_inside 0)": dict(noise_inside=0),
    "pick among inside states (pick_all 0)": dict(pick_all=0),
    "no region rule (territory 0)": dict(territory=0),
    "printed noise p(1+dp eps), dp 0.05, every step": dict(noise_mode=0, delta_p=0.05, noise_inside=0),
    "clustering off": dict(clustering=0),
    "round-1 reading (dp 0.2 refresh every step, inside pick, no region rule)": dict(delta_p=0.2, noise_inside=0, pick_all=0, territory=0),
}

def one(args):
    name, rid = args
    import oracle
    from paper_2312_03911_gb300 import workloads as W
    w = W.workload("c2")
    lik = oracle.Likelihood.from_spec(w["spec"])
    cfg = oracle.make_cfg(**dict(w["cfg"], run_id=rid, **VARIANTS[name]))
    r = oracle.run(lik, w["lo"], w["hi"], cfg)
    return name, rid, r["logz"], r["logz_err"], r["n_like"], r["status"]

if __name__ == "__main__":
    import oracle
    oracle.build()
    from paper_2312_03911_gb300 import workloads as W
    truth = W.truth_logz(W.workload("c2"))
    jobs = [(n, 100 + r) for n in VARIANTS for r in range(16)]
    t0 = time.time()
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        res = pool.map(one, jobs, chunksize=1)
    out = {}
    for name in VARIANTS:
        z = np.array([r[2] for r in res if r[0] == name])
        nl = np.array([r[4] for r in res if r[0] == name])
        e = np.array([r[3] for r in res if r[0] == name])
        out[name] = dict(bias=float(z.mean() - truth), se=float(z.std(ddof=1) / math.sqrt(len(z))), sd=float(z.std(ddof=1)),
                         err=float(e.mean()), n_like=float(nl.mean()), runs=len(z))
        print(f"{name:75s} bias {z.mean()-truth:+.3f} +- {z.std(ddof=1)/math.sqrt(len(z)):.3f}  sd {z.std(ddof=1):.3f}  stated {e.mean():.3f}  n_like {nl.mean():.3g}", flush=True)
    print("took", time.time() - t0)
