"""Benchmark: HSS point-steps/s and time-to-log-Z of gradient-guided nested sampling.

One step = one complete pass of the hot path over one batch: R seeded replicas of
the d=32 four-component mixture workload (n_live=1000, clustering on) run to
termination in one context -- prior draws, per iteration cluster finding,
selection, FP64 statistics, spawn, the three HSS phases and the tail, then the
final sweep, the posterior information and d log Z / d means of every replica.
The replicas are the R = ceil((3 sigma / 0.2)^2) runs whose mean meets the
0.2-nat criterion.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ggns|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs its own R
replicas (independent runs: no collective on the data path, weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2312_03911_gb300 import workloads as W  # noqa: E402

METRIC = "HSS point-steps/s"
UNIT = "point-steps/s"
WORKLOAD = "c2"
DEFAULT_REPLICAS = 17
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM bytes (read + write) per k_hss1 launch from one ncu capture of this workload
# (profiles/k_hss1_c2x17.md), valid only for the kernel sources with these hashes.
HSS_TRAFFIC_BYTES = 130.85e6
HSS_TRAFFIC_SOURCES = {"paper_2312_03911_gb300/csrc/ggns_kernels.cuh": "29d4e8cec9657d33",
                       "paper_2312_03911_gb300/csrc/ggns_internal.cuh": "2215bb2dc5d7ffc3"}
SMS = 152
FP32_LANES_PER_SM = 128


def lane_ops_per_point_step(d: int, K: int, out_frac: float, rng: bool = True) -> float:
    """Algorithmic lane operations of one walker step of the isotropic-mixture HSS
    (the per-unit figure of the roofline; derivation in the design notes):
    move d FMA; likelihood 2Kd (difference, FMA) + K exp + 1 log + 12 scalar;
    score Kd FMA + d scale; box test 2d; reflection 3d on outside steps; noise
    2d (scale, FMA).  With rng: the step's d normals, d/4 Philox4x32-10 blocks x
    100 integer ops + 4 ops per uniform + 4 ops per normal (log/sqrt/sincos
    shared by pairs); the reservoir word rides on the noise block's spare bits.
    Without rng: the normals were drawn ahead by k_noise."""
    move = d
    lik = 2 * K * d + K + 1 + 12
    score = K * d + d
    box = 2 * d
    refl = 3 * d * out_frac
    noise = 2 * d
    draw = (d / 4) * 100 + 4 * d + 4 * d if rng else 0.0
    return move + lik + score + box + refl + noise + draw


class ClockSampler:
    """nvidia-smi clock and throttle sampling during the timed region."""

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            dev = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0] or str(
                int(os.environ.get("LOCAL_RANK", "0")))
            self.p = subprocess.Popen(["nvidia-smi", "-i", dev, f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        try:
            for line in open(self.f.name):
                parts = [t.strip() for t in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def replicas(R: int, rank: int):
    w = W.workload(WORKLOAD)
    return w, [dict(w, cfg=dict(w["cfg"], run_id=rank * R + r)) for r in range(R)]


def max_over_ranks(t: float, dist, device: str) -> float:
    """A step ends when the slowest rank ends: the maximum of the ranks' step times."""
    if dist is None:
        return t
    import torch
    tt = torch.tensor([t], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def sum_over_ranks(x: float, dist, device: str) -> float:
    """Whole-job totals (point-steps of every rank's replicas)."""
    if dist is None:
        return x
    import torch
    tt = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(tt)
    return float(tt.item())


def measured_traffic():
    """The profiled traffic per launch, or None once the kernel sources differ from the profiled ones."""
    import hashlib
    for rel, h in HSS_TRAFFIC_SOURCES.items():
        with open(os.path.join(ROOT, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != h:
                return None
    return HSS_TRAFFIC_BYTES


def load_peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return {}


# --------------------------------------------------------------------------- #
# Oracle leg (CPU baseline / reference arm)                                     #
# --------------------------------------------------------------------------- #
def oracle_sample(n_runs: int, threads: int, seed_base: int = 0):
    """Run n_runs full oracle runs of the workload on `threads` host threads (the
    oracle is single-threaded per run; ctypes releases the GIL).  Returns
    (point-steps, seconds, logZs)."""
    import oracle
    w = W.workload(WORKLOAD)
    lik = oracle.Likelihood.from_spec(w["spec"])
    out = [None] * n_runs
    nxt = [0]
    lock = threading.Lock()

    def worker():
        while True:
            with lock:
                i = nxt[0]
                nxt[0] += 1
            if i >= n_runs:
                return
            cfg = oracle.make_cfg(**dict(w["cfg"], run_id=seed_base + i))
            r = oracle.run(lik, w["lo"], w["hi"], cfg)
            out[i] = (r["n_steps_total"], r["logz"])

    t0 = time.perf_counter()
    ths = [threading.Thread(target=worker) for _ in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    dt = time.perf_counter() - t0
    return sum(o[0] for o in out), dt, [o[1] for o in out]


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    threads = min(os.cpu_count() or 1, args.replicas)
    cfg_desc = workload_config(args)
    for i in range(args.warmup):
        oracle_sample(1, 1, seed_base=10_000 + i)
    times, steps = [], []
    for i in range(args.steps):
        n, t, _ = oracle_sample(threads, threads, seed_base=20_000 + i * threads)
        times.append(t)
        steps.append(n)
    value = sum(steps) / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg_desc,
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{threads} complete oracle runs of the workload per step, one per thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args):
    return {"workload": f"{WORKLOAD}x{args.replicas}: {args.replicas} seeded replicas of the d=32 equal mixture of "
                        f"4 isotropic Gaussians (sigma 0.05), prior U[-1,1]^32, n_live=1000, clustering on, "
                        f"XL-peak tol 0.01", "replicas": args.replicas, "d": 32, "n_live": 1000, "n_comp": 4,
            "noise_mode": 1, "delta_p": 0.2, "l2": "flushed between steps (256 MiB write)"}


# --------------------------------------------------------------------------- #
# GPU leg                                                                       #
# --------------------------------------------------------------------------- #
def gpu_arm(args):
    import torch
    from paper_2312_03911_gb300 import build as B
    from paper_2312_03911_gb300 import ggns

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if dist is not None:
        dist.barrier()
    ggns.load()
    stream = torch.cuda.current_stream()
    R = args.replicas
    w, runs = replicas(R, rank)
    s = ggns.Sampler(runs, stream=stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    truth = W.truth_logz(w)

    def one_step(seed):
        s.restart(seed)
        s.run()
        res = [s.result(r) for r in range(R)]
        for r in range(R):
            s.grad_logz(r)
        return res

    for i in range(args.warmup):
        one_step(W.SEED_BASE + 1000 + i)
    s.profile(reset=True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    times, pts, logz, errs = [], [], [], []
    with ClockSampler() as clk:
        for i in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            ev0.record(stream)
            res = one_step(W.SEED_BASE + 2000 + i)
            ev1.record(stream)
            torch.cuda.synchronize()
            t = max_over_ranks(ev0.elapsed_time(ev1) / 1000.0, dist, "cuda")
            times.append(t)
            pts.append(sum(r["n_steps_total"] for r in res))
            logz.append([r["logz"] for r in res])
            errs.append([r["logz_err"] for r in res])
    prof = s.profile(reset=True)
    clocks = clk.summary()
    tot_pts = sum_over_ranks(float(sum(pts)), dist, "cuda")
    value = tot_pts / sum(times)
    ms = 1000.0 * sum(times) / len(times)
    # roofline of the dominant kernel (HSS): algorithmic lane-ops / HSS time
    zall = np.array(logz)
    out_frac_est = 0.12
    drawn_ahead = prof.get("noise_steps", 0) > 0
    ops = lane_ops_per_point_step(32, 4, out_frac_est, rng=not drawn_ahead)
    hss_s = prof["hss_ms"] / 1000.0  # time during which HSS kernels of any run were executing
    achieved = ops * (sum(pts)) / hss_s if hss_s > 0 else None
    f_sm = (clocks.get("sm_mhz") or 1447.0) * 1e6
    peak = SMS * FP32_LANES_PER_SM * f_sm
    hss_iters = max(prof["hss_iters"], 1)
    roof = {"bound": "alu", "achieved": achieved / 1e12 if achieved else None, "peak": peak / 1e12,
            "unit": "Tlane-op/s", "frac": (achieved / peak) if achieved else None, "traffic": measured_traffic(),
            "traffic_unit": "bytes per launch (DRAM read + write)",
            "kernel": ("k_hss1 + k_hss_pick (single pass)" if prof.get("rec_len", 0) > 0 else "k_hss (phases 0-2)"),
            "hss_rec_overflows": prof.get("rec_overflows"), "ops_per_point_step": ops,
            "noise": ("drawn ahead by k_noise on a side stream (not in this kernel's count): "
                      f"{lane_ops_per_point_step(32, 4, 0.0) - lane_ops_per_point_step(32, 4, 0.0, rng=False):.0f} "
                      "lane-ops per point-step") if drawn_ahead else "drawn in the walk",
            "hss_ms_per_run_iteration": prof["hss_ms_sum"] / hss_iters,
            "hss_busy_fraction_of_step": prof["hss_ms"] / (1000.0 * sum(times)),
            "peak_note": f"{SMS} SMs x {FP32_LANES_PER_SM} lanes x median SM clock {f_sm / 1e6:.0f} MHz"}
    # e2e: through the C ABI from host buffers (create = H2D of parameters, result = D2H)
    e2e_t = []
    h2d = 0
    for r in runs:
        sp = r["spec"]
        h2d += 8 * (2 * sp["d"] + np.size(sp["means"]) + np.size(sp["sigma"]) + np.size(sp.get("log_weights", [])))
    d2h = R * 96
    for i in range(max(1, min(2, args.steps))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = ggns.Sampler(runs)
        s2.run()
        _ = [s2.result(r) for r in range(R)]
        s2.close()
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_pts = pts[-1]
    e2e_value = e2e_pts / (sum(e2e_t) / len(e2e_t))
    # the plain GPU path: one run per context, one host-synchronised launch chain per iteration
    plain_ms = None
    if not args.no_plain:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r in runs:
            sp = ggns.Sampler([r])
            while not sp.step(1):
                pass
            sp.run(0)
            sp.result(0)
            sp.close()
        torch.cuda.synchronize()
        plain_ms = 1000.0 * (time.perf_counter() - t0)
    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            threads = min(os.cpu_count() or 1, R)
            n, t, _ = oracle_sample(threads, threads, seed_base=50_000)
            cpu = {"value": n / t, "unit": UNIT, "cores": threads, "kind": "oracle",
                   "sample": f"{threads} complete oracle runs of the workload on {threads} host threads "
                             f"({n} point-steps in {t:.1f} s)"}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(args),
                "time_to_logz_ms": ms,
                "plain": None if plain_ms is None else {
                    "time_to_logz_ms": plain_ms,
                    "what": "same replicas one after another, one context each, one host-synchronised launch "
                            "chain per iteration (no graph, no batching)",
                    "speedup": plain_ms / ms},
                "logz_mean": float(zall.mean()), "logz_truth": truth,
                "dlogz_mean": float(zall.mean() - truth), "logz_err_mean": float(np.mean(errs)),
                "logz_sd": float(zall.std()),
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": d2h},
                "gpu_launches": int(prof["launches"] / max(args.steps, 1)),
                "clocks": {"sm_mhz": clocks.get("sm_mhz"), "sm_max_mhz": clocks.get("sm_max_mhz"),
                           "reasons": clocks.get("reasons")},
                "peaks": {k: load_peaks().get(k) for k in ("hbm_gbs", "bf16_tflops")}}
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ggns", choices=["ggns", "reference"])
    ap.add_argument("--replicas", type=int, default=DEFAULT_REPLICAS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
