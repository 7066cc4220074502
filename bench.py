"""Benchmark: HSS point-steps/s of gradient-guided nested sampling, and time-to-log-Z.

Headline workload c5 (the largest single-GPU configuration): d=512, an equal mixture
of 8 Gaussians sharing one dense precision matrix, n_live=4000.  One step = one
complete run in one context: prior draws, every iteration (selection, FP64
statistics, spawn, the HSS walk, the step-size tail), the final sweep, the
posterior weights and d log Z / d means.  value = HSS point-steps/s over the step.

Beside it, time-to-log-Z on c2x17: 17 seeded replicas of the d=32 four-component
mixture (n_live=1000, clustering on) in one batch, the R = ceil((3 sigma / 0.2)^2)
replicas whose mean meets the 0.2-nat criterion; its time is reported only when
the replicas' mean is within 0.2 nats of the closed form.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ggns|reference]
                  [--workload c5|c2]
  python bench.py --profile-case [--workload c5|c2] [--iters N] [--n-steps S]   (ncu captures)

Prints one JSON line (rank 0).  Under torchrun each rank runs its own runs
(independent runs: no collective on the data path, weak scaling).
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
C2_REPLICAS = 17
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SMS = 152
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) of the dominant kernel from one ncu capture, valid only for the kernel
# sources with these hashes: c5 per walker point-step (the records of the steps dominate, so the
# traffic of a launch grows with the point-steps it takes; scaled to the timed launches' mean),
# c2 per launch (one launch of the timed batch).
TRAFFIC = {
    "c5": {"bytes_per_point_step": 1656.15,
           "sources": {"paper_2312_03911_gb300/csrc/ggns_kernels.cuh": "377883e806dbcbd2",
                       "paper_2312_03911_gb300/csrc/ggns_internal.cuh": "2cb53c1f2bf11a28",
                       "paper_2312_03911_gb300/csrc/ggns_tc.cuh": "c425a27c121efb13"}},
    "c2": {"bytes_per_launch": 83.198208e6,
           "sources": {"paper_2312_03911_gb300/csrc/ggns_kernels.cuh": "377883e806dbcbd2",
                       "paper_2312_03911_gb300/csrc/ggns_internal.cuh": "2cb53c1f2bf11a28"}},
}


def lane_ops_per_point_step(d: int, K: int, out_frac: float, rng: bool = True) -> float:
    """Algorithmic lane operations of one walker step of the isotropic-mixture HSS:
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


def dense_mix_flops_per_point_step(d: int, K: int) -> float:
    """Algorithmic FLOPs of one walker step of the dense-mixture likelihood: the contraction
    y = P x (2 d^2; the mixture shares P, so P mu_k is precomputed) and the K quadratic forms
    and score terms (x - mu_k).(y - P mu_k), about 4 K d."""
    return 2.0 * d * d + 4.0 * K * d


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


def runs_of(name: str, n: int, rank: int):
    """n seeded runs of a workload (rank r takes run ids r*n .. r*n+n-1)."""
    w = W.workload(name)
    return w, [dict(w, cfg=dict(w["cfg"], run_id=rank * n + r)) for r in range(n)]


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


def measured_traffic(name: str, point_steps_per_launch: float):
    """The profiled DRAM traffic of one launch of the workload's dominant kernel (c5: scaled to
    the mean point-steps of the timed launches), or None when it was not captured for the
    current kernel sources."""
    import hashlib
    t = TRAFFIC.get(name)
    if not t or not t["sources"]:
        return None
    for rel, h in t["sources"].items():
        with open(os.path.join(ROOT, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != h:
                return None
    if "bytes_per_point_step" in t:
        return t["bytes_per_point_step"] * point_steps_per_launch if t["bytes_per_point_step"] else None
    return t["bytes_per_launch"]


def load_peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return {}


# --------------------------------------------------------------------------- #
# Oracle leg (CPU baseline / reference arm)                                     #
# --------------------------------------------------------------------------- #
def oracle_sample(name: str, threads: int, seed_base: int = 0):
    """A bounded sample of the workload on the oracle, on `threads` host threads (the oracle is
    single-threaded per call; ctypes releases the GIL).  c2: one complete run per thread.  c5 (a
    complete run takes hours on a core): per thread, one HSS call of Algorithm 5 of 4 walkers
    started at prior points, 40 steps, on the c5 likelihood.  Returns (point-steps, seconds)."""
    import numpy as np
    import oracle
    w = W.workload(name)
    lik = oracle.Likelihood.from_spec(w["spec"])
    ld = lik.logdet()
    out = [0] * threads
    lock = threading.Lock()

    def worker(i):
        if name == "c5":
            d = w["spec"]["d"]
            rng = np.random.default_rng(seed_base + i)
            x0 = rng.uniform(-1, 1, size=(4, d))
            l0 = np.array([lik.loglik(v) for v in x0])
            cfg = oracle.make_cfg(**dict(w["cfg"], run_id=seed_base + i, n_steps=40, min_steps=40,
                                         max_ref=10**6))
            o = oracle.hss_batch(lik, w["lo"], w["hi"], cfg, 1, x0, l0, float(l0.min()) - 50.0, 0.002)
            n = 4 * o["t_stop"]
        else:
            cfg = oracle.make_cfg(**dict(w["cfg"], run_id=seed_base + i))
            n = oracle.run(lik, w["lo"], w["hi"], cfg)["n_steps_total"]
        with lock:
            out[i] = n

    del ld
    t0 = time.perf_counter()
    ths = [threading.Thread(target=worker, args=(i,)) for i in range(threads)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    return sum(out), time.perf_counter() - t0


def sample_note(name: str, threads: int, n: int, t: float) -> str:
    if name == "c5":
        return (f"{threads} host threads, each one HSS call (Algorithm 5) of 4 walkers x 40 steps on the c5 "
                f"likelihood from prior points ({n} point-steps in {t:.1f} s)")
    return f"{threads} complete oracle runs of c2, one per host thread ({n} point-steps in {t:.1f} s)"


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    if args.workload == "c2":
        threads = min(threads, C2_REPLICAS)
    for i in range(args.warmup):
        oracle_sample(args.workload, 1, seed_base=10_000 + i)
    times, steps = [], []
    for i in range(args.steps):
        n, t = oracle_sample(args.workload, threads, seed_base=20_000 + i * threads)
        times.append(t)
        steps.append(n)
    value = sum(steps) / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample_note(args.workload, threads, steps[-1], times[-1])},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(name: str):
    if name == "c5":
        return {"workload": "c5: d=512 equal mixture of 8 Gaussians sharing one dense precision P = Sigma^-1, "
                            "Sigma = Q diag(lambda) Q^T (Q from QR of a seeded normal matrix, lambda log-uniform "
                            "in [1e-3, 1e-1]), means U[-0.5,0.5]^512, prior U[-1,1]^512, n_live=4000, one complete "
                            "run per step (prior draws to the final sweep, posterior weights, d logZ/d means)",
                "d": 512, "n_live": 4000, "n_comp": 8, "runs": 1,
                "l2": "inputs larger than L2 (P and the 4000 x 512 live points are re-read every iteration; "
                      "256 MiB written between steps)"}
    return {"workload": f"c2x{C2_REPLICAS}: {C2_REPLICAS} seeded replicas of the d=32 equal mixture of 4 "
                        "isotropic Gaussians (sigma 0.05), prior U[-1,1]^32, n_live=1000, clustering on, "
                        "XL-peak tol 0.01", "replicas": C2_REPLICAS, "d": 32, "n_live": 1000, "n_comp": 4,
            "l2": "flushed between steps (256 MiB write)"}


# --------------------------------------------------------------------------- #
# GPU leg                                                                       #
# --------------------------------------------------------------------------- #
def _timed_steps(s, R, steps, stream, flush, dist, seed0, grad=True):
    """Complete runs of the context's R runs per step (restart with a new seed, run to the final
    sweep, posterior information and d log Z / d means of every run), timed with CUDA events on
    the context's stream; max over ranks."""
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    times, pts, logz, errs = [], [], [], []
    for i in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        ev0.record(stream)
        s.restart(seed0 + i)
        s.run()
        res = [s.result(r) for r in range(R)]
        if grad:
            for r in range(R):
                s.grad_logz(r)
        ev1.record(stream)
        torch.cuda.synchronize()
        times.append(max_over_ranks(ev0.elapsed_time(ev1) / 1000.0, dist, "cuda"))
        pts.append(sum(r["n_steps_total"] for r in res))
        logz.append([r["logz"] for r in res])
        errs.append([r["logz_err"] for r in res])
    return times, pts, logz, errs


def _c2_throughput(ggns, stream, flush, rank, reps, f_sm):
    """Throughput mode of the c2 walk: reps seeded replicas in one batch (more walkers than the
    GPU holds at once), one warm-up batch and one timed batch; the walker kernel's lane-op rate
    against the ALU peak at the sampled SM clock."""
    w, runs = runs_of("c2", reps, rank)
    s = ggns.Sampler(runs, stream=stream.cuda_stream)
    s.restart(W.SEED_BASE + 5000)
    s.run()
    s.profile(reset=True)
    times, pts, _, _ = _timed_steps(s, reps, 1, stream, flush, None, W.SEED_BASE + 6000, grad=False)
    prof = s.profile(reset=True)
    s.close()
    ops = lane_ops_per_point_step(32, 4, 0.12, rng=not prof.get("noise_steps", 0) > 0)
    hss_s = prof["hss_ms"] / 1000.0
    ach = ops * sum(pts) / hss_s if hss_s > 0 else None
    peak = SMS * FP32_LANES_PER_SM * f_sm
    return {"replicas": reps, "point_steps_per_s": sum(pts) / sum(times), "ms_per_batch": 1000.0 * sum(times),
            "hss_achieved": ach / 1e12 if ach else None, "hss_peak": peak / 1e12, "unit": "Tlane-op/s",
            "hss_frac": ach / peak if ach else None,
            "hss_busy_fraction_of_step": prof["hss_ms"] / (1000.0 * sum(times))}


def _c2_time_to_logz(ggns, torch, stream, flush, rank, warmup, f_sm):
    """c2x17 in one batch: time to a mean log Z of the 17 replicas, against the plain path."""
    w, runs = runs_of("c2", C2_REPLICAS, rank)
    s = ggns.Sampler(runs, stream=stream.cuda_stream)
    for i in range(max(1, warmup)):
        s.restart(W.SEED_BASE + 3000 + i)
        s.run()
    s.profile(reset=True)
    times, pts, logz, errs = _timed_steps(s, C2_REPLICAS, 2, stream, flush, None, W.SEED_BASE + 4000)
    prof = s.profile(reset=True)
    s.close()
    truth = W.truth_logz(w)
    z = np.array(logz)
    ms = 1000.0 * sum(times) / len(times)
    dz = float(z.mean() - truth)
    sem = float(z.std(ddof=1) / math.sqrt(z.size))
    meets = abs(dz) < 0.2
    # the plain GPU path: the same replicas one after another, one pre-created context each,
    # one host-synchronised launch chain per iteration (no graph, no batching); CUDA events on
    # the default stream bracket the whole sequence
    plains = [ggns.Sampler([r]) for r in runs]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for sp in plains:
        while not sp.step(1):
            pass
        sp.run(0)
        sp.result(0)
    e1.record()
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    for sp in plains:
        sp.close()
    hss_s = prof["hss_ms"] / 1000.0
    ops = lane_ops_per_point_step(32, 4, 0.12, rng=not prof.get("noise_steps", 0) > 0)
    return {"workload": workload_config("c2")["workload"], "point_steps_per_s": sum(pts) / sum(times),
            "ms_per_batch": ms, "logz_mean": float(z.mean()), "logz_truth": truth, "dlogz_mean": dz,
            "dlogz_sem": sem, "logz_sd": float(z.std(ddof=1)), "logz_err_mean": float(np.mean(errs)),
            "runs": int(z.size), "meets_0p2": meets,
            "time_to_logz_ms": ms if meets else None,
            "time_to_logz_note": None if meets else f"mean log Z of the replicas is {dz:+.2f} nats off the closed form",
            "plain": {"time_to_logz_ms": plain_ms if meets else None, "ms": plain_ms,
                      "what": "the 17 replicas one after another, one pre-created context each, one "
                              "host-synchronised launch chain per iteration (no graph, no batching), CUDA events",
                      "speedup": plain_ms / ms},
            "hss_roofline": {"bound": "alu", "achieved": ops * sum(pts) / hss_s / 1e12 if hss_s > 0 else None,
                             "peak": SMS * FP32_LANES_PER_SM * f_sm / 1e12,
                             "frac": ops * sum(pts) / hss_s / (SMS * FP32_LANES_PER_SM * f_sm) if hss_s > 0 else None,
                             "unit": "Tlane-op/s", "ops_per_point_step": ops,
                             "hss_busy_fraction_of_step": prof["hss_ms"] / (1000.0 * sum(times))},
            "throughput_mode": _c2_throughput(ggns, stream, flush, rank, 8 * C2_REPLICAS, f_sm)}


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
    name = args.workload
    R = 1 if name == "c5" else C2_REPLICAS
    w, runs = runs_of(name, R, rank)
    s = ggns.Sampler(runs, stream=stream.cuda_stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for i in range(args.warmup):
        s.restart(W.SEED_BASE + 1000 + i)
        s.run()
        for r in range(R):
            s.grad_logz(r)
    s.profile(reset=True)
    with ClockSampler() as clk:
        times, pts, logz, errs = _timed_steps(s, R, args.steps, stream, flush, dist, W.SEED_BASE + 2000)
    prof = s.profile(reset=True)
    clocks = clk.summary()
    tot_pts = sum_over_ranks(float(sum(pts)), dist, "cuda")
    value = tot_pts / sum(times)
    ms = 1000.0 * sum(times) / len(times)
    peaks = load_peaks()
    f_sm = (clocks.get("sm_mhz") or 1447.0) * 1e6
    hss_s = prof["hss_ms"] / 1000.0
    if name == "c5":
        d, K = 512, 8
        flops = dense_mix_flops_per_point_step(d, K)
        tensor = prof.get("tensor_classes", 0) > 0
        achieved = flops * sum(pts) / hss_s if hss_s > 0 else None
        if tensor:
            # FP16 tcgen05 (kind::f16): the measured BF16 peak, sustained (the kernel runs inside a
            # long step); FP16 and BF16 share the nominal dense rate
            peak = float(peaks.get("bf16_tflops_sustained") or 1700.0) * 1e12
            bound, pnote = "tensor", "FP16 = measured BF16 sustained (same nominal dense rate)"
        else:
            peak = SMS * FP32_LANES_PER_SM * 2.0 * f_sm
            bound, pnote = "alu", f"FP32 FMA: {SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 x {f_sm / 1e6:.0f} MHz"
        roof = {"bound": bound, "achieved": achieved / 1e12 if achieved else None, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                "traffic": measured_traffic(name, sum(pts) / max(prof["hss_iters"], 1)),
                "kernel": "dense-mixture HSS walk (k_hss1, CTA-cooperative)", "flops_per_point_step": flops,
                "hss_busy_fraction_of_step": prof["hss_ms"] / (1000.0 * sum(times)),
                "hss_ms_per_iteration": prof["hss_ms_sum"] / max(prof["hss_iters"], 1), "peak_note": pnote}
    else:
        ops = lane_ops_per_point_step(32, 4, 0.12, rng=not prof.get("noise_steps", 0) > 0)
        achieved = ops * sum(pts) / hss_s if hss_s > 0 else None
        peak = SMS * FP32_LANES_PER_SM * f_sm
        roof = {"bound": "alu", "achieved": achieved / 1e12 if achieved else None, "peak": peak / 1e12,
                "unit": "Tlane-op/s", "frac": (achieved / peak) if achieved else None,
                "traffic": measured_traffic(name, 0.0), "kernel": "k_hss1 + k_hss_pick", "ops_per_point_step": ops,
                "hss_busy_fraction_of_step": prof["hss_ms"] / (1000.0 * sum(times)),
                "peak_note": f"{SMS} SMs x {FP32_LANES_PER_SM} lanes x median SM clock {f_sm / 1e6:.0f} MHz"}
    # e2e: through the C ABI from host buffers: create (H2D of the problem), run, results and the
    # gradient read back (D2H)
    h2d = 0
    for r in runs:
        sp = r["spec"]
        h2d += 8 * (2 * sp["d"] + np.size(sp["means"]) + np.size(sp.get("sigma", [])) +
                    np.size(sp.get("log_weights", [])) + np.size(sp.get("precision", [])))
    d2h = R * (96 + 8 * np.size(w["spec"]["means"]))
    e2e_t = []
    for i in range(max(1, min(2, args.steps))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = ggns.Sampler(runs)
        s2.run()
        _ = [s2.result(r) for r in range(R)]
        _ = [s2.grad_logz(r) for r in range(R)]
        s2.close()
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = pts[-1] / (sum(e2e_t) / len(e2e_t))
    c2leg = None
    if name == "c5" and world == 1 and not args.no_c2:
        c2leg = _c2_time_to_logz(ggns, torch, stream, flush, rank, args.warmup, f_sm)
    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            threads = os.cpu_count() or 1
            if name == "c2":
                threads = min(threads, C2_REPLICAS)
            n, t = oracle_sample(name, threads, seed_base=50_000)
            cpu = {"value": n / t, "unit": UNIT, "cores": threads, "kind": "oracle",
                   "sample": sample_note(name, threads, n, t)}
        z = np.array(logz)
        truth = W.truth_logz(w)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(name),
                "logz_mean": float(z.mean()),
                "logz_truth_box_mass_1": truth,
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": int(prof["launches"] / max(args.steps, 1)),
                "clocks": {"sm_mhz": clocks.get("sm_mhz"), "sm_max_mhz": clocks.get("sm_max_mhz"),
                           "reasons": clocks.get("reasons")},
                "peaks": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained")}}
        if c2leg is not None:
            line["time_to_logz"] = c2leg
        if name == "c2":
            line["dlogz_mean"] = float(z.mean() - truth)
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def profile_case(args):
    """A bounded case for ncu captures (not a benchmark line): one run of the workload with the
    HSS step cap lowered to --n-steps (so the step records stay small) stepped --iters
    iterations through ns_step."""
    import torch
    from paper_2312_03911_gb300 import build as B
    from paper_2312_03911_gb300 import ggns
    torch.cuda.set_device(0)
    B.build()
    ggns.load()
    w = W.workload(args.workload, n_steps=args.n_steps)
    s = ggns.Sampler([w])
    # one iteration per ns_step: iteration i launches the walker kernel once, so the
    # point-steps of launch i are the growth of n_like over iteration i
    steps, last = [], s.result(0, check=False)["n_like"]
    for _ in range(args.iters):
        done = s.step(1)
        nl = s.result(0, check=False)["n_like"]
        steps.append(nl - last)
        last = nl
        if done:
            break
    torch.cuda.synchronize()
    r = s.result(0, check=False)
    print(json.dumps({"profile_case": args.workload, "n_steps": args.n_steps, "n_iter": r["n_iter"],
                      "n_like": r["n_like"], "status": r["status"], "point_steps_per_iteration": steps}), flush=True)
    s.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ggns", choices=["ggns", "reference"])
    ap.add_argument("--workload", default="c5", choices=["c5", "c2"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-c2", action="store_true", help="skip the c2x17 time-to-log-Z leg")
    ap.add_argument("--profile-case", action="store_true",
                    help="run a bounded case for ncu captures instead of the benchmark (see --iters, --n-steps)")
    ap.add_argument("--iters", type=int, default=100, help="--profile-case: iterations to step")
    ap.add_argument("--n-steps", type=int, default=200, help="--profile-case: HSS step cap")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args)
    if args.impl == "reference":
        return reference_arm(args)
    return gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
