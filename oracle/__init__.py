"""FP64 CPU oracle for gradient-guided nested sampling (arXiv 2312.03911).

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package; the product library never does.

The arithmetic lives in ``ggns_oracle.c`` (plain C, FP64, single-threaded); this
module compiles it with gcc and wraps it with ctypes.  It shares no code with the
CUDA path.  Every function cites the passage of the paper it follows in the C
source; the readings taken where the paper is ambiguous are stated in the header of
``ggns_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ggns_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libggns_oracle.so")
_lock = threading.Lock()
_lib = None

LIK_ISO, LIK_MIX_ISO, LIK_DENSE, LIK_DENSE_MIX, LIK_ROSEN, LIK_TORUS = 0, 1, 2, 3, 4, 5
P_INIT, P_MOM, P_NOISE, P_RES, P_CLUSTER, P_START, P_PRUNE = 0, 1, 2, 3, 4, 5, 6


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libggns_oracle.so`` (gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class LikT(C.Structure):
    _fields_ = [("kind", C.c_int), ("d", C.c_int), ("n_comp", C.c_int),
                ("means", C.POINTER(C.c_double)), ("log_weights", C.POINTER(C.c_double)),
                ("sigma", C.POINTER(C.c_double)), ("precision", C.POINTER(C.c_double)),
                ("rosen_scale", C.c_double), ("torus_alpha", C.c_double), ("torus_beta", C.c_double),
                ("torus_c", C.c_double)]


class CfgT(C.Structure):
    _fields_ = [("n_live", C.c_int), ("n_steps", C.c_int), ("min_steps", C.c_int), ("dt_init", C.c_double),
                ("delta_p", C.c_double), ("tol", C.c_double), ("min_ref", C.c_int),
                ("max_ref", C.c_int), ("prune_after", C.c_int), ("termination", C.c_int),
                ("clustering", C.c_int), ("seed", C.c_uint64), ("run_id", C.c_uint32),
                ("max_iters", C.c_int), ("noise_mode", C.c_int),
                ("out_lo", C.c_double), ("out_hi", C.c_double), ("periodic", C.c_int), ("keep_last", C.c_int),
                ("noise_inside", C.c_int), ("pick_all", C.c_int), ("territory", C.c_int),
                ("box_fold", C.c_int), ("fold_counts", C.c_int), ("midpoint", C.c_int)]


class BatchStatsT(C.Structure):
    _fields_ = [("n_in", C.c_long), ("n_out", C.c_long), ("t_save", C.c_int), ("t_stop", C.c_int),
                ("n_fallback", C.c_int), ("n_fold", C.c_long)]


class ResultT(C.Structure):
    _fields_ = [("logz", C.c_double), ("logz_err", C.c_double), ("logz_skilling_err", C.c_double),
                ("info_h", C.c_double), ("n_iter", C.c_long), ("n_dead", C.c_long),
                ("n_like", C.c_long), ("n_steps_total", C.c_long), ("n_fallback", C.c_long),
                ("n_region_rejected", C.c_long), ("dt", C.c_double),
                ("n_clusters_final", C.c_int), ("max_clusters", C.c_int),
                ("terminated", C.c_int), ("status", C.c_int)]


class IterTraceT(C.Structure):
    _fields_ = [("lstar", C.c_double), ("dt", C.c_double), ("out_frac", C.c_double),
                ("logz", C.c_double), ("log_xl", C.c_double), ("n_clusters", C.c_double)]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.orc_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                      C.c_uint32, C.c_int, C.POINTER(C.c_double)]
            L.orc_loglik.restype = C.c_double
            L.orc_loglik.argtypes = [C.POINTER(LikT), C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.orc_logdet_spd.restype = C.c_double
            L.orc_logdet_spd.argtypes = [C.c_int, C.POINTER(C.c_double)]
            L.orc_loglik_dmeans.argtypes = [C.POINTER(LikT), C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.orc_hss_batch.argtypes = [C.POINTER(LikT), C.c_double, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.POINTER(CfgT), C.c_uint32, C.c_int,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_double, C.c_double,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int),
                                        C.POINTER(BatchStatsT), C.POINTER(C.c_double)]
            L.orc_reflect.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.orc_walk_step.argtypes = [C.POINTER(LikT), C.c_double, C.c_int, C.c_double, C.c_double,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.orc_walk_step.restype = C.c_int
            L.orc_sort_by_logl.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)]
            L.orc_knn_components.restype = C.c_int
            L.orc_knn_components.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_int)]
            L.orc_stats_sequence.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                             C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int,
                                             C.POINTER(C.c_int), C.POINTER(C.c_double),
                                             C.POINTER(C.c_double), C.POINTER(C.c_double),
                                             C.POINTER(C.c_double), C.POINTER(C.c_double),
                                             C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.orc_stats_program.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                            C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.orc_run.restype = C.c_int
            L.orc_run.argtypes = [C.POINTER(CfgT), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(LikT), C.POINTER(ResultT), C.c_long, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int),
                                  C.POINTER(IterTraceT)]
            L.orc_territory.restype = C.c_int
            L.orc_territory.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_int), C.c_int,
                                        C.POINTER(C.c_float), C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.orc_grad_logz_means.argtypes = [C.POINTER(LikT), C.c_long, C.POINTER(C.c_double),
                                              C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_double,
                                              C.POINTER(C.c_double)]
            _lib = L
    return _lib


# --------------------------------------------------------------------------- #
# Python-side wrappers                                                          #
# --------------------------------------------------------------------------- #

class Likelihood:
    """Holds contiguous FP64 parameter arrays alive for the ctypes struct."""

    def __init__(self, kind, d, means=None, sigma=None, log_weights=None, precision=None,
                 rosen_scale=0.05, torus=None):
        self.kind, self.d = int(kind), int(d)
        self.means = None if means is None else np.ascontiguousarray(np.atleast_2d(means), dtype=np.float64)
        self.n_comp = 1 if self.means is None else self.means.shape[0]
        self.sigma = None if sigma is None else np.ascontiguousarray(np.atleast_1d(sigma), dtype=np.float64)
        self.log_weights = None if log_weights is None else np.ascontiguousarray(log_weights, dtype=np.float64)
        self.precision = None if precision is None else np.ascontiguousarray(precision, dtype=np.float64)
        self.rosen_scale = float(rosen_scale)
        # torus reward (Section 4, eq. torus): (alpha, beta, c)
        self.torus = (0.0, 0.0, 0.0) if torus is None else tuple(float(v) for v in torus)
        self.struct = LikT(self.kind, self.d, self.n_comp, _dp(self.means), _dp(self.log_weights),
                           _dp(self.sigma), _dp(self.precision), self.rosen_scale, *self.torus)

    @classmethod
    def from_spec(cls, spec: dict) -> "Likelihood":
        return cls(spec["kind"], spec["d"], means=spec.get("means"), sigma=spec.get("sigma"),
                   log_weights=spec.get("log_weights"), precision=spec.get("precision"),
                   rosen_scale=spec.get("rosen_scale", 0.05), torus=spec.get("torus"))

    def logdet(self) -> float:
        if self.precision is None:
            return 0.0
        return lib().orc_logdet_spd(self.d, _dp(self.precision))

    def loglik(self, x, grad=False):
        x = np.ascontiguousarray(x, dtype=np.float64)
        g = np.zeros(self.d) if grad else None
        v = lib().orc_loglik(C.byref(self.struct), _dp(x), _dp(g))
        return (v, g) if grad else v

    def dmeans(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros((self.n_comp, self.d))
        lib().orc_loglik_dmeans(C.byref(self.struct), _dp(x), _dp(out))
        return out


def make_cfg(**kw) -> CfgT:
    c = dict(n_live=200, n_steps=1000, min_steps=0, dt_init=0.1, delta_p=0.05, tol=0.01, min_ref=1, max_ref=3,
             prune_after=10, termination=0, clustering=0, seed=0, run_id=0, max_iters=100000,
             noise_mode=0, out_lo=0.05, out_hi=0.15, periodic=0, keep_last=0, noise_inside=0, pick_all=0, territory=0, box_fold=0,
             fold_counts=0, midpoint=0)
    c.update(kw)
    return CfgT(**c)


def philox(ctr, key):
    a = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(a, k, o)
    return [int(v) for v in o]


def normals(seed, run_id, it, purpose, slot, step, d):
    z = np.zeros(d)
    lib().orc_normals(int(seed), int(run_id), int(it), int(purpose), int(slot), int(step), int(d), _dp(z))
    return z


def hss_batch(lik: Likelihood, lo, hi, cfg: CfgT, it, x0, logl0, lstar, dt, trace=False):
    """Algorithm 5 on n walkers starting at x0[n][d]; returns outputs and batch statistics."""
    d = lik.d
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    x0 = np.ascontiguousarray(np.atleast_2d(x0), dtype=np.float64)
    logl0 = np.ascontiguousarray(logl0, dtype=np.float64)
    n = x0.shape[0]
    xo = np.zeros((n, d))
    lo_out = np.zeros(n)
    steps = np.zeros(n, dtype=np.int32)
    st = BatchStatsT()
    tr = np.zeros((cfg.n_steps, n, 2 * d + 2)) if trace else None
    lib().orc_hss_batch(C.byref(lik.struct), lik.logdet(), _dp(lo), _dp(hi), C.byref(cfg), int(it), n,
                        _dp(x0), _dp(logl0), float(lstar), float(dt), _dp(xo), _dp(lo_out), _ip(steps),
                        C.byref(st), _dp(tr))
    out = dict(x=xo, logl=lo_out, n_in=st.n_in, n_out=st.n_out, t_save=st.t_save, t_stop=st.t_stop,
               n_fallback=st.n_fallback, n_fold=st.n_fold)
    if trace:
        out["trace"] = tr[: st.t_stop]
    return out


def walk_step(lik: Likelihood, mode: int, lstar: float, dt: float, x, p):
    """One deterministic step of the walk without noise or box (orc_walk_step): mode 0 as
    Algorithm 5 prints it, mode 1 the symmetric splitting.  Returns (x', p', reflected)."""
    x = np.array(x, dtype=np.float64)
    p = np.array(p, dtype=np.float64)
    r = lib().orc_walk_step(C.byref(lik.struct), lik.logdet(), int(mode), float(lstar), float(dt), _dp(x), _dp(p))
    return x, p, bool(r)


def reflect(p, n):
    p = np.array(p, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    lib().orc_reflect(len(p), _dp(p), _dp(n))
    return p


def sort_by_logl(logl):
    logl = np.ascontiguousarray(logl, dtype=np.float64)
    order = np.zeros(len(logl), dtype=np.int32)
    lib().orc_sort_by_logl(len(logl), _dp(logl), _ip(order))
    return order


def knn_components(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    m, d = x.shape
    comp = np.zeros(m, dtype=np.int32)
    n = lib().orc_knn_components(m, d, x.ctypes.data_as(C.POINTER(C.c_float)), _ip(comp))
    return n, comp


def stats_sequence(counts, logx0, labels, logl, logzx0=None, logxx0=None):
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    nc = len(counts)
    logx0 = np.ascontiguousarray(logx0, dtype=np.float64)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    logl = np.ascontiguousarray(logl, dtype=np.float64)
    zx = None if logzx0 is None else np.ascontiguousarray(logzx0, dtype=np.float64)
    xx = None if logxx0 is None else np.ascontiguousarray(logxx0, dtype=np.float64)
    k = len(labels)
    oz, oz2 = C.c_double(), C.c_double()
    ox, ox2, ozx = np.zeros(nc), np.zeros(nc), np.zeros(nc)
    ow = np.zeros(k)
    lib().orc_stats_sequence(nc, _ip(counts), _dp(logx0), _dp(zx), _dp(xx), k, _ip(labels), _dp(logl),
                             C.byref(oz), C.byref(oz2), _dp(ox), _dp(ox2), _dp(ozx), _dp(ow))
    return dict(logz=oz.value, logz2=oz2.value, logx=ox, logx2=ox2, logzx=ozx, logw=ow)


def stats_program(cap, n0, ops):
    """ops: list of ("kill", cluster, logL) or ("split", cluster, size_of_part_kept)."""
    op = np.array([0 if o[0] == "kill" else 1 for o in ops], dtype=np.int32)
    arg = np.array([o[1] for o in ops], dtype=np.int32)
    val = np.array([o[2] for o in ops], dtype=np.float64)
    out = np.zeros(2 + 7 * cap + cap * cap)
    lib().orc_stats_program(cap, n0, len(ops), _ip(op), _ip(arg), _dp(val), _dp(out))
    per = out[2:2 + 7 * cap].reshape(cap, 7)
    return dict(logz=out[0], logz2=out[1], logx=per[:, 0], logx2=per[:, 1], logzx=per[:, 2], logzp=per[:, 3],
                logzp2=per[:, 4], logzpxp=per[:, 5], n=per[:, 6].astype(int),
                logxx=out[2 + 7 * cap:].reshape(cap, cap))


def run(lik: Likelihood, lo, hi, cfg: CfgT, dead_cap=None, trace=False):
    """One full GGNS run (Algorithm 3).  Returns a dict with the result and dead points."""
    d = lik.d
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    if dead_cap is None:
        dead_cap = cfg.n_live * 4000
    dx = np.zeros((dead_cap, d))
    dl = np.zeros(dead_cap)
    dw = np.zeros(dead_cap)
    dlab = np.zeros(dead_cap, dtype=np.int32)
    tr = (IterTraceT * cfg.max_iters)() if trace else None
    res = ResultT()
    lib().orc_run(C.byref(cfg), _dp(lo), _dp(hi), C.byref(lik.struct), C.byref(res), dead_cap, _dp(dx),
                  _dp(dl), _dp(dw), _ip(dlab), tr)
    n = res.n_dead
    out = dict(logz=res.logz, logz_err=res.logz_err, logz_skilling_err=res.logz_skilling_err,
               info_h=res.info_h, n_iter=res.n_iter, n_dead=n, n_like=res.n_like,
               n_steps_total=res.n_steps_total, n_fallback=res.n_fallback,
               n_region_rejected=res.n_region_rejected, dt=res.dt, n_clusters_final=res.n_clusters_final,
               max_clusters=res.max_clusters, terminated=res.terminated, status=res.status,
               dead_x=dx[:n], dead_logl=dl[:n], dead_logw=dw[:n], dead_label=dlab[:n])
    if trace:
        it = res.n_iter
        out["trace"] = {f: np.array([getattr(tr[i], f) for i in range(it)]) for f, _ in IterTraceT._fields_}
    return out


def territory(surv, surv_label, xn, want):
    """Which new points stay in the region of the cluster they were spawned in (1) or are rejected (0)."""
    surv = np.ascontiguousarray(surv, dtype=np.float32)
    xn = np.ascontiguousarray(xn, dtype=np.float32)
    sl = np.ascontiguousarray(surv_label, dtype=np.int32)
    wl = np.ascontiguousarray(want, dtype=np.int32)
    keep = np.zeros(len(xn), dtype=np.int32)
    lib().orc_territory(len(surv), surv.shape[1], surv.ctypes.data_as(C.POINTER(C.c_float)), _ip(sl), len(xn),
                        xn.ctypes.data_as(C.POINTER(C.c_float)), _ip(wl), _ip(keep))
    return keep


def grad_logz_means(lik: Likelihood, xs, logl, logw, logz):
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    logl = np.ascontiguousarray(logl, dtype=np.float64)
    logw = np.ascontiguousarray(logw, dtype=np.float64)
    g = np.zeros((lik.n_comp, lik.d))
    lib().orc_grad_logz_means(C.byref(lik.struct), len(logl), _dp(xs), _dp(logl), _dp(logw), float(logz), _dp(g))
    return g
