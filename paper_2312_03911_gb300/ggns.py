"""Thin ctypes binding of libggns (include/ggns.h).

Argument marshalling only: every step of the sampler runs in the CUDA library.
The library is loaded on first use from ``paper_2312_03911_gb300/_build`` and
this module raises if it is missing or if no CUDA device is present; there is
no CPU fallback.

A run is a dict ``{spec, lo, hi, cfg}``: ``spec`` holds ``kind`` (LIK_*), ``d`` and the
parameters of that kind (``means`` [n_comp][d], ``sigma``, ``log_weights``, ``precision``
[d][d], ``rosen_scale``, ``torus`` = (alpha, beta, c)); ``lo``/``hi`` bound the uniform
prior (a torus for LIK_TORUS); ``cfg`` overrides fields of ``ns_config`` by name.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

NS_OK, NS_ERR_ARG, NS_ERR_CUDA, NS_ERR_OOM, NS_ERR_TIMEOUT, NS_ERR_STUCK, NS_ERR_NUMERIC, NS_ERR_NOT_DONE, \
    NS_ERR_CAPACITY, NS_ERR_BOUNDS = range(10)
STATUS_NAMES = ["NS_OK", "NS_ERR_ARG", "NS_ERR_CUDA", "NS_ERR_OOM", "NS_ERR_TIMEOUT", "NS_ERR_STUCK",
                "NS_ERR_NUMERIC", "NS_ERR_NOT_DONE", "NS_ERR_CAPACITY", "NS_ERR_BOUNDS"]
LIK_ISO_GAUSS, LIK_MIX_ISO, LIK_DENSE_GAUSS, LIK_DENSE_MIX, LIK_ROSENBROCK, LIK_TORUS = range(6)


class PriorBox(C.Structure):
    _fields_ = [("d", C.c_int), ("lo", C.POINTER(C.c_double)), ("hi", C.POINTER(C.c_double))]


class LikSpec(C.Structure):
    _fields_ = [("kind", C.c_int), ("d", C.c_int), ("n_comp", C.c_int), ("means", C.POINTER(C.c_double)),
                ("log_weights", C.POINTER(C.c_double)), ("sigma", C.POINTER(C.c_double)),
                ("precision", C.POINTER(C.c_double)), ("rosen_scale", C.c_double),
                ("torus_alpha", C.c_double), ("torus_beta", C.c_double), ("torus_c", C.c_double)]


class Config(C.Structure):
    _fields_ = [("n_live", C.c_int), ("n_steps", C.c_int), ("min_steps", C.c_int), ("dt_init", C.c_double),
                ("delta_p", C.c_double), ("tol", C.c_double), ("min_ref", C.c_int), ("max_ref", C.c_int),
                ("prune_after", C.c_int), ("termination", C.c_int), ("clustering", C.c_int),
                ("noise_mode", C.c_int), ("out_lo", C.c_double), ("out_hi", C.c_double), ("seed", C.c_uint64),
                ("run_id", C.c_uint32), ("max_iters", C.c_long), ("dead_cap", C.c_long),
                ("noise_inside", C.c_int), ("pick_all", C.c_int), ("territory", C.c_int), ("keep_last", C.c_int),
                ("box_fold", C.c_int), ("fold_counts", C.c_int),
                ("tile", C.c_int), ("hss_mode", C.c_int), ("rec_len", C.c_int), ("noise_ahead", C.c_int),
                ("coop", C.c_int), ("runs_per_group", C.c_int), ("midpoint", C.c_int)]


class Result(C.Structure):
    _fields_ = [("logz", C.c_double), ("logz_err", C.c_double), ("logz_skilling_err", C.c_double),
                ("info_h", C.c_double), ("n_iter", C.c_long), ("n_dead", C.c_long), ("n_like", C.c_long),
                ("n_steps_total", C.c_long), ("dt", C.c_double), ("n_clusters", C.c_int),
                ("max_clusters", C.c_int), ("terminated", C.c_int), ("status", C.c_int)]


# every symbol include/ggns.h declares
EXPORTS = ["ns_config_default", "ns_create", "ns_batch_create", "ns_set_stream", "ns_step", "ns_run", "ns_restart",
           "ns_profile", "ns_result",
           "ns_result_run", "ns_samples", "ns_grad_logz", "ns_state_save", "ns_state_load", "ns_last_error",
           "ns_destroy", "ns_philox", "ns_lik_forward", "ns_lik_backward", "ns_hss", "ns_knn_components",
           "ns_sort_logl", "ns_stats_update", "ns_knn_components_noalloc", "ns_set_means", "ns_territory"]

_lib = None
_lock = threading.Lock()
_vp = C.c_void_p


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def load(path: str | None = None, build_if_missing: bool = False):
    """Load libggns.so (without touching the GPU).  Raises if the library is absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or _build.LIB
        if not os.path.exists(path):
            if build_if_missing:
                _build.build()
            else:
                raise RuntimeError(f"libggns.so not found at {path}: run __graft_entry__.build() first")
        L = C.CDLL(path)
        L.ns_config_default.argtypes = [C.POINTER(Config)]
        L.ns_config_default.restype = None
        L.ns_create.argtypes = [C.POINTER(PriorBox), C.POINTER(LikSpec), C.POINTER(Config), C.POINTER(_vp)]
        L.ns_batch_create.argtypes = [C.c_int, C.POINTER(PriorBox), C.POINTER(LikSpec), C.POINTER(Config),
                                      C.POINTER(_vp)]
        L.ns_set_stream.argtypes = [_vp, _vp]
        L.ns_step.argtypes = [_vp, C.c_int, C.POINTER(C.c_int)]
        L.ns_run.argtypes = [_vp, C.c_long]
        L.ns_restart.argtypes = [_vp, C.c_uint64]
        L.ns_profile.argtypes = [_vp, C.POINTER(C.c_double), C.c_int]
        L.ns_result.argtypes = [_vp, C.POINTER(Result)]
        L.ns_result_run.argtypes = [_vp, C.c_int, C.POINTER(Result)]
        L.ns_samples.argtypes = [_vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_long,
                                 C.POINTER(C.c_long)]
        L.ns_grad_logz.argtypes = [_vp, C.c_int, C.POINTER(C.c_double), C.c_long]
        L.ns_state_save.argtypes = [_vp, _vp, C.c_size_t, C.POINTER(C.c_size_t)]
        L.ns_state_load.argtypes = [_vp, _vp, C.c_size_t]
        L.ns_last_error.argtypes = [_vp]
        L.ns_last_error.restype = C.c_char_p
        L.ns_destroy.argtypes = [_vp]
        L.ns_destroy.restype = None
        L.ns_philox.argtypes = [_vp, C.c_uint32, C.c_uint32, _vp, C.c_long, _vp]
        L.ns_lik_forward.argtypes = [_vp, _vp, C.c_long, _vp, _vp, _vp]
        L.ns_lik_backward.argtypes = [_vp, _vp, C.c_long, _vp, _vp, _vp, _vp]
        L.ns_set_means.argtypes = [_vp, C.c_int, C.POINTER(C.c_double)]
        L.ns_hss.argtypes = [_vp, _vp, _vp, C.c_long, C.c_float, C.c_double, C.c_uint32, _vp, _vp, _vp,
                             C.POINTER(C.c_long), _vp]
        L.ns_knn_components.argtypes = [_vp, C.c_int, C.c_int, _vp, C.POINTER(C.c_int), _vp]
        L.ns_sort_logl.argtypes = [_vp, C.c_int, _vp, _vp]
        L.ns_territory.argtypes = [_vp, _vp, C.c_int, _vp, _vp, C.c_int, C.c_int, _vp, _vp]
        L.ns_knn_components_noalloc.argtypes = [_vp, C.c_int, C.c_int, _vp, C.POINTER(C.c_int), _vp]
        L.ns_stats_update.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double)]
        for name in EXPORTS:
            if name not in ("ns_config_default", "ns_last_error", "ns_destroy"):
                getattr(L, name).restype = C.c_int
        _lib = L
        return L


class GGNSError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


def _check(st, ctx=None):
    if st != NS_OK:
        msg = load().ns_last_error(ctx)
        raise GGNSError(st, msg.decode() if msg else "")


def default_config(**kw) -> Config:
    c = Config()
    load().ns_config_default(C.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


class _Keep:
    """Holds the numpy arrays referenced by the ctypes structs of one create call."""

    def __init__(self):
        self.items = []

    def arr(self, a, dtype=np.float64):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dtype)
        self.items.append(a)
        return a


def _structs(keep: _Keep, spec: dict, lo, hi, cfg: dict):
    d = int(spec["d"])
    lo = keep.arr(lo)
    hi = keep.arr(hi)
    box = PriorBox(d, _dp(lo), _dp(hi))
    means = keep.arr(None if spec.get("means") is None else np.atleast_2d(spec["means"]))
    n_comp = 1 if means is None else means.shape[0]
    lk = LikSpec(int(spec["kind"]), d, n_comp, _dp(means), _dp(keep.arr(spec.get("log_weights"))),
                 _dp(keep.arr(None if spec.get("sigma") is None else np.atleast_1d(spec["sigma"]))),
                 _dp(keep.arr(spec.get("precision"))), float(spec.get("rosen_scale", 0.05)),
                 *[float(v) for v in spec.get("torus", (0.0, 0.0, 0.0))])
    c = default_config()
    for k, v in cfg.items():
        if hasattr(c, k) or k in dict(Config._fields_):
            setattr(c, k, v)
    return box, lk, c


class Sampler:
    """One context holding one or more independent runs (ns_batch_create)."""

    def __init__(self, runs: list[dict], stream=None):
        L = load()
        self._keep = _Keep()
        n = len(runs)
        boxes = (PriorBox * n)()
        liks = (LikSpec * n)()
        cfgs = (Config * n)()
        self.d = []
        self.n_comp = []
        for i, w in enumerate(runs):
            b, lk, c = _structs(self._keep, w["spec"], w["lo"], w["hi"], w["cfg"])
            boxes[i], liks[i], cfgs[i] = b, lk, c
            self.d.append(lk.d)
            self.n_comp.append(lk.n_comp)
        h = _vp()
        st = L.ns_batch_create(n, boxes, liks, cfgs, C.byref(h))
        _check(st, None)
        self.h = h
        self.n_runs = n
        if stream is not None:
            _check(L.ns_set_stream(self.h, _vp(stream)), self.h)

    def close(self):
        if getattr(self, "h", None):
            load().ns_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        _check(load().ns_set_stream(self.h, _vp(stream)), self.h)

    def step(self, n_iters: int) -> bool:
        done = C.c_int()
        _check(load().ns_step(self.h, int(n_iters), C.byref(done)), self.h)
        return bool(done.value)

    def run(self, max_iters: int = 10**9):
        _check(load().ns_run(self.h, int(max_iters)), self.h)

    def restart(self, seed: int):
        _check(load().ns_restart(self.h, int(seed) & 0xFFFFFFFFFFFFFFFF), self.h)

    def profile(self, reset: bool = False) -> dict:
        out = (C.c_double * 10)()
        _check(load().ns_profile(self.h, out, int(reset)), self.h)
        return dict(hss_ms=out[0], hss_iters=int(out[1]), launches=int(out[2]), replays=int(out[3]),
                    hss_ms_sum=out[4], rec_overflows=int(out[5]), rec_len=int(out[6]), noise_steps=int(out[7]),
                    coop_classes=int(out[8]), tensor_classes=int(out[9]))

    def result(self, run: int = 0, check: bool = True) -> dict:
        r = Result()
        st = load().ns_result_run(self.h, int(run), C.byref(r))
        if check:
            _check(st, self.h)
        return {f: getattr(r, f) for f, _ in Result._fields_}

    def samples(self, run: int = 0):
        L = load()
        n = C.c_long()
        _check(L.ns_samples(self.h, run, None, None, 0, C.byref(n)), self.h)
        x = np.zeros((n.value, self.d[run]))
        lp = np.zeros(n.value)
        _check(L.ns_samples(self.h, run, _dp(x), _dp(lp), n.value, C.byref(n)), self.h)
        return x, lp

    def grad_logz(self, run: int = 0):
        g = np.zeros((self.n_comp[run], self.d[run]))
        _check(load().ns_grad_logz(self.h, run, _dp(g), g.size), self.h)
        return g

    def state_save(self) -> bytes:
        L = load()
        n = C.c_size_t()
        _check(L.ns_state_save(self.h, None, 0, C.byref(n)), self.h)
        buf = C.create_string_buffer(n.value)
        _check(L.ns_state_save(self.h, buf, n.value, C.byref(n)), self.h)
        return buf.raw[: n.value]

    def state_load(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        _check(load().ns_state_load(self.h, buf, len(data)), self.h)

    # ---- component calls (device pointers as ints)
    def lik_forward(self, x_ptr, n, logl_ptr, grad_ptr=None, stream=None):
        _check(load().ns_lik_forward(self.h, _vp(x_ptr), int(n), _vp(logl_ptr), _vp(grad_ptr), _vp(stream)), self.h)

    def set_means(self, means, run: int = 0):
        """Replace the component means of run `run` (n_comp x d, FP64 copy taken)."""
        m = np.ascontiguousarray(np.asarray(means, dtype=np.float64))
        _check(load().ns_set_means(self.h, int(run), _dp(m)), self.h)

    def lik_backward(self, x_ptr, n, gout_ptr, gx_ptr=None, gmu_ptr=None, stream=None):
        _check(load().ns_lik_backward(self.h, _vp(x_ptr), int(n), _vp(gout_ptr), _vp(gx_ptr), _vp(gmu_ptr),
                                      _vp(stream)), self.h)

    def hss(self, x0_ptr, logl0_ptr, n, lstar, dt, it, x_out_ptr, logl_out_ptr, steps_ptr=None, stream=None):
        st = (C.c_long * 5)()
        _check(load().ns_hss(self.h, _vp(x0_ptr), _vp(logl0_ptr), int(n), float(lstar), float(dt), int(it),
                             _vp(x_out_ptr), _vp(logl_out_ptr), _vp(steps_ptr), st, _vp(stream)), self.h)
        return dict(n_in=st[0], n_out=st[1], t_save=st[2], t_stop=st[3], n_fold=st[4])


def philox(ctr_ptr, key0, key1, out_ptr, n, stream=None):
    _check(load().ns_philox(_vp(ctr_ptr), int(key0) & 0xFFFFFFFF, int(key1) & 0xFFFFFFFF, _vp(out_ptr), int(n),
                            _vp(stream)))


def knn_components(x_ptr, m, d, comp_ptr, stream=None) -> int:
    nc = C.c_int()
    _check(load().ns_knn_components(_vp(x_ptr), int(m), int(d), _vp(comp_ptr), C.byref(nc), _vp(stream)))
    return nc.value


def knn_components_noalloc(x_ptr, m, d, comp_ptr, stream=None) -> int:
    """ns_knn_components_noalloc: the same result without allocating device memory (m <= 4096)."""
    nc = C.c_int()
    _check(load().ns_knn_components_noalloc(_vp(x_ptr), int(m), int(d), _vp(comp_ptr), C.byref(nc), _vp(stream)))
    return nc.value


def territory(surv_ptr, surv_label_ptr, m_s, xn_ptr, want_ptr, k, d, keep_ptr, stream=None):
    """ns_territory: keep[j] = 1 when new point j's nearest survivor carries label want[j]."""
    _check(load().ns_territory(_vp(surv_ptr), _vp(surv_label_ptr), int(m_s), _vp(xn_ptr), _vp(want_ptr), int(k),
                               int(d), _vp(keep_ptr), _vp(stream)))


def sort_logl(logl_ptr, n, order_ptr, stream=None):
    _check(load().ns_sort_logl(_vp(logl_ptr), int(n), _vp(order_ptr), _vp(stream)))


def stats_update(counts, logx0, labels, logl, logzx0=None, logxx0=None):
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    nc = len(counts)
    logx0 = np.ascontiguousarray(logx0, dtype=np.float64)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    logl = np.ascontiguousarray(logl, dtype=np.float64)
    zx = None if logzx0 is None else np.ascontiguousarray(logzx0, dtype=np.float64)
    xx = None if logxx0 is None else np.ascontiguousarray(logxx0, dtype=np.float64)
    k = len(labels)
    out = np.zeros(3 + 3 * nc + k)
    ip = lambda a: a.ctypes.data_as(C.POINTER(C.c_int))
    _check(load().ns_stats_update(nc, ip(counts), _dp(logx0), _dp(zx), _dp(xx), k, ip(labels), _dp(logl), _dp(out)))
    per = out[3:3 + 3 * nc].reshape(nc, 3)
    return dict(logz=out[0], logz2=out[1], logx=per[:, 0], logx2=per[:, 1], logzx=per[:, 2], logw=out[3 + 3 * nc:])
