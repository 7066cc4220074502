"""Failure detection through the C ABI: every failure ends a normal GPU run with a status
the host reads (no trap, no fault), and the runs beside the failing one in the same
context finish normally.  Also the checks ns_state_load makes on a saved state before
anything reaches the device."""
import math

import numpy as np
import pytest

from paper_2312_03911_gb300 import ggns
from paper_2312_03911_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_03911_gb300 import build
    build.build()
    ggns.load()


def _healthy():
    return W.small_workload("iso", 4, 100, seed=1)


def _status(s, run):
    return s.result(run, check=False)["status"]


def test_nan_parameters_report_numeric():
    """Means poisoned with NaN make every log-likelihood NaN: the run stops with
    NS_ERR_NUMERIC; the healthy run of the same context terminates normally."""
    bad = W.small_workload("iso", 4, 100, seed=2)
    bad = dict(bad, spec=dict(bad["spec"], means=np.full((1, 4), np.nan)), cfg=dict(bad["cfg"], max_iters=50))
    s = ggns.Sampler([bad, _healthy()])
    s.run()
    assert _status(s, 0) == ggns.NS_ERR_NUMERIC
    with pytest.raises(ggns.GGNSError) as e:
        s.result(0)
    assert e.value.status == ggns.NS_ERR_NUMERIC
    ok = s.result(1)
    assert ok["status"] == ggns.NS_OK and ok["terminated"] == 1


def test_iteration_cap_reports_not_done():
    capped = dict(_healthy(), cfg=dict(_healthy()["cfg"], max_iters=3))
    s = ggns.Sampler([capped, _healthy()])
    s.run()
    r = s.result(0, check=False)
    assert r["status"] == ggns.NS_ERR_NOT_DONE and r["terminated"] == 0 and r["n_iter"] == 3
    assert s.result(1)["terminated"] == 1


def test_more_clusters_than_slots_report_capacity():
    """The torus reward with frequencies 9 on [0, 2 pi)^2 has 81 separated maxima: with
    clustering on, Algorithm 4 finds more clusters than the 64 slots of a run and the run
    stops with NS_ERR_CAPACITY."""
    d = 2
    spec = dict(kind=W.LIK_TORUS, d=d, torus=(9.0, 9.0, d + 0.5))
    lo, hi = np.zeros(d), np.full(d, 2 * math.pi)
    cfg = dict(W.DEFAULT_CFG, n_live=4000, clustering=1, seed=5, max_iters=400)
    s = ggns.Sampler([dict(spec=spec, lo=lo, hi=hi, cfg=cfg), _healthy()])
    s.run()
    r = s.result(0, check=False)
    assert r["status"] == ggns.NS_ERR_CAPACITY, r
    assert s.result(1)["terminated"] == 1


def test_host_side_capacity_errors():
    s = ggns.Sampler([_healthy()])
    s.run()
    L = ggns.load()
    import ctypes as C
    n = C.c_long()
    x = np.zeros((2, 4))
    lp = np.zeros(2)
    st = L.ns_samples(s.h, 0, ggns._dp(x), ggns._dp(lp), 2, C.byref(n))
    assert st == ggns.NS_ERR_CAPACITY and n.value > 2
    need = C.c_size_t()
    assert L.ns_state_save(s.h, None, 0, C.byref(need)) == ggns.NS_OK
    buf = C.create_string_buffer(need.value)
    assert L.ns_state_save(s.h, buf, need.value - 1, C.byref(need)) == ggns.NS_ERR_CAPACITY


def _long_at(b, pos):
    return int.from_bytes(b[pos:pos + 8], "little", signed=True)


def _patch_long(b, pos, v):
    return b[:pos] + int(v).to_bytes(8, "little", signed=True) + b[pos + 8:]


def test_state_load_rejects_inconsistent_buffers():
    """A truncated or padded state, a dead-point count patched negative or too large, and a
    run state whose dead-point count disagrees with the rows that follow are refused with
    NS_ERR_ARG before any copy; the context keeps its state, steps on, and reaches the same
    result as a clean resume."""
    w = W.small_workload("mix", 6, 200, seed=12, clustering=1)
    a = ggns.Sampler([w])
    a.step(5)
    blob = a.state_save()
    nd = a.result(0, check=False)["n_dead"]
    # layout: a 40-byte header, then the run state, whose dead-point count follows 16 ints'
    # and doubles' worth (64 bytes) of iteration fields
    assert _long_at(blob, 104) == nd
    # the per-run dead-point count in front of the dead rows: the last position holding nd
    # from which the remaining bytes split into nd rows of (4 d_pad + 16) bytes
    pos = None
    for p in range(len(blob) - 8, 104, -1):
        if _long_at(blob, p) == nd:
            rest = len(blob) - p - 8
            if rest % nd == 0 and (rest // nd - 16) % 4 == 0 and rest // nd > 16:
                pos = p
                break
    assert pos is not None
    bad = [blob[:-1], blob + b"\0", _patch_long(blob, pos, -1), _patch_long(blob, pos, 1 << 40),
           _patch_long(blob, pos, nd - 1), _patch_long(blob, 104, nd + 50)]
    for b in bad:
        with pytest.raises(ggns.GGNSError) as e:
            a.state_load(b)
        assert e.value.status == ggns.NS_ERR_ARG
    # the context kept its state: it resumes from iteration 5 like a clean load would
    a.run()
    ra = a.result(0)
    b2 = ggns.Sampler([w])
    b2.state_load(blob)
    b2.run()
    rb = b2.result(0)
    assert ra["logz"] == rb["logz"] and ra["n_iter"] == rb["n_iter"]
