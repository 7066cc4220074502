"""The checked build (GGNS_CHECKED): the library compiled with index checks on the
dead-point arena, the step records and the live slots, each of which reports
NS_ERR_BOUNDS in the run's status instead of touching memory out of range.  It is
the stand-in for a device memory checker: the workloads below, run through the
checked library in a process of its own, must end with status 0 (no check fired)
and give the same log Z, bit for bit, as the default library (the checks change no
arithmetic)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2312_03911_gb300 import build as B  # noqa: E402
from paper_2312_03911_gb300 import ggns  # noqa: E402
from paper_2312_03911_gb300 import workloads as W  # noqa: E402

# the isotropic d = 2 run, the 4-mode mixture with clustering and the region rule, the
# dense mixture on the tensor-core walk (d = 128), the torus
CASES = [("c1", None), ("mix", 8), ("dense_mix", 128), ("torus", 4)]

SCRIPT = r"""
import json, sys
sys.path.insert(0, {root!r})
from paper_2312_03911_gb300 import ggns
sys.path.insert(0, {tests!r})
import test_gpu_checked as T
ggns.load({lib!r})
print(json.dumps(T.run_cases()))
"""


def _runs(name, d):
    if name == "c1":
        w = W.workload("c1")
    elif name == "mix":
        w = W.small_workload("mix", d, 200, seed=5, clustering=1)
    elif name == "dense_mix":
        w = W.small_workload("dense_mix", d, 200, seed=5)
    else:
        w = W.small_workload("torus", d, 100, seed=5)
    return [dict(w, cfg=dict(w["cfg"], run_id=r)) for r in range(4)]


def run_cases():
    """Every case as one batch of 4 runs through the library loaded in this process:
    per case the statuses and log Z of its runs."""
    torch.cuda.set_device(0)
    out = {}
    for name, d in CASES:
        s = ggns.Sampler(_runs(name, d))
        s.run()
        res = [s.result(r, check=False) for r in range(4)]
        out[name] = dict(status=[int(r["status"]) for r in res], logz=[float(r["logz"]) for r in res],
                         n_like=[int(r["n_like"]) for r in res])
        s.close()
    return out


def test_checked_build_runs_clean_and_bit_identical():
    lib = B.build(checked=True)
    script = SCRIPT.format(root=ROOT, tests=os.path.dirname(os.path.abspath(__file__)), lib=lib)
    p = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    checked = json.loads(p.stdout.strip().splitlines()[-1])
    ggns.load()
    plain = run_cases()
    for name, _ in CASES:
        assert checked[name]["status"] == [0, 0, 0, 0], (name, checked[name]["status"])
        assert plain[name]["status"] == [0, 0, 0, 0], (name, plain[name]["status"])
        assert checked[name]["n_like"] == plain[name]["n_like"], name
        np.testing.assert_array_equal(checked[name]["logz"], plain[name]["logz"], err_msg=name)
