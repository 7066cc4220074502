"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared symbol."""
import os
import re

import pytest

from paper_2312_03911_gb300 import build as B
from paper_2312_03911_gb300 import ggns

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ns_[a-z_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = ggns.load(path)
    declared = _declared()
    assert declared == set(ggns.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_config_defaults_without_gpu():
    c = ggns.default_config()
    assert (c.n_live, c.n_steps, c.min_ref, c.max_ref, c.termination, c.clustering, c.noise_mode) == \
        (200, 1000, 1, 3, 0, 1, 1)
    assert c.tol == pytest.approx(0.01) and c.dt_init == pytest.approx(0.1) and c.delta_p == pytest.approx(0.5)
    # the readings of Algorithm 5 the library defaults to, and the library's own launch choices
    assert (c.noise_inside, c.pick_all, c.territory, c.keep_last, c.box_fold, c.fold_counts) == (1, 1, 1, 0, 0, 0)
    assert (c.tile, c.hss_mode, c.rec_len, c.noise_ahead, c.coop, c.runs_per_group) == (0, 0, 0, 0, 0, 0)


def test_config_struct_matches_the_header():
    """The binding's ns_config mirrors include/ggns.h field by field (names in order)."""
    import re
    src = open(os.path.join(ROOT, "include", "ggns.h")).read()
    body = src[src.index("typedef struct {\n    int n_live;"):]
    body = body[:body.index("} ns_config;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"(\w+)\s*;", body)
    assert names == [f for f, _ in ggns.Config._fields_]


def test_create_rejects_bad_arguments_without_touching_the_gpu():
    import numpy as np
    w = dict(spec=dict(kind=0, d=2, means=np.zeros((1, 2)), sigma=np.array([0.1])), lo=-np.ones(2), hi=np.ones(2),
             cfg=dict(n_live=1))
    with pytest.raises(ggns.GGNSError) as e:
        ggns.Sampler([w])
    assert e.value.status == ggns.NS_ERR_ARG
    w["cfg"] = dict(n_live=100, min_ref=4, max_ref=3)
    with pytest.raises(ggns.GGNSError):
        ggns.Sampler([w])


def test_autotune_candidates_hold_d_without_doubling_the_padding():
    from paper_2312_03911_gb300 import autotune
    for d in (2, 3, 8, 17, 32, 64, 100, 256, 512):
        c = autotune.candidates(d)
        assert c, d
        for t in c:
            g, e = autotune.TILES[t]
            assert d <= g * e <= 2 * max(d, 2)
    run = dict(spec=dict(kind=1, d=32), cfg=dict(n_live=100))
    out = autotune.apply({(1, 32): (4, 0)}, [run])
    assert out[0]["cfg"]["tile"] == 5 and out[0]["cfg"]["coop"] == 0 and "tile" not in run["cfg"]
