"""d log Z / d mu on the GPU, against the closed form and against central finite differences
of log Z over seeded runs (the evidence of Section 2.1 as a function of the component means).

A dense mixture whose shared precision is diagonal has a closed-form evidence under the box
prior,
    log Z = log sum_k w_k prod_i [Phi((hi_i - mu_ki) / s_i) - Phi((lo_i - mu_ki) / s_i)]
            - sum_i log(hi_i - lo_i),
so the derivative in any mean is known exactly.  One mean sits near a face of the box, where the
derivative is far from zero; the other component lies inside, where it nearly vanishes.  The
likelihood runs through the dense-mixture code path (P as a full matrix)."""
import math

import numpy as np
import pytest

from paper_2312_03911_gb300 import ggns
from paper_2312_03911_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

D = 8
SIG = np.array([0.15, 0.2, 0.25, 0.3, 0.15, 0.2, 0.25, 0.3])
MEANS = np.array([[0.85, 0.2, -0.3, 0.1, 0.0, 0.0, 0.0, 0.0],
                  [-0.2, 0.1, 0.3, -0.1, 0.2, -0.3, 0.0, 0.1]])
LO, HI = -np.ones(D), np.ones(D)
R = 48
H = 0.1


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_03911_gb300 import build
    build.build()
    ggns.load()


def _phi(z):
    return math.exp(-0.5 * z * z) / math.sqrt(2 * math.pi)


def _Phi(z):
    return 0.5 * math.erfc(-z / math.sqrt(2))


def _mass(mu, s, lo, hi):
    return _Phi((hi - mu) / s) - _Phi((lo - mu) / s)


def logz_exact(means):
    """The closed form above (equal weights)."""
    K = means.shape[0]
    terms = [sum(math.log(_mass(means[k, i], SIG[i], LO[i], HI[i])) for i in range(D)) - math.log(K)
             for k in range(K)]
    m = max(terms)
    return m + math.log(sum(math.exp(t - m) for t in terms)) - float(np.sum(np.log(HI - LO)))


def dlogz_exact(means, k, i):
    """d log Z / d mu_ki of the closed form: the component's share of Z times the derivative of the
    log of its one-dimensional box mass."""
    K = means.shape[0]
    logm = np.array([sum(math.log(_mass(means[j, c], SIG[c], LO[c], HI[c])) for c in range(D)) for j in range(K)])
    share = math.exp(logm[k] - np.logaddexp.reduce(logm))
    mu, s = means[k, i], SIG[i]
    dlogmass = (_phi((LO[i] - mu) / s) - _phi((HI[i] - mu) / s)) / s / _mass(mu, s, LO[i], HI[i])
    return share * dlogmass


def _workload(means):
    spec = dict(kind=W.LIK_DENSE_MIX, d=D, means=means, precision=np.diag(1.0 / SIG**2),
                log_weights=np.full(len(means), -math.log(len(means))))
    cfg = dict(W.DEFAULT_CFG, n_live=500, clustering=0, seed=4242)
    return dict(spec=spec, lo=LO, hi=HI, cfg=cfg)


def _runs(means):
    w = _workload(means)
    s = ggns.Sampler([dict(w, cfg=dict(w["cfg"], run_id=r)) for r in range(R)])
    s.run()
    res = [s.result(r) for r in range(R)]
    assert all(r["terminated"] == 1 for r in res)
    return s, np.array([r["logz"] for r in res])


def test_logz_of_the_diagonal_dense_mixture_matches_the_closed_form():
    s, z = _runs(MEANS)
    se = z.std(ddof=1) / math.sqrt(R)
    assert abs(z.mean() - logz_exact(MEANS)) < max(0.1, 4 * se), (z.mean(), logz_exact(MEANS), se)


def test_grad_logz_matches_the_closed_form_derivative():
    """The posterior-weighted score estimate of d log Z / d mu (ns_grad_logz), averaged over 48
    seeded runs, matches the exact derivative for the mean near the face (about -0.88) and for the
    interior component (about 0) within 4 standard errors."""
    s, _ = _runs(MEANS)
    g = np.array([s.grad_logz(r) for r in range(R)])  # R x K x D
    for k, i in ((0, 0), (0, 1), (1, 0), (1, 5)):
        est = g[:, k, i]
        se = est.std(ddof=1) / math.sqrt(R)
        exact = dlogz_exact(MEANS, k, i)
        assert abs(est.mean() - exact) < max(0.03, 4 * se), (k, i, est.mean(), exact, se)
    assert dlogz_exact(MEANS, 0, 0) < -0.5  # the test has a derivative to find


def test_central_differences_of_logz_match_the_closed_form():
    """log Z at mu_00 +- h over the same 48 seeds: the difference quotient of the means matches the
    closed-form difference quotient within 4 standard errors of the paired differences, and the
    gradient estimate at mu agrees with both."""
    up, dn = MEANS.copy(), MEANS.copy()
    up[0, 0] += H
    dn[0, 0] -= H
    _, zu = _runs(up)
    _, zd = _runs(dn)
    fd = (zu - zd) / (2 * H)
    se = fd.std(ddof=1) / math.sqrt(R)
    exact = (logz_exact(up) - logz_exact(dn)) / (2 * H)
    assert abs(fd.mean() - exact) < max(0.05, 4 * se), (fd.mean(), exact, se)
    s, _ = _runs(MEANS)
    g = np.array([s.grad_logz(r)[0, 0] for r in range(R)])
    sg = g.std(ddof=1) / math.sqrt(R)
    assert abs(g.mean() - fd.mean()) < max(0.05, 4 * math.hypot(se, sg)), (g.mean(), fd.mean(), se, sg)
