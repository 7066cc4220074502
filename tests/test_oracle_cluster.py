"""Pins of the oracle's cluster finding (Algorithm 4) and ordering."""
import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components

import oracle


def _scipy_alg4(x):
    """Algorithm 4 through SciPy's connected-components routine: k-NN graphs for k = 2, 3, ...
    (symmetric union, ties to the lower index, k capped at m - 1) until the size multiset repeats."""
    x = np.asarray(x, np.float32)
    m = len(x)
    if m < 3:
        return np.arange(m) * 0
    dist = np.zeros((m, m), np.float32)
    for t in range(x.shape[1]):  # FP32 fused multiply-add per coordinate, in coordinate order
        diff = (x[:, None, t] - x[None, :, t]).astype(np.float32)
        # fmaf(diff, diff, dist): the product of two FP32 values is exact in FP64
        dist = (diff.astype(np.float64) * diff.astype(np.float64) + dist.astype(np.float64)).astype(np.float32)
    order = []
    for i in range(m):
        js = [j for j in range(m) if j != i]
        js.sort(key=lambda j: (dist[i, j], j))
        order.append(js)
    prev = None
    labels = None
    for k in range(2, m + 1):
        kk = min(k, m - 1)
        rows, cols = [], []
        for i in range(m):
            for j in order[i][:kk]:
                rows.append(i); cols.append(j)
        g = csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(m, m))
        nc, lab = connected_components(g, directed=False)
        sizes = sorted(np.bincount(lab).tolist(), reverse=True)
        if sizes == prev:
            break
        prev, labels = sizes, lab
    # canonical id: smallest member index
    out = np.zeros(m, int)
    for c in np.unique(labels):
        mem = np.where(labels == c)[0]
        out[mem] = mem.min()
    return out


def test_separated_blobs_are_found():
    rng = np.random.default_rng(0)
    centers = np.array([[0, 0, 0, 0], [3, 0, 0, 0], [0, 3, 3, 0]], float)
    x = np.concatenate([c + 0.1 * rng.standard_normal((25, 4)) for c in centers])
    perm = rng.permutation(len(x))
    x = x[perm]
    n, comp = oracle.knn_components(x)
    assert n == 3
    blob = perm // 25
    for b in range(3):
        mem = np.where(blob == b)[0]
        assert np.all(comp[mem] == mem.min())


@pytest.mark.parametrize("seed,m,d", [(1, 40, 3), (2, 60, 2), (3, 25, 8), (4, 80, 5), (5, 3, 2), (6, 4, 1)])
def test_matches_library_components(seed, m, d):
    rng = np.random.default_rng(seed)
    k = rng.integers(1, 4)
    centers = rng.uniform(-2, 2, (k, d))
    x = centers[rng.integers(0, k, m)] + 0.3 * rng.standard_normal((m, d))
    x = x.astype(np.float32)
    _, comp = oracle.knn_components(x)
    np.testing.assert_array_equal(comp, _scipy_alg4(x))


def test_ties_break_to_lower_index():
    # points on a lattice produce many equal distances
    g = np.array([[i, j] for i in range(5) for j in range(5)], np.float32)
    x = np.concatenate([g, g + 10.0])
    _, comp = oracle.knn_components(x)
    np.testing.assert_array_equal(comp, _scipy_alg4(x))


def test_sort_order_nan_first_then_index():
    logl = np.array([0.5, np.nan, -1.0, 0.5, -np.inf, np.nan, 2.0])
    order = oracle.sort_by_logl(logl)
    assert list(order) == [1, 5, 4, 2, 0, 3, 6]
