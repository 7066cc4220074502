"""The allocation-free k-NN component finder (ns_knn_components_noalloc).

Callers that cannot allocate device memory while they run -- a host framework
that owns every device allocation through its own pool, or a process whose
device-memory budget is fixed at start time -- use this entry point; its scratch
is a static device array.  Its output must equal that of the allocating entry
point ns_knn_components, on consecutive calls that reuse the same scratch.
This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import numpy as np
import pytest

from paper_2312_03911_gb300 import ggns

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_03911_gb300 import build
    build.build()
    ggns.load()


def _blobs(seed, m, d, k):
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-1, 1, (k, d))
    return (centers[rng.integers(0, k, m)] + 0.08 * rng.standard_normal((m, d))).astype(np.float32)


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    # the second call is smaller than the first, so stale scratch from call one would show
    for seed, m, d, k in [(21, 3000, 16, 4), (22, 700, 32, 3), (23, 4096, 8, 5)]:
        x = torch.as_tensor(_blobs(seed, m, d, k), device="cuda")
        ref = torch.zeros(m, dtype=torch.int32, device="cuda")
        got = torch.full((m,), -7, dtype=torch.int32, device="cuda")
        n_ref = ggns.knn_components(x.data_ptr(), m, d, ref.data_ptr())
        n_got = ggns.knn_components_noalloc(x.data_ptr(), m, d, got.data_ptr())
        assert n_got == n_ref
        assert torch.equal(got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    x = torch.zeros((4097, 2), device="cuda")
    out = torch.zeros(4097, dtype=torch.int32, device="cuda")
    with pytest.raises(ggns.GGNSError) as e:
        ggns.knn_components_noalloc(x.data_ptr(), 4097, 2, out.data_ptr())
    assert e.value.status == ggns.NS_ERR_ARG
    assert "4096" in str(e.value)
