"""The FP64 direct summation on the GPU (the reference of the bench's error
measurements) against the oracle's direct sum (O1)."""
import numpy as np
import pytest

import oracle as O
from paper_1005_5384_gb300 import octgrav as G
from paper_1005_5384_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.load()


@pytest.mark.parametrize("n,eps", [(1, 0.01), (2, 0.0), (300, 0.05), (40000, 0.01)])
def test_direct_sum_equals_oracle(n, eps):
    pos, m = W.plummer(n, seed=n) if n > 2 else (np.array([[0.0, 0, 0], [1, 2, 2]])[:n], np.array([1.0, 2.0])[:n])
    samp = W.sample_indices(n, min(n, 700), seed=3)
    a, p = G.direct(pos, m, eps, G=2.0, targets=samp)
    ra, rp = O.direct(pos, m, eps, G=2.0, targets=samp)
    if n == 1:
        assert np.all(a == 0) and np.all(p == 0)
        return
    assert np.abs(a - ra).max() <= 1e-12 * np.abs(ra).max()
    assert np.abs(p - rp).max() <= 1e-12 * np.abs(rp).max()


def test_all_targets_and_errors():
    pos, m = W.plummer(3000, seed=5)
    a, p = G.direct(pos, m, 0.01)
    ra, rp = O.direct(pos, m, 0.01)
    assert np.abs(a - ra).max() <= 1e-12 * np.abs(ra).max()
    with pytest.raises(G.OctgravError) as e:
        G.direct(pos, m, 0.01, targets=[0, 3000])
    assert e.value.code == G.ERR_ARG
