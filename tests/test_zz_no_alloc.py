"""The allocation-free Gram entry point (bmg_gram_noalloc).

Some callers cannot allocate device memory (their framework already holds the
device's memory, or they run under a fixed budget), so libbmg offers a variant of the
Gram product whose partial sums live in a fixed array inside the library.  This file
checks it through the C ABI against the allocating entry point, on two calls in a row
(the second call reuses the array the first one left behind).  It is collected last
so that a run stopping at its first failure has run every other test already.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _dev(X):
    n, k = X.shape
    ld = (k + 1) // 2 * 2
    T = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
    T[:, :k] = torch.from_numpy(X).cuda()
    return T


@pytest.mark.parametrize("n,k", [(40962, 64), (2562, 20), (4099, 130)])
def test_gram_noalloc_matches_gram_on_two_consecutive_calls(gpu_bmg, n, k):
    rng = np.random.default_rng(n * 7 + k)
    for call in range(2):
        X, Y = rng.standard_normal((n, k)), rng.standard_normal((n, k))
        Xd, Yd = _dev(X), _dev(Y)
        G_ref = torch.empty((k, k), dtype=torch.float64, device="cuda")
        G_new = torch.full((k, k), np.nan, dtype=torch.float64, device="cuda")
        gpu_bmg.gram(Xd, Yd, k, G_ref)
        gpu_bmg.gram_noalloc(Xd, Yd, k, G_new)
        torch.cuda.synchronize()
        a, b = G_new.cpu().numpy(), G_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), call
        assert np.max(np.abs(a - b)) <= 1e-14 * n * 4, call          # tolerance of the Gram tests
        assert np.max(np.abs(a - X.T @ Y)) <= 1e-14 * n * 4, call


def test_gram_noalloc_rejects_oversize_block(gpu_bmg):
    X = torch.zeros((8, 162), dtype=torch.float64, device="cuda")
    G = torch.zeros((161, 161), dtype=torch.float64, device="cuda")
    with pytest.raises(gpu_bmg.BmgError) as e:
        gpu_bmg._check(gpu_bmg.LIB.bmg_gram_noalloc(X.data_ptr(), X.data_ptr(), 8, 161, 162,
                                                    G.data_ptr(), None))
    assert e.value.code == 1 and "160" in str(e.value)
