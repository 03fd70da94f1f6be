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


def test_gram_noalloc_allocates_nothing_on_a_side_stream(gpu_bmg):
    """The entry point's contract: after a first call (which looks up the array's
    address), repeated calls on a non-default stream leave the device's free memory
    unchanged; only the end is synchronised."""
    n, k = 40962, 64
    rng = np.random.default_rng(5)
    Xd, Yd = _dev(rng.standard_normal((n, k))), _dev(rng.standard_normal((n, k)))
    G = torch.empty((k, k), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        gpu_bmg.gram_noalloc(Xd, Yd, k, G)          # first call on this device
    side.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with torch.cuda.stream(side):
        for _ in range(5):
            gpu_bmg.gram_noalloc(Xd, Yd, k, G)
        free1 = torch.cuda.mem_get_info()[0]
    side.synchronize()
    assert free1 == free0 and torch.cuda.mem_get_info()[0] == free0
    ref = torch.empty_like(G)
    gpu_bmg.gram(Xd, Yd, k, ref)
    assert torch.max(torch.abs(G - ref)).item() <= 1e-14 * n * 4      # tolerance of the Gram tests


def test_gram_noalloc_wide_leading_dimension(gpu_bmg):
    """A k = 20 column slice of a 200-wide block (shared-memory rows wider than the
    default 48 KB allowance) against bmg_gram and the host product."""
    n, k, ld = 4099, 20, 200
    rng = np.random.default_rng(9)
    Xw = torch.from_numpy(rng.standard_normal((n, ld))).cuda()
    Yw = torch.from_numpy(rng.standard_normal((n, ld))).cuda()
    G1 = torch.empty((k, k), dtype=torch.float64, device="cuda")
    G2 = torch.full((k, k), np.nan, dtype=torch.float64, device="cuda")
    gpu_bmg.gram(Xw, Yw, k, G1)
    gpu_bmg.gram_noalloc(Xw, Yw, k, G2)
    torch.cuda.synchronize()
    ref = Xw[:, :k].cpu().numpy().T @ Yw[:, :k].cpu().numpy()
    assert np.max(np.abs(G1.cpu().numpy() - ref)) <= 1e-14 * n * 4
    assert torch.equal(G1, G2)


def test_gram_noalloc_rejects_oversize_block(gpu_bmg):
    X = torch.zeros((8, 162), dtype=torch.float64, device="cuda")
    G = torch.zeros((161, 161), dtype=torch.float64, device="cuda")
    with pytest.raises(gpu_bmg.BmgError) as e:
        gpu_bmg._check(gpu_bmg.LIB.bmg_gram_noalloc(X.data_ptr(), X.data_ptr(), 8, 161, 162,
                                                    G.data_ptr(), None))
    assert e.value.code == 1 and "160" in str(e.value)
