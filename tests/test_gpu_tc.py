"""Tensor-core (tcgen05) Gram products and Ritz-vector expansion from exact digit
slices, against float64 references on the CPU.

The claimed error (include/bmg.h, bmg_gram_tc): each window of K <= 256 rows
contributes at most about 2^-53 K max|x| max|y| (float64 blocks) or 2^-33 K max|x|
max|y| (float64 accumulation of float32 blocks), the maxima over the window's column;
the expansion likewise with k terms and the maxima over a row of X and a column of Yx.
The tests allow 2^-50 (2^-31) of that bound plus the rounding of the float64 reference
(2^-51 of sum |x||y|), on Gaussian blocks and on blocks with spikes, tiny and zero
columns, on ragged sizes from one row to several windows and parts."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def dev(X, dtype=torch.float64):
    n, k = X.shape
    align = 2 if dtype == torch.float64 else 4
    ld = (k + align - 1) // align * align
    T = torch.zeros((n, ld), dtype=dtype, device="cuda")
    T[:, :k] = torch.from_numpy(np.ascontiguousarray(X)).to(dtype).cuda()
    return T


def window_bound(X, Y, w=256):
    """sum over windows of w rows of w_rows * max|x_i| * max|y_j| (k x k)."""
    n = X.shape[0]
    b = np.zeros((X.shape[1], Y.shape[1]))
    for r0 in range(0, n, w):
        xs, ys = np.abs(X[r0:r0 + w]), np.abs(Y[r0:r0 + w])
        b += xs.shape[0] * np.outer(xs.max(axis=0), ys.max(axis=0))
    return b


def blocks(n, k, seed, spiky):
    rng = np.random.default_rng(seed)
    X, Y = rng.standard_normal((n, k)), rng.standard_normal((n, k))
    if spiky and k >= 4:
        X[:, 1] *= 1e-9
        Y[:, 2] *= 1e7
        X[:, 3] = 0.0
        X[n // 2, 0] = 1e4
        Y[0, k - 1] = -3e-5
    return X, Y


CASES = [(1, 1), (7, 3), (130, 8), (2562, 20), (10242, 64), (4099, 100), (40962, 128), (163842, 128)]


@pytest.mark.parametrize("n,k", CASES)
@pytest.mark.parametrize("spiky", [False, True])
def test_gram_tc_fp64(gpu_bmg, n, k, spiky):
    X, Y = blocks(n, k, n + k, spiky)
    G = torch.full((k, k), np.nan, dtype=torch.float64, device="cuda")
    gpu_bmg.gram_tc(dev(X), dev(Y), k, G)
    err = np.abs(G.cpu().numpy() - X.T @ Y)
    tol = 2.0 ** -50 * window_bound(X, Y) + 2.0 ** -51 * (np.abs(X).T @ np.abs(Y))
    assert np.all(err <= tol), (err / tol).max()


@pytest.mark.parametrize("n,k", CASES)
@pytest.mark.parametrize("spiky", [False, True])
def test_gram_tc_fp32(gpu_bmg, n, k, spiky):
    X, Y = blocks(n, k, 3 * n + k, spiky)
    X32, Y32 = X.astype(np.float32), Y.astype(np.float32)
    G = torch.full((k, k), np.nan, dtype=torch.float64, device="cuda")
    gpu_bmg.gram_tc_f32(dev(X32, torch.float32), dev(Y32, torch.float32), k, G)
    Xd, Yd = X32.astype(np.float64), Y32.astype(np.float64)
    err = np.abs(G.cpu().numpy() - Xd.T @ Yd)
    tol = 2.0 ** -31 * window_bound(Xd, Yd) + 2.0 ** -51 * (np.abs(Xd).T @ np.abs(Yd))
    assert np.all(err <= tol), (err / tol).max()


@pytest.mark.parametrize("n,k", CASES)
@pytest.mark.parametrize("with_z", [True, False])
def test_expand_tc_fp64(gpu_bmg, n, k, with_z):
    rng = np.random.default_rng(7 * n + k)
    X, _ = blocks(n, k, n + 2 * k, True)
    Yx = rng.standard_normal((k, k))
    Yx[:, 0] *= 1e-5
    Z = rng.standard_normal((n, k)) if with_z else np.zeros((n, k))
    Xd, Zd = dev(X), dev(Z)
    U = torch.full_like(Xd, np.nan)
    gpu_bmg.expand(Zd if with_z else None, Xd, torch.from_numpy(Yx).cuda(), k, U, True)
    ref = Z + X @ Yx
    err = np.abs(U[:, :k].cpu().numpy() - ref)
    bound = k * np.outer(np.abs(X).max(axis=1), np.abs(Yx).max(axis=0))
    tol = 2.0 ** -50 * bound + 2.0 ** -51 * (np.abs(Z) + np.abs(X) @ np.abs(Yx))
    assert np.all(err <= tol), (err / tol).max()
    assert torch.all(U[:, k:] == 0)            # padding columns stay zero
    # the CUDA-core form of the same call
    U2 = torch.full_like(Xd, np.nan)
    gpu_bmg.expand(Zd if with_z else None, Xd, torch.from_numpy(Yx).cuda(), k, U2, False)
    err2 = np.abs(U2[:, :k].cpu().numpy() - ref)
    assert np.all(err2 <= 2.0 ** -45 * (np.abs(Z) + np.abs(X) @ np.abs(Yx)))


@pytest.mark.parametrize("n,k", CASES)
def test_expand_tc_fp32(gpu_bmg, n, k):
    rng = np.random.default_rng(11 * n + k)
    X, _ = blocks(n, k, n + 3 * k, False)
    Yx = rng.standard_normal((k, k))
    Z = rng.standard_normal((n, k))
    X32, Z32 = X.astype(np.float32), Z.astype(np.float32)
    Xd, Zd = dev(X32, torch.float32), dev(Z32, torch.float32)
    U = torch.full_like(Xd, np.nan)
    gpu_bmg.expand(Zd, Xd, torch.from_numpy(Yx).cuda(), k, U, True)
    ref = Z32.astype(np.float64) + X32.astype(np.float64) @ Yx
    scale = np.abs(Z32) + np.abs(X32.astype(np.float64)) @ np.abs(Yx)
    bound = k * np.outer(np.abs(X32).max(axis=1), np.abs(Yx).max(axis=0))
    err = np.abs(U[:, :k].cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= 2.0 ** -31 * bound + 2.0 ** -23 * scale), (err / (bound + scale)).max()
    assert torch.all(U[:, k:] == 0)


def test_tc_rejects_large_k(gpu_bmg):
    X = torch.zeros((8, 130), dtype=torch.float64, device="cuda")
    G = torch.zeros((129, 129), dtype=torch.float64, device="cuda")
    with pytest.raises(gpu_bmg.BmgError) as e:
        gpu_bmg._check(gpu_bmg.LIB.bmg_gram_tc(X.data_ptr(), X.data_ptr(), 8, 129, 130, G.data_ptr(), None))
    assert e.value.code == 1


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_tc_non_finite_inputs_give_nan(gpu_bmg, dtype):
    """A NaN or Inf in a column (Gram) or row (expansion) makes the outputs it feeds NaN."""
    n, k = 300, 20
    rng = np.random.default_rng(3)
    X, Y = rng.standard_normal((n, k)), rng.standard_normal((n, k))
    X[200, 4] = np.nan
    Y[17, 9] = np.inf
    Xd, Yd = dev(X, dtype), dev(Y, dtype)
    G = torch.zeros((k, k), dtype=torch.float64, device="cuda")
    (gpu_bmg.gram_tc if dtype == torch.float64 else gpu_bmg.gram_tc_f32)(Xd, Yd, k, G)
    Gh = G.cpu().numpy()
    bad = np.zeros((k, k), bool)
    bad[4, :] = True
    bad[:, 9] = True
    assert np.all(np.isnan(Gh[bad])) and np.all(np.isfinite(Gh[~bad]))
    Yx = torch.from_numpy(rng.standard_normal((k, k))).cuda()
    U = torch.zeros_like(Xd)
    gpu_bmg.expand(None, Xd, Yx, k, U, True)
    Uh = U[:, :k].cpu().numpy()
    assert np.all(np.isnan(Uh[200])) and np.all(np.isfinite(np.delete(Uh, 200, axis=0)))


def test_bounded_wait_expiry_returns_timeout_and_context_stays_usable(gpu_bmg):
    """A Gram whose MMA warp issues nothing, with waits of about 1 ms: the workers'
    waits for the commits expire, the kernel frees its tensor memory and returns, and
    the host sees BMG_ERR_TIMEOUT (9).  A normal Gram afterwards is exact."""
    assert gpu_bmg.tc_timeout_selftest() == 9
    assert "bounded wait" in gpu_bmg.LIB.bmg_last_error().decode()
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    n, k = 4099, 64
    X, Y = rng.standard_normal((n, k)), rng.standard_normal((n, k))
    G = torch.empty((k, k), dtype=torch.float64, device="cuda")
    gpu_bmg.gram_tc(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), k, G)
    err = np.abs(G.cpu().numpy() - X.T @ Y)
    assert np.all(err <= 2.0 ** -48 * (np.abs(X).T @ np.abs(Y)))
