"""Per-step GPU parity against the FP64 oracle: fused SpMM, smoothers, transfers,
Gram, and the enriched eigensolve, on blocks that span several tiles with ragged
column counts."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import bmg as obmg, multilevel
from paper_1511_07042_gb300 import inputs

pytestmark = pytest.mark.gpu
R = 4


@pytest.fixture(scope="module")
def env(gpu_bmg):
    v, t = inputs.icosahedron()
    prob = gpu_bmg.Problem(v, t, R)
    prob.hierarchy(R)
    H = obmg.build_hierarchy(v, t, R, colour2=True)
    return gpu_bmg, prob, H


def dev(X, ld=None):
    n, k = X.shape
    ld = ld or (k + 1) // 2 * 2
    T = torch.zeros((n, ld), dtype=torch.float64, device="cuda")
    T[:, :k] = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    return T


def host(T, k):
    torch.cuda.synchronize()
    return T[:, :k].cpu().numpy()


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


KS = [3, 20, 64, 130]


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("f,l", [(4, 4), (4, 2), (3, 1)])
def test_spmm(env, k, f, l):
    bmg, prob, H = env
    A = H.A[l] if f == l else H.GA[f][l]
    M = H.M[l] if f == l else H.GM[f][l]
    X = np.random.default_rng(k + 10 * l).standard_normal((A.shape[0], k))
    Xd = dev(X)
    AX, MX = torch.empty_like(Xd), torch.empty_like(Xd)
    prob.spmm(f, l, Xd, k, AX, MX)
    assert rel(host(AX, k), A @ X) < 1e-14 and rel(host(MX, k), M @ X) < 1e-14
    assert torch.all(AX[:, k:] == 0) and torch.all(MX[:, k:] == 0)


@pytest.mark.parametrize("k", [3, 20, 64])
@pytest.mark.parametrize("smoother,nu,omega", [("jacobi", 2, 2 / 3), ("mcgs", 1, 1.0), ("mcsgs", 2, 1.0),
                                               ("kaczmarz", 2, 1.0), ("kaczmarz", 1, 0.8)])
@pytest.mark.parametrize("f,l", [(4, 4), (4, 3)])
@pytest.mark.parametrize("with_b", [True, False])
def test_smoothers(env, k, smoother, nu, omega, f, l, with_b):
    bmg, prob, H = env
    A = H.A[l] if f == l else H.GA[f][l]
    M = H.M[l] if f == l else H.GM[f][l]
    rng = np.random.default_rng(100 + k)
    X = rng.standard_normal((A.shape[0], k))
    B = rng.standard_normal((A.shape[0], k)) if with_b else np.zeros_like(X)
    s = rng.uniform(0.0, 20.0, k)
    Xd, Bd = dev(X), dev(B)
    sd = torch.zeros(Xd.shape[1], dtype=torch.float64, device="cuda")
    sd[:k] = torch.from_numpy(s).cuda()
    work = torch.empty_like(Xd)
    prob.smooth(f, l, Xd, Bd if with_b else None, sd, k, smoother, nu, omega, work)
    if smoother == "jacobi":
        ref = multilevel.jacobi(A, M, X, B, s, omega, nu)
    elif smoother == "kaczmarz":
        ref = multilevel.kaczmarz(A, M, X, B, s, H.colour2[l], nu, omega)
    else:
        ref = multilevel.mc_gauss_seidel(A, M, X, B, s, H.colour[l], nu, symmetric=(smoother == "mcsgs"))
    assert rel(host(Xd, k), ref) < 1e-12
    assert torch.all(Xd[:, k:] == 0)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("l", [2, 3, 4])
def test_prolong_restrict_bit_exact(env, k, l):
    bmg, prob, H = env
    P = H.P[l]
    rng = np.random.default_rng(7 * k + l)
    Xc = rng.standard_normal((P.shape[1], k))
    Rf = rng.standard_normal((P.shape[0], k))
    Y0 = rng.standard_normal((P.shape[0], k))
    Xcd, Rfd = dev(Xc), dev(Rf)
    Y = torch.empty_like(Rfd)
    prob.prolong(l, Xcd, Y, k)
    assert np.array_equal(host(Y, k), P @ Xc)
    Yadd = dev(Y0)
    prob.prolong(l, Xcd, Yadd, k, add=True)
    assert np.array_equal(host(Yadd, k), Y0 + P @ Xc)
    Z = torch.empty_like(Xcd)
    prob.restrict(l, Rfd, Z, k)
    assert np.array_equal(host(Z, k), P.T @ Rf)


@pytest.mark.parametrize("n,k", [(1, 1), (17, 3), (2562, 20), (10242, 64), (4099, 130)])
def test_gram(env, n, k):
    bmg, prob, H = env
    rng = np.random.default_rng(n + k)
    X, Y = rng.standard_normal((n, k)), rng.standard_normal((n, k))
    G = torch.empty((k, k), dtype=torch.float64, device="cuda")
    bmg.gram(dev(X), dev(Y), k, G)
    ref = X.T @ Y
    assert np.max(np.abs(G.cpu().numpy() - ref)) <= 1e-14 * n * 4


def _dense(bmg, Ah, Mh, sigma, k):
    A = torch.from_numpy(Ah).cuda()
    M = torch.from_numpy(Mh).cuda()
    th = torch.empty(k, dtype=torch.float64, device="cuda")
    Y = torch.empty((Ah.shape[0], k), dtype=torch.float64, device="cuda")
    rk = torch.zeros(1, dtype=torch.int32, device="cuda")
    bmg.dense_eig(A, M, sigma, k, th, Y, rk)
    return th.cpu().numpy(), Y.cpu().numpy(), int(rk.item())


@pytest.mark.parametrize("n,k,sigma", [(10, 4, 0.0), (62, 20, 0.0), (106, 64, 1.5), (170, 128, 0.0), (192, 150, 0.0),
                                         (194, 150, 0.5), (200, 160, 0.0), (202, 160, 0.0)])
def test_dense_eig_well_conditioned(env, n, k, sigma):
    bmg, prob, H = env
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    Mh = B @ B.T + n * np.eye(n)
    S = rng.standard_normal((n, n))
    Ah = S + S.T
    th, Y, rk = _dense(bmg, Ah, Mh, sigma, k)
    thr, Yr = obmg.svqb_eig(Ah, Mh, sigma, k)
    assert rk == n
    assert np.allclose(th, thr, rtol=1e-11, atol=1e-11 * np.abs(thr).max())
    assert np.allclose(Y.T @ Mh @ Y, np.eye(k), atol=1e-11)
    assert np.max(np.abs(Ah @ Y - Mh @ Y * (th + sigma)[None, :])) < 1e-9


def test_dense_eig_enriched_space_rank_deficient(env):
    """Enriched matrices of a real level where X holds the constant vector, which
    lies in span(Q) exactly (P 1 = 1): the pivoted factorisation must drop it."""
    bmg, prob, H = env
    f, k = 3, 12
    rng = np.random.default_rng(5)
    X = rng.standard_normal((H.A[f].shape[0], k))
    X[:, 0] = 1.0
    Ah, Mh = obmg.enriched_matrices(H, f, X, H.A[f] @ X, H.M[f] @ X)
    th, Y, rk = _dense(bmg, Ah, Mh, 0.0, k)
    thr, _ = obmg.svqb_eig(Ah, Mh, 0.0, k)
    assert rk == Ah.shape[0] - 1
    assert np.allclose(th, thr, rtol=1e-10, atol=1e-10)
