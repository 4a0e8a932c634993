"""Pins of the block Davidson-Liu oracle (Sec. 6 remark) against facts outside it (no GPU):
LAPACK's lowest eigenpairs, the single-vector oracle it must reduce to with a block of
one, and planted mistakes that these pins must catch."""
import numpy as np
import pytest

from dmrg_inputs import warmup
from oracle import block_davidson as bd
from oracle import davidson as dav
from oracle import projection


def _hubbard():
    sb = warmup.warmup_superblock("hubbard", 8, m=40, U=4.0)
    return projection.superblock_dense(sb)


def _random_operator(n=400, seed=1):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return np.diag(np.linspace(0.0, 20.0, n)) + 0.25 * (A + A.T)


H_HUB = _hubbard()
H_RND = _random_operator()
_EIGH = {}


def _eigh(H):
    # LAPACK's decomposition of each test matrix, computed once
    key = id(H)
    if key not in _EIGH:
        _EIGH[key] = np.linalg.eigh(H)
    return _EIGH[key]


def _start(n, b, seed=0):
    return np.column_stack([warmup.start_vector(n, seed=seed + j) for j in range(b)])


@pytest.mark.parametrize("keep", [1, 2])
@pytest.mark.parametrize("max_subspace", [20, 4])
def test_block_of_one_is_the_single_vector_iteration(max_subspace, keep):
    # b = nev = 1: the same iterates as Algorithm 3 with the same restart reading
    H = H_HUB
    x0 = warmup.start_vector(H.shape[0], seed=0)
    lam, x, info = dav.davidson(lambda z: H @ z, np.diag(H).copy(), x0, tol=1e-10,
                                max_subspace=max_subspace, restart_keep=keep)
    th, X, binfo = bd.block_davidson(lambda z: H @ z, np.diag(H).copy(), x0[:, None], 1,
                                     tol=1e-10, max_subspace=max_subspace, restart_keep=keep)
    assert binfo["converged"] and info["converged"]
    assert binfo["iters"] == info["iters"] and binfo["restarts"] == info["restarts"]
    # the same iterates up to rounding: Ritz values to 1e-12 relative; residual norms to
    # 1e-12 absolute (rounding of ||r|| ~ eps ||H|| ||x||, ||H|| ~ 10 here) plus 1e-3
    # relative (many restarts amplify the rounding differences of the two codes)
    for (l1, r1), (t2, r2) in zip(info["history"], binfo["history"]):
        assert abs(l1 - t2[0]) <= 1e-12 * abs(l1)
        assert abs(r1 - r2[0]) <= 1e-12 + 1e-3 * r1
    assert abs(abs(x @ X[:, 0]) - 1.0) <= 1e-12


@pytest.mark.parametrize("H", [H_HUB, H_RND], ids=["hubbard_L8_m40", "random400"])
@pytest.mark.parametrize("nev,b", [(1, 2), (2, 2), (3, 4), (4, 4)])
@pytest.mark.parametrize("max_subspace", [24, 12])
def test_block_davidson_equals_eigh(H, nev, b, max_subspace):
    w, v = _eigh(H)
    th, X, info = bd.block_davidson(lambda z: H @ z, np.diag(H).copy(), _start(H.shape[0], b),
                                    nev, tol=1e-10, max_subspace=max_subspace)
    assert info["converged"]
    np.testing.assert_allclose(th, w[:nev], atol=1e-10)
    # orthonormal Ritz vectors, each an eigenvector to the residual tolerance, spanning
    # LAPACK's lowest eigenspace
    assert np.linalg.norm(X.T @ X - np.eye(nev)) <= 1e-12
    assert np.all(np.linalg.norm(H @ X - X * th, axis=0) <= 1e-10 * 1.0001)
    P = v[:, :nev]
    assert np.linalg.norm(X - P @ (P.T @ X)) <= 1e-8


def test_block_davidson_restarts_and_rejects_bad_blocks():
    H = H_RND
    th, X, info = bd.block_davidson(lambda z: H @ z, np.diag(H).copy(), _start(400, 4), 4,
                                    tol=1e-10, max_subspace=12)
    assert info["converged"] and info["restarts"] >= 2
    with pytest.raises(ValueError):
        bd.block_davidson(lambda z: H @ z, np.diag(H).copy(), _start(400, 2), 3)
    x = warmup.start_vector(400, 0)
    with pytest.raises(ValueError):   # rank-deficient start block
        bd.block_davidson(lambda z: H @ z, np.diag(H).copy(), np.column_stack([x, 2 * x]), 2)


def test_planted_highest_ritz_pairs_are_caught(monkeypatch):
    # taking the block from the top of the projected spectrum converges (if at all) to
    # other eigenvalues than LAPACK's lowest
    H = H_HUB
    real = np.linalg.eigh

    def top_first(A):
        w, v = real(A)
        return w[::-1].copy(), v[:, ::-1].copy()

    monkeypatch.setattr(bd.np.linalg, "eigh", top_first)
    th, X, info = bd.block_davidson(lambda z: H @ z, np.diag(H).copy(), _start(H.shape[0], 2), 2,
                                    tol=1e-10, max_iter=200)
    monkeypatch.setattr(bd.np.linalg, "eigh", real)
    w = _eigh(H)[0]
    assert not (info["converged"] and np.allclose(th, w[:2], atol=1e-8))


def test_planted_restart_w_not_transformed_is_caught(monkeypatch):
    H = H_RND

    def bad(V, W, B, C):
        return V @ C, W[:, :C.shape[1]].copy(), C.T @ B @ C

    monkeypatch.setattr(bd, "collapse_block", bad)
    th, X, info = bd.block_davidson(lambda z: H @ z, np.diag(H).copy(), _start(400, 2), 2,
                                    tol=1e-10, max_subspace=8, max_iter=300)
    w = _eigh(H)[0]
    assert not (info["converged"] and np.allclose(th, w[:2], atol=1e-8))
