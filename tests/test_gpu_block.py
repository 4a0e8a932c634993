"""Block Davidson-Liu on the GPU (dmrg_davidson_solve_block) against the block oracle,
LAPACK and the golden energies.

The nev lowest Ritz values must equal the oracle's (and, on problems small enough for a
dense eigensolver, LAPACK's lowest eigenvalues) to |dE| <= 1e-10; every returned vector
must be an eigenvector of the oracle's projection to ||H x - theta x|| <= 1.5e-10 and the
returned block orthonormal to 1e-10.  Eigenvectors are compared through the subspace they
span (a vector is unique only up to sign, and up to rotation inside a degenerate space).
"""
import numpy as np
import pytest

from dmrg_inputs import warmup
from oracle import block_davidson as obd
from oracle import davidson as odav
from oracle import projection as oproj

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_1309_5571_gb300 import Plan, capi  # noqa: E402

from _workloads import golden, workload  # noqa: E402
from test_gpu_parity import problem  # noqa: E402

E_TOL = 1e-10
R_TOL = 1.5e-10


def start_block(n, b, seed=0):
    return np.stack([warmup.start_vector(n, seed=seed + j) for j in range(b)])


def check_pairs(sb, X, th):
    X = X.cpu().numpy()
    assert np.linalg.norm(X @ X.T - np.eye(len(th))) <= 1e-10
    for x, t in zip(X, th):
        assert np.linalg.norm(oproj.project_blocks(sb, x) - t * x) <= R_TOL
    return X


@pytest.mark.parametrize("nev,b", [(1, 1), (1, 2), (2, 2), (3, 4)])
@pytest.mark.parametrize("prec", ["fp64", "fp64tc"])
@pytest.mark.parametrize("name", ["heis_L16_m64", "hub_L8_m40", "ragged"])
def test_block_davidson_matches_oracle(name, prec, nev, b):
    sb = problem(name)
    X0 = start_block(sb.n, b)
    plan = Plan(sb, prec=prec)
    X, th, rn, info = plan.solve_block(torch.from_numpy(X0).cuda(), nev)
    assert info["converged"] == 1 and max(rn) <= 1e-10
    th_o, X_o, oinfo = obd.block_davidson(lambda v: oproj.project_blocks(sb, v), oproj.diagonal(sb),
                                          X0.T.copy(), nev, tol=1e-10, max_subspace=20)
    assert oinfo["converged"]
    np.testing.assert_allclose(th, th_o, atol=E_TOL, rtol=0)
    X = check_pairs(sb, X, th)
    # the same eigenspace as the oracle's Ritz vectors
    P = X_o / np.linalg.norm(X_o, axis=0)
    assert np.linalg.norm(X.T - P @ (P.T @ X.T)) <= 1e-7


@pytest.mark.parametrize("name", ["heis_L16_m64", "hub_quarter_L12_m48"])
def test_block_davidson_lowest_eigenvalues_equal_lapack(name):
    sb = problem(name)
    H = oproj.superblock_dense(sb)
    w = np.linalg.eigvalsh(H)
    X, th, rn, info = Plan(sb, prec="fp64").solve_block(torch.from_numpy(start_block(sb.n, 4)).cuda(), 4)
    np.testing.assert_allclose(th, w[:4], atol=E_TOL, rtol=0)
    check_pairs(sb, X, th)


def test_block_of_one_matches_single_vector_solve():
    # b = nev = 1 is the single-vector iteration: the same energy as the FP64 solve
    sb = problem("hub_L8_m40")
    x0 = warmup.start_vector(sb.n, seed=0)
    plan = Plan(sb, prec="fp64")
    X, th, rn, info = plan.solve_block(torch.from_numpy(x0[None, :].copy()).cuda(), 1)
    x1, info1 = plan.solve(torch.from_numpy(x0).cuda())
    lam = odav.davidson(lambda v: oproj.project_blocks(sb, v), oproj.diagonal(sb), x0)[0]
    assert abs(th[0] - info1["energy"]) <= E_TOL and abs(th[0] - lam) <= E_TOL
    assert abs(info["iters"] - info1["iters"]) <= max(3, info1["iters"] // 10)


def test_block_davidson_small_subspace_restarts():
    # max_subspace = 8 with a block of 4: every iteration that adds corrections restarts
    sb = problem("hub_L8_m40")
    X0 = start_block(sb.n, 4, seed=3)
    X, th, rn, info = Plan(sb, prec="fp64", max_subspace=8).solve_block(torch.from_numpy(X0).cuda(), 3)
    assert info["converged"] == 1 and info["restarts"] >= 3
    w = np.linalg.eigvalsh(oproj.superblock_dense(sb))
    np.testing.assert_allclose(th, w[:3], atol=E_TOL, rtol=0)
    check_pairs(sb, X, th)


def test_block_davidson_rejects_bad_arguments():
    sb = problem("heis_L16_m64")
    plan = Plan(sb, prec="fp64")
    X0 = torch.from_numpy(start_block(sb.n, 2)).cuda()
    with pytest.raises(capi.DmrgError):
        plan.solve_block(X0, 3)                       # nev > block
    x = warmup.start_vector(sb.n, 0)
    with pytest.raises(capi.DmrgError):               # rank-deficient start block
        plan.solve_block(torch.from_numpy(np.stack([x, 3 * x])).cuda(), 2)
    with pytest.raises(capi.DmrgError):               # 2 block > max_subspace
        Plan(sb, prec="fp64", max_subspace=6).solve_block(
            torch.from_numpy(start_block(sb.n, 4)).cuda(), 2)


def test_block_davidson_full_size_golden():
    # hub_L64_m2048, the two lowest pairs with a block of two (FP64-accurate tensor-core
    # projections): the lowest equals the oracle's golden ground-state energy
    sb = workload("hub_L64_m2048")
    g = golden()["hub_L64_m2048"]
    X0 = start_block(sb.n, 2)
    X, th, rn, info = Plan(sb, prec="fp64tc").solve_block(torch.from_numpy(X0).cuda(), 2)
    assert info["converged"] == 1
    assert abs(th[0] - g["energy"]) <= E_TOL, (th, g["energy"])
    assert th[1] > th[0]
    check_pairs(sb, X, th)
