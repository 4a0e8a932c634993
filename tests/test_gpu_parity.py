"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, on the GPU.

Tolerances: FP64 projection relative error <= 1e-12 (element-wise, relative to the
largest output magnitude); ground-state energy |dE| <= 1e-10; eigenvector overlap
|<x_gpu, x_oracle>| >= 1 - 1e-8 (the sign of an eigenvector is not unique).
"""
import numpy as np
import pytest

from dmrg_inputs import warmup
from dmrg_inputs.superblock import BlockOp, Superblock
from oracle import davidson as odav
from oracle import projection as oproj

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_1309_5571_gb300 import Plan, capi, gemv_trans  # noqa: E402

PROJ_TOL = 1e-12
E_TOL = 1e-10


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel_err(y, y_ref):
    return float(np.max(np.abs(y - y_ref)) / max(np.max(np.abs(y_ref)), 1e-300))


def ragged_superblock(seed=0):
    """Hand-built superblock with ragged sectors (1, 3, 17, 70, 129, 200 states), a
    missing block, an empty sector and an identity-identity term."""
    rng = np.random.default_rng(seed)
    dL = np.array([1, 3, 17, 70, 129, 0, 200])
    dR = np.array([200, 129, 70, 17, 3, 1, 5])
    qL = [(q,) for q in range(7)]
    qR = [(6 - q,) for q in range(7)]
    # right sector k has quantum number 6 - k, so (i, k) is valid iff i == k; the pairs
    # are stored in reverse order to exercise arbitrary segment offsets
    pairs = [(i, i) for i in range(7)][::-1]
    def sym(d):
        a = rng.standard_normal((d, d))
        return a + a.T
    HL = BlockOp({(i, i): sym(d) for i, d in enumerate(dL) if d > 0}, "H_L")
    HR = BlockOp({(k, k): sym(d) for k, d in enumerate(dR) if d > 0}, "H_R")
    # raising on the left (i -> i+1), lowering on the right (k -> k+1 lowers q_R)
    up = BlockOp({(i, i + 1): rng.standard_normal((dL[i + 1], dL[i]))
                  for i in range(6) if i != 2}, "up")            # block 2->3 missing
    dn = BlockOp({(k, k + 1): rng.standard_normal((dR[k + 1], dR[k])) for k in range(6)}, "dn")
    upT = BlockOp({(j, i): M.T.copy() for (i, j), M in up.blocks.items()}, "upT")
    dnT = BlockOp({(j, i): M.T.copy() for (i, j), M in dn.blocks.items()}, "dnT")
    sb = Superblock(qL=qL, dL=dL, qR=qR, dR=dR, Q=(6,), pairs=pairs,
                    opsL=[HL, up, upT], opsR=[HR, dn, dnT],
                    terms=[(1.0, 0, -1), (0.7, -1, 0), (0.5, 1, 1), (0.5, 2, 2), (-0.3, -1, -1)])
    sb.validate()
    return sb


PROBLEMS = {
    "heis_L16_m64": lambda: warmup.warmup_superblock("heisenberg", 16, m=64),
    "hub_L8_m40": lambda: warmup.warmup_superblock("hubbard", 8, m=40, U=4.0),
    "hub_quarter_L12_m48": lambda: warmup.warmup_superblock("hubbard", 12, m=48, U=8.0,
                                                            filling=0.5),
    "heis_L6_exact": lambda: warmup.warmup_superblock("heisenberg", 6, m=1000),
    "ragged": ragged_superblock,
}
_cache = {}


def problem(name):
    if name not in _cache:
        _cache[name] = PROBLEMS[name]()
    return _cache[name]


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_projection_fp64_matches_oracle(name):
    sb = problem(name)
    plan = Plan(sb, prec="fp64")
    for seed in (0, 1):
        x = np.random.default_rng(seed).standard_normal(sb.n)
        y = plan.project(cuda(x)).cpu().numpy()
        y_ref = oproj.project_blocks(sb, x)
        assert rel_err(y, y_ref) <= PROJ_TOL


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_diagonal_matches_oracle(name):
    sb = problem(name)
    plan = Plan(sb)
    d = plan.diagonal().cpu().numpy()
    np.testing.assert_allclose(d, oproj.diagonal(sb), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 1000, 4099, 100003])
@pytest.mark.parametrize("k", [1, 7, 24])
def test_gemv_trans_matches_numpy(n, k):
    rng = np.random.default_rng(n + k)
    ldv = n + 5
    V = rng.standard_normal((k, ldv))
    w = rng.standard_normal(n)
    s = gemv_trans(cuda(V), k, cuda(w)).cpu().numpy()
    ref = V[:, :n] @ w
    np.testing.assert_allclose(s, ref, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(V).max() * n))


@pytest.mark.parametrize("name,max_subspace,keep", [("heis_L16_m64", 20, 2), ("hub_L8_m40", 20, 2),
                                                    ("hub_quarter_L12_m48", 20, 2),
                                                    ("heis_L16_m64", 4, 2), ("heis_L16_m64", 4, 1),
                                                    ("hub_L8_m40", 8, 1), ("hub_L8_m40", 8, 2),
                                                    ("ragged", 20, 2), ("heis_L6_exact", 20, 2)])
def test_davidson_fp64_matches_oracle(name, max_subspace, keep):
    # keep: vectors kept at a subspace-limit restart (the Ritz vector; or also the previous one)
    sb = problem(name)
    x0 = warmup.start_vector(sb.n, seed=0)
    plan = Plan(sb, prec="fp64", max_subspace=max_subspace, restart_keep=keep)
    x, info = plan.solve(cuda(x0))
    x = x.cpu().numpy()
    lam, xo, oinfo = odav.davidson(lambda v: oproj.project_blocks(sb, v), oproj.diagonal(sb),
                                   x0, max_subspace=max_subspace, restart_keep=keep)
    assert oinfo["converged"] and info["converged"]
    assert abs(info["energy"] - lam) <= E_TOL
    assert abs(x @ xo) / (np.linalg.norm(x) * np.linalg.norm(xo)) >= 1 - 1e-8
    # the returned pair satisfies the stopping rule when re-checked by the oracle
    r = oproj.project_blocks(sb, x) - info["energy"] * x
    assert np.linalg.norm(r) <= 1.5e-10
    assert info["fp64_projections"] == info["iters"]
    # same algorithm, same readings: the iteration counts agree closely
    assert abs(info["iters"] - oinfo["iters"]) <= max(3, 0.1 * oinfo["iters"])


def test_davidson_step_api_and_ritz():
    sb = problem("heis_L16_m64")
    x0 = warmup.start_vector(sb.n, seed=3)
    plan = Plan(sb, prec="fp64")
    st = plan.state(cuda(x0))
    conv, it = False, 0
    while not conv and it < 500:
        conv = st.step()
        it += 1
    assert conv
    info = st.info()
    x = st.ritz().cpu().numpy()
    lam = float(x @ oproj.project_blocks(sb, x)) / float(x @ x)
    assert abs(lam - info["energy"]) <= E_TOL
    st.close()


def test_nonconvergence_is_reported():
    sb = problem("heis_L16_m64")
    plan = Plan(sb, prec="fp64", max_iter=3)
    x, info = plan.solve(cuda(warmup.start_vector(sb.n, 0)), raise_on_nonconvergence=False)
    assert not info["converged"] and info["iters"] == 3
    with pytest.raises(capi.NotConverged):
        plan.solve(cuda(warmup.start_vector(sb.n, 0)))


def test_solve_host_matches_device_solve():
    sb = problem("hub_L8_m40")
    x0 = warmup.start_vector(sb.n, seed=1)
    plan = Plan(sb)
    xd, infod = plan.solve(cuda(x0))
    xh, infoh = plan.solve_host(x0)
    assert infoh["energy"] == infod["energy"]
    np.testing.assert_array_equal(xh, xd.cpu().numpy())


def test_zero_start_vector_rejected():
    sb = problem("heis_L6_exact")
    plan = Plan(sb)
    with pytest.raises(capi.DmrgError):
        plan.solve(torch.zeros(sb.n, dtype=torch.float64, device="cuda"))


# ---------------------------------------------------------------- full-size workloads
@pytest.fixture(scope="module")
def heis_L100_m1024():
    return warmup.workload("heis_L100_m1024")


def test_full_size_projection_heisenberg_m1024(heis_L100_m1024):
    sb = heis_L100_m1024
    plan = Plan(sb, prec="fp64")
    x = warmup.start_vector(sb.n, seed=7)
    y = plan.project(cuda(x)).cpu().numpy()
    y_ref = oproj.project_blocks(sb, x)
    assert rel_err(y, y_ref) <= PROJ_TOL


def test_full_size_solve_heisenberg_m1024_properties(heis_L100_m1024):
    # the oracle cannot run the whole solve in seconds at n ~ 8e5; it re-checks the
    # returned pair instead: residual and Rayleigh quotient with its own projection
    sb = heis_L100_m1024
    plan = Plan(sb, prec="fp64")
    x0 = warmup.start_vector(sb.n, seed=0)
    x, info = plan.solve(cuda(x0))
    x = x.cpu().numpy()
    Hx = oproj.project_blocks(sb, x)
    rq = float(x @ Hx) / float(x @ x)
    assert abs(rq - info["energy"]) <= E_TOL
    assert np.linalg.norm(Hx - info["energy"] * x) <= 1.5e-10


@pytest.mark.parametrize("vector_arith", ["fp64", "df", "split"])
def test_vector_arithmetic_options_match_oracle(vector_arith):
    # Davidson vector passes on the FP64 units or in double-float FP32-pair arithmetic
    # ("split" is the FP64 path in an FP64 solve)
    sb = problem("hub_quarter_L12_m48")
    x0 = warmup.start_vector(sb.n, seed=2)
    x, info = Plan(sb, prec="fp64", vector_arith=vector_arith).solve(cuda(x0))
    lam = odav.davidson(lambda v: oproj.project_blocks(sb, v), oproj.diagonal(sb), x0)[0]
    assert abs(info["energy"] - lam) <= E_TOL
    x = x.cpu().numpy()
    assert np.linalg.norm(oproj.project_blocks(sb, x) - info["energy"] * x) <= 1.5e-10
