"""The l-1-1-r strategy on the GPU (dmrg_plan_create_l11r; Sec. 4.2, Eqs. 12-13) against
the l-1-1-r oracle, the LR plan of the same superblock and the golden energy.

The l-1-1-r and LR superblocks of a workload are one Hamiltonian in two bases, so a
solve in either form reaches the same ground-state energy; the full-size case is checked
against the oracle-written golden energy of hub_L64_m2048.  Tolerances are those of the
LR parity tests (the same GEMM arithmetic on smaller blocks).
"""
import numpy as np
import pytest

from dmrg_inputs import warmup
from oracle import davidson as odav
from oracle import l11r as ol11r

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_1309_5571_gb300 import Plan  # noqa: E402

from _workloads import golden, workload_l11r  # noqa: E402

TOL = {"fp64": 1e-12, "fp64tc": 1e-12, "bf16x3": 2e-5, "bf16x2": 2e-4, "tf32": 5e-3}
E_TOL = 1e-10
PROBLEMS = {
    "heis_L6_exact": dict(model="heisenberg", L=6, m=1000),
    "heis_L16_m64": dict(model="heisenberg", L=16, m=64),
    "hub_L8_m40": dict(model="hubbard", L=8, m=40, U=4.0),
    "hub_quarter_L12_m48": dict(model="hubbard", L=12, m=48, U=8.0, filling=0.5),
}
_cache = {}


def pair(name):
    if name not in _cache:
        kw = PROBLEMS[name]
        _cache[name] = (warmup.warmup_superblock_l11r(**kw), warmup.warmup_superblock(**kw))
    return _cache[name]


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel_err(y, y_ref):
    return float(np.max(np.abs(y - y_ref)) / max(np.max(np.abs(y_ref)), 1e-300))


@pytest.mark.parametrize("prec", list(TOL))
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_l11r_projection_matches_oracle(name, prec):
    sb, _ = pair(name)
    plan = Plan(sb, prec=prec)
    for seed in (0, 1):
        x = np.random.default_rng(seed).standard_normal(sb.n)
        y = plan.project(cuda(x)).cpu().numpy()
        assert rel_err(y, ol11r.project_blocks(sb, x)) <= TOL[prec], (name, prec)
    assert plan.stats["records"] == ol11r.flop_count(sb)["records"]
    assert plan.stats["flops"] == ol11r.flop_count(sb)["flops"]


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_l11r_diagonal_matches_oracle(name):
    sb, _ = pair(name)
    d = Plan(sb).diagonal().cpu().numpy()
    np.testing.assert_allclose(d, ol11r.diagonal(sb), rtol=0, atol=1e-14 * max(1.0, np.max(np.abs(d))))


@pytest.mark.parametrize("opts", [dict(prec="fp64"), dict(prec="bf16x2", anchor_prec="fp64tc"),
                                  dict(prec="bf16x3", anchor_prec="fp64")], ids=["fp64", "bf16x2", "bf16x3"])
@pytest.mark.parametrize("name", ["heis_L16_m64", "hub_L8_m40", "hub_quarter_L12_m48"])
def test_l11r_solve_matches_oracle_and_lr(name, opts):
    sb, sb_lr = pair(name)
    x0 = warmup.start_vector(sb.n, seed=0)
    x, info = Plan(sb, **opts).solve(cuda(x0))
    lam, _, _ = odav.davidson(lambda v: ol11r.project_blocks(sb, v), ol11r.diagonal(sb), x0)
    assert info["converged"] and abs(info["energy"] - lam) <= E_TOL, (info, lam)
    x = x.cpu().numpy()
    assert np.linalg.norm(ol11r.project_blocks(sb, x) - info["energy"] * x) <= 1.5e-10
    # the LR form of the same superblock: the same lowest eigenvalue
    _, info_lr = Plan(sb_lr, prec="fp64").solve(cuda(warmup.start_vector(sb_lr.n, seed=0)))
    assert abs(info["energy"] - info_lr["energy"]) <= E_TOL


def test_l11r_batched_solve():
    from paper_1309_5571_gb300 import solve_batched
    sbs = [pair(n)[0] for n in ("heis_L16_m64", "hub_L8_m40", "hub_quarter_L12_m48")]
    plans = [Plan(sb, prec="bf16x2", anchor_prec="fp64tc") for sb in sbs]
    x0s = [cuda(warmup.start_vector(sb.n, seed=i)) for i, sb in enumerate(sbs)]
    outs, infos = solve_batched(plans, x0s)
    for sb, x0, info in zip(sbs, x0s, infos):
        lam = odav.davidson(lambda v: ol11r.project_blocks(sb, v), ol11r.diagonal(sb),
                            x0.cpu().numpy())[0]
        assert info["converged"] == 1 and abs(info["energy"] - lam) <= E_TOL


@pytest.fixture(scope="module")
def hub_l11r():
    return workload_l11r("hub_L64_m2048")


def test_l11r_full_size_projection(hub_l11r):
    sb = hub_l11r
    x = warmup.start_vector(sb.n, seed=5)
    y_ref = ol11r.project_blocks(sb, x)
    for prec in ("fp64tc", "bf16x2"):
        y = Plan(sb, prec=prec).project(cuda(x)).cpu().numpy()
        assert rel_err(y, y_ref) <= TOL[prec], prec


@pytest.mark.parametrize("opts", [dict(prec="bf16x2", anchor_prec="fp64tc"), dict(prec="fp64tc")],
                         ids=["bf16x2", "fp64tc"])
def test_l11r_full_size_solve_matches_golden(hub_l11r, opts):
    sb = hub_l11r
    g = golden()["hub_L64_m2048"]
    assert sb.n == g["n"]
    x, info = Plan(sb, **opts).solve(cuda(warmup.start_vector(sb.n, seed=0)))
    assert info["converged"] == 1 and abs(info["energy"] - g["energy"]) <= E_TOL, (info, g["energy"])
    x = x.cpu().numpy()
    assert np.linalg.norm(ol11r.project_blocks(sb, x) - info["energy"] * x) <= 1.5e-10
