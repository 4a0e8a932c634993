"""Full-size solves of the benchmark superblocks on the GPU against the golden energies
that the FP64 oracle wrote (tests/golden/energies.json: the oracle's Davidson iteration,
cross-checked by ARPACK on the oracle's projection).

Every arithmetic of the library must reach the oracle's ground-state energy to
|dE| <= 1e-10 from the same start vector (seed 0), and the returned vector must be an
eigenvector of the oracle's projection to ||H x - E x|| <= 1.5e-10: the mixed modes end
only on an FP64-accurate residual, so low-precision projections never decide the answer.
"""
import numpy as np
import pytest

from dmrg_inputs import warmup
from oracle import projection as oproj

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_1309_5571_gb300 import Plan, solve_batched  # noqa: E402

from _workloads import golden, superblock, workload  # noqa: E402

E_TOL = 1e-10
R_TOL = 1.5e-10

# (projection arithmetic, FP64-accurate anchor arithmetic of the mixed modes)
VARIANTS = {
    "fp64": dict(prec="fp64"),
    "fp64tc": dict(prec="fp64tc"),
    "bf16x3+fp64tc": dict(prec="bf16x3", anchor_prec="fp64tc"),
    "bf16x3+fp64": dict(prec="bf16x3", anchor_prec="fp64"),
    "bf16x2+fp64tc": dict(prec="bf16x2", anchor_prec="fp64tc"),
    "tf32+fp64tc": dict(prec="tf32", anchor_prec="fp64tc"),
    # every anchor a full FP64_TC projection (no anchor update)
    "bf16x2+fp64tc/full-anchors": dict(prec="bf16x2", anchor_prec="fp64tc", anchor_update=False),
}


def _check_solve(sb, E_gold, opts):
    x0 = warmup.start_vector(sb.n, seed=0)
    plan = Plan(sb, **opts)
    x, info = plan.solve(torch.from_numpy(x0).cuda())
    plan.close()
    x = x.cpu().numpy()
    assert info["converged"] == 1
    assert abs(info["energy"] - E_gold) <= E_TOL, (opts, info["energy"], E_gold)
    r = oproj.project_blocks(sb, x) - info["energy"] * x
    assert np.linalg.norm(r) <= R_TOL * np.linalg.norm(x), (opts, np.linalg.norm(r))
    return info


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("name", ["hub_L64_m2048", "heis_L100_m1024"])
def test_full_size_solve_matches_golden_energy(name, variant):
    g = golden()[name]
    sb = workload(name)
    assert sb.n == g["n"]
    opts = VARIANTS[variant]
    info = _check_solve(sb, g["energy"], opts)
    if variant not in ("fp64", "fp64tc"):
        assert info["fp64_projections"] >= 1 and info["projections"] >= 1
    if opts.get("anchor_prec") != "fp64tc" or opts.get("anchor_update") is False:
        assert info["anchor_updates"] == 0
    elif name == "hub_L64_m2048":
        # later anchors of this solve are formed from the previous one (a few digits suffice)
        assert 1 <= info["anchor_updates"] <= info["fp64_projections"]


def test_golden_file_is_the_oracles():
    # the stored energies are the oracle Davidson's, and ARPACK on the oracle's projection
    # agrees with each of them
    for name, g in golden().items():
        assert g["davidson"]["converged"] and g["davidson"]["resnorm"] <= 1e-10, name
        assert abs(g["energy"] - g["arpack_energy"]) <= 1e-9, name


# ---------------------------------------------------------------- uneven batch, full size
def test_full_size_uneven_batch_matches_golden_energies():
    # 64 Heisenberg superblocks (L = 100), m drawn from {256, 512, 1024, 2048} (seed 1234),
    # one plan per problem, BF16x3 projections grouped into shared launches with FP64_TC
    # anchors; every problem reaches the oracle's energy for its m
    sbs, ms, x0s = warmup.batched_workload(count=64)
    g = golden()
    plans = [Plan(sb, prec="bf16x3", anchor_prec="fp64tc") for sb in sbs]
    xs = [torch.from_numpy(x).cuda() for x in x0s]
    outs, infos = solve_batched(plans, xs)
    checked = set()
    for sb, m, x, info in zip(sbs, ms, outs, infos):
        assert info["converged"] == 1
        assert abs(info["energy"] - g[f"heis_L100_m{m}"]["energy"]) <= E_TOL, (m, info)
        if m not in checked:  # one residual check per operator set
            checked.add(m)
            xh = x.cpu().numpy()
            r = oproj.project_blocks(sb, xh) - info["energy"] * xh
            assert np.linalg.norm(r) <= R_TOL
    assert checked == {256, 512, 1024, 2048}
    for p in plans:
        p.close()


def test_full_size_uneven_batch_equals_one_by_one():
    # one problem per m, batched and then alone on the same plans: bit for bit, with an
    # unsplit tile schedule (the grouped launch takes no K split)
    sbs, ms, x0s = warmup.batched_workload(count=64)
    first = {}
    for i, m in enumerate(ms):
        first.setdefault(m, i)
    idx = sorted(first.values())
    plans = [Plan(sbs[i], prec="bf16x3", anchor_prec="fp64tc") for i in idx]
    for p in plans:
        p.set_tile_schedule(0, 0)
    xs = [torch.from_numpy(x0s[i]).cuda() for i in idx]
    outs, infos = solve_batched(plans, xs)
    for p, x0, x, info in zip(plans, xs, outs, infos):
        x1, info1 = p.solve(x0)
        assert info["energy"] == info1["energy"] and info["iters"] == info1["iters"]
        assert torch.equal(x, x1)
    for p in plans:
        p.close()


# ---------------------------------------------------------------- large quarter-filled Hubbard
@pytest.fixture(scope="module")
def quarter():
    return workload("hub_L100_m4096_quarter")


def test_large_quarter_filling_projection_fp64tc(quarter):
    # FP64-accurate tensor-core projection at n = 1.2e7 against the oracle: the FP64 bar
    sb = quarter
    plan = Plan(sb, prec="fp64tc")
    x = warmup.start_vector(sb.n, seed=5)
    y = plan.project(torch.from_numpy(x).cuda()).cpu().numpy()
    plan.close()
    y_ref = oproj.project_blocks(sb, x)
    assert np.max(np.abs(y - y_ref)) <= 1e-12 * np.max(np.abs(y_ref))


def test_large_quarter_filling_solve_matches_golden_energy(quarter):
    g = golden()
    assert quarter.n == g["hub_L100_m4096_quarter"]["n"]
    _check_solve(quarter, g["hub_L100_m4096_quarter"]["energy"],
                 dict(prec="bf16x3", anchor_prec="fp64tc"))
