"""Batched solves of independent, uneven superblocks (dmrg_davidson_solve_batched) on the
GPU: identical to solving them one by one, and equal to the FP64 oracle."""
import numpy as np
import pytest

from dmrg_inputs import warmup
from oracle import davidson as odav
from oracle import projection as oproj

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_1309_5571_gb300 import Plan, solve_batched  # noqa: E402

from test_gpu_parity import ragged_superblock  # noqa: E402


def _mixed_bag():
    sbs = [warmup.warmup_superblock("heisenberg", 20, m=32),
           warmup.warmup_superblock("heisenberg", 24, m=64),
           warmup.warmup_superblock("hubbard", 10, m=40, U=4.0),
           warmup.warmup_superblock("heisenberg", 6, m=1000),
           ragged_superblock(3)]
    return sbs


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_batched_equals_one_by_one(prec):
    sbs = _mixed_bag()
    plans = [Plan(sb, prec=prec) for sb in sbs]
    x0s = [torch.from_numpy(warmup.start_vector(sb.n, seed=i)).cuda() for i, sb in enumerate(sbs)]
    if prec == "bf16x3":
        # the grouped launch takes no K split; neither does this schedule (a split changes
        # the FP32 summation order; every unsplit schedule gives the same bits)
        for p in plans:
            p.set_tile_schedule(0, 0)
    xs, infos = solve_batched(plans, x0s)
    for p, x0, x, info in zip(plans, x0s, xs, infos):
        x1, info1 = p.solve(x0)
        assert info["converged"] == 1
        assert info["energy"] == info1["energy"]
        assert info["iters"] == info1["iters"]
        assert torch.equal(x, x1)


def test_batched_problems_sharing_a_plan_stay_ordered():
    # several problems on ONE plan (shared projection scratch) give the same results as
    # solving them one by one
    sb = warmup.warmup_superblock("heisenberg", 24, m=64)
    plan = Plan(sb, prec="bf16x3")
    x0s = [torch.from_numpy(warmup.start_vector(sb.n, seed=i)).cuda() for i in range(6)]
    plan.set_tile_schedule(0, 0)  # the same tile schedule in both runs
    xs, infos = solve_batched([plan] * 6, x0s)
    for x0, x, info in zip(x0s, xs, infos):
        x1, info1 = plan.solve(x0)
        assert info["energy"] == info1["energy"] and torch.equal(x, x1)


def test_batched_uneven_heisenberg_matches_oracle():
    # scaled-down uneven batch: 12 Heisenberg superblocks (L = 40), m drawn from
    # {32, 64, 128, 256} with a fixed seed
    sbs, ms, x0s = warmup.batched_workload(count=12, ms=(32, 64, 128, 256), L=40, seed=1234)
    plans = {}
    for sb, m in zip(sbs, ms):
        if m not in plans:
            plans[m] = Plan(sb, prec="bf16x3")
    plist = [plans[m] for m in ms]
    xs, infos = solve_batched(plist, [torch.from_numpy(x).cuda() for x in x0s])
    ref = {}
    for sb, m, x, x0, info in zip(sbs, ms, xs, x0s, infos):
        assert info["converged"] == 1
        if m not in ref:
            ref[m] = odav.davidson(lambda v: oproj.project_blocks(sb, v), oproj.diagonal(sb), x0)[0]
        assert abs(info["energy"] - ref[m]) <= 1e-10
        xh = x.cpu().numpy()
        assert np.linalg.norm(oproj.project_blocks(sb, xh) - info["energy"] * xh) <= 1.5e-10


def test_batched_reports_nonconvergence_per_problem():
    sbs = _mixed_bag()[:2]
    plans = [Plan(sbs[0], max_iter=3), Plan(sbs[1])]
    x0s = [torch.from_numpy(warmup.start_vector(sb.n, seed=0)).cuda() for sb in sbs]
    xs, infos = solve_batched(plans, x0s, raise_on_nonconvergence=False)
    assert infos[0]["converged"] == 0 and infos[0]["iters"] == 3
    assert infos[1]["converged"] == 1
