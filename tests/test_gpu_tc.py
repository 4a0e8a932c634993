"""Tensor-core (tcgen05) projections and the mixed-precision Davidson against the FP64
oracle, on the GPU.

Tolerances, derived from the arithmetic (all relative to max|y|):

* BF16x3 keeps 24 significant bits per operand (dropped products are below 2^-24
  relative) and accumulates in FP32, whose rounding grows with the accumulation length;
  two chained stages with K up to ~900 give a bound of a few hundred units of
  u = 2^-24: 2e-5.
* BF16x2 represents each operand as x0 + x1 to 2^-18 relative (x0 = rn(x) to 2^-9, x1 =
  rn(x - x0) to 2^-9 of the remainder) and drops x1 y1 (below 2^-18 |x y|): at most
  3 * 2^-18 = 1.1e-5 per product and per stage, twice (the stage-1 result is split
  again), times the cancellation of the sums (sum |terms| / max|y|, a few on these
  operators), plus the FP32 accumulation of BF16x3: 2e-4.
* TF32 rounds each operand to 11 significant bits (2^-11 = 4.9e-4 relative): two
  operands and the rounded intermediate, times the same cancellation: 5e-3.

The mixed Davidson ends only on an FP64 residual, so its energy meets |dE| <= 1e-10.
"""
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
from paper_1309_5571_gb300 import Plan, capi  # noqa: E402

from test_gpu_parity import PROBLEMS, problem, rel_err, cuda  # noqa: E402

TOL = {"bf16x3": 2e-5, "bf16x2": 2e-4, "tf32": 5e-3}
LOWPREC = ["bf16x3", "bf16x2", "tf32"]
E_TOL = 1e-10


@pytest.mark.parametrize("prec", LOWPREC)
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_projection_tensor_core_matches_oracle(name, prec):
    sb = problem(name)
    plan = Plan(sb, prec=prec)
    for seed in (0, 1):
        x = np.random.default_rng(seed).standard_normal(sb.n)
        y = plan.project(cuda(x)).cpu().numpy()
        y_ref = oproj.project_blocks(sb, x)
        assert rel_err(y, y_ref) <= TOL[prec], (name, prec, rel_err(y, y_ref))


def test_projection_tensor_core_repeatable():
    sb = problem("hub_L8_m40")
    plan = Plan(sb, prec="bf16x3")
    x = cuda(np.random.default_rng(3).standard_normal(sb.n))
    y1 = plan.project(x).cpu().numpy()
    y2 = plan.project(x).cpu().numpy()
    np.testing.assert_array_equal(y1, y2)


@pytest.mark.parametrize("name", ["heis_L16_m64", "hub_L8_m40", "hub_quarter_L12_m48", "ragged"])
@pytest.mark.parametrize("prec", LOWPREC)
def test_mixed_davidson_matches_oracle(name, prec):
    sb = problem(name)
    x0 = warmup.start_vector(sb.n, seed=0)
    plan = Plan(sb, prec=prec)
    x, info = plan.solve(cuda(x0))
    x = x.cpu().numpy()
    lam, xo, oinfo = odav.davidson(lambda v: oproj.project_blocks(sb, v), oproj.diagonal(sb), x0)
    assert info["converged"]
    assert abs(info["energy"] - lam) <= E_TOL, (info, lam)
    assert abs(x @ xo) / (np.linalg.norm(x) * np.linalg.norm(xo)) >= 1 - 1e-8
    r = oproj.project_blocks(sb, x) - info["energy"] * x
    assert np.linalg.norm(r) <= 1.5e-10
    assert info["fp64_projections"] >= 1 and info["projections"] >= 1


NSCHED = capi.TILE_SCHEDULES  # (3 s + w) 3 + o: K split s, tile width w, order o


def candidates(prec, stage):
    """Tile schedules of a GEMM stage: stage 1 takes no K split, TF32 only 128-column tiles."""
    return [c for c in range(NSCHED)
            if (stage == 2 or c // 9 == 0) and (prec != "tf32" or (c // 3) % 3 == 0)]


@pytest.mark.parametrize("prec", LOWPREC)
def test_autotuned_schedule(prec):
    # the tuner times exactly the candidates of each stage and keeps one of them; schedules
    # without a K split compute every output element in the same CTA arithmetic, so the
    # tuned plan agrees with the untuned one bit for bit unless stage 2 took a split
    sb = problem("ragged")
    xh = np.random.default_rng(11).standard_normal(sb.n)
    x = cuda(xh)
    fixed = Plan(sb, prec=prec, autotune=False)
    y0 = fixed.project(x).cpu().numpy()
    assert fixed.get_stats()["tc_schedule"] == [0, 0]
    tuned = Plan(sb, prec=prec)
    st = tuned.autotune(prec)
    for g in (0, 1):
        cand = candidates(prec, g + 1)
        assert st["tc_schedule"][g] in cand
        assert all((t > 0) == (c in cand) for c, t in enumerate(st["tc_tune_us"][g]))
    y1 = tuned.project(x).cpu().numpy()
    assert rel_err(y1, oproj.project_blocks(sb, xh)) <= TOL[prec]
    if st["tc_schedule"][1] < 9:
        np.testing.assert_array_equal(y0, y1)
    # tuning on first use, inside the projection call, picks a candidate too
    p2 = Plan(sb, prec=prec)
    assert rel_err(p2.project(x).cpu().numpy(), oproj.project_blocks(sb, xh)) <= TOL[prec]
    assert all(c in candidates(prec, g + 1) for g, c in enumerate(p2.get_stats()["tc_schedule"]))


@pytest.mark.parametrize("prec", LOWPREC)
@pytest.mark.parametrize("name", ["hub_L8_m40", "ragged", "heis_L16_m64"])
def test_every_tile_schedule_matches_oracle(name, prec):
    # each candidate schedule of each stage (the other stage on schedule 0) against the
    # oracle; every schedule is repeatable bit for bit, and the unsplit ones agree with
    # schedule (0, 0) bit for bit (small problems: the K split cuts most stage-2 tiles)
    sb = problem(name)
    xh = np.random.default_rng(7).standard_normal(sb.n)
    y_ref = oproj.project_blocks(sb, xh)
    x = cuda(xh)
    plan = Plan(sb, prec=prec, autotune=False)
    base = plan.project(x).cpu().numpy()
    pairs = [(c, 0) for c in candidates(prec, 1)] + [(0, c) for c in candidates(prec, 2)]
    for s1, s2 in pairs:
        assert plan.set_tile_schedule(s1, s2, prec=prec)["tc_schedule"] == [s1, s2]
        y = plan.project(x).cpu().numpy()
        assert rel_err(y, y_ref) <= TOL[prec], (s1, s2, rel_err(y, y_ref))
        np.testing.assert_array_equal(y, plan.project(x).cpu().numpy())
        if s2 < 9:
            np.testing.assert_array_equal(y, base)


def test_tile_schedule_rejects_non_candidates():
    sb = problem("ragged")
    plan = Plan(sb, prec="bf16x3", autotune=False)
    for bad in ((9, 0), (-1, 0), (0, NSCHED)):
        with pytest.raises(capi.DmrgError):
            plan.set_tile_schedule(*bad)
    tf = Plan(sb, prec="tf32", autotune=False)
    with pytest.raises(capi.DmrgError):
        tf.set_tile_schedule(0, 3, prec="tf32")   # 256-column tiles: BF16 splits only


@pytest.mark.parametrize("name", ["heis_L16_m64", "hub_quarter_L12_m48", "ragged"])
def test_mixed_davidson_vector_arithmetic(name):
    # split arithmetic (FP64 anchor column, FP32 low-precision columns) reaches the same
    # FP64 answer as FP64 vector passes, in about the same number of iterations
    sb = problem(name)
    x0 = warmup.start_vector(sb.n, seed=0)
    lam = odav.davidson(lambda v: oproj.project_blocks(sb, v), oproj.diagonal(sb), x0)[0]
    iters = {}
    for arith in ("fp64", "split", "df"):
        x, info = Plan(sb, prec="bf16x3", vector_arith=arith).solve(cuda(x0))
        assert info["converged"] and abs(info["energy"] - lam) <= E_TOL, (arith, info, lam)
        x = x.cpu().numpy()
        assert np.linalg.norm(oproj.project_blocks(sb, x) - info["energy"] * x) <= 1.5e-10
        iters[arith] = info["iters"]
    assert iters["split"] <= 1.25 * iters["fp64"] + 3, iters


@pytest.fixture(scope="module")
def hub_L64_m2048():
    from _workloads import workload
    return workload("hub_L64_m2048")


def test_full_size_projection_hubbard_m2048_bf16x3(hub_L64_m2048):
    sb = hub_L64_m2048
    plan = Plan(sb, prec="bf16x3")
    x = warmup.start_vector(sb.n, seed=5)
    y = plan.project(cuda(x)).cpu().numpy()
    y_ref = oproj.project_blocks(sb, x)
    assert rel_err(y, y_ref) <= TOL["bf16x3"]
    y64 = plan.project(cuda(x), prec="fp64").cpu().numpy()
    assert rel_err(y64, y_ref) <= 1e-12
    # the K-split schedules of stage 2 (both split bounds, LPT order, narrow and wide tiles)
    for s2 in (9, 18, 24, 25):
        plan.set_tile_schedule(4, s2)
        ys = plan.project(cuda(x)).cpu().numpy()
        assert rel_err(ys, y_ref) <= TOL["bf16x3"], (s2, rel_err(ys, y_ref))


@pytest.mark.parametrize("prec", ["bf16x2", "tf32"])
def test_full_size_projection_hubbard_m2048_lowprec(hub_L64_m2048, prec):
    # the other low-precision arithmetics at full size, on every schedule family the
    # autotuner may pick for stage 2 (LPT order, K split), against the oracle
    sb = hub_L64_m2048
    plan = Plan(sb, prec=prec)
    x = warmup.start_vector(sb.n, seed=5)
    y_ref = oproj.project_blocks(sb, x)
    y = plan.project(cuda(x)).cpu().numpy()
    assert rel_err(y, y_ref) <= TOL[prec], (prec, rel_err(y, y_ref))
    for s2 in (9, 18):
        plan.set_tile_schedule(0, s2, prec=prec)
        ys = plan.project(cuda(x)).cpu().numpy()
        assert rel_err(ys, y_ref) <= TOL[prec], (prec, s2, rel_err(ys, y_ref))


def test_full_size_mixed_solve_hubbard_m2048_properties(hub_L64_m2048):
    sb = hub_L64_m2048
    plan = Plan(sb, prec="bf16x3")
    x, info = plan.solve(cuda(warmup.start_vector(sb.n, seed=0)))
    x = x.cpu().numpy()
    Hx = oproj.project_blocks(sb, x)
    rq = float(x @ Hx) / float(x @ x)
    assert abs(rq - info["energy"]) <= E_TOL
    assert np.linalg.norm(Hx - info["energy"] * x) <= 1.5e-10


# ---------------------------------------------------------------- FP64-accurate tensor cores
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_projection_fp64tc_matches_oracle(name):
    # exact digit products: the FP64 bar of 1e-12 (relative to max|y|) applies
    sb = problem(name)
    plan = Plan(sb, prec="fp64tc")
    for seed in (0, 1):
        x = np.random.default_rng(seed).standard_normal(sb.n)
        y = plan.project(cuda(x)).cpu().numpy()
        assert rel_err(y, oproj.project_blocks(sb, x)) <= 1e-12


def test_projection_fp64tc_scaled_inputs():
    # rows whose magnitudes differ by many orders: per-row, per-chunk scales
    sb = problem("hub_L8_m40")
    plan = Plan(sb, prec="fp64tc")
    x = np.random.default_rng(9).standard_normal(sb.n) * np.exp(np.random.default_rng(8).uniform(-20, 20, sb.n))
    y = plan.project(cuda(x)).cpu().numpy()
    y_ref = oproj.project_blocks(sb, x)
    assert rel_err(y, y_ref) <= 1e-12


@pytest.mark.parametrize("name", ["heis_L16_m64", "hub_quarter_L12_m48", "ragged"])
def test_davidson_fp64tc_matches_oracle(name):
    sb = problem(name)
    x0 = warmup.start_vector(sb.n, seed=0)
    x, info = Plan(sb, prec="fp64tc").solve(cuda(x0))
    lam, xo, _ = odav.davidson(lambda v: oproj.project_blocks(sb, v), oproj.diagonal(sb), x0)
    assert abs(info["energy"] - lam) <= E_TOL
    x = x.cpu().numpy()
    assert np.linalg.norm(oproj.project_blocks(sb, x) - info["energy"] * x) <= 1.5e-10


@pytest.mark.parametrize("name", ["heis_L16_m64", "hub_L8_m40"])
def test_mixed_davidson_with_fp64tc_anchors(name):
    sb = problem(name)
    x0 = warmup.start_vector(sb.n, seed=0)
    x, info = Plan(sb, prec="bf16x3", anchor_prec="fp64tc").solve(cuda(x0))
    lam = odav.davidson(lambda v: oproj.project_blocks(sb, v), oproj.diagonal(sb), x0)[0]
    assert abs(info["energy"] - lam) <= E_TOL and info["fp64_projections"] >= 1


def test_full_size_projection_hubbard_m2048_fp64tc(hub_L64_m2048):
    sb = hub_L64_m2048
    plan = Plan(sb, prec="fp64tc")
    x = warmup.start_vector(sb.n, seed=5)
    y = plan.project(cuda(x)).cpu().numpy()
    assert rel_err(y, oproj.project_blocks(sb, x)) <= 1e-12


# ---------------------------------------------------------------- CUDA-graph replay
@pytest.mark.parametrize("prec", LOWPREC)
def test_graph_replay_is_bit_identical(prec):
    # a projection replayed from its captured graph equals the direct launches bit for bit,
    # for several vector pairs (one graph each) and after a schedule change (graphs dropped)
    sb = problem("hub_L8_m40")
    direct = Plan(sb, prec=prec, graphs=False)
    graphed = Plan(sb, prec=prec, graphs=True)
    for pl in (direct, graphed):
        pl.set_tile_schedule(3, 12, prec=prec) if prec != "tf32" else pl.set_tile_schedule(1, 10, prec=prec)
    xs = [cuda(np.random.default_rng(s).standard_normal(sb.n)) for s in range(3)]
    ys = [torch.empty_like(x) for x in xs]
    for rep in range(2):
        for x, y in zip(xs, ys):
            ref = direct.project(x, prec=prec).cpu().numpy()
            out = graphed.project(x, y, prec=prec).cpu().numpy()
            np.testing.assert_array_equal(out, ref)
    for pl in (direct, graphed):
        pl.set_tile_schedule(0, 9, prec=prec)
    np.testing.assert_array_equal(graphed.project(xs[0], ys[0], prec=prec).cpu().numpy(),
                                  direct.project(xs[0], prec=prec).cpu().numpy())


def test_graph_projection_inside_a_caller_capture():
    # while the caller's stream is being captured the projection launches its kernels into
    # that capture (no nested capture); replaying the caller's graph gives the same bits
    sb = problem("ragged")
    plan = Plan(sb, prec="bf16x2")
    x = cuda(np.random.default_rng(4).standard_normal(sb.n))
    ref = plan.project(x).cpu().numpy()      # builds and tunes the plan outside the capture
    y = torch.zeros_like(x)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.project(x, y, stream=s)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(y.cpu().numpy(), ref)


def test_graph_solve_equals_direct_solve():
    sb = problem("heis_L16_m64")
    x0 = cuda(warmup.start_vector(sb.n, seed=0))
    res = {}
    for gflag in (False, True):
        plan = Plan(sb, prec="bf16x2", anchor_prec="fp64tc", graphs=gflag)
        plan.set_tile_schedule(0, 0, prec="bf16x2")
        x, info = plan.solve(x0)
        res[gflag] = (x.cpu().numpy(), info)
    np.testing.assert_array_equal(res[False][0], res[True][0])
    assert res[False][1]["energy"] == res[True][1]["energy"]
    assert res[False][1]["iters"] == res[True][1]["iters"]
