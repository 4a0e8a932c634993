"""The allocation-free overlap entry point (dmrg_gemv_trans_noalloc) against the allocating
one (dmrg_gemv_trans), through the C ABI; and repeated solves on one plan, which reuse the
workspace their plan keeps (dmrg_plan_trim releases it).

Some callers cannot let the library allocate device memory (their allocator owns all of
it, or cudaMalloc's synchronisation is not acceptable in their loop); for them the library
keeps the cross-block partial sums in a fixed scratch array.  This file is collected last
so that a failure here leaves every other test already run.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_1309_5571_gb300 import capi  # noqa: E402


def _call(fn, V, k, w):
    s = torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
    st = fn(V.data_ptr(), V.shape[1], w.numel(), k, w.data_ptr(), s.data_ptr(),
            torch.cuda.current_stream().cuda_stream)
    assert st == 0, capi.load().dmrg_last_error()
    torch.cuda.synchronize()
    return s.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice():
    lib = capi.load()
    rng = np.random.default_rng(11)
    for n, k in ((100003, 24), (4099, 7)):       # two calls in a row, different shapes
        ldv = n + 3
        V = torch.from_numpy(rng.standard_normal((k, ldv))).cuda()
        w = torch.from_numpy(rng.standard_normal(n)).cuda()
        ref = _call(lib.dmrg_gemv_trans, V, k, w)
        got = _call(lib.dmrg_gemv_trans_noalloc, V, k, w)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * n)
        exact = V.cpu().numpy()[:, :n] @ w.cpu().numpy()
        np.testing.assert_allclose(got, exact, rtol=1e-12, atol=1e-12 * n)


def test_noalloc_rejects_more_columns_than_its_scratch_holds():
    lib = capi.load()
    V = torch.zeros((25, 8), dtype=torch.float64, device="cuda")
    w = torch.zeros(8, dtype=torch.float64, device="cuda")
    s = torch.zeros(25, dtype=torch.float64, device="cuda")
    st = lib.dmrg_gemv_trans_noalloc(V.data_ptr(), 8, 8, 25, w.data_ptr(), s.data_ptr(), None)
    assert st == 1
    assert b"outside [1, 24]" in lib.dmrg_last_error()


@pytest.mark.parametrize("n,k", [(0, 1), (1, 24), (300, 5), (1, 1)])
def test_noalloc_edge_shapes_match_numpy(n, k):
    # empty input (s = 0), one row, and fewer rows than the grid has threads (most blocks
    # write zero partial sums), against NumPy and against the allocating entry point
    lib = capi.load()
    rng = np.random.default_rng(100 + n + k)
    ldv = max(n, 1) + 5
    Vh = rng.standard_normal((k, ldv))
    wh = rng.standard_normal(max(n, 1))[:n]
    V = torch.from_numpy(Vh).cuda()
    w = torch.from_numpy(np.ascontiguousarray(wh)).cuda() if n else torch.zeros(1, dtype=torch.float64, device="cuda")
    s = torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.dmrg_gemv_trans_noalloc(V.data_ptr(), ldv, n, k, w.data_ptr(), s.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.dmrg_last_error()
    torch.cuda.synchronize()
    got = s.cpu().numpy()
    exact = Vh[:, :n] @ wh
    np.testing.assert_allclose(got, exact, rtol=1e-12, atol=1e-12 * max(n, 1))
    if n:
        np.testing.assert_allclose(got, _call(lib.dmrg_gemv_trans, V, k, w[:n]), rtol=1e-12,
                                   atol=1e-12 * n)


def test_noalloc_allocates_no_device_memory():
    # the call's contract: no device allocation.  After a warm-up call (which loads the
    # kernel and looks up the scratch address), repeated calls leave the free device memory
    # exactly where it was; the output and inputs are allocated by the caller beforehand
    lib = capi.load()
    rng = np.random.default_rng(5)
    n, k = 200003, 17
    V = torch.from_numpy(rng.standard_normal((k, n))).cuda()
    w = torch.from_numpy(rng.standard_normal(n)).cuda()
    s = torch.empty(k, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.dmrg_gemv_trans_noalloc(V.data_ptr(), n, n, k, w.data_ptr(), s.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert lib.dmrg_gemv_trans_noalloc(V.data_ptr(), n, n, k, w.data_ptr(), s.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    np.testing.assert_allclose(s.cpu().numpy(), V.cpu().numpy() @ w.cpu().numpy(), rtol=1e-12,
                               atol=1e-12 * n)


@pytest.mark.parametrize("prec", ["fp64", "bf16x2"])
def test_repeated_solves_allocate_nothing(prec):
    from dmrg_inputs import warmup
    from paper_1309_5571_gb300 import Plan
    sb = warmup.warmup_superblock("heisenberg", 40, m=300)
    plan = Plan(sb, prec=prec)
    x0 = torch.from_numpy(warmup.start_vector(sb.n, seed=0)).cuda()
    x1, x2 = torch.empty_like(x0), torch.empty_like(x0)
    _, i1 = plan.solve(x0, x1)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    _, i2 = plan.solve(x0, x2)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free1
    # the same workspace and tile schedule: the same iterations, bit for bit
    assert torch.equal(x1, x2)
    assert (i1["iters"], i1["energy"]) == (i2["iters"], i2["energy"])
    # host-buffer solves keep their two device vectors as well
    xh0 = x0.cpu().numpy()
    plan.solve_host(xh0)
    torch.cuda.synchronize()
    free3 = torch.cuda.mem_get_info()[0]
    xh, _ = plan.solve_host(xh0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free3
    np.testing.assert_array_equal(xh, x1.cpu().numpy())
    plan.trim()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] > free3
    # and the plan still solves after the trim
    x3 = torch.empty_like(x0)
    _, i3 = plan.solve(x0, x3)
    assert torch.equal(x3, x1)
    plan.close()
