"""The allocation-free overlap entry point (dmrg_gemv_trans_noalloc) against the allocating
one (dmrg_gemv_trans), through the C ABI.

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
