"""The FP64_TC projection with fewer digits (dmrg_project_digits) and the Davidson anchor
update that uses it, on the GPU against the FP64 oracle.

With its leading d base-128 digits, every operand of the digit-product projection is
truncated to about 7 d bits of its row-chunk scale, so the error relative to max|y| falls
by about 2^-7 per digit until d = 7 reaches the FP64 level.  A mixed solve whose anchors are
formed as H x = y_0 W(:,0) + H d (the correction d projected with the digits its norm needs)
must end at the same energy and FP64-accurate residual as one that projects every anchor in
full.
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
from paper_1309_5571_gb300 import Plan  # noqa: E402

from _workloads import superblock  # noqa: E402


@pytest.mark.parametrize("model,L,m", [("hubbard", 16, 160), ("heisenberg", 40, 300)])
def test_project_digits_accuracy(model, L, m):
    sb = superblock(model, L, m)
    x = warmup.start_vector(sb.n, seed=3)
    y_ref = oproj.project_blocks(sb, x)
    scale = np.max(np.abs(y_ref))
    plan = Plan(sb, prec="fp64tc")
    xt = torch.from_numpy(x).cuda()
    errs = {}
    for d in range(2, 8):
        y = plan.project_digits(xt, d).cpu().numpy()
        errs[d] = float(np.max(np.abs(y - y_ref)) / scale)
        # about 2^(1 - 7 d) relative to the row-chunk scales, with room for the sums
        assert errs[d] <= 2.0 ** (8 - 7 * d), (d, errs)
    for d in range(2, 6):
        assert errs[d + 1] < errs[d] / 16, errs
    assert errs[7] <= 1e-12
    # seven digits are the FP64_TC projection itself, bit for bit
    y7 = plan.project_digits(xt, 7)
    assert torch.equal(y7, plan.project(xt, prec="fp64tc"))
    plan.close()


def test_project_digits_rejects_bad_counts():
    sb = superblock("heisenberg", 16, 64)
    plan = Plan(sb, prec="fp64tc")
    xt = torch.from_numpy(warmup.start_vector(sb.n, seed=0)).cuda()
    for d in (1, 8):
        with pytest.raises(Exception):
            plan.project_digits(xt, d)
    plan.close()


@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3"])
def test_anchor_update_matches_full_anchors(prec):
    sb = superblock("hubbard", 24, 400)
    x0 = warmup.start_vector(sb.n, seed=0)
    lam, _, _ = odav.davidson(lambda v: oproj.project_blocks(sb, v), oproj.diagonal(sb), x0)
    out = {}
    for upd in (True, False):
        plan = Plan(sb, prec=prec, anchor_prec="fp64tc", anchor_update=upd)
        x, info = plan.solve(torch.from_numpy(x0).cuda())
        plan.close()
        x = x.cpu().numpy()
        assert info["converged"] == 1
        r = oproj.project_blocks(sb, x) - info["energy"] * x
        assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(x), (upd, np.linalg.norm(r))
        assert abs(info["energy"] - lam) <= 1e-10, (upd, info["energy"], lam)
        out[upd] = info
    assert out[False]["anchor_updates"] == 0
    assert out[True]["anchor_updates"] <= out[True]["fp64_projections"]
