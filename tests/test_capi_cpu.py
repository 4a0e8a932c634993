"""The C ABI library loads, exports every declared symbol and validates its inputs on the
host (no GPU needed: no call here reaches a kernel or a device allocation)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import __graft_entry__
from paper_1309_5571_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return capi.load()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dmrg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dmrg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dmrg_project", "dmrg_davidson_step", "dmrg_davidson_solve",
                     "dmrg_plan_create", "dmrg_gemv_trans"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    # and the binding declares a signature for each of them
    assert set(declared_functions()) <= set(capi.SIGNATURES)


def test_status_strings_and_defaults(lib):
    assert lib.dmrg_status_string(0) == b"ok"
    assert lib.dmrg_status_string(5) == b"not converged"
    assert b"sm_103a" in lib.dmrg_version()
    o = capi.Options()
    lib.dmrg_options_default(C.byref(o))
    assert (o.prec, o.tol, o.max_iter, o.max_subspace, o.fp64_refine) == (0, 1e-10, 1000, 20, 1)
    assert o.refine_ratio == 0.0
    assert o.anchor_prec == 0 and o.vector_arith == 2  # DMRG_VEC_SPLIT
    assert o.autotune == 1 and o.restart_keep == 2 and o.graphs == 1 and o.anchor_update == 1


def _desc_from(sb):
    return capi.marshal(sb)


def _tiny():
    from dmrg_inputs import warmup
    return warmup.warmup_superblock("heisenberg", 6, m=100)


def _create(lib, m, opt=None):
    h = C.c_void_p()
    st = lib.dmrg_plan_create(C.byref(m.desc), C.byref(opt) if opt else None, None, C.byref(h))
    return st, h


def test_null_desc_rejected(lib):
    h = C.c_void_p()
    assert lib.dmrg_plan_create(None, None, None, C.byref(h)) == 1
    assert b"NULL" in lib.dmrg_last_error()


def test_bad_pair_rejected(lib):
    m = _desc_from(_tiny())
    m.desc.pair_i[0] = 99
    st, _ = _create(lib, m)
    assert st == 1 and b"out of range" in lib.dmrg_last_error()


def test_repeated_pair_rejected(lib):
    sb = _tiny()
    sb.pairs = sb.pairs + [sb.pairs[0]]
    st, _ = _create(lib, _desc_from(sb))
    assert st == 2 and b"twice" in lib.dmrg_last_error()


def test_block_shape_mismatch_rejected(lib):
    sb = _tiny()
    op = sb.opsL[0]
    key = next(iter(op.blocks))
    op.blocks[key] = np.zeros((op.blocks[key].shape[0] + 1, op.blocks[key].shape[1]))
    st, _ = _create(lib, _desc_from(sb))
    assert st == 2 and b"does not match" in lib.dmrg_last_error()


def test_bad_term_rejected(lib):
    sb = _tiny()
    sb.terms = sb.terms + [(1.0, 57, -1)]
    st, _ = _create(lib, _desc_from(sb))
    assert st == 1 and b"missing operator" in lib.dmrg_last_error()


def test_bad_options_rejected(lib):
    m = _desc_from(_tiny())
    opt = capi.options(max_subspace=30)
    st, _ = _create(lib, m, opt)
    assert st == 1 and b"max_subspace" in lib.dmrg_last_error()


def test_gemv_trans_argument_checks(lib):
    assert lib.dmrg_gemv_trans(None, 10, 10, 3, None, None, None) == 1
    buf = (C.c_double * 4)()
    assert lib.dmrg_gemv_trans(buf, 1, 4, 1, buf, buf, None) == 1     # ldv < n
    assert lib.dmrg_gemv_trans(buf, 4, 4, 25, buf, buf, None) == 1    # k > 24


def test_trim_rejects_a_null_plan(lib):
    assert lib.dmrg_plan_trim(None) == 1


def test_schedule_calls_check_arguments(lib):
    # NULL plan and precisions without tile schedules are rejected on the host
    assert lib.dmrg_plan_set_tile_schedule(None, 2, 0, 0, None) == 1
    assert lib.dmrg_plan_autotune(None, 2, None) == 1


def test_binding_structs_match_the_header(tmp_path):
    # the ctypes mirrors have the size and field offsets that a C compiler gives the
    # header's structs (compiled with the host C compiler, no GPU)
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    pairs = [(capi.Block, "dmrg_block"), (capi.Operator, "dmrg_operator"),
             (capi.Term, "dmrg_term"), (capi.SuperblockDesc, "dmrg_superblock_desc"),
             (capi.Options, "dmrg_options"), (capi.SolveInfo, "dmrg_solve_info"),
             (capi.PlanStats, "dmrg_plan_stats"), (capi.Term4, "dmrg_term4"),
             (capi.L11rDesc, "dmrg_l11r_desc")]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dmrg.h"', "int main(void) {",
             '  printf("%d\\n", (int)DMRG_TILE_SCHEDULES);']
    expect = [str(capi.TILE_SCHEDULES)]
    for cls, cname in pairs:
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        expect.append(str(C.sizeof(cls)))
        for f, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {f}));')
            expect.append(str(getattr(cls, f).offset))
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert got == expect
