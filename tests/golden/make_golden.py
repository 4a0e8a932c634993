"""Writes tests/golden/energies.json: ground-state energies of the benchmark superblocks,
computed by the FP64 oracle alone.

For every case the seeded synthetic superblock is generated (dmrg_inputs), and its lowest
eigenvalue in the target sector is computed twice, by independent routes that share only
the projection of Eq. 11 (oracle.projection.project_blocks):

* the oracle's Davidson iteration (Algorithm 3 with the readings of the oracle: diagonal
  correction, CGS2, two-vector restart at 20 columns, ||r|| <= 1e-10), from start vector
  seed 0;
* ARPACK's implicitly restarted Lanczos (scipy.sparse.linalg.eigsh, smallest algebraic
  eigenvalue) on the same projection, from the same start vector.

The file records both and their difference; the GPU tests compare the CUDA library's
energies with the Davidson value.  Nothing here touches the CUDA library.

  python tests/golden/make_golden.py [case ...]     (default: every case; existing
                                                     entries of other cases are kept)
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
from scipy.sparse.linalg import LinearOperator, eigsh  # noqa: E402

from dmrg_inputs import warmup  # noqa: E402
from oracle import davidson as odav  # noqa: E402
from oracle import projection as oproj  # noqa: E402

OUT = os.path.join(HERE, "energies.json")

# name -> generator arguments (dmrg_inputs.warmup.warmup_superblock)
CASES = {
    "heis_L100_m256": dict(model="heisenberg", L=100, m=256),
    "heis_L100_m512": dict(model="heisenberg", L=100, m=512),
    "heis_L100_m1024": dict(model="heisenberg", L=100, m=1024),
    "heis_L100_m2048": dict(model="heisenberg", L=100, m=2048),
    "hub_L64_m2048": dict(model="hubbard", L=64, m=2048, U=4.0, t=1.0),
    "hub_L100_m4096_quarter": dict(model="hubbard", L=100, m=4096, U=8.0, t=1.0, filling=0.5),
}


def solve_case(name: str, args: dict) -> dict:
    t0 = time.time()
    sb = warmup.warmup_superblock(**args)
    t_gen = time.time() - t0
    x0 = warmup.start_vector(sb.n, seed=0)
    D = oproj.diagonal(sb)
    t0 = time.time()
    lam, x, info = odav.davidson(lambda v: oproj.project_blocks(sb, v), D, x0, tol=1e-10)
    t_dav = time.time() - t0
    count = [0]

    def mv(v):
        count[0] += 1
        return oproj.project_blocks(sb, np.ascontiguousarray(v).ravel())

    op = LinearOperator((sb.n, sb.n), matvec=mv, dtype=np.float64)
    t0 = time.time()
    w, v = eigsh(op, k=1, which="SA", v0=x0, tol=1e-14, ncv=40, maxiter=2000)
    t_arp = time.time() - t0
    e_arp = float(w[0])
    v = v[:, 0]
    r_arp = float(np.linalg.norm(mv(v) - e_arp * v))
    return {
        "generator": {"function": "dmrg_inputs.warmup.warmup_superblock", "args": args},
        "n": int(sb.n), "start_vector_seed": 0,
        "energy": float(lam),
        "davidson": {"resnorm": float(info["resnorm"]), "iters": int(info["iters"]),
                     "restarts": int(info["restarts"]), "converged": bool(info["converged"]),
                     "tol": 1e-10, "max_subspace": 20, "restart_keep": 2},
        "arpack_energy": e_arp, "arpack_resnorm": r_arp, "arpack_matvecs": count[0],
        "abs_diff_davidson_arpack": abs(float(lam) - e_arp),
        "eigvec_overlap": float(abs(x @ v) / (np.linalg.norm(x) * np.linalg.norm(v))),
        "seconds": {"generate": t_gen, "davidson": t_dav, "arpack": t_arp},
        "source": "oracle.davidson.davidson (Algorithm 3) and scipy eigsh over "
                  "oracle.projection.project_blocks (Eq. 11); written by tests/golden/make_golden.py",
    }


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names:
        print(f"{name} ...", flush=True)
        data[name] = solve_case(name, CASES[name])
        print(json.dumps({name: data[name]}, indent=1), flush=True)
        with open(OUT + ".tmp", "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
