"""Per-process cache of the full-size benchmark superblocks and the oracle-written golden
energies (tests/golden/energies.json), shared by the GPU test modules so that each
workload is generated once per pytest session."""
import functools
import json
import os

from dmrg_inputs import warmup

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "energies.json")


@functools.lru_cache(maxsize=None)
def workload(name):
    return warmup.workload(name)


@functools.lru_cache(maxsize=None)
def workload_l11r(name):
    return warmup.workload_l11r(name)


@functools.lru_cache(maxsize=None)
def superblock(model, L, m, **kw):
    return warmup.warmup_superblock(model, L, m, **kw)


def golden():
    with open(GOLDEN) as f:
        return json.load(f)
