"""Stored analyses of fixed synthetic patterns (integer structure only).

The Erdos-Renyi workload (n = 5000, p = 0.001, seed 1) is ordered by the
library's minimum-degree ordering and partitioned into relaxed supernodes
(at most 16 explicit zeros per merge).  Programs that must not load the
library -- the CPU oracle's timing arm of the benchmark -- rebuild the
analysed pattern from two stored integer arrays: the permutation
(perm[new] = old) and the first column of every relaxed supernode (before
any splitting of wide supernodes, which leaves the pattern unchanged).  The
oracle's own fill and supernodal pattern of that partition give the same
pattern as the library (checked on the host by
``tests/test_symbolic_host.py::test_stored_er5000_analysis``).

Regenerate the file with ``python -m workloads.analysed`` (needs the built
library).
"""
from __future__ import annotations

import os

import numpy as np

from .patterns import erdos_renyi, pattern_hash

ER5000_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "er5000_mindeg_relax16.npz")


def er5000_pattern():
    """The input pattern of the Erdos-Renyi workload (lower CSC)."""
    return erdos_renyi(5000, 0.001, np.random.default_rng(1))


def load_er5000():
    """(pattern, perm, snode_ptr) of the stored analysis; the pattern's hash
    must match the one recorded with it."""
    pattern = er5000_pattern()
    with np.load(ER5000_FILE) as z:
        perm = np.asarray(z["perm"], dtype=np.int64)
        snode_ptr = np.asarray(z["snode_ptr"], dtype=np.int64)
        h = str(z["pattern_hash"])
    if h != pattern_hash(pattern):
        raise ValueError("stored analysis belongs to another pattern")
    return pattern, perm, snode_ptr


def write_er5000():
    from paper_1203_2742_gb300 import build
    build.build()
    from paper_1203_2742_gb300 import binding as B
    pattern = er5000_pattern()
    sym = B.Symbolic(*pattern, ordering="mindeg", relax=16, split_cols=-1)
    sp = np.asarray(sym.supernodes()[0], dtype=np.int32)
    np.savez_compressed(ER5000_FILE, perm=np.asarray(sym.perm, dtype=np.int32), snode_ptr=sp,
                        pattern_hash=np.asarray(pattern_hash(pattern)))


if __name__ == "__main__":
    write_er5000()
