"""Shared helpers for the library tests (no barrier arithmetic here)."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    """Names of the functions declared in include/*.h."""
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(chd_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def lib():
    from paper_1203_2742_gb300 import build
    build.build()
    from paper_1203_2742_gb300 import binding
    return binding


def product_structure(B, sym):
    """Supernodes of an analysed pattern in the USER numbering:
    list of (N_k, A_k, parent index) with N_k, A_k sorted lists."""
    sp, par, rp, rows = sym.supernodes()
    perm = sym.perm
    out = []
    for k in range(len(sp) - 1):
        nk = int(sp[k + 1] - sp[k])
        J = rows[rp[k]:rp[k + 1]]
        out.append((sorted(int(perm[v]) for v in J[:nk]), sorted(int(perm[v]) for v in J[nk:]), int(par[k])))
    return out
