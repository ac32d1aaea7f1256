import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def load_paper_tables():
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", "paper_tables.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            t, form, d, N, k, memA, memAT, memAh, memAhT, nnzB, meff, ceff = line.split()
            rows.append(dict(table=int(t), form=form, d=int(d), N=int(N), k=int(k),
                             memA=int(memA), memA_T=int(memAT), memAhat=int(memAh),
                             memAhat_T=int(memAhT), nnzB=int(nnzB), mem_eff=float(meff),
                             comp_eff=float(ceff)))
    return rows
