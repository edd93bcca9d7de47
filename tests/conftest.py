"""Shared pytest set-up: markers, import path and fixture loaders."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the CUDA extension")
    config.addinivalue_line("markers", "slow: long-running physics check")


def load_int_matrix(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(v) for v in line.split()])
    return np.array(rows, dtype=np.float64)


def load_expr_matrix(name):
    """Matrix of polynomial entries in ux, uy, uz (as printed in the paper's appendix)."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            cells = [c.strip() for c in line.split(";")]
            rows.append([compile(c, name, "eval") for c in cells])

    def evaluate(u):
        env = {"__builtins__": {}, "ux": float(u[0]), "uy": float(u[1]), "uz": float(u[2])}
        return np.array([[eval(c, env) for c in r] for r in rows], dtype=np.float64)

    return evaluate
