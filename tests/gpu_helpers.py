"""Shared set-up for GPU parity tests (CUDA path vs FP64 CPU oracle)."""
import numpy as np

import oracle
import paper_1805_03981_gb300 as dgw


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def pair(cfg, prec=dgw.DG_FP64, alpha=None):
    """(GPU solver, oracle) on the same seeded instance."""
    a = cfg["alpha"] if alpha is None else alpha
    s = dgw.Solver(cfg["mesh"], cfg["k"], prec, a, cfg["rho"], cfg["c"])
    o = oracle.Oracle(cfg["mesh"], cfg["k"], cfg["rho"], cfg["c"], a)
    return s, o
