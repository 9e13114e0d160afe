"""Helpers shared by the GPU tests (no arithmetic of the method here)."""
import numpy as np
import pytest


def solver_module():
    import paper_1603_00279_gb300 as P
    from paper_1603_00279_gb300 import build
    build.build()
    return P


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)
