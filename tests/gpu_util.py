"""Helpers for the GPU parity tests."""
import numpy as np


def rel_err(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_rel_err(a, b):
    """max_i |a_i - b_i| / max_i |b_i| (element by element, scaled by the largest entry)."""
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return float(np.abs(a - b).max() / np.abs(b).max())
