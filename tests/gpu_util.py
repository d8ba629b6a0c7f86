"""Helpers shared by the GPU parity tests (test-side only)."""
import numpy as np


def rel_fro(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64)) /
                 max(np.linalg.norm(np.asarray(b, np.float64)), 1e-300))
