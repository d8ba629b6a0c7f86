"""Helpers shared by the GPU parity tests (test-side only)."""
import numpy as np


def rel_fro(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64)) /
                 max(np.linalg.norm(np.asarray(b, np.float64)), 1e-300))


# Hertz's law for a layer bonded to a rigid base (Dimitriadis et al.,
# Biophys. J. 82, 2002): the factor multiplying the half-space force.
def bonded_layer_factor(chi, nu):
    a0 = -(1.2876 - 1.4678 * nu + 1.3442 * nu ** 2) / (1 - nu)
    b0 = (0.6387 - 1.0277 * nu + 1.5164 * nu ** 2) / (1 - nu)
    pi = np.pi
    c1 = -2 * a0 / pi
    c2 = 4 * a0 ** 2 / pi ** 2
    c3 = -8 / pi ** 3 * (a0 ** 3 + 4 * pi ** 2 * b0 / 15)
    c4 = -16 * a0 / pi ** 4 * (a0 ** 3 + 3 * pi ** 2 * b0 / 5)
    return 1 + c1 * chi + c2 * chi ** 2 + c3 * chi ** 3 + c4 * chi ** 4
