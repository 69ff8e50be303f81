"""Central finite differences of a scalar function (test infrastructure only)."""

import numpy as np


def directional(f, x, delta, h):
    """(f(x + h delta) - f(x - h delta)) / (2 h)."""
    x = np.asarray(x, dtype=np.float64)
    delta = np.asarray(delta, dtype=np.float64)
    return (f(x + h * delta) - f(x - h * delta)) / (2.0 * h)


def gradient(f, x, rel_step=1e-6):
    """Coordinate-wise central differences with step h_i = rel_step * max(1, |x_i|)."""
    x = np.asarray(x, dtype=np.float64)
    g = np.empty_like(x)
    flat = x.reshape(-1)
    for i in range(flat.size):
        h = rel_step * max(1.0, abs(flat[i]))
        e = np.zeros_like(flat)
        e[i] = 1.0
        g.reshape(-1)[i] = directional(f, flat, e, h)
    return g
