"""Initial data u0 evaluated at the nodes (V^0_i = u0(x_i), Algorithm 2)."""
import numpy as np


def cosine_bump(xy, cx=0.5, cy=0.75, radius=0.15):
    """0.5 (1 + cos(pi min(r / radius, 1))): peak 1 at the centre, 0 outside."""
    r = np.hypot(xy[:, 0] - cx, xy[:, 1] - cy)
    return 0.5 * (1.0 + np.cos(np.pi * np.minimum(r / radius, 1.0)))


def gaussian(xy, cx=0.5, cy=0.75, sigma=0.05):
    r2 = (xy[:, 0] - cx) ** 2 + (xy[:, 1] - cy) ** 2
    return np.exp(-r2 / (2.0 * sigma * sigma))


def linear(xy, a=0.25, b=1.0, c=-0.5):
    return a + b * xy[:, 0] + c * xy[:, 1]


def constant(xy, value=0.75):
    return np.full(xy.shape[0], value, dtype=np.float64)
