"""Advecting fields f(x, t) as (kind, parameter vector) pairs.

Only the parameters live here; each consumer evaluates f with its own code.
Kind codes and parameter layouts (p = 48 doubles):

  ZERO      f = 0
  AFFINE    f_x = p0 + p1 x + p2 y + p3 t,   f_y = p4 + p5 x + p6 y + p7 t
  ROTATION  f = p0 (p2 - y, x - p1)          (solid rotation about (p1, p2))
  SWIRL     f = cos(pi t / p0) (sin^2(pi x) sin(2 pi y), -sin^2(pi y) sin(2 pi x))
  FOURIER8  psi = sum_m a_m cos(2 pi t + phi_m) sin(k_m pi x) sin(l_m pi y),
            f = (d psi/dy, -d psi/dx); mode m in 0..7 stores
            p[4m] = k_m, p[4m+1] = l_m, p[4m+2] = a_m, p[4m+3] = phi_m
  PAPER     f = (cos(p0 r + p1 t), sin(p0 r + p1 t)), r = |x - (p2, p3)|
            (the test field of the paper's Sec. 4, with C0 = p0, C1 = p1)
"""
from dataclasses import dataclass, field as dc_field
import numpy as np

from .rng import uniform01, normal01, splitmix64

FIELD_ZERO, FIELD_AFFINE, FIELD_ROTATION, FIELD_SWIRL, FIELD_FOURIER8, FIELD_PAPER = range(6)
N_PARAMS = 48


@dataclass
class Field:
    kind: int
    params: np.ndarray = dc_field(default_factory=lambda: np.zeros(N_PARAMS))
    scale: float = 0.0     # an upper estimate of max |f| over the unit square (for choosing dt)

    def packed(self):
        p = np.zeros(N_PARAMS, dtype=np.float64)
        p[: len(self.params)] = self.params
        return p


def zero_field():
    return Field(FIELD_ZERO, np.zeros(N_PARAMS), 0.0)


def affine_field(p):
    q = np.zeros(N_PARAMS)
    q[:8] = p
    return Field(FIELD_AFFINE, q, float(np.abs(q[:8]).sum()))


def rotation_field(omega=2.0 * np.pi, cx=0.5, cy=0.5):
    q = np.zeros(N_PARAMS)
    q[:3] = (omega, cx, cy)
    r = max(np.hypot(cx, cy), np.hypot(1 - cx, cy), np.hypot(cx, 1 - cy), np.hypot(1 - cx, 1 - cy))
    return Field(FIELD_ROTATION, q, abs(omega) * r)


def swirl_field(period=1.0):
    q = np.zeros(N_PARAMS)
    q[0] = period
    return Field(FIELD_SWIRL, q, 1.0)


def fourier8_field(seed):
    """k_m, l_m ~ U{1..4}; a_m = z_m / (k_m^2 + l_m^2), z_m ~ N(0,1);
    phi_m ~ U[0, 2 pi)."""
    m = np.arange(8)
    k = 1 + (splitmix64(seed, 20, m) % np.uint64(4)).astype(np.float64)
    l = 1 + (splitmix64(seed, 21, m) % np.uint64(4)).astype(np.float64)
    z = normal01(seed, 22, m)
    a = z / (k * k + l * l)
    phi = 2.0 * np.pi * uniform01(seed, 23, m)
    q = np.zeros(N_PARAMS)
    q[0:32:4] = k
    q[1:32:4] = l
    q[2:32:4] = a
    q[3:32:4] = phi
    scale = float(np.sum(np.abs(a) * np.pi * np.hypot(k, l)))
    return Field(FIELD_FOURIER8, q, scale)


def paper_field(c0=2.0 * np.pi, c1=2.0 * np.pi, cx=0.5, cy=0.5):
    q = np.zeros(N_PARAMS)
    q[:4] = (c0, c1, cx, cy)
    return Field(FIELD_PAPER, q, 1.0)
