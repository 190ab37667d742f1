"""The five benchmark / parity workloads.

  C1  64^2 jittered (+-0.25h) grid, swirl, cosine bump r=0.15 at (0.5,0.75),
      dt = 1/20, 20 steps (to t = 1), FP64.                       seed 1
  C2  1024^2, same construction, dt = 0.05, 20 steps, FP64.        seed 2
  C3  4096^2 graded (x + 0.3 sin(2 pi x)/(2 pi)) grid jittered +-0.2h,
      solid rotation 2 pi (0.5 - y, x - 0.5), Gaussian sigma 0.05 at
      (0.5, 0.75), dt = 0.02, 50 steps, FP64.                      seed 3
  C4  the C3 mesh, swirl, cosine bump, dt = 0.05, 20 steps, FP32.  seed 3
  C5  256 independent meshes, (M_p+1)^2 nodes with N_p log-uniform in
      [2e3, 2e5] and M_p = round(sqrt(N_p)) - 1, jitter +-0.25h; field drawn
      uniformly from {rotation, swirl, fourier8}; Gaussian sigma 0.05 at a
      centre drawn in [0.3, 0.7]^2; dt_p = C_p h_p / scale_p with
      C_p ~ U[5, 30] and scale_p the field's analytic bound on |f|;
      50 steps.  Problem p uses seed 5*1000 + p.
"""
from dataclasses import dataclass
import numpy as np

from .meshes import grid_mesh, Mesh
from .fields import Field, swirl_field, rotation_field, fourier8_field
from .initial import cosine_bump, gaussian
from .rng import uniform01, splitmix64

CONFIG_NAMES = ("C1", "C2", "C3", "C4", "C5")


@dataclass
class Problem:
    name: str
    mesh: Mesh
    field: Field
    dt: float
    n_steps: int
    v0: np.ndarray      # float64 initial values at the nodes
    precision: str      # "fp64" or "fp32"
    seed: int


def _single(name, M, jitter, graded, seed, field, u0, dt, steps, precision):
    mesh = grid_mesh(M, jitter=jitter, seed=seed, graded=graded)
    return Problem(name, mesh, field, float(dt), int(steps), u0(mesh.xy), precision, seed)


def config(name, M=None):
    """Build config `name`; `M` overrides the cells per side (for scaled-down
    parity cases with the same construction)."""
    if name == "C1":
        return _single("C1", M or 64, 0.25, False, 1, swirl_field(), cosine_bump, 1.0 / 20.0, 20, "fp64")
    if name == "C2":
        return _single("C2", M or 1024, 0.25, False, 2, swirl_field(), cosine_bump, 0.05, 20, "fp64")
    if name == "C3":
        return _single("C3", M or 4096, 0.2, True, 3, rotation_field(), gaussian, 0.02, 50, "fp64")
    if name == "C4":
        return _single("C4", M or 4096, 0.2, True, 3, swirl_field(), cosine_bump, 0.05, 20, "fp32")
    raise ValueError(f"unknown single-mesh config {name!r}")


def batch_config(n_problems=256, seed=5, nmin=2e3, nmax=2e5, steps=50, precision="fp64"):
    """C5: a list of independent Problems (see the module docstring)."""
    probs = []
    for p in range(n_problems):
        s = seed * 1000 + p
        u = uniform01(s, 30, np.arange(6))
        n_p = float(np.exp(np.log(nmin) + u[0] * (np.log(nmax) - np.log(nmin))))
        M = max(2, int(round(np.sqrt(n_p))) - 1)
        kind = int(splitmix64(s, 31, 0) % np.uint64(3))
        if kind == 0:
            field = rotation_field()
        elif kind == 1:
            field = swirl_field()
        else:
            field = fourier8_field(s)
        courant = 5.0 + 25.0 * u[1]
        dt = courant * (1.0 / M) / field.scale
        cx, cy = 0.3 + 0.4 * u[2], 0.3 + 0.4 * u[3]
        mesh = grid_mesh(M, jitter=0.25, seed=s, graded=False)
        v0 = gaussian(mesh.xy, cx, cy, 0.05)
        probs.append(Problem(f"C5[{p}]", mesh, field, dt, steps, v0, precision, s))
    return probs
