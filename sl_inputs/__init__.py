"""Seeded synthetic inputs for the semi-Lagrangian foot / locate / P1 path.

This module only *generates inputs*: meshes (node coordinates, CCW triangles),
field parameters (the numbers a field definition needs, including the random
draws of the Fourier field), time steps and initial data V^0 = u0(x_i).
It contains none of the method's arithmetic (no foot, no clip, no point
location, no interpolation, no field evaluation), so both the CPU oracle and
the CUDA library can consume it without sharing computation.

Random numbers come from a counter-based SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): the value for
(seed, stream, i) is mix64(mix64(seed*G + stream) + (i+1)*G) with
G = 0x9E3779B97F4A7C15, so any element can be regenerated independently.

The paper's own experiments (Sec. 4) ran on Delaunay meshes from the Triangle
library on [-1/2, 1/2]^2; those are not available here.  Jittered,
shorter-diagonal-split grids on [0,1]^2 stand in for them (same node density,
same quasi-uniform triangle shapes, same regular valence ~6).
"""
from .rng import splitmix64, uniform01, normal01
from .meshes import Mesh, grid_mesh, courant_grid
from .fields import (FIELD_ZERO, FIELD_AFFINE, FIELD_ROTATION, FIELD_SWIRL,
                     FIELD_FOURIER8, FIELD_PAPER, Field, zero_field,
                     affine_field, rotation_field, swirl_field,
                     fourier8_field, paper_field, N_PARAMS)
from .initial import cosine_bump, gaussian, linear, constant
from .configs import Problem, config, CONFIG_NAMES, batch_config

__all__ = [
    "splitmix64", "uniform01", "normal01", "Mesh", "grid_mesh", "courant_grid",
    "FIELD_ZERO", "FIELD_AFFINE", "FIELD_ROTATION", "FIELD_SWIRL",
    "FIELD_FOURIER8", "FIELD_PAPER", "Field", "zero_field", "affine_field",
    "rotation_field", "swirl_field", "fourier8_field", "paper_field",
    "N_PARAMS", "cosine_bump", "gaussian", "linear", "constant", "Problem",
    "config", "CONFIG_NAMES", "batch_config",
]
