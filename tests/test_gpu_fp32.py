"""The FP32 path (float coordinates and values, FP32-certified walk with a
double / exact fallback) against the oracle.

Triangles: the oracle locates the GPU's own float feet (exact in double)
exactly on the float-rounded mesh (reading c19); a foot strictly inside a
triangle must be in the GPU's triangle, a foot on an edge or vertex must lie
in it by the exact signs.  Feet: within float rounding of the double Euler
foot of the same float nodes.  Values: compared with the FP64 oracle on the
FP64 mesh; the error is reported and must stay below 1e-5 (max)."""
import numpy as np
import pytest

import oracle
import paper_2104_09189_gb300 as sl
import sl_inputs as si
from gpu_helpers import DeviceRun, exact_triangle_parity

pytestmark = pytest.mark.gpu

# The float foot against the double foot of the same float nodes: the
# field's factors and the Euler step each round once or twice in float
# (|X| <= 1, so a rounding is at most 2^-25), the trig tables once more.
FOOT_TOL32 = 8 * 2.0 ** -24


def _fp32_parity(prob, steps, curve=sl.SL_CURVE_HILBERT):
    mesh = prob.mesh
    xy32 = mesh.xy.astype(np.float32)
    om32 = oracle.OracleMesh(xy32.astype(np.float64), mesh.tri)
    om64 = oracle.OracleMesh(mesh.xy, mesh.tri)
    g = DeviceRun(mesh, prob.field, prob.dt, curve=curve, precision=sl.SL_FP32)
    v_dev = g.to_dev(prob.v0.astype(np.float32))
    v64 = prob.v0.copy()
    worst = 0.0
    on_edge = 0
    for n in range(steps):
        v_dev, res = g.step(n, v_dev)
        v64, _, _, _ = om64.step(prob.field.kind, prob.field.packed(), prob.dt, n, v64, want_feet=False)
        f64, _ = oracle.feet(prob.field.kind, prob.field.packed(), prob.dt, n, xy32.astype(np.float64))
        assert np.abs(res["feet"] - f64).max() <= FOOT_TOL32
        assert np.array_equal(res["feet"], res["feet"].astype(np.float32).astype(np.float64))
        assert not res["feet_lo"].any()
        on_edge += exact_triangle_parity(om32, res["tri"], res["feet"], None, res["flags"])
        worst = max(worst, np.abs(res["v"] - v64).max())
    g.close()
    return worst, on_edge


def test_fp32_parity_c4_construction():
    prob = si.config("C4", M=256)
    worst, near = _fp32_parity(prob, 6)
    assert worst <= 1e-5, worst


def test_fp32_parity_other_fields():
    mesh = si.grid_mesh(96, 0.25, 12)
    v0 = si.gaussian(mesh.xy, 0.45, 0.55, 0.1)
    for fld, dt in [(si.rotation_field(), 0.02), (si.fourier8_field(7), 0.03), (si.paper_field(), 0.02)]:
        prob = si.Problem("x", mesh, fld, dt, 4, v0, "fp32", 12)
        worst, _ = _fp32_parity(prob, 4)
        assert worst <= 1e-5, (fld.kind, worst)
