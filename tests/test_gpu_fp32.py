"""The FP32 path (float coordinates and values, FP32-certified walk with a
double / exact fallback) against the oracle.

Triangles: the oracle's FP32 feet (same float arithmetic) located exactly on
the float mesh must give the GPU's triangle, except for feet within a few
float ulps of an edge line, which must be contained.  Values: compared with
the FP64 oracle on the FP64 mesh; the error is reported and must stay below
1e-5 (max)."""
import numpy as np
import pytest

import oracle
import paper_2104_09189_gb300 as sl
import sl_inputs as si
from gpu_helpers import DeviceRun

pytestmark = pytest.mark.gpu

DELTA32 = 8 * 2.0 ** -24       # feet of the two sides may differ by float rounding of the field tables


def _fp32_parity(prob, steps, curve=sl.SL_CURVE_HILBERT):
    mesh = prob.mesh
    xy32 = mesh.xy.astype(np.float32)
    om32 = oracle.OracleMesh(xy32.astype(np.float64), mesh.tri)
    om64 = oracle.OracleMesh(mesh.xy, mesh.tri)
    g = DeviceRun(mesh, prob.field, prob.dt, curve=curve, precision=sl.SL_FP32)
    v_dev = g.to_dev(prob.v0.astype(np.float32))
    v64 = prob.v0.copy()
    worst = 0.0
    near_total = 0
    for n in range(steps):
        v_dev, res = g.step(n, v_dev)
        v64, _, _, _ = om64.step(prob.field.kind, prob.field.packed(), prob.dt, n, v64, want_feet=False)
        f32, _ = oracle.feet_f32(prob.field.kind, prob.field.packed(), prob.dt, n, xy32)
        ft = f32.astype(np.float64)
        otri, _ = om32.locate(ft)
        margin = om32.margins(otri, ft)
        safe = margin > DELTA32
        assert np.all(res["tri"][safe] == otri[safe]), np.nonzero(safe & (res["tri"] != otri))[0][:5]
        near = np.nonzero(~safe)[0]
        if near.size:
            assert np.all(om32.margins(res["tri"][near].astype(np.int32), ft[near]) >= -DELTA32)
        near_total += near.size
        worst = max(worst, np.abs(res["v"] - v64).max())
    g.close()
    return worst, near_total


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


def test_fp32_rotation_feet_bitwise():
    """Trig-free fields: the GPU's float feet equal the oracle's FP32 feet bit
    for bit (same operations in the same order)."""
    prob = si.config("C3", M=128)
    mesh = prob.mesh
    g = DeviceRun(mesh, prob.field, prob.dt, curve=sl.SL_CURVE_NONE, precision=sl.SL_FP32)
    v_dev = g.to_dev(prob.v0.astype(np.float32))
    for n in range(3):
        v_dev, res = g.step(n, v_dev)
        f32, _ = oracle.feet_f32(prob.field.kind, prob.field.packed(), prob.dt, n, mesh.xy.astype(np.float32))
        assert np.array_equal(res["feet"], f32.astype(np.float64))
    g.close()


@pytest.mark.slow
def test_fp32_full_c4_error_vs_fp64_oracle():
    """C4 at full size (16.8M nodes, 20 steps): max and L2 error of the FP32
    path against the FP64 oracle; the target is a max error <= 1e-5."""
    import torch
    prob = si.config("C4")
    mesh = prob.mesh
    no, to, xy, tri = sl.pack_meshes([(mesh.xy, mesh.tri)])
    h = sl.sl_mesh_create(no, to, xy, tri, precision=sl.SL_FP32, seed=prob.seed)
    perm, _ = sl.sl_mesh_reorder(h, sl.SL_CURVE_HILBERT)
    probs = sl.problems([(prob.field.kind, prob.dt, prob.field.packed())])
    v = torch.tensor(prob.v0[perm], dtype=torch.float32, device="cuda")
    w = torch.empty_like(v)
    stats = sl.sl_run(h, probs, 0, prob.n_steps, v, w)
    got = np.empty(mesh.n_nodes)
    got[perm] = v.double().cpu().numpy()
    sl.sl_mesh_destroy(h)
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    want = om.run(prob.field.kind, prob.field.packed(), prob.dt, 0, prob.n_steps, prob.v0)
    err = np.abs(got - want)
    print(f"C4 FP32 vs FP64 oracle: max {err.max():.3e}  L2 {np.sqrt((err ** 2).mean()):.3e}  stats {stats}")
    assert err.max() <= 1e-5
