"""Parity at the benchmark's full sizes, on the path bench.py times
(sl_autotune, then sl_run recorded as a CUDA graph): every node of the
16.8M-node C3 mesh and of the 256-problem C5 batch against the oracle, and
ragged batches down to the smallest mesh (one cell, two triangles)."""
import numpy as np
import pytest

import oracle
import paper_2104_09189_gb300 as sl
import sl_inputs as si
from gpu_helpers import FOOT_DELTA, REL_TOL_FP64

pytestmark = pytest.mark.gpu


def _device_run(probs, steps, precision=sl.SL_FP64, curve=sl.SL_CURVE_HILBERT, debug_first=False):
    import torch
    no, to, xy, tri = sl.pack_meshes([(p.mesh.xy, p.mesh.tri) for p in probs])
    h = sl.sl_mesh_create(no, to, xy, tri, precision=precision, seed=probs[0].seed)
    lperm, tperm = sl.sl_mesh_reorder(h, curve)
    perm = lperm.astype(np.int64) + np.repeat(no[:-1], np.diff(no))         # global new -> old
    tperm_g = tperm.astype(np.int64) + np.repeat(to[:-1], np.diff(to))
    pr = sl.problems([(p.field.kind, p.dt, p.field.packed()) for p in probs])
    vt = torch.float64 if precision == sl.SL_FP64 else torch.float32
    v0 = np.concatenate([p.v0 for p in probs])
    v = torch.tensor(v0[perm], dtype=vt, device="cuda")
    w = torch.empty_like(v)
    sl.sl_autotune(h, pr, 2, v, w)
    tri_first = None
    if debug_first:
        N = int(no[-1])
        dbg = {"tri": torch.full((N,), -1, dtype=torch.int32, device="cuda"),
               "feet": torch.zeros(2 * N, dtype=torch.float64, device="cuda")}
        sl.sl_step(h, pr, 0, v, w, debug=dbg)
        sl.sl_mesh_status(h)
        t = dbg["tri"].cpu().numpy()
        tri_first = np.empty(N, dtype=np.int64)
        tri_first[perm] = tperm_g[t]
        sl.sl_mesh_reset_t0(h)
    sl.sl_run(h, pr, 0, steps, v, w, use_graph=True)
    out = np.empty(len(v0))
    out[perm] = v.double().cpu().numpy()
    sl.sl_mesh_destroy(h)
    return out, no, tri_first


def test_c3_full_size_parity():
    """C3 at 4096^2 (16 785 409 nodes): the first step's located triangles
    (every non-degenerate foot) and V after 3 steps (every node)."""
    prob = si.config("C3")
    got, _, tri_first = _device_run([prob], 3, debug_first=True)
    om = oracle.OracleMesh(prob.mesh.xy, prob.mesh.tri)
    v1, otri, _, oft = om.step(prob.field.kind, prob.field.packed(), prob.dt, 0, prob.v0)
    safe = om.margins(otri.astype(np.int32), oft) > FOOT_DELTA
    # ~4% of the feet are clipped onto the boundary (margin 0 by construction)
    assert safe.sum() > 0.9 * prob.mesh.n_nodes
    assert np.array_equal(tri_first[safe], otri[safe])
    near = np.nonzero(~safe)[0]
    assert np.all(om.margins(tri_first[near].astype(np.int32), oft[near]) >= -FOOT_DELTA)
    want = om.run(prob.field.kind, prob.field.packed(), prob.dt, 0, 3, prob.v0)
    assert np.abs(got - want).max() <= REL_TOL_FP64 * np.abs(want).max()


def test_c5_full_batch_parity():
    """The 256-problem batch (log-uniform sizes 2e3..2e5): every problem after
    3 steps."""
    probs = si.batch_config(256)
    got, no, _ = _device_run(probs, 3)
    for k, p in enumerate(probs):
        om = oracle.OracleMesh(p.mesh.xy, p.mesh.tri)
        want = om.run(p.field.kind, p.field.packed(), p.dt, 0, 3, p.v0)
        seg = got[no[k]:no[k + 1]]
        assert np.abs(seg - want).max() <= REL_TOL_FP64 * max(np.abs(want).max(), 1e-300), k
        om.close()


@pytest.mark.parametrize("precision", [sl.SL_FP64, sl.SL_FP32], ids=["fp64", "fp32"])
def test_ragged_batch_down_to_one_cell(precision):
    """Problems of 1, 2, 3, 5, 40 and 7 cells per side in one launch, every
    field kind: the one-cell mesh has 4 nodes (all on the boundary) and two
    triangles."""
    fields = [si.rotation_field(), si.swirl_field(), si.fourier8_field(3), si.paper_field(),
              si.affine_field([0.1, 0.2, -0.1, 0.3, -0.2, 0.1, 0.05, -0.4]), si.zero_field()]
    probs = []
    for k, (M, f) in enumerate(zip((1, 2, 3, 5, 40, 7), fields)):
        mesh = si.grid_mesh(M, 0.25 if M > 1 else 0.0, 30 + k)
        v0 = si.gaussian(mesh.xy, 0.4, 0.6, 0.2)
        probs.append(si.Problem(f"m{M}", mesh, f, 0.07, 4, v0, "fp64", 30 + k))
    got, no, _ = _device_run(probs, 4, precision=precision)
    for k, p in enumerate(probs):
        om = oracle.OracleMesh(p.mesh.xy, p.mesh.tri)
        want = om.run(p.field.kind, p.field.packed(), p.dt, 0, 4, p.v0)
        seg = got[no[k]:no[k + 1]]
        tol = REL_TOL_FP64 if precision == sl.SL_FP64 else 1e-5
        assert np.abs(seg - want).max() <= tol * max(np.abs(want).max(), 1e-300), p.name
        om.close()
