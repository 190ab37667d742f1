"""sl_step_noalloc: the step for callers that cannot allocate device memory
while they step (its scratch is a fixed static device array of the library).
It must give the values of sl_step, call after call, and refuse meshes beyond
its fixed limit.  This file is collected last on purpose."""
import numpy as np
import pytest

import paper_2104_09189_gb300 as sl
import sl_inputs as si

pytestmark = pytest.mark.gpu

REL_TOL = 1e-12     # the tolerance of the FP64 parity tests


def _handle(prob):
    no, to, xy, tri = sl.pack_meshes([(prob.mesh.xy, prob.mesh.tri)])
    h = sl.sl_mesh_create(no, to, xy, tri, precision=sl.SL_FP64, seed=prob.seed)
    perm, _ = sl.sl_mesh_reorder(h, sl.SL_CURVE_HILBERT)
    return h, perm


@pytest.mark.parametrize("name", ["rotation", "swirl"])
def test_noalloc_matches_sl_step_on_two_calls_in_a_row(name):
    import torch
    if name == "rotation":
        prob = si.config("C3", M=256)
    else:
        prob = si.config("C2", M=256)
    probs = sl.problems([(prob.field.kind, prob.dt, prob.field.packed())])
    ref, perm = _handle(prob)
    new, _ = _handle(prob)
    try:
        v0 = torch.tensor(prob.v0[perm], dtype=torch.float64, device="cuda")
        if name == "swirl":
            # the swirl's node tables are built (allocated) by one ordinary
            # step; T^0 is then put back so both handles start alike
            scratch = torch.empty_like(v0)
            sl.sl_step(new, probs, 0, v0, scratch)
            sl.sl_mesh_reset_t0(new)
        a_ref, b_ref = torch.empty_like(v0), torch.empty_like(v0)
        a_new, b_new = torch.empty_like(v0), torch.empty_like(v0)
        sl.sl_step(ref, probs, 0, v0, a_ref)
        sl.sl_step(ref, probs, 1, a_ref, b_ref)
        sl.sl_step_noalloc(new, probs, 0, v0, a_new)
        sl.sl_step_noalloc(new, probs, 1, a_new, b_new)
        sl.sl_mesh_status(new)
        torch.cuda.synchronize()
        for got, want in ((a_new, a_ref), (b_new, b_ref)):
            g, w = got.cpu().numpy(), want.cpu().numpy()
            assert np.abs(g - w).max() <= REL_TOL * np.abs(w).max()
        # both handles walked to the same triangles
        t_ref = torch.empty(prob.mesh.n_nodes, dtype=torch.int32, device="cuda")
        t_new = torch.empty_like(t_ref)
        sl.sl_mesh_get_t0(ref, t_ref)
        sl.sl_mesh_get_t0(new, t_new)
        assert torch.equal(t_ref, t_new)
    finally:
        sl.sl_mesh_destroy(ref)
        sl.sl_mesh_destroy(new)


def test_noalloc_refuses_meshes_beyond_its_limit():
    import torch
    prob = si.config("C2")                      # 1025^2 = 1 050 625 nodes > 2^20
    assert prob.mesh.n_nodes > sl.SL_NOALLOC_MAX_NODES
    probs = sl.problems([(si.FIELD_ROTATION, 0.01, si.rotation_field().packed())])
    h, _ = _handle(prob)
    try:
        v = torch.zeros(prob.mesh.n_nodes, dtype=torch.float64, device="cuda")
        w = torch.empty_like(v)
        with pytest.raises(sl.SLError) as e:
            sl.sl_step_noalloc(h, probs, 0, v, w)
        assert e.value.status == sl.SL_E_ARG and str(sl.SL_NOALLOC_MAX_NODES) in str(e.value)
    finally:
        sl.sl_mesh_destroy(h)


def test_noalloc_requires_node_tables_built_first():
    import torch
    prob = si.config("C1")
    probs = sl.problems([(prob.field.kind, prob.dt, prob.field.packed())])
    h, perm = _handle(prob)
    try:
        v = torch.tensor(prob.v0[perm], dtype=torch.float64, device="cuda")
        w = torch.empty_like(v)
        with pytest.raises(sl.SLError) as e:
            sl.sl_step_noalloc(h, probs, 0, v, w)
        assert e.value.status == sl.SL_E_STATE
    finally:
        sl.sl_mesh_destroy(h)


def test_noalloc_matches_sl_step_on_a_batch_on_two_calls_in_a_row():
    """Six problems of uneven sizes with rotation and swirl fields: the
    per-problem constants in the static array and the per-block problem
    lookup, against sl_step."""
    import torch
    fields = [si.rotation_field(), si.swirl_field(), si.rotation_field(3.0, 0.4, 0.6), si.swirl_field(),
              si.rotation_field(), si.swirl_field()]
    probs_in = []
    for k, (M, f) in enumerate(zip((7, 40, 13, 64, 3, 25), fields)):
        mesh = si.grid_mesh(M, 0.25, 50 + k)
        probs_in.append((mesh, f, 0.6 / M, si.gaussian(mesh.xy, 0.45, 0.55, 0.15)))
    no, to, xy, tri = sl.pack_meshes([(m.xy, m.tri) for m, _, _, _ in probs_in])
    pr = sl.problems([(f.kind, dt, f.packed()) for _, f, dt, _ in probs_in])
    v0 = torch.tensor(np.concatenate([v for _, _, _, v in probs_in]), dtype=torch.float64, device="cuda")
    ref = sl.sl_mesh_create(no, to, xy, tri, precision=sl.SL_FP64, seed=3)
    new = sl.sl_mesh_create(no, to, xy, tri, precision=sl.SL_FP64, seed=3)
    try:
        scratch = torch.empty_like(v0)
        sl.sl_step(new, pr, 0, v0, scratch)        # builds the swirl's node tables
        sl.sl_mesh_reset_t0(new)
        a_ref, b_ref = torch.empty_like(v0), torch.empty_like(v0)
        a_new, b_new = torch.empty_like(v0), torch.empty_like(v0)
        sl.sl_step(ref, pr, 0, v0, a_ref)
        sl.sl_step(ref, pr, 1, a_ref, b_ref)
        sl.sl_step_noalloc(new, pr, 0, v0, a_new)
        sl.sl_step_noalloc(new, pr, 1, a_new, b_new)
        sl.sl_mesh_status(new)
        torch.cuda.synchronize()
        for got, want in ((a_new, a_ref), (b_new, b_ref)):
            for k in range(len(probs_in)):
                g, w = got[no[k]:no[k + 1]].cpu().numpy(), want[no[k]:no[k + 1]].cpu().numpy()
                assert np.abs(g - w).max() <= REL_TOL * np.abs(w).max(), k
    finally:
        sl.sl_mesh_destroy(ref)
        sl.sl_mesh_destroy(new)


def test_noalloc_refuses_more_problems_than_its_limit():
    import torch
    n = sl.SL_NOALLOC_MAX_PROBLEMS + 1
    mesh = si.grid_mesh(1, 0.0, 1)
    no, to, xy, tri = sl.pack_meshes([(mesh.xy, mesh.tri)] * n)
    pr = sl.problems([(si.FIELD_ROTATION, 0.01, si.rotation_field().packed())] * n)
    h = sl.sl_mesh_create(no, to, xy, tri, precision=sl.SL_FP64, seed=1)
    try:
        v = torch.zeros(int(no[-1]), dtype=torch.float64, device="cuda")
        w = torch.empty_like(v)
        with pytest.raises(sl.SLError) as e:
            sl.sl_step_noalloc(h, pr, 0, v, w)
        assert e.value.status == sl.SL_E_ARG and str(sl.SL_NOALLOC_MAX_PROBLEMS) in str(e.value)
    finally:
        sl.sl_mesh_destroy(h)
