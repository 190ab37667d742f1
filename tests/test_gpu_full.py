"""Parity at the benchmark's full sizes, on the path bench.py times
(sl_autotune, then sl_run recorded as a CUDA graph), and step by step on the
same launch configuration with the per-node outputs: every node of the
16.8M-node C3 mesh over all 50 steps, the FP32 C4 run over its 20 steps,
every problem of the 256-problem C5 batch over its 50 steps, and ragged
batches down to the smallest mesh (one cell, two triangles).

Triangles are checked on the GPU's own feet with the oracle's exact
location (tests/gpu_helpers.exact_triangle_parity); the numbers of feet on
an edge or a vertex are reported at the end of the pytest run."""
import numpy as np
import pytest

import oracle
import paper_2104_09189_gb300 as sl
import sl_inputs as si
from gpu_helpers import FOOT_TOL_FP64, REL_TOL_FP64, exact_triangle_parity, report

pytestmark = pytest.mark.gpu


class FullRun:
    """A reordered (Hilbert) mesh on the GPU, autotuned like bench.py's, with
    the permutations to the original numbering."""

    def __init__(self, probs, precision=sl.SL_FP64, curve=sl.SL_CURVE_HILBERT):
        import torch
        self.torch = torch
        no, to, xy, tri = sl.pack_meshes([(p.mesh.xy, p.mesh.tri) for p in probs])
        self.no, self.to = no, to
        self.N = int(no[-1])
        self.h = sl.sl_mesh_create(no, to, xy, tri, precision=precision, seed=probs[0].seed)
        lperm, tperm = sl.sl_mesh_reorder(self.h, curve)
        self.perm = lperm.astype(np.int64) + np.repeat(no[:-1], np.diff(no))           # global new -> old
        self.tperm = tperm.astype(np.int64) + np.repeat(to[:-1], np.diff(to))
        self.pr = sl.problems([(p.field.kind, p.dt, p.field.packed()) for p in probs])
        self.vt = torch.float64 if precision == sl.SL_FP64 else torch.float32
        self.v0 = np.concatenate([p.v0 for p in probs])

    def dev(self, v_orig):
        return self.torch.tensor(np.asarray(v_orig)[self.perm], dtype=self.vt, device="cuda")

    def host(self, v_dev):
        out = np.empty(self.N)
        out[self.perm] = v_dev.double().cpu().numpy()
        return out

    def autotune(self):
        v, w = self.dev(self.v0), self.dev(self.v0)
        sl.sl_autotune(self.h, self.pr, 2, v, w)

    def graph_run(self, steps):
        """The timed path: sl_run of `steps` steps as one CUDA graph from V^0
        and the initial start triangles."""
        sl.sl_mesh_reset_t0(self.h)
        v, w = self.dev(self.v0), self.dev(self.v0)
        sl.sl_run(self.h, self.pr, 0, steps, v, w, use_graph=True)
        return self.host(v)

    def step(self, n, v, debug):
        """One sl_step; with debug the per-node outputs in the original
        numbering (triangles as original global indices)."""
        t = self.torch
        w = t.empty_like(v)
        if not debug:
            sl.sl_step(self.h, self.pr, n, v, w)
            return w, None
        N = self.N
        dbg = {"feet": t.zeros(2 * N, dtype=t.float64, device="cuda"),
               "feet_lo": t.zeros(2 * N, dtype=t.float64, device="cuda"),
               "tri": t.full((N,), -1, dtype=t.int32, device="cuda"),
               "flags": t.zeros(N, dtype=t.uint8, device="cuda")}
        sl.sl_step(self.h, self.pr, n, v, w, debug=dbg)
        sl.sl_mesh_status(self.h)
        res = {}
        for k, c in (("feet", 2), ("feet_lo", 2)):
            a = np.empty((N, 2))
            a[self.perm] = dbg[k].cpu().numpy().reshape(N, 2)
            res[k] = a
        tri = np.empty(N, dtype=np.int64)
        tri[self.perm] = self.tperm[dbg["tri"].cpu().numpy()]
        flags = np.empty(N, dtype=np.uint8)
        flags[self.perm] = dbg["flags"].cpu().numpy()
        res.update(tri=tri, flags=flags)
        return w, res

    def close(self):
        if self.h:
            sl.sl_mesh_destroy(self.h)
            self.h = None


def test_c3_full_size_parity_all_steps():
    """C3 at 4096^2 (16 785 409 nodes), all 50 steps of the bench's run:
    V after every step within 1e-12 of the oracle (step by step, autotuned
    launch shape and split form), the located triangles exactly at steps 1,
    2 and 50, and V^50 of the CUDA graph the bench replays."""
    prob = si.config("C3")
    om = oracle.OracleMesh(prob.mesh.xy, prob.mesh.tri)
    run = FullRun([prob])
    run.autotune()
    v50_graph = run.graph_run(prob.n_steps)
    sl.sl_mesh_reset_t0(run.h)
    v = run.dev(prob.v0)
    vo = prob.v0.copy()
    worst, on_edge, precise = 0.0, {}, {}
    kind, par, dt = prob.field.kind, prob.field.packed(), prob.dt
    for n in range(prob.n_steps):
        debug = n in (0, 1, prob.n_steps - 1)
        v, res = run.step(n, v, debug)
        got = run.host(v)
        if debug:
            precise[n + 1] = int(((res["flags"] & sl.SL_NODE_PRECISE) != 0).sum())
        ov, _, _, oft = om.step(kind, par, dt, n, vo, want_feet=debug)
        err = np.abs(got - ov).max() / np.abs(ov).max()
        assert err <= REL_TOL_FP64, (n, err)
        worst = max(worst, err)
        if debug:
            assert np.abs(res["feet"] - oft).max() <= FOOT_TOL_FP64
            on_edge[n + 1] = exact_triangle_parity(om, res["tri"], res["feet"], res["feet_lo"], res["flags"])
        vo = ov
    gerr = np.abs(v50_graph - vo).max() / np.abs(vo).max()
    assert gerr <= REL_TOL_FP64
    run.close()
    report("C3 full size, 50 steps", max_rel_err=f"{max(worst, gerr):.2e}",
           feet_on_edge_or_vertex_at_step=on_edge, fp64_value_path_nodes_at_step=precise,
           nodes=prob.mesh.n_nodes)


@pytest.mark.slow
def test_c4_full_size_fp32_parity_and_error_vs_fp64_oracle():
    """C4 at full size (16.8M nodes, FP32, 20 steps): the located triangles
    of the GPU's float feet exactly at steps 1, 2 and 20, and the max and L2
    error of V against the FP64 oracle after every step (target max <=
    1e-5), step by step and through the bench's CUDA graph."""
    prob = si.config("C4")
    mesh = prob.mesh
    om64 = oracle.OracleMesh(mesh.xy, mesh.tri)
    om32 = oracle.OracleMesh(mesh.xy.astype(np.float32).astype(np.float64), mesh.tri)
    run = FullRun([prob], precision=sl.SL_FP32)
    run.autotune()
    v20_graph = run.graph_run(prob.n_steps)
    sl.sl_mesh_reset_t0(run.h)
    v = run.dev(prob.v0.astype(np.float32))
    vo = prob.v0.copy()
    worst, on_edge = 0.0, {}
    kind, par, dt = prob.field.kind, prob.field.packed(), prob.dt
    for n in range(prob.n_steps):
        debug = n in (0, 1, prob.n_steps - 1)
        v, res = run.step(n, v, debug)
        got = run.host(v)
        vo, _, _, _ = om64.step(kind, par, dt, n, vo, want_feet=False)
        worst = max(worst, np.abs(got - vo).max())
        assert worst <= 1e-5, (n, worst)
        if debug:
            on_edge[n + 1] = exact_triangle_parity(om32, res["tri"], res["feet"], None, res["flags"])
    err = np.abs(v20_graph - vo)
    assert err.max() <= 1e-5
    run.close()
    report("C4 full size FP32, 20 steps", max_err_vs_fp64_oracle=f"{max(worst, err.max()):.2e}",
           l2_err=f"{np.sqrt((err ** 2).mean()):.2e}", feet_on_edge_or_vertex_at_step=on_edge)


# Accumulated drift of the double-float path over a run, relative to max
# |V^0|.  Its foot and barycentric numerators round at about 2^-48 (the
# foot's (grid, remainder) form, the remainder differences and the cross
# terms of the numerators, each equivalent to moving the foot by a few
# 2^-49), so one step can differ from the oracle's by about
# 5 * 2^-48 * |grad V|; where the gradient exceeds SL_OPT_PRECISE's bound
# G = 32 the value is evaluated in FP64, so a step stays below about
# 5 * 2^-48 * 32 ~ 5.7e-13, and on a time-constant field the same node
# repeats the same rounding at every step: 50 steps could add up to 2.8e-11,
# the measured drift is far smaller.  The 1e-12 tolerance holds for every
# single step.
DRIFT_TOL_FP64 = 1e-11


def test_c5_full_batch_parity():
    """The 256-problem batch (log-uniform sizes 2e3..2e5), all 50 steps:
    every step of every problem within 1e-12 of one oracle step applied to
    the GPU's own V^n (relative to the problem's max |V^0|); the located
    triangles of the first step exactly, problem by problem; V^50 of the
    bench's CUDA graph against the oracle's 50-step run within the drift
    bound above (the largest drift is reported).

    The scale is max |V^0|: P1 interpolation is a convex combination (theta
    >= 0, sum 1), so every value a run carries is at most max |V^0|, while on
    some coarse meshes the stretched Gaussian's maximum decays a
    thousandfold in 50 steps."""
    probs = si.batch_config(256)
    run = FullRun(probs)
    run.autotune()
    got = run.graph_run(50)
    sl.sl_mesh_reset_t0(run.h)
    no, to = run.no, run.to
    oms = [oracle.OracleMesh(p.mesh.xy, p.mesh.tri) for p in probs]
    scale = [max(np.abs(p.v0).max(), 1e-300) for p in probs]
    vo = [p.v0.copy() for p in probs]
    v = run.dev(run.v0)
    on_edge, worst_step = 0, 0.0
    for n in range(50):
        vin = run.host(v)
        v, res = run.step(n, v, n == 0)
        out = run.host(v)
        for k, p in enumerate(probs):
            sel = slice(no[k], no[k + 1])
            kind, par = p.field.kind, p.field.packed()
            one, _, _, _ = oms[k].step(kind, par, p.dt, n, vin[sel], want_feet=False)
            e = np.abs(out[sel] - one).max() / scale[k]
            assert e <= REL_TOL_FP64, (n, k, e)
            worst_step = max(worst_step, e)
            vo[k], _, _, _ = oms[k].step(kind, par, p.dt, n, vo[k], want_feet=False)
            if n == 0:
                on_edge += exact_triangle_parity(oms[k], res["tri"][sel] - to[k], res["feet"][sel],
                                                 res["feet_lo"][sel], res["flags"][sel])
    run.close()
    drift = max(np.abs(got[no[k]:no[k + 1]] - vo[k]).max() / scale[k] for k in range(len(probs)))
    for om in oms:
        om.close()
    assert drift <= DRIFT_TOL_FP64, drift
    report("C5 batch, 256 problems, 50 steps", max_rel_err_one_step=f"{worst_step:.2e}",
           max_rel_drift_50_steps=f"{drift:.2e}", feet_on_edge_or_vertex_at_step_1=on_edge)


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
    run = FullRun(probs, precision=precision)
    run.autotune()
    got = run.graph_run(4)
    run.close()
    for k, p in enumerate(probs):
        om = oracle.OracleMesh(p.mesh.xy, p.mesh.tri)
        want = om.run(p.field.kind, p.field.packed(), p.dt, 0, 4, p.v0)
        seg = got[run.no[k]:run.no[k + 1]]
        tol = REL_TOL_FP64 if precision == sl.SL_FP64 else 1e-5
        assert np.abs(seg - want).max() <= tol * max(np.abs(want).max(), 1e-300), p.name
        om.close()
