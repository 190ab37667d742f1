"""Helpers for the GPU parity tests: run the library step by step with its
per-node debug outputs, run the oracle on the same seeded inputs, compare."""
import numpy as np

import oracle
import paper_2104_09189_gb300 as sl

REL_TOL_FP64 = 1e-12          # normwise relative, at every step
FOOT_DELTA = 1e-12            # feet may differ by rounding of the field's
                              # trig functions (CUDA vs libm): triangles of
                              # feet closer than this to an edge line may differ


class DeviceRun:
    """A single-problem mesh on the GPU, optionally renumbered, with the
    permutations kept so results can be compared in the original numbering."""

    def __init__(self, mesh, field, dt, curve=sl.SL_CURVE_NONE, seed=1, precision=sl.SL_FP64, kernel=0):
        import torch
        self.torch = torch
        self.mesh, self.field, self.dt = mesh, field, dt
        no, to, xy, tri = sl.pack_meshes([(mesh.xy, mesh.tri)])
        self.h = sl.sl_mesh_create(no, to, xy, tri, precision=precision, seed=seed)
        if kernel:
            sl.sl_mesh_set_option(self.h, sl.SL_OPT_KERNEL, kernel)
        n, nt = mesh.n_nodes, mesh.n_tri
        if curve != sl.SL_CURVE_NONE:
            self.node_perm, self.tri_perm = sl.sl_mesh_reorder(self.h, curve)
        else:
            self.node_perm, self.tri_perm = np.arange(n, dtype=np.int32), np.arange(nt, dtype=np.int32)
        self.probs = sl.problems([(field.kind, dt, field.packed())])
        self.dev = torch.device("cuda:0")
        self.vt = torch.float64 if precision == sl.SL_FP64 else torch.float32

    def close(self):
        if self.h:
            sl.sl_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def to_dev(self, v_orig):
        return self.torch.tensor(np.asarray(v_orig)[self.node_perm], dtype=self.vt, device=self.dev)

    def from_dev(self, v_dev):
        out = np.empty(self.mesh.n_nodes, dtype=np.float64)
        out[self.node_perm] = v_dev.double().cpu().numpy()
        return out

    def step(self, n, v_dev):
        """One sl_step with debug outputs; returns (v_out_dev, dict in original numbering)."""
        t = self.torch
        N = self.mesh.n_nodes
        vout = t.empty_like(v_dev)
        dbg = {"feet": t.zeros(2 * N, dtype=t.float64, device=self.dev),
               "tri": t.full((N,), -7, dtype=t.int32, device=self.dev),
               "moves": t.zeros(N, dtype=t.int32, device=self.dev),
               "flags": t.zeros(N, dtype=t.uint8, device=self.dev)}
        sl.sl_step(self.h, self.probs, n, v_dev, vout, debug=dbg)
        sl.sl_mesh_status(self.h)
        res = {}
        feet = np.empty((N, 2))
        feet[self.node_perm] = dbg["feet"].cpu().numpy().reshape(N, 2)
        tri = np.empty(N, dtype=np.int64)
        d = dbg["tri"].cpu().numpy()
        tri[self.node_perm] = np.where(d < 0, -1, self.tri_perm[np.maximum(d, 0)])   # -1: excluded
        moves = np.empty(N, dtype=np.int64)
        moves[self.node_perm] = dbg["moves"].cpu().numpy()
        flags = np.empty(N, dtype=np.uint8)
        flags[self.node_perm] = dbg["flags"].cpu().numpy()
        res.update(feet=feet, tri=tri, moves=moves, flags=flags, v=self.from_dev(vout))
        return vout, res


def compare_step(om, gpu, orc_v, orc_tri, orc_feet, rel_tol=REL_TOL_FP64, delta=FOOT_DELTA):
    """Value parity (normwise relative) and triangle parity: exact for feet
    farther than `delta` from every edge line of the oracle's triangle;
    closer feet (on or next to an edge or a vertex) are counted and the GPU's
    triangle must contain the oracle's foot up to `delta`.
    Returns (max relative error, number of near-degenerate feet)."""
    scale = max(np.abs(orc_v).max(), 1e-300)
    err = np.abs(gpu["v"] - orc_v).max() / scale
    assert err <= rel_tol, f"value error {err:.3e} > {rel_tol:.1e}"
    margin = om.margins(orc_tri.astype(np.int32), orc_feet)
    safe = margin > delta
    bad = np.nonzero(safe & (gpu["tri"] != orc_tri))[0]
    assert bad.size == 0, f"{bad.size} non-degenerate feet located in a different triangle, e.g. node {bad[:5]}"
    near = np.nonzero(~safe)[0]
    if near.size:
        m2 = om.margins(gpu["tri"][near].astype(np.int32), orc_feet[near])
        assert np.all(m2 >= -delta), f"GPU triangle does not contain the foot for nodes {near[m2 < -delta][:5]}"
    return err, int(near.size)
