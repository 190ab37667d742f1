"""Helpers for the GPU parity tests: run the library step by step with its
per-node debug outputs, run the oracle on the same seeded inputs, compare."""
import numpy as np

import oracle
import paper_2104_09189_gb300 as sl

REL_TOL_FP64 = 1e-12          # normwise relative, at every step
FOOT_TOL_FP64 = 1e-12         # the GPU's foot against the oracle's: both are
                              # Eq. 4 in (about) double precision; they differ
                              # by rounding and by the trig functions of CUDA
                              # and libm, never by more than this
ON_EDGE = oracle.FLAG_DEGENERATE | oracle.FLAG_MULTI
NODE_DEGENERATE = 2           # SL_NODE_DEGENERATE

REPORT = []                   # (test, figures) lines printed at the end of the run


def report(name, **figures):
    """Record figures of a parity test (error, feet on an edge or vertex) for
    the summary printed at the end of the pytest run."""
    REPORT.append((name, figures))


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
               "feet_lo": t.full((2 * N,), 7.0, dtype=t.float64, device=self.dev),
               "tri": t.full((N,), -7, dtype=t.int32, device=self.dev),
               "moves": t.zeros(N, dtype=t.int32, device=self.dev),
               "flags": t.zeros(N, dtype=t.uint8, device=self.dev)}
        sl.sl_step(self.h, self.probs, n, v_dev, vout, debug=dbg)
        sl.sl_mesh_status(self.h)
        res = {}
        feet = np.empty((N, 2))
        feet[self.node_perm] = dbg["feet"].cpu().numpy().reshape(N, 2)
        feet_lo = np.empty((N, 2))
        feet_lo[self.node_perm] = dbg["feet_lo"].cpu().numpy().reshape(N, 2)
        tri = np.empty(N, dtype=np.int64)
        d = dbg["tri"].cpu().numpy()
        tri[self.node_perm] = np.where(d < 0, -1, self.tri_perm[np.maximum(d, 0)])   # -1: excluded
        moves = np.empty(N, dtype=np.int64)
        moves[self.node_perm] = dbg["moves"].cpu().numpy()
        flags = np.empty(N, dtype=np.uint8)
        flags[self.node_perm] = dbg["flags"].cpu().numpy()
        res.update(feet=feet, feet_lo=feet_lo, tri=tri, moves=moves, flags=flags, v=self.from_dev(vout))
        return vout, res


def exact_triangle_parity(om, tri, feet, feet_lo=None, gpu_flags=None, keep=None):
    """Triangle parity on the GPU's own feet, with no tolerance.

    The oracle locates exactly the point each GPU thread located (feet +
    feet_lo, summed exactly).  A foot strictly inside one triangle (neither
    DEGENERATE nor MULTI) must be in the GPU's triangle: the same index.  A
    foot on an edge or a vertex, where several triangles are correct
    (reading c4), must be contained in the GPU's triangle: its three exact
    orientation signs >= 0.  With gpu_flags, the GPU's SL_NODE_DEGENERATE bit
    must be set exactly where a sign of its triangle is zero.  keep selects
    the nodes to check (excluded nodes have no triangle).
    Returns the number of feet on an edge or a vertex."""
    idx = np.arange(len(tri)) if keep is None else np.nonzero(keep)[0]
    q = feet[idx]
    ql = None if feet_lo is None else feet_lo[idx]
    otri, oflags = om.locate(q, ql)
    on_edge = (oflags & ON_EDGE) != 0
    gt = np.asarray(tri)[idx]
    bad = np.nonzero(~on_edge & (gt != otri))[0]
    assert bad.size == 0, (f"{bad.size} feet strictly inside a triangle located elsewhere, e.g. nodes "
                           f"{idx[bad[:5]]}: GPU {gt[bad[:5]]} oracle {otri[bad[:5]]}")
    sg = om.signs(gt.astype(np.int32), q, ql)
    outside = np.nonzero((sg < 0).any(axis=1))[0]
    assert outside.size == 0, f"GPU triangle does not contain the foot of nodes {idx[outside[:5]]}"
    if gpu_flags is not None:
        zero = (sg == 0).any(axis=1)
        gdeg = (np.asarray(gpu_flags)[idx] & NODE_DEGENERATE) != 0
        wrong = np.nonzero(zero != gdeg)[0]
        assert wrong.size == 0, f"SL_NODE_DEGENERATE differs from the exact signs at nodes {idx[wrong[:5]]}"
    return int(on_edge.sum())


def compare_step(om, gpu, orc_v, orc_feet=None, rel_tol=REL_TOL_FP64, foot_tol=FOOT_TOL_FP64, keep=None):
    """One step of the GPU against the oracle: the values normwise (relative
    to max |V|), the feet to rounding, and the located triangles exactly
    (exact_triangle_parity on the GPU's feet).
    Returns (max relative value error, number of feet on an edge or vertex)."""
    scale = max(np.abs(orc_v).max(), 1e-300)
    err = np.abs(gpu["v"] - orc_v).max() / scale
    assert err <= rel_tol, f"value error {err:.3e} > {rel_tol:.1e}"
    sel = slice(None) if keep is None else keep
    if orc_feet is not None:
        d = np.abs(gpu["feet"][sel] - orc_feet[sel]).max()
        assert d <= foot_tol, f"foot differs from the oracle's by {d:.3e}"
    on_edge = exact_triangle_parity(om, gpu["tri"], gpu["feet"], gpu.get("feet_lo"), gpu.get("flags"), keep)
    return err, on_edge
