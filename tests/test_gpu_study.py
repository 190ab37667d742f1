"""GPU tests of the paper's experimental setup (Sec. 4): exclusion of the
nodes whose foot leaves the domain, and the start strategies (a) and (b) of
Sec. 3.  Results must not depend on the strategy: the walk locates the
triangle that contains the foot whichever triangle it starts from."""
import numpy as np
import pytest

import oracle
import paper_2104_09189_gb300 as sl
import sl_inputs as si
from gpu_helpers import REL_TOL_FP64, DeviceRun, exact_triangle_parity

pytestmark = pytest.mark.gpu


def _bump(xy):
    return np.exp(-((xy[:, 0] - 0.45) ** 2 + (xy[:, 1] - 0.6) ** 2) / (2 * 0.12 ** 2))


@pytest.mark.parametrize("kernel", [1, 2], ids=["plain", "fast"])
def test_exclusion_matches_the_oracle(kernel):
    m = si.grid_mesh(96, 0.25, 11)
    f = si.paper_field(2 * np.pi, 2 * np.pi)
    dt = 0.04
    om = oracle.OracleMesh(m.xy, m.tri)
    g = DeviceRun(m, f, dt, curve=sl.SL_CURVE_HILBERT, kernel=kernel)
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_OUTSIDE, 1)
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_STATS, 1)
    sl.sl_mesh_stats(g.h, reset=True)
    vo = _bump(m.xy)
    v = g.to_dev(vo)
    n_out = 0
    for n in range(4):
        v_prev = g.from_dev(v)
        v, res = g.step(n, v)
        ov, otri, ofl, oft = om.step(f.kind, f.packed(), dt, n, vo, exclude=True)
        out = (ofl & oracle.FLAG_EXCLUDED) != 0
        gout = (res["flags"] & sl.SL_NODE_EXCLUDED) != 0
        # no unclipped foot within rounding of the boundary, so the decisions agree exactly
        margin = np.minimum(np.minimum(np.abs(oft[:, 0]), np.abs(oft[:, 0] - 1)),
                            np.minimum(np.abs(oft[:, 1]), np.abs(oft[:, 1] - 1)))
        assert margin.min() > 1e-12
        assert np.array_equal(out, gout)
        assert out.sum() > 0.02 * m.n_nodes
        n_out += int(out.sum())
        # excluded: V unchanged (bitwise in double; the fast kernel carries
        # values as (hi, lo) float pairs, a 48-bit significand)
        if kernel == 1:
            assert np.array_equal(res["v"][out], v_prev[out])
        else:
            assert np.all(np.abs(res["v"][out] - v_prev[out]) <= 2.0 ** -46 * np.abs(v_prev[out]))
        assert np.all(res["tri"][out] == -1)
        keep = ~out
        err = np.abs(res["v"][keep] - ov[keep]).max() / np.abs(ov).max()
        assert err <= REL_TOL_FP64
        exact_triangle_parity(om, res["tri"], res["feet"], res["feet_lo"], res["flags"], keep=keep)
        vo = ov
    st = sl.sl_mesh_stats(g.h)
    assert st["excluded"] == n_out
    assert st["node_updates"] == 4 * m.n_nodes
    g.close()


@pytest.mark.parametrize("prec", [sl.SL_FP64, sl.SL_FP32], ids=["fp64", "fp32"])
def test_strategy_a_locates_the_same_triangles_with_more_hops(prec):
    # Courant 6.4: (a) walks ~ the whole characteristic every step, (b) only
    # the foot's drift ~ L_t dt^2 / h (Sec. 4)
    m = si.grid_mesh(128, 0.25, 12)
    f = si.paper_field(2 * np.pi, 2 * np.pi)
    dt = 0.05
    runs = {}
    for strategy in (0, 1):
        g = DeviceRun(m, f, dt, curve=sl.SL_CURVE_HILBERT, precision=prec)
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_STRATEGY, strategy)
        t0_init = g.torch.empty(m.n_nodes, dtype=g.torch.int32, device=g.dev)
        sl.sl_mesh_get_t0(g.h, t0_init)
        v = g.to_dev(_bump(m.xy))
        hist = []
        for n in range(6):
            v, res = g.step(n, v)
            hist.append(res)
        t0_end = g.torch.empty_like(t0_init)
        sl.sl_mesh_get_t0(g.h, t0_end)
        runs[strategy] = (hist, bool(g.torch.equal(t0_init, t0_end)))
        g.close()
    hb, b_kept = runs[0]
    ha, a_kept = runs[1]
    assert a_kept and not b_kept          # (a) never overwrites T^0 (Sec. 3); (b) does
    for n, (rb, ra) in enumerate(zip(hb, ha)):
        clean = ((rb["flags"] | ra["flags"]) & sl.SL_NODE_DEGENERATE) == 0
        assert np.array_equal(rb["tri"][clean], ra["tri"][clean])
        tol = REL_TOL_FP64 if prec == sl.SL_FP64 else 1e-6
        assert np.abs(rb["v"] - ra["v"]).max() <= tol * np.abs(rb["v"]).max()
        if n == 0:
            # the first step: (a) and (b) coincide (Sec. 3)
            assert np.array_equal(rb["moves"], ra["moves"])
        else:
            # later steps: (b) starts next to the foot, (a) at the node
            assert ra["moves"].mean() > 1.5 * rb["moves"].mean()
    # (a) walks the same path every step for a time-constant reach: step 1 vs
    # step 2 hop counts differ only through the field's time dependence
    assert ha[1]["moves"].mean() > 0.5 * ha[0]["moves"].mean()


def test_strategy_option_resets_t0():
    m = si.grid_mesh(48, 0.25, 13)
    f = si.rotation_field()
    g = DeviceRun(m, f, 0.03)
    t0_init = g.torch.empty(m.n_nodes, dtype=g.torch.int32, device=g.dev)
    sl.sl_mesh_get_t0(g.h, t0_init)
    v = g.to_dev(_bump(m.xy))
    for n in range(2):
        v, _ = g.step(n, v)
    t0 = g.torch.empty_like(t0_init)
    sl.sl_mesh_get_t0(g.h, t0)
    assert not g.torch.equal(t0, t0_init)
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_STRATEGY, 1)
    sl.sl_mesh_get_t0(g.h, t0)
    assert g.torch.equal(t0, t0_init)
    with pytest.raises(sl.SLError):
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_STRATEGY, 2)
    with pytest.raises(sl.SLError):
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_OUTSIDE, 5)
    g.close()


def test_courant_study_shows_the_paper_trends():
    """Sec. 4: hops of strategy (a) grow linearly with the Courant number,
    those of (b) grow like L_t alpha^2 dx and stay below (a) while
    L_t alpha dx < 1; a larger L_t costs (b) more hops."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    p = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--study", "courant", "--study-cells", "64"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert p.returncode == 0, p.stderr[-2000:]
    d = json.loads(p.stdout.strip().splitlines()[-1])

    def hops(lt, strategy):
        r = [x for x in d["rows"] if x["Lt"] == lt and x["strategy"] == strategy]
        return np.array([x["alpha"] for x in r]), np.array([x["mean_hops"] for x in r])

    al, a2 = hops("2pi", "a")
    _, b2 = hops("2pi", "b")
    _, b8 = hops("8pi", "b")
    big = al >= 1
    assert np.all(np.diff(a2[big]) > 0)
    mid = (al >= 2) & (al <= 6)              # L_t alpha dx < 1 for L_t = 2 pi, dx = 1/64
    assert np.all(b2[mid] < a2[mid])
    assert b8[mid].mean() > b2[mid].mean()
    # (c): nearly flat in alpha while L_x dt < 1 (the uniform bound of Sec. 3)
    _, c2 = hops("2pi", "c")
    flat = (al >= 1) & (al <= 6)
    assert c2[flat].max() < 2.0 * c2[flat].min() + 0.5
    assert np.all(c2[al >= 8] < a2[al >= 8])
    assert all(0.0 <= x["excluded_fraction"] < 1.0 for x in d["rows"])


@pytest.mark.parametrize("kernel,prec,curve,shuffle", [
    (2, sl.SL_FP64, sl.SL_CURVE_HILBERT, False),
    (1, sl.SL_FP64, sl.SL_CURVE_NONE, False),
    (2, sl.SL_FP64, sl.SL_CURVE_NONE, True),
    (0, sl.SL_FP32, sl.SL_CURVE_MORTON, False),
], ids=["fast-hilbert", "plain", "fast-shuffled", "fp32-morton"])
def test_direct_location_on_the_courant_grid(kernel, prec, curve, shuffle):
    """Strategy 2: the walk starts at the triangle of the paper's direct
    formula (Sec. 4); results equal the oracle's and almost no walk is left."""
    from sl_inputs.meshes import shuffled
    M = 80
    m = si.courant_grid(M)
    if shuffle:
        m = shuffled(m, 5)
    f = si.paper_field(2 * np.pi, 2 * np.pi)
    dt = 5.0 / M
    om = oracle.OracleMesh(m.xy, m.tri)
    g = DeviceRun(m, f, dt, curve=curve, kernel=kernel, precision=prec)
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_STRATEGY, 2)
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_OUTSIDE, 1)
    vo = _bump(m.xy)
    v = g.to_dev(vo)
    hops = []
    for n in range(3):
        v, res = g.step(n, v)
        if prec == sl.SL_FP64:
            ov, otri, ofl, oft = om.step(f.kind, f.packed(), dt, n, vo, exclude=True)
            out = (ofl & oracle.FLAG_EXCLUDED) != 0
            assert np.array_equal(out, (res["flags"] & sl.SL_NODE_EXCLUDED) != 0)
            keep = ~out
            assert np.abs(res["v"][keep] - ov[keep]).max() <= REL_TOL_FP64 * np.abs(ov).max()
            exact_triangle_parity(om, res["tri"], res["feet"], res["feet_lo"], res["flags"], keep=keep)
            vo = ov
        else:
            # FP32: a node is excluded when its own float foot (reported
            # unclipped) leaves the square, which agrees with the double
            # Euler foot wherever that is farther than float rounding from
            # the boundary; the kept feet are located exactly on the
            # float-rounded mesh
            xy32 = m.xy.astype(np.float32)
            om32 = oracle.OracleMesh(xy32.astype(np.float64), m.tri)
            out = (res["flags"] & sl.SL_NODE_EXCLUDED) != 0
            ft = res["feet"]
            assert np.array_equal(out, ~((ft >= 0.0) & (ft <= 1.0)).all(axis=1))
            _, _, ofl, oft = om32.step(f.kind, f.packed(), dt, n, vo, exclude=True)
            margin = np.minimum(np.abs(oft), np.abs(oft - 1.0)).min(axis=1)
            sure = margin > 8 * 2.0 ** -24
            assert np.array_equal(out[sure], ((ofl & oracle.FLAG_EXCLUDED) != 0)[sure])
            exact_triangle_parity(om32, res["tri"], ft, None, res["flags"], keep=~out)
            om32.close()
        hops.append(res["moves"][(res["flags"] & sl.SL_NODE_EXCLUDED) == 0].mean())
    assert max(hops) < 0.01
    g.close()


def test_direct_location_rejects_other_meshes():
    m = si.grid_mesh(32, 0.25, 3)
    g = DeviceRun(m, si.rotation_field(), 0.01)
    with pytest.raises(sl.SLError):
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_STRATEGY, 2)
    g.close()
    # a Courant grid keeps its table through a renumbering
    c = si.courant_grid(24)
    g = DeviceRun(c, si.rotation_field(), 0.01)
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_STRATEGY, 2)
    sl.sl_mesh_reorder(g.h, sl.SL_CURVE_HILBERT)
    g.close()


@pytest.mark.parametrize("kernel,prec", [(2, sl.SL_FP64), (1, sl.SL_FP64), (0, sl.SL_FP32)],
                         ids=["fast", "plain", "fp32"])
def test_strategy_c_matches_the_oracle_and_walks_little(kernel, prec):
    """Strategy (c) (Sec. 3): every node starts at its spanning-tree parent's
    triangle of the same step.  Results equal the oracle's, T^0 holds every
    node's own foot triangle, and the walks stay short (the feet of
    neighbouring nodes are within (1 + L_x dt) dx of each other)."""
    m = si.grid_mesh(72, 0.25, 21)
    f = si.paper_field(2 * np.pi, 2 * np.pi)
    dt = 6.0 / 72
    om = oracle.OracleMesh(m.xy, m.tri)
    g = DeviceRun(m, f, dt, curve=sl.SL_CURVE_HILBERT, kernel=kernel, precision=prec)
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_STRATEGY, 3)
    vo = _bump(m.xy)
    v = g.to_dev(vo)
    t0 = g.torch.empty(m.n_nodes, dtype=g.torch.int32, device=g.dev)
    for n in range(3):
        v, res = g.step(n, v)
        if prec == sl.SL_FP64:
            ov, otri, ofl, oft = om.step(f.kind, f.packed(), dt, n, vo)
            assert np.abs(res["v"] - ov).max() <= REL_TOL_FP64 * np.abs(ov).max()
            exact_triangle_parity(om, res["tri"], res["feet"], res["feet_lo"], res["flags"])
            vo = ov
        # T^0_i is the triangle located for node i (Algorithm 1, strategy (c))
        sl.sl_mesh_get_t0(g.h, t0)
        got = np.empty(m.n_nodes, dtype=np.int64)
        got[g.node_perm] = g.tri_perm[t0.cpu().numpy()]
        assert np.array_equal(got, res["tri"])
        if n > 0:
            assert res["moves"].mean() < 3.0
    g.close()


def test_strategy_c_on_a_batch_with_exclusion():
    """Tree levels of several problems run together; exclusion passes the
    parent's start on to the children.  Values equal the oracle's."""
    probs = si.batch_config(5, nmin=2e3, nmax=3e4, steps=3)
    meshes = [(p.mesh.xy, p.mesh.tri) for p in probs]
    no, to, xy, tri = sl.pack_meshes(meshes)
    import torch
    h = sl.sl_mesh_create(no, to, xy, tri)
    sl.sl_mesh_set_option(h, sl.SL_OPT_STRATEGY, 3)
    sl.sl_mesh_set_option(h, sl.SL_OPT_OUTSIDE, 1)
    pr = sl.problems([(p.field.kind, 2.0 * p.dt, p.field.packed()) for p in probs])
    v = torch.tensor(np.concatenate([p.v0 for p in probs]), dtype=torch.float64, device="cuda:0")
    w = torch.empty_like(v)
    sl.sl_run(h, pr, 0, 3, v, w, use_graph=True)        # (c) runs eagerly whatever use_graph says
    got = v.cpu().numpy()
    sl.sl_mesh_destroy(h)
    for k, p in enumerate(probs):
        om = oracle.OracleMesh(p.mesh.xy, p.mesh.tri)
        want = om.run(p.field.kind, p.field.packed(), 2.0 * p.dt, 0, 3, p.v0, exclude=True)
        seg = got[no[k]:no[k + 1]]
        assert np.abs(seg - want).max() <= 1e-12 * np.abs(want).max()
