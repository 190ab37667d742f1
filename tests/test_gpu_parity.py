"""GPU path vs the CPU oracle, through the C ABI (sl_step / sl_run).

Values: normwise relative error <= 1e-12 at every step (FP64).
Triangles: the oracle locates the GPU's own feet exactly; a foot strictly
inside a triangle must be located in that triangle, a foot on an edge or a
vertex (counted) must lie in the GPU's triangle by the exact signs.
"""
import numpy as np
import pytest

import oracle
import paper_2104_09189_gb300 as sl
import sl_inputs as si
from gpu_helpers import DeviceRun, compare_step, exact_triangle_parity

pytestmark = pytest.mark.gpu


def _parity_run(prob, steps, curve=sl.SL_CURVE_NONE, kernel=0, seed=1, check_every=1):
    mesh = prob.mesh
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    g = DeviceRun(mesh, prob.field, prob.dt, curve=curve, kernel=kernel, seed=seed)
    v_dev = g.to_dev(prob.v0)
    v_orc = prob.v0.copy()
    worst, near_total = 0.0, 0
    for n in range(steps):
        v_dev, res = g.step(n, v_dev)
        ov, otri, oflags, ofeet = om.step(prob.field.kind, prob.field.packed(), prob.dt, n, v_orc)
        v_orc = ov
        if n % check_every == 0 or n == steps - 1:
            err, near = compare_step(om, res, ov, ofeet)
            worst = max(worst, err)
            near_total += near
    g.close()
    return worst, near_total, res


KERNELS = [pytest.param(1, id="plain"), pytest.param(2, id="fast")]


@pytest.mark.parametrize("kernel", [1, 2], ids=["plain", "fast"])
def test_c1_swirl_full_parity(kernel):
    prob = si.config("C1")
    worst, near, res = _parity_run(prob, prob.n_steps, kernel=kernel)
    assert worst <= 1e-12
    # boundary nodes of the swirl have f = 0 (or ~1e-16): their feet are
    # vertices and must be flagged degenerate
    assert near >= 4 * 64


@pytest.mark.parametrize("kernel", [1, 2], ids=["plain", "fast"])
@pytest.mark.parametrize("curve", [sl.SL_CURVE_NONE, sl.SL_CURVE_HILBERT, sl.SL_CURVE_MORTON])
def test_c2_construction_swirl_parity(curve, kernel):
    prob = si.config("C2", M=256)
    _parity_run(prob, 6, curve=curve, kernel=kernel)


@pytest.mark.parametrize("kernel", [1, 2], ids=["plain", "fast"])
def test_c2_full_size_parity_hilbert(kernel):
    prob = si.config("C2")
    _parity_run(prob, 3, curve=sl.SL_CURVE_HILBERT, kernel=kernel)


@pytest.mark.parametrize("kernel", [1, 2], ids=["plain", "fast"])
def test_c3_construction_rotation_parity_and_zero_hops(kernel):
    """Graded mesh, solid rotation.  The plain kernel computes the feet with
    the same rounded operations as the oracle, so they agree bit for bit; the
    fast kernel's double-float feet agree to rounding.  A time-constant field
    needs no walk move after the first step (Sec. 3, strategy (b))."""
    prob = si.config("C3", M=256)
    mesh = prob.mesh
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    g = DeviceRun(mesh, prob.field, prob.dt, curve=sl.SL_CURVE_HILBERT, kernel=kernel)
    v_dev = g.to_dev(prob.v0)
    v_orc = prob.v0.copy()
    for n in range(4):
        v_dev, res = g.step(n, v_dev)
        ov, otri, oflags, ofeet = om.step(prob.field.kind, prob.field.packed(), prob.dt, n, v_orc)
        v_orc = ov
        if kernel == 1:
            assert np.array_equal(res["feet"], ofeet)
            compare_step(om, res, ov, ofeet, foot_tol=0.0)
        else:
            assert np.abs(res["feet"] - ofeet).max() < 1e-13   # double-float feet: ~2^-46
            compare_step(om, res, ov, ofeet)
        if n == 0:
            assert res["moves"].mean() > 5      # strategy (a) on the first step: ~ Courant number
        else:
            assert res["moves"].max() == 0
    g.close()


@pytest.mark.parametrize("kernel", [1, 2], ids=["plain", "fast"])
def test_other_fields_parity(kernel):
    mesh = si.grid_mesh(96, 0.25, 12)
    v0 = si.gaussian(mesh.xy, 0.45, 0.55, 0.1)
    p = np.zeros(48)
    p[:8] = (0.3, -1.0, 0.5, 2.0, -0.2, 0.7, 0.4, -1.5)
    for fld, dt in [(si.fourier8_field(77), 0.03), (si.paper_field(), 0.02), (si.swirl_field(), 0.1),
                    (si.Field(si.FIELD_AFFINE, p, 3.0), 0.05), (si.rotation_field(3.0, 0.3, 0.6), 0.04)]:
        prob = si.Problem("x", mesh, fld, dt, 4, v0, "fp64", 12)
        _parity_run(prob, 4, kernel=kernel)


@pytest.mark.parametrize("kernel", [1, 2], ids=["plain", "fast"])
def test_linear_data_closed_form_on_gpu(kernel):
    """Contracting affine field with linear data: V^n = u0(c + (1-k dt)^n (x - c))."""
    mesh = si.grid_mesh(128, 0.25, 4)
    k, cx, cy, dt, steps = 3.0, 0.4, 0.6, 0.05, 10
    p = np.zeros(48)
    p[:8] = (-k * cx, k, 0.0, 0.0, -k * cy, 0.0, k, 0.0)
    fld = si.Field(si.FIELD_AFFINE, p, 1.0)
    g = DeviceRun(mesh, fld, dt, curve=sl.SL_CURVE_HILBERT, kernel=kernel)
    lin = lambda q: 0.25 + q[:, 0] - 0.5 * q[:, 1]
    v = g.to_dev(lin(mesh.xy))
    w = g.torch.empty_like(v)
    sl.sl_run(g.h, g.probs, 0, steps, v, w, use_graph=True)
    r = (1 - k * dt) ** steps
    want = lin(np.stack([cx + r * (mesh.xy[:, 0] - cx), cy + r * (mesh.xy[:, 1] - cy)], 1))
    assert np.abs(g.from_dev(v) - want).max() < 1e-13
    g.close()


def test_zero_field_leaves_values_bitwise():
    """f = 0: every foot is its own node.  Both kernels return each node's
    own value and flag every foot degenerate (it lies on a vertex of its
    start triangle, an incident triangle of the node).  The plain kernel
    reproduces V bit for bit; the fast kernel takes a foot equal to its
    node's coordinate pair as the node, walks no step, and returns the value
    as it holds it between steps, a (hi, lo) float pair: V rounded to the
    pair, bit for bit."""
    mesh = si.grid_mesh(64, 0.25, 2)
    v0 = si.cosine_bump(mesh.xy)
    g = DeviceRun(mesh, si.zero_field(), 0.1, kernel=1)
    v_dev = g.to_dev(v0)
    for n in range(3):
        v_dev, res = g.step(n, v_dev)
        assert np.array_equal(res["v"], v0)
        assert np.all(res["flags"] & sl.SL_NODE_DEGENERATE)
    g.close()
    hi = v0.astype(np.float32).astype(np.float64)
    v_pair = hi + (v0 - hi).astype(np.float32).astype(np.float64)
    assert np.abs(v_pair - v0).max() <= 2.0 ** -48 * np.abs(v0).max()
    for split in (0, 1):
        g = DeviceRun(mesh, si.zero_field(), 0.1, kernel=2)
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_SPLIT, split)
        v_dev = g.to_dev(v0)
        for n in range(3):
            v_dev, res = g.step(n, v_dev)
            assert np.array_equal(res["v"], v_pair)
            assert np.all(res["flags"] & sl.SL_NODE_DEGENERATE)
            assert not np.any(res["flags"] & sl.SL_NODE_EXACT)
            assert np.all(res["moves"] == 0)
            assert np.all(np.any(mesh.tri[res["tri"]] == np.arange(mesh.n_nodes)[:, None], axis=1))
            assert np.abs(res["feet"] - mesh.xy).max() <= 2.0 ** -48
        g.close()


def test_value_pairs_round_to_nearest_at_every_magnitude():
    """The fast FP64 path carries V as (hi, lo) float pairs: hi = V rounded to
    the nearest float (ties to even), lo = V - hi rounded likewise, and back
    as hi + lo in double.  With f = 0 every value comes back as that round
    trip; checked bit for bit against numpy's conversions on values of every
    magnitude from 2^-1000 to 2^126, exact ties, both signs, zero and the
    subnormal range, in sl_step and in a graph-recorded sl_run."""
    mesh = si.grid_mesh(64, 0.25, 2)
    n = mesh.n_nodes
    rng = np.random.default_rng(7)
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-1000, 127, n)
    v = np.ldexp(mant, expo) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    # exact ties of the float rounding (a float plus half its ulp), either parity
    k = n // 8
    base = np.ldexp(rng.uniform(1.0, 2.0, k).astype(np.float32).astype(np.float64), rng.integers(-60, 100, k))
    v[:k] = base + np.ldexp(np.float64(1.0), np.frexp(base)[1] - 25)
    v[k] = 0.0
    v[k + 1] = -0.0
    v[k + 2] = 5e-324
    v[k + 3] = 2.0 ** -75 * 1.75
    v[k + 4] = 2.0 ** -74 * 1.25
    v[k + 5] = (2.0 - 2.0 ** -52) * 2.0 ** 126
    hi = v.astype(np.float32).astype(np.float64)
    want = hi + (v - hi).astype(np.float32).astype(np.float64)
    g = DeviceRun(mesh, si.zero_field(), 0.1, kernel=2)
    vd = g.to_dev(v)
    _, res = g.step(0, vd)
    assert np.array_equal(res["v"].view(np.int64), want.view(np.int64))
    w = g.torch.empty_like(vd)
    vd = g.to_dev(v)
    sl.sl_run(g.h, g.probs, 0, 2, vd, w, use_graph=True)
    assert np.array_equal(g.from_dev(vd).view(np.int64), want.view(np.int64))
    g.close()


def test_async_runs_queue_back_to_back_with_the_same_results():
    """SL_OPT_ASYNC = 1: sl_run without statistics returns before its steps
    finish; several runs queued back to back end with the values of
    synchronous runs, and sl_mesh_status reports the device status."""
    prob = si.config("C2", M=128)
    outs = []
    for asy in (0, 1):
        g = DeviceRun(prob.mesh, prob.field, prob.dt, curve=sl.SL_CURVE_HILBERT)
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_ASYNC, asy)
        v = g.to_dev(prob.v0)
        w = g.torch.empty_like(v)
        for _ in range(3):
            sl.sl_mesh_reset_t0(g.h)
            assert sl.sl_run(g.h, g.probs, 0, 4, v, w, stats=False) is None
        sl.sl_mesh_status(g.h)
        outs.append(g.from_dev(v))
        g.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("kernel", [1, 2], ids=["plain", "fast"])
def test_graph_eager_reorder_and_resume_are_bitwise_identical(kernel):
    prob = si.config("C2", M=192)
    mesh = prob.mesh
    outs = []
    for curve, graph in [(sl.SL_CURVE_NONE, False), (sl.SL_CURVE_NONE, True), (sl.SL_CURVE_HILBERT, True),
                         (sl.SL_CURVE_MORTON, False)]:
        g = DeviceRun(mesh, prob.field, prob.dt, curve=curve, kernel=kernel)
        v = g.to_dev(prob.v0)
        w = g.torch.empty_like(v)
        sl.sl_run(g.h, g.probs, 0, 7, v, w, use_graph=graph)
        outs.append(g.from_dev(v))
        g.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    # resume: 3 steps, export T^0 and V; a new handle imports them and runs
    # 4 more steps, exactly like the first handle continuing
    g = DeviceRun(mesh, prob.field, prob.dt, kernel=kernel)
    v = g.to_dev(prob.v0)
    w = g.torch.empty_like(v)
    sl.sl_run(g.h, g.probs, 0, 3, v, w)
    t0 = g.torch.empty(mesh.n_nodes, dtype=g.torch.int32, device=g.dev)
    sl.sl_mesh_get_t0(g.h, t0)
    v_resume = v.clone()
    sl.sl_run(g.h, g.probs, 3, 4, v, w)
    g2 = DeviceRun(mesh, prob.field, prob.dt, kernel=kernel)
    sl.sl_mesh_set_t0(g2.h, t0)
    sl.sl_run(g2.h, g2.probs, 3, 4, v_resume, w)
    assert np.array_equal(g2.from_dev(v_resume), g.from_dev(v))
    if kernel == 1:
        assert np.array_equal(g.from_dev(v), outs[0])
    else:
        assert np.abs(g.from_dev(v) - outs[0]).max() <= 1e-14
    g.close()
    g2.close()


@pytest.mark.parametrize("precision", [sl.SL_FP64, sl.SL_FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("steps", [5, 6])
def test_run_host_matches_device_run(precision, steps):
    """sl_run_host on pageable and on page-locked host memory, recorded and
    eager: bitwise the device run, for an odd and an even number of steps,
    and again on the same handle."""
    import torch
    prob = si.config("C1")
    dt = np.float64 if precision == sl.SL_FP64 else np.float32
    g = DeviceRun(prob.mesh, prob.field, prob.dt, precision=precision)
    v = g.to_dev(prob.v0)
    w = g.torch.empty_like(v)
    sl.sl_run(g.h, g.probs, 0, steps, v, w)
    dev_result = g.from_dev(v)
    g.close()
    for pinned in (False, True):
        for use_graph in (True, False):
            g = DeviceRun(prob.mesh, prob.field, prob.dt, precision=precision)
            for _ in range(2):
                sl.sl_mesh_reset_t0(g.h)
                if pinned:
                    host = torch.tensor(prob.v0.astype(dt)).pin_memory().numpy()
                else:
                    host = prob.v0.astype(dt).copy()
                sl.sl_run_host(g.h, g.probs, 0, steps, host, use_graph=use_graph)
                assert np.array_equal(host.astype(np.float64), dev_result), (pinned, use_graph)
            g.close()


@pytest.mark.parametrize("kernel", [1, 2], ids=["plain", "fast"])
def test_walk_cap_reports_status_without_hanging(kernel):
    """A tiny hop cap (debug knob) must end in SL_E_WALK_LIMIT, not a hang."""
    prob = si.config("C2", M=128)
    g = DeviceRun(prob.mesh, prob.field, prob.dt, kernel=kernel)
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_WALK_CAP, 1)
    v = g.to_dev(prob.v0)
    w = g.torch.empty_like(v)
    with pytest.raises(sl.SLError) as e:
        sl.sl_run(g.h, g.probs, 0, 1, v, w, use_graph=False)
    assert e.value.status == sl.SL_E_WALK_LIMIT
    # the handle stays usable
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_WALK_CAP, 0)
    sl.sl_run(g.h, g.probs, 1, 1, v, w, use_graph=False)
    g.close()


def test_async_run_defers_the_walk_limit_status_to_mesh_status():
    """With SL_OPT_ASYNC = 1 a run that hits the hop cap returns at once;
    sl_mesh_status then reports SL_E_WALK_LIMIT, and the handle stays usable."""
    prob = si.config("C2", M=128)
    g = DeviceRun(prob.mesh, prob.field, prob.dt)
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_WALK_CAP, 1)
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_ASYNC, 1)
    v = g.to_dev(prob.v0)
    w = g.torch.empty_like(v)
    assert sl.sl_run(g.h, g.probs, 0, 1, v, w, use_graph=False, stats=False) is None
    with pytest.raises(sl.SLError) as e:
        sl.sl_mesh_status(g.h)
    assert e.value.status == sl.SL_E_WALK_LIMIT
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_WALK_CAP, 0)
    sl.sl_run(g.h, g.probs, 1, 1, v, w, use_graph=False, stats=False)
    sl.sl_mesh_status(g.h)
    g.close()


def test_split_steps_on_a_batch_are_bitwise_identical():
    """Split steps on a batch of meshes with different fields (the settle
    pass that finds each node's problem): values, T^0 and statistics are
    bitwise those of the fused steps."""
    probs = si.batch_config(6, nmin=2e3, nmax=2e4, steps=5)
    no, to, xy, tri = sl.pack_meshes([(p.mesh.xy, p.mesh.tri) for p in probs])
    import torch
    pr = sl.problems([(p.field.kind, p.dt, p.field.packed()) for p in probs])
    outs = []
    for split in (0, 1):
        h = sl.sl_mesh_create(no, to, xy, tri)
        sl.sl_mesh_set_option(h, sl.SL_OPT_SPLIT, split)
        sl.sl_mesh_set_option(h, sl.SL_OPT_STATS, 1)
        v = torch.tensor(np.concatenate([p.v0 for p in probs]), dtype=torch.float64, device="cuda:0")
        w = torch.empty_like(v)
        st = sl.sl_run(h, pr, 0, 5, v, w)
        t0 = torch.empty(v.numel(), dtype=torch.int32, device="cuda:0")
        sl.sl_mesh_get_t0(h, t0)
        outs.append((v.cpu().numpy(), t0.cpu().numpy(), st))
        sl.sl_mesh_destroy(h)
    (v0, t00, s0), (v1, t01, s1) = outs
    assert np.array_equal(v0.view(np.int64), v1.view(np.int64))
    assert np.array_equal(t00, t01)
    for k in ("node_updates", "walk_moves", "max_moves", "exact_tests", "clipped", "fallbacks"):
        assert s0[k] == s1[k], k


@pytest.mark.parametrize("kernel", [1, 2], ids=["plain", "fast"])
def test_batched_problems_match_single_runs(kernel):
    probs = si.batch_config(6, nmin=2e3, nmax=2e4, steps=3)
    meshes = [(p.mesh.xy, p.mesh.tri) for p in probs]
    no, to, xy, tri = sl.pack_meshes(meshes)
    import torch
    h = sl.sl_mesh_create(no, to, xy, tri)
    sl.sl_mesh_set_option(h, sl.SL_OPT_KERNEL, kernel)
    pr = sl.problems([(p.field.kind, p.dt, p.field.packed()) for p in probs])
    v = torch.tensor(np.concatenate([p.v0 for p in probs]), dtype=torch.float64, device="cuda:0")
    w = torch.empty_like(v)
    sl.sl_run(h, pr, 0, 3, v, w)
    got = v.cpu().numpy()
    sl.sl_mesh_destroy(h)
    for k, p in enumerate(probs):
        om = oracle.OracleMesh(p.mesh.xy, p.mesh.tri)
        want = om.run(p.field.kind, p.field.packed(), p.dt, 0, 3, p.v0)
        seg = got[no[k]:no[k + 1]]
        assert np.abs(seg - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("form", ["fp64", "fp64_split", "fp32"])
def test_many_tiny_problems_match_single_runs(form):
    """A batch of 40 problems of 9 to 100 nodes, so that a block of nodes and
    a chunk of the problem table span several problems: every problem's
    values after 3 steps are those of the same problem run alone (its field
    constants found through the table; a wrong problem would change them
    entirely), and within the precision's tolerance of the oracle, both
    relative to the problem's max |V^0|.  (Not bitwise: the initial start
    triangle hashes the global node index, reading c5, so a foot on an edge
    may end its walk in the other triangle, which rounds differently.)"""
    import torch
    prec = sl.SL_FP32 if form == "fp32" else sl.SL_FP64
    probs = si.batch_config(40, seed=11, nmin=9, nmax=100, steps=3)
    meshes = [(p.mesh.xy, p.mesh.tri) for p in probs]
    no, to, xy, tri = sl.pack_meshes(meshes)
    vt = torch.float32 if prec == sl.SL_FP32 else torch.float64

    def run(meshes_, problems, v0):
        n_, t_, x_, r_ = sl.pack_meshes(meshes_)
        h = sl.sl_mesh_create(n_, t_, x_, r_, precision=prec)
        if form == "fp64_split":
            sl.sl_mesh_set_option(h, sl.SL_OPT_SPLIT, 1)
        pr = sl.problems([(p.field.kind, p.dt, p.field.packed()) for p in problems])
        v = torch.tensor(v0, dtype=vt, device="cuda:0")
        w = torch.empty_like(v)
        sl.sl_run(h, pr, 0, 3, v, w)
        out = v.double().cpu().numpy()
        sl.sl_mesh_destroy(h)
        return out

    got = run(meshes, probs, np.concatenate([p.v0 for p in probs]))
    assert int(np.diff(no).max()) <= 100 and len(probs) == 40
    # the batch tolerance scales with each problem's max |V^0| (a step of
    # several domain widths decays some of these values a billionfold)
    same, orc = (1e-13, 1e-12) if prec == sl.SL_FP64 else (1e-6, 1e-5)
    for k, p in enumerate(probs):
        scale = np.abs(p.v0).max()
        alone = run([meshes[k]], [p], p.v0)
        seg = got[no[k]:no[k + 1]]
        assert np.abs(seg - alone).max() <= same * scale, k
        om = oracle.OracleMesh(p.mesh.xy, p.mesh.tri)
        want = om.run(p.field.kind, p.field.packed(), p.dt, 0, 3, p.v0)
        assert np.abs(seg - want).max() <= orc * scale, k


def test_bad_step_arguments():
    prob = si.config("C1", M=8)
    g = DeviceRun(prob.mesh, prob.field, prob.dt)
    v = g.to_dev(prob.v0)
    with pytest.raises(sl.SLError) as e:
        sl.sl_step(g.h, g.probs, 0, v, v)
    assert e.value.status == sl.SL_E_ARG
    bad = sl.problems([(prob.field.kind, float("nan"), prob.field.packed())])
    w = g.torch.empty_like(v)
    with pytest.raises(sl.SLError) as e:
        sl.sl_step(g.h, bad, 0, v, w)
    assert e.value.status == sl.SL_E_ARG
    g.close()


def test_autotune_restores_state_and_keeps_results():
    """sl_autotune measures every launch configuration, keeps the fastest
    and leaves values, T^0 and the results of a following run unchanged."""
    prob = si.config("C2", M=256)
    g = DeviceRun(prob.mesh, prob.field, prob.dt, curve=sl.SL_CURVE_HILBERT)
    v = g.to_dev(prob.v0)
    w = g.torch.empty_like(v)
    before = v.clone()
    tune = sl.sl_autotune(g.h, g.probs, 2, v, w)
    assert g.torch.equal(v, before)
    assert 0 <= tune["config_first"] < len(tune["first_ms"]) and 0 <= tune["config_rest"] < len(tune["rest_ms"])
    assert all(t > 0 for t in tune["first_ms"] + tune["rest_ms"])
    sl.sl_run(g.h, g.probs, 0, 5, v, w)
    tuned = g.from_dev(v)
    g.close()
    ref = DeviceRun(prob.mesh, prob.field, prob.dt, curve=sl.SL_CURVE_HILBERT)
    v2 = ref.to_dev(prob.v0)
    w2 = ref.torch.empty_like(v2)
    sl.sl_run(ref.h, ref.probs, 0, 5, v2, w2)
    assert np.abs(ref.from_dev(v2) - tuned).max() <= 1e-12 * np.abs(tuned).max()
    ref.close()


def test_gather_probe_times_and_leaves_state():
    """sl_probe_gather returns a positive mean time, reads v without
    changing it, leaves T^0 alone and refuses bad arguments."""
    prob = si.config("C2", M=256)
    g = DeviceRun(prob.mesh, prob.field, prob.dt, curve=sl.SL_CURVE_HILBERT)
    v = g.to_dev(prob.v0)
    w = g.torch.empty_like(v)
    sl.sl_run(g.h, g.probs, 0, 3, v, w)
    before = v.clone()
    n = v.numel()
    t0 = g.torch.empty(n, dtype=g.torch.int32, device="cuda")
    sl.sl_mesh_get_t0(g.h, t0)
    ms = sl.sl_probe_gather(g.h, v, w, reps=5)
    assert ms > 0
    assert g.torch.equal(v, before)
    t1 = g.torch.empty_like(t0)
    sl.sl_mesh_get_t0(g.h, t1)
    assert g.torch.equal(t0, t1)
    for reps in (0, 1001):
        with pytest.raises(sl.SLError) as e:
            sl.sl_probe_gather(g.h, v, w, reps=reps)
        assert e.value.status == sl.SL_E_ARG
    with pytest.raises(sl.SLError):
        sl.sl_probe_gather(g.h, v, v, reps=1)
    g.close()


@pytest.mark.parametrize("kernel", [1, 2], ids=["plain", "fast"])
@pytest.mark.parametrize("fx", [-1e-17, 1e-17])
def test_boundary_nodes_with_nearly_tangent_velocity(kernel, fx):
    """A boundary node whose velocity is tangent to within 1e-17: x - dt f_x
    rounds (in double, Eq. 4) onto the boundary or across it.  The clip is
    discontinuous there, so the fast kernel must decide on the foot rounded
    to double like the oracle: the same nodes are clipped and the values
    agree."""
    mesh = si.grid_mesh(40, 0.25, 9)
    p = np.zeros(48)
    p[0], p[4] = fx, -1.0                     # f = (fx, -1): feet move up by dt
    fld = si.Field(si.FIELD_AFFINE, p, 1.0)
    dt = 0.05
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    g = DeviceRun(mesh, fld, dt, curve=sl.SL_CURVE_HILBERT, kernel=kernel)
    v0 = np.cos(2.0 * mesh.xy[:, 0]) + mesh.xy[:, 1] ** 2
    v = g.to_dev(v0)
    v, res = g.step(0, v)
    ov, otri, ofl, oft = om.step(fld.kind, fld.packed(), dt, 0, v0)
    on_side = (mesh.xy[:, 0] == 0.0) | (mesh.xy[:, 0] == 1.0)
    assert on_side.sum() > 40
    assert np.array_equal((res["flags"] & sl.SL_NODE_CLIPPED) != 0, (ofl & oracle.FLAG_CLIPPED) != 0)
    assert np.abs(res["v"] - ov).max() <= 1e-12 * np.abs(ov).max()
    g.close()


@pytest.mark.parametrize("steps", [5, 6])
@pytest.mark.parametrize("name", ["C2", "C3"])
def test_split_steps_are_bitwise_identical(name, steps):
    """SL_OPT_SPLIT: the settle pass finishes the nodes whose foot is
    certainly inside their start triangle and the finish pass the rest, with
    the same arithmetic as the fused kernel: values, T^0 and the walk
    statistics are bitwise those of the fused step (moving feet: swirl;
    stationary ones: rotation).  A split last step writes the run's doubles
    itself; an odd and an even number of steps place the buffers
    differently."""
    prob = si.config(name, M=192)
    outs = []
    for split in (0, 1):
        g = DeviceRun(prob.mesh, prob.field, prob.dt, curve=sl.SL_CURVE_HILBERT)
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_SPLIT, split)
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_STATS, 1)
        v = g.to_dev(prob.v0)
        w = g.torch.empty_like(v)
        sl.sl_run(g.h, g.probs, 0, steps, v, w, use_graph=True)
        t0 = g.torch.empty(prob.mesh.n_nodes, dtype=g.torch.int32, device=g.dev)
        sl.sl_mesh_get_t0(g.h, t0)
        st = sl.sl_mesh_stats(g.h)
        outs.append((g.from_dev(v), t0.cpu().numpy(), st))
        g.close()
    (v0, t00, s0), (v1, t01, s1) = outs
    assert np.array_equal(v0, v1)
    assert np.array_equal(t00, t01)
    for k in ("node_updates", "walk_moves", "max_moves", "exact_tests", "clipped", "fallbacks"):
        assert s0[k] == s1[k], k


def test_split_steps_settle_clipped_feet_like_the_fused_step():
    """Rotation about the centre carries the corner nodes out of the square:
    their feet are clipped onto a side, on the boundary edge of their start
    triangle, where one sign is exactly zero.  The settle pass finishes them
    by the boundary side codes; every debug output (foot, triangle, hops,
    flags including DEGENERATE) is bitwise that of the fused step."""
    prob = si.config("C3", M=160)
    outs = []
    for split in (0, 1):
        g = DeviceRun(prob.mesh, prob.field, prob.dt, curve=sl.SL_CURVE_HILBERT)
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_SPLIT, split)
        v = g.to_dev(prob.v0)
        steps = []
        for n in range(3):
            v, res = g.step(n, v)
            steps.append(res)
        outs.append(steps)
        g.close()
    for a, b in zip(*outs):
        for k in ("feet", "tri", "moves", "flags", "v"):
            assert np.array_equal(a[k], b[k]), k
    last = outs[1][-1]
    clipped = (last["flags"] & sl.SL_NODE_CLIPPED) != 0
    assert clipped.sum() > 100
    settled_on_side = clipped & (last["moves"] == 0) & ((last["flags"] & sl.SL_NODE_DEGENERATE) != 0)
    assert settled_on_side.sum() > 0.5 * clipped.sum()


@pytest.mark.parametrize("split", [0, 1])
def test_boundary_nodes_moving_out_keep_their_value(split):
    """Rotation about the centre: a boundary node whose velocity points out
    of the square is clipped at the start of its segment (Eq. 4 with the
    boundary clip), so its foot is the node itself.  The P1 value there is
    the node's own value (bit for bit as the kernel holds it, a (hi, lo)
    float pair), found in its start triangle (an incident triangle) without
    a walk or an exact test, at every step; the oracle agrees to rounding."""
    prob = si.config("C3", M=160)
    mesh = prob.mesh
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    g = DeviceRun(prob.mesh, prob.field, prob.dt, curve=sl.SL_CURVE_HILBERT)
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_SPLIT, split)
    v = g.to_dev(prob.v0)
    prev = prob.v0
    for n in range(3):
        v, res = g.step(n, v)
        ov, otri, ofl, oft = om.step(prob.field.kind, prob.field.packed(), prob.dt, n, prev)
        compare_step(om, res, ov, oft)
        out = np.all(oft == mesh.xy, axis=1) & ((ofl & oracle.FLAG_CLIPPED) != 0)
        assert out.sum() > 100
        hi = prev[out].astype(np.float32).astype(np.float64)
        assert np.array_equal(res["v"][out], hi + (prev[out] - hi).astype(np.float32).astype(np.float64))
        assert np.all(res["moves"][out] == 0)
        assert not np.any(res["flags"][out] & sl.SL_NODE_EXACT)
        assert np.all(res["flags"][out] & sl.SL_NODE_DEGENERATE)
        assert np.all(np.any(mesh.tri[res["tri"][out]] == np.nonzero(out)[0][:, None], axis=1))
        prev = res["v"]
    g.close()


def test_split_steps_match_the_oracle_with_debug_outputs():
    prob = si.config("C2", M=128)
    om = oracle.OracleMesh(prob.mesh.xy, prob.mesh.tri)
    g = DeviceRun(prob.mesh, prob.field, prob.dt, curve=sl.SL_CURVE_HILBERT)
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_SPLIT, 1)
    v = g.to_dev(prob.v0)
    vo = prob.v0
    for n in range(4):
        v, res = g.step(n, v)
        ov, otri, _, oft = om.step(prob.field.kind, prob.field.packed(), prob.dt, n, vo)
        compare_step(om, res, ov, oft)
        if n > 0:
            assert (res["moves"] == 0).mean() > 0.05      # both passes did work
            assert (res["moves"] > 0).mean() > 0.05
        vo = ov
    g.close()


def test_steep_data_takes_the_fp64_value_path():
    """A narrow Gaussian (sigma = 0.01, |grad V| up to 61) in the Fourier
    stream-function field: where V^n is steeper than SL_OPT_PRECISE's bound
    the value is evaluated in FP64 (flag SL_NODE_PRECISE) and every step
    stays within 1e-12 of one oracle step on the same V^n; with the bound at
    0 no node takes that path.  In the split form the settle pass leaves the
    steep nodes to the finish pass: values and flags agree bitwise with the
    fused form."""
    mesh = si.grid_mesh(400, 0.25, 41)
    fld = si.fourier8_field(11)
    dt = 0.01
    v0 = si.gaussian(mesh.xy, 0.5, 0.5, 0.01)
    om = oracle.OracleMesh(mesh.xy, mesh.tri)
    outs = {}
    for split, bound in ((0, 32), (1, 32), (0, 0)):
        g = DeviceRun(mesh, fld, dt, curve=sl.SL_CURVE_HILBERT)
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_SPLIT, split)
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_PRECISE, bound)
        v = g.to_dev(v0)
        steps = []
        for n in range(3):
            vin = g.from_dev(v)
            v, res = g.step(n, v)
            one, _, _, _ = om.step(fld.kind, fld.packed(), dt, n, vin, want_feet=False)
            err = np.abs(res["v"] - one).max() / np.abs(v0).max()
            precise = (res["flags"] & sl.SL_NODE_PRECISE) != 0
            steps.append((err, int(precise.sum()), res["v"], res["flags"]))
            exact_triangle_parity(om, res["tri"], res["feet"], res["feet_lo"], res["flags"])
        outs[(split, bound)] = steps
        g.close()
    for key in ((0, 32), (1, 32)):
        for err, n_precise, _, _ in outs[key]:
            assert err <= 1e-12
            assert n_precise > 100
    assert all(n == 0 for _, n, _, _ in outs[(0, 0)])
    # the FP64 path is what keeps the steep nodes within the tolerance
    assert max(e for e, _, _, _ in outs[(0, 32)]) < max(e for e, _, _, _ in outs[(0, 0)])
    for (_, _, va, fa), (_, _, vb, fb) in zip(outs[(0, 32)], outs[(1, 32)]):
        assert np.array_equal(va, vb)
        assert np.array_equal(fa, fb)


@pytest.mark.parametrize("split", [0, 1])
def test_compact_walk_records_give_identical_results(split):
    """The 8-byte half-edge records of fine meshes (SL_OPT_RECORDS) make the
    same hops as the 16-byte ones: values, located triangles, hop counts
    and flags bitwise equal over steps from the initial start triangles and
    later ones, on a mesh fine enough for them (the C2 construction at 512^2);
    a coarse mesh keeps 16-byte records."""
    prob = si.config("C2", M=512)
    runs = []
    for records in (0, 1):
        g = DeviceRun(prob.mesh, prob.field, prob.dt, curve=sl.SL_CURVE_HILBERT)
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_SPLIT, split)
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_RECORDS, records)
        assert sl.sl_mesh_get_option(g.h, sl.SL_OPT_RECORDS) == (16 if records == 0 else 8)
        v = g.to_dev(prob.v0)
        out = []
        for n in range(3):
            v, res = g.step(n, v)
            out.append(res)
        runs.append(out)
        g.close()
    for a, b in zip(*runs):
        for key in ("v", "tri", "moves", "flags", "feet", "feet_lo"):
            assert np.array_equal(a[key], b[key]), key
    assert runs[0][0]["moves"].mean() > 5          # the first step walks
    coarse = DeviceRun(si.grid_mesh(100, 0.25, 3), prob.field, prob.dt)
    sl.sl_mesh_set_option(coarse.h, sl.SL_OPT_RECORDS, 1)      # too coarse: 16-byte records stay
    assert sl.sl_mesh_get_option(coarse.h, sl.SL_OPT_RECORDS) == 16
    coarse.close()


def test_split_graph_replays_are_identical():
    """A recorded run of split steps (settle pass, then the finish pass over
    the nodes it queued), replayed three times from the same V^0 and start
    triangles: the same values, T^0 and statistics every time, equal to eager
    steps."""
    prob = si.config("C2", M=160)
    g = DeviceRun(prob.mesh, prob.field, prob.dt, curve=sl.SL_CURVE_HILBERT)
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_SPLIT, 1)
    sl.sl_mesh_set_option(g.h, sl.SL_OPT_STATS, 1)
    v0 = g.to_dev(prob.v0)
    w = g.torch.empty_like(v0)
    results = []
    for use_graph in (True, True, True, False):
        sl.sl_mesh_reset_t0(g.h)
        sl.sl_mesh_stats(g.h, reset=True)
        v = v0.clone()
        sl.sl_run(g.h, g.probs, 0, 5, v, w, use_graph=use_graph)
        t0 = g.torch.empty(prob.mesh.n_nodes, dtype=g.torch.int32, device=g.dev)
        sl.sl_mesh_get_t0(g.h, t0)
        results.append((v.cpu().numpy(), t0.cpu().numpy(), sl.sl_mesh_stats(g.h)))
    g.close()
    assert results[0][2]["walk_moves"] > 0
    for v, t0, st in results[1:]:
        assert np.array_equal(v, results[0][0])
        assert np.array_equal(t0, results[0][1])
        assert st == results[0][2]


@pytest.mark.parametrize("form", ["split", "fused", "fp32"])
def test_programmatic_launches_give_identical_results(form):
    """SL_OPT_PDL: the step kernels of a run launched with programmatic stream
    serialization (each computes its feet while the kernel before it
    finishes, then waits for it) give bitwise the values, T^0 and statistics
    of plain launches, recorded as a graph and eager, in the split form (the
    finish pass has queued nodes to walk here), the fused form and FP32."""
    prob = si.config("C2", M=160)
    precision = sl.SL_FP32 if form == "fp32" else sl.SL_FP64
    g = DeviceRun(prob.mesh, prob.field, prob.dt, precision=precision, curve=sl.SL_CURVE_HILBERT)
    if form == "split":
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_SPLIT, 1)
    v0 = g.to_dev(prob.v0)
    w = g.torch.empty_like(v0)
    results = []
    for pdl, stats, use_graph in ((0, 1, True), (1, 1, True), (1, 1, False), (0, 0, True), (1, 0, True)):
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_PDL, pdl)
        sl.sl_mesh_set_option(g.h, sl.SL_OPT_STATS, stats)
        assert sl.sl_mesh_get_option(g.h, sl.SL_OPT_PDL) == pdl
        sl.sl_mesh_reset_t0(g.h)
        sl.sl_mesh_stats(g.h, reset=True)
        v = v0.clone()
        sl.sl_run(g.h, g.probs, 0, 6, v, w, use_graph=use_graph)
        t0 = g.torch.empty(prob.mesh.n_nodes, dtype=g.torch.int32, device=g.dev)
        sl.sl_mesh_get_t0(g.h, t0)
        results.append((v.cpu().numpy(), t0.cpu().numpy(), sl.sl_mesh_stats(g.h) if stats else None))
    g.close()
    assert results[0][2]["walk_moves"] > 0
    for k, (v, t0, st) in enumerate(results[1:], 1):
        assert np.array_equal(v, results[0][0]), k
        assert np.array_equal(t0, results[0][1]), k
        if st is not None:
            assert st == results[0][2], k


@pytest.mark.parametrize("precision", [sl.SL_FP64, sl.SL_FP32], ids=["fp64", "fp32"])
def test_layout_autotuner_renumbers_consistently(precision):
    """sl_autotune_layout on a shuffled mesh with the swirl field (whose node
    tables are built by the timed steps and must follow every renumbering):
    it times the numbering as given, Hilbert and Morton, keeps the fastest,
    permutes V^0 in place and returns the permutation; a run afterwards,
    mapped back through it, is bitwise a run on an untuned copy of the mesh
    in its own numbering."""
    import torch
    from sl_inputs.meshes import shuffled
    prob = si.config("C2", M=160)
    mesh = shuffled(prob.mesh, 17)
    v0 = si.gaussian(mesh.xy, 0.5, 0.75, 0.05)
    dt = torch.float64 if precision == sl.SL_FP64 else torch.float32
    no, to, xy, tri = sl.pack_meshes([(mesh.xy, mesh.tri)])
    pr = sl.problems([(prob.field.kind, prob.dt, prob.field.packed())])
    h = sl.sl_mesh_create(no, to, xy, tri, precision=precision, seed=4)
    v = torch.tensor(v0, dtype=dt, device="cuda")
    w = torch.empty_like(v)
    node_perm, tri_perm, tune = sl.sl_autotune_layout(h, pr, 2, v, w)
    assert tune["curve"] in ("as given", "hilbert", "morton")
    assert set(tune["curve_ms"]) == {"as given", "hilbert", "morton"}
    assert np.array_equal(v.cpu().numpy(), v0.astype(v.cpu().numpy().dtype)[node_perm])
    assert np.array_equal(np.sort(node_perm), np.arange(mesh.n_nodes))
    sl.sl_run(h, pr, 0, 4, v, w)
    got = np.empty(mesh.n_nodes)
    got[node_perm] = v.cpu().numpy()
    sl.sl_mesh_destroy(h)
    h2 = sl.sl_mesh_create(no, to, xy, tri, precision=precision, seed=4)
    v2 = torch.tensor(v0, dtype=dt, device="cuda")
    sl.sl_run(h2, pr, 0, 4, v2, torch.empty_like(v2))
    want = v2.cpu().numpy()
    sl.sl_mesh_destroy(h2)
    assert np.array_equal(got, want)
