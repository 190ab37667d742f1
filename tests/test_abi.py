"""The C-ABI library: it loads on a machine without a GPU, exports every
entry point include/sl.h declares, and its host-side mesh handling
(validation, neighbour list of Sec. 3, initial start triangles) is right.
No GPU compute is called here."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2104_09189_gb300 as sl
import sl_inputs as si
from sl_inputs.meshes import shuffled

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sl_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = sl.library()
    names = _declared()
    assert "sl_step" in names and "sl_run" in names and "sl_mesh_create" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(sl.EXPORTED)


def _brute_nbr(tri):
    owner = {}
    for j, t in enumerate(tri):
        for k in range(3):
            owner[(int(t[(k + 1) % 3]), int(t[(k + 2) % 3]))] = j
    nbr = np.full(tri.shape, -1, dtype=np.int32)
    for j, t in enumerate(tri):
        for k in range(3):
            nbr[j, k] = owner.get((int(t[(k + 2) % 3]), int(t[(k + 1) % 3])), -1)
    return nbr


@pytest.mark.parametrize("shuffle", [False, True])
def test_validate_builds_neighbours_and_incident_start(shuffle):
    m = si.grid_mesh(7, 0.25, 3)
    if shuffle:
        m = shuffled(m, 5)
    no, to, xy, tri = sl.pack_meshes([(m.xy, m.tri)])
    nbr, t0 = sl.sl_mesh_validate(no, to, xy, tri, seed=9)
    assert np.array_equal(nbr, _brute_nbr(m.tri))
    for i in range(m.n_nodes):
        assert i in m.tri[t0[i]]
    nbr2, t02 = sl.sl_mesh_validate(no, to, xy, tri, seed=9)
    assert np.array_equal(t0, t02)
    _, t03 = sl.sl_mesh_validate(no, to, xy, tri, seed=10)
    assert not np.array_equal(t0, t03)
    # a supplied, consistent neighbour list is accepted
    sl.sl_mesh_validate(no, to, xy, tri, nbr=nbr)


def test_validate_batch_local_indices():
    a, b = si.grid_mesh(3, 0.2, 1), si.grid_mesh(5, 0.2, 2)
    no, to, xy, tri = sl.pack_meshes([(a.xy, a.tri), (b.xy, b.tri)])
    nbr, t0 = sl.sl_mesh_validate(no, to, xy, tri)
    assert np.array_equal(nbr[: a.n_tri], _brute_nbr(a.tri))
    assert np.array_equal(nbr[a.n_tri:], _brute_nbr(b.tri))
    assert t0[: a.n_nodes].max() < a.n_tri and t0[a.n_nodes:].max() < b.n_tri


def _expect(status, fn):
    with pytest.raises(sl.SLError) as e:
        fn()
    assert e.value.status == status, str(e.value)
    return str(e.value)


def test_malformed_meshes_are_rejected():
    m = si.grid_mesh(4, 0.2, 3)
    no, to = np.array([0, m.n_nodes]), np.array([0, m.n_tri])
    # clockwise triangle
    t = m.tri.copy()
    t[5] = t[5, ::-1]
    assert "counter-clockwise" in _expect(sl.SL_E_MESH, lambda: sl.sl_mesh_validate(no, to, m.xy, t))
    # index out of range
    t = m.tri.copy()
    t[2, 1] = m.n_nodes
    _expect(sl.SL_E_MESH, lambda: sl.sl_mesh_validate(no, to, m.xy, t))
    # node outside the square
    xy = m.xy.copy()
    xy[0, 0] = -1e-9
    _expect(sl.SL_E_MESH, lambda: sl.sl_mesh_validate(no, to, xy, m.tri))
    xy[0, 0] = np.nan
    _expect(sl.SL_E_MESH, lambda: sl.sl_mesh_validate(no, to, xy, m.tri))
    # a hole: drop two triangles -> area != 1 and interior boundary edges
    _expect(sl.SL_E_MESH, lambda: sl.sl_mesh_validate(np.array([0, m.n_nodes]), np.array([0, m.n_tri - 2]),
                                                       m.xy, m.tri[:-2]))
    # asymmetric supplied neighbours
    nbr, _ = sl.sl_mesh_validate(no, to, m.xy, m.tri)
    bad = nbr.copy()
    bad[0, 0] = 3 if bad[0, 0] != 3 else 4
    _expect(sl.SL_E_MESH, lambda: sl.sl_mesh_validate(no, to, m.xy, m.tri, nbr=bad))
    # a duplicated triangle (edge shared three times)
    t = np.vstack([m.tri, m.tri[:1]])
    _expect(sl.SL_E_MESH, lambda: sl.sl_mesh_validate(no, np.array([0, m.n_tri + 1]), m.xy, t))


def test_bad_arguments():
    m = si.grid_mesh(3, 0.0, 0)
    _expect(sl.SL_E_ARG, lambda: sl.sl_mesh_validate(np.array([1, m.n_nodes]), np.array([0, m.n_tri]), m.xy, m.tri))
    _expect(sl.SL_E_ARG, lambda: sl.sl_mesh_validate(np.array([0, m.n_nodes, 3]), np.array([0, m.n_tri, 2]),
                                                      m.xy, m.tri))


def test_python_constants_match_the_header_enums():
    # every "SL_NAME = value" enumerator of include/sl.h has the same value in
    # the binding (options, node flags, field kinds, statuses, ...)
    import re
    hdr = open(os.path.join(ROOT, "include", "sl.h")).read()
    hdr = re.sub(r"/\*.*?\*/", " ", hdr, flags=re.S)     # comments mention values too
    pairs = re.findall(r"\b(SL_[A-Z0-9_]+)\s*=\s*(\d+)", hdr)
    assert len(pairs) > 20
    missing = []
    for name, val in pairs:
        if hasattr(sl, name):
            assert getattr(sl, name) == int(val), name
        else:
            missing.append(name)
    # field kinds live on the input side; everything else must be exported
    assert all(n.startswith("SL_FIELD_") for n in missing), missing


def test_stats_struct_matches_the_header():
    import re
    hdr = open(os.path.join(ROOT, "include", "sl.h")).read()
    body = hdr[hdr.index("typedef struct {\n    uint64_t node_updates;"):]
    body = body[:body.index("} sl_stats;")]
    names = re.findall(r"uint64_t\s+(\w+);", body)
    assert [n for n, _ in sl.sl_stats._fields_] == names


def test_size_limits_are_rejected_before_any_array_is_read():
    # int32 node ids and int32 half-edge codes (3 t + k): more than 2^31 - 1
    # nodes or 715 827 882 triangles is SL_E_ARG; the check runs on the
    # offsets alone (the arrays passed here are tiny and never read)
    L = sl.library()
    xy = np.zeros(8, dtype=np.float64)
    tri = np.zeros(6, dtype=np.int32)
    for n_nodes, n_tri in [(1 << 31, 2), (4, 715827883), (4, 1 << 30)]:
        no = np.array([0, n_nodes], dtype=np.int64)
        to = np.array([0, n_tri], dtype=np.int64)
        st = L.sl_mesh_validate(1, no.ctypes.data, to.ctypes.data, xy.ctypes.data, tri.ctypes.data, None, 1,
                                None, None)
        assert st == sl.SL_E_ARG, (n_nodes, n_tri)
        assert "more than" in sl.sl_last_error()
