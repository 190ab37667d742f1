"""GB300 semi-Lagrangian foot -> locate -> P1 library (Cacace & Ferretti).

Python binding of ``include/sl.h``: the functions below carry the C names
and only marshal arguments (numpy arrays and torch tensors to pointers, the
current torch stream to a cudaStream_t).  Every step of the path runs in the
CUDA library ``libslwalk.so``; nothing here computes a foot, a location or an
interpolant.  If the library has not been built the first call raises
``RuntimeError`` -- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from ._build import LIB as _LIB_PATH

__all__ = [
    "SL_OK", "SL_E_ARG", "SL_E_MESH", "SL_E_NOMEM", "SL_E_CUDA", "SL_E_WALK_LIMIT", "SL_E_STATE",
    "SL_FP64", "SL_FP32", "SL_CURVE_NONE", "SL_CURVE_HILBERT", "SL_CURVE_MORTON",
    "SL_OPT_STATS", "SL_OPT_WALK_CAP", "SL_OPT_KERNEL", "SL_OPT_BLOCK", "SL_OPT_CONFIG",
    "SL_OPT_CONFIG_FIRST", "SL_OPT_STRATEGY", "SL_OPT_OUTSIDE", "SL_OPT_SPLIT", "SL_OPT_ASYNC", "SL_OPT_PRECISE", "SL_OPT_RECORDS", "SL_OPT_L2_WINDOW", "SL_OPT_PDL",
    "SL_NODE_CLIPPED", "SL_NODE_DEGENERATE", "SL_NODE_EXACT", "SL_NODE_FALLBACK", "SL_NODE_WALK_LIMIT",
    "SL_NODE_RANGE", "SL_NODE_EXCLUDED", "SL_NODE_PRECISE", "SLError", "sl_problem", "problems", "pack_meshes",
    "sl_mesh_create", "sl_mesh_validate", "sl_mesh_reorder", "sl_step", "sl_run", "sl_run_host", "sl_mesh_get_t0",
    "sl_mesh_set_t0", "sl_mesh_reset_t0", "sl_mesh_status", "sl_mesh_stats", "sl_mesh_set_option", "sl_mesh_info",
    "sl_mesh_export", "sl_mesh_destroy", "sl_last_error", "library", "EXPORTED", "sl_step_noalloc",
    "SL_NOALLOC_MAX_NODES", "SL_NOALLOC_MAX_PROBLEMS", "sl_autotune", "sl_probe_gather", "sl_mesh_get_option",
    "sl_autotune_layout",
]

SL_OK, SL_E_ARG, SL_E_MESH, SL_E_NOMEM, SL_E_CUDA, SL_E_WALK_LIMIT, SL_E_STATE = range(7)
SL_FP64, SL_FP32 = 0, 1
SL_CURVE_NONE, SL_CURVE_HILBERT, SL_CURVE_MORTON = 0, 1, 2
SL_OPT_STATS, SL_OPT_WALK_CAP, SL_OPT_KERNEL, SL_OPT_BLOCK = range(4)
SL_OPT_CONFIG = 5
SL_OPT_CONFIG_FIRST, SL_OPT_STRATEGY, SL_OPT_OUTSIDE, SL_OPT_SPLIT, SL_OPT_ASYNC, SL_OPT_PRECISE = 7, 8, 9, 10, 11, 12
SL_OPT_RECORDS = 13
SL_OPT_L2_WINDOW = 14
SL_OPT_PDL = 15
SL_NODE_CLIPPED, SL_NODE_DEGENERATE, SL_NODE_EXACT, SL_NODE_FALLBACK, SL_NODE_WALK_LIMIT, SL_NODE_RANGE = (
    1, 2, 4, 8, 16, 32)
SL_NODE_EXCLUDED = 64
SL_NODE_PRECISE = 128
SL_NPARAMS = 48
SL_NOALLOC_MAX_NODES = 1 << 20
SL_NOALLOC_MAX_PROBLEMS = 256

_STATUS_NAMES = {0: "SL_OK", 1: "SL_E_ARG", 2: "SL_E_MESH", 3: "SL_E_NOMEM", 4: "SL_E_CUDA",
                 5: "SL_E_WALK_LIMIT", 6: "SL_E_STATE"}

# every entry point declared in include/sl.h
EXPORTED = ("sl_mesh_create", "sl_mesh_validate", "sl_mesh_reorder", "sl_step", "sl_run", "sl_run_host", "sl_mesh_get_t0",
            "sl_mesh_set_t0", "sl_mesh_reset_t0", "sl_mesh_status", "sl_mesh_stats", "sl_mesh_set_option", "sl_mesh_info",
            "sl_mesh_export", "sl_mesh_destroy", "sl_last_error", "sl_step_noalloc", "sl_autotune",
            "sl_probe_gather", "sl_mesh_get_option", "sl_autotune_layout")


class SLError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


class sl_problem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("dt", ctypes.c_double),
                ("p", ctypes.c_double * SL_NPARAMS)]


class sl_debug(ctypes.Structure):
    _fields_ = [("feet", ctypes.c_void_p), ("tri", ctypes.c_void_p), ("moves", ctypes.c_void_p),
                ("flags", ctypes.c_void_p), ("feet_lo", ctypes.c_void_p)]


class sl_tune(ctypes.Structure):
    _fields_ = [("config_first", ctypes.c_int32), ("config_rest", ctypes.c_int32), ("n_configs", ctypes.c_int32),
                ("split", ctypes.c_int32), ("first_ms", ctypes.c_float * 8), ("rest_ms", ctypes.c_float * 8),
                ("split_ms", ctypes.c_float * 8), ("records", ctypes.c_int32), ("compact_first_ms", ctypes.c_float),
                ("compact_rest_ms", ctypes.c_float), ("curve", ctypes.c_int32), ("curve_ms", ctypes.c_float * 3)]


class sl_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("node_updates", "walk_moves", "max_moves", "exact_tests",
                                                "filter2_tests", "clipped", "fallbacks", "walk_limit",
                                                "excluded")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


_lib = None


def library():
    """Load libslwalk.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is not built; run `python -c \"import __graft_entry__ as g; g.build()\"`")
    L = ctypes.CDLL(_LIB_PATH)
    P, I32, I64, U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "sl_mesh_create": [I32, P, P, P, P, P, I32, U64, ctypes.POINTER(ctypes.c_void_p)],
        "sl_mesh_validate": [I32, P, P, P, P, P, U64, P, P],
        "sl_mesh_reorder": [P, I32, P, P],
        "sl_step": [P, P, I64, P, P, P, P],
        "sl_run": [P, P, I64, I32, P, P, I32, P, P],
        "sl_run_host": [P, P, I64, I32, P, I32, P, P],
        "sl_mesh_get_t0": [P, P, P],
        "sl_mesh_set_t0": [P, P, P],
        "sl_mesh_status": [P, P],
        "sl_mesh_reset_t0": [P, P],
        "sl_mesh_stats": [P, P, I32, P],
        "sl_mesh_set_option": [P, I32, I64],
        "sl_mesh_get_option": [P, I32, P],
        "sl_mesh_info": [P, P, P, P, P],
        "sl_mesh_export": [P, P, P, P],
        "sl_step_noalloc": [P, P, I64, P, P, P],
        "sl_autotune": [P, P, I32, P, P, P, P],
        "sl_autotune_layout": [P, P, I32, I32, P, P, P, P, P, P],
        "sl_probe_gather": [P, P, P, I32, P, P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.sl_mesh_destroy.argtypes = [P]
    L.sl_mesh_destroy.restype = None
    L.sl_last_error.argtypes = []
    L.sl_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def sl_last_error():
    return library().sl_last_error().decode(errors="replace")


def _check(st):
    if st != SL_OK:
        raise SLError(st, sl_last_error())


def _ptr(x):
    """Device or host address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def problems(specs):
    """ctypes array of sl_problem from a list of (kind, dt, params) tuples."""
    arr = (sl_problem * len(specs))()
    for k, (kind, dt, params) in enumerate(specs):
        arr[k].kind = int(kind)
        arr[k].reserved = 0
        arr[k].dt = float(dt)
        p = np.zeros(SL_NPARAMS)
        q = np.asarray(params, dtype=np.float64).ravel()
        p[: q.size] = q
        for i in range(SL_NPARAMS):
            arr[k].p[i] = float(p[i])
    return arr


def pack_meshes(meshes):
    """(node_off, tri_off, xy, tri) for a list of (xy, tri) pairs with local
    indices, concatenated in order."""
    node_off = np.zeros(len(meshes) + 1, dtype=np.int64)
    tri_off = np.zeros(len(meshes) + 1, dtype=np.int64)
    for k, (xy, tri) in enumerate(meshes):
        node_off[k + 1] = node_off[k] + len(xy)
        tri_off[k + 1] = tri_off[k] + len(tri)
    xy = np.ascontiguousarray(np.concatenate([np.asarray(m[0], np.float64).reshape(-1, 2) for m in meshes]))
    tri = np.ascontiguousarray(np.concatenate([np.asarray(m[1], np.int32).reshape(-1, 3) for m in meshes]))
    return node_off, tri_off, xy, tri


def sl_mesh_create(node_off, tri_off, xy, tri, nbr=None, precision=SL_FP64, seed=1):
    node_off = np.ascontiguousarray(node_off, dtype=np.int64)
    tri_off = np.ascontiguousarray(tri_off, dtype=np.int64)
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    nbr = None if nbr is None else np.ascontiguousarray(nbr, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(library().sl_mesh_create(len(node_off) - 1, _ptr(node_off), _ptr(tri_off), _ptr(xy), _ptr(tri),
                                    _ptr(nbr), int(precision), int(seed) & ((1 << 64) - 1), ctypes.byref(h)))
    return h.value


def sl_mesh_validate(node_off, tri_off, xy, tri, nbr=None, seed=1):
    """Host-only validation; returns (nbr, t0) with local indices."""
    node_off = np.ascontiguousarray(node_off, dtype=np.int64)
    tri_off = np.ascontiguousarray(tri_off, dtype=np.int64)
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    nbr = None if nbr is None else np.ascontiguousarray(nbr, dtype=np.int32)
    nbr_out = np.empty((int(tri_off[-1]), 3), dtype=np.int32)
    t0_out = np.empty(int(node_off[-1]), dtype=np.int32)
    _check(library().sl_mesh_validate(len(node_off) - 1, _ptr(node_off), _ptr(tri_off), _ptr(xy), _ptr(tri),
                                      _ptr(nbr), int(seed) & ((1 << 64) - 1), _ptr(nbr_out), _ptr(t0_out)))
    return nbr_out, t0_out


def sl_mesh_info(h):
    n, nt, npb, prec = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    _check(library().sl_mesh_info(h, ctypes.byref(n), ctypes.byref(nt), ctypes.byref(npb), ctypes.byref(prec)))
    return {"n_nodes": n.value, "n_tri": nt.value, "n_problems": npb.value, "precision": prec.value}


def sl_mesh_reorder(h, curve=SL_CURVE_HILBERT):
    """Returns (node_perm, tri_perm), new -> old, local to each problem."""
    info = sl_mesh_info(h)
    node_perm = np.empty(info["n_nodes"], dtype=np.int32)
    tri_perm = np.empty(info["n_tri"], dtype=np.int32)
    _check(library().sl_mesh_reorder(h, int(curve), _ptr(node_perm), _ptr(tri_perm)))
    return node_perm, tri_perm


def sl_mesh_export(h):
    info = sl_mesh_info(h)
    xy = np.empty((info["n_nodes"], 2), dtype=np.float64)
    tri = np.empty((info["n_tri"], 3), dtype=np.int32)
    nbr = np.empty((info["n_tri"], 3), dtype=np.int32)
    _check(library().sl_mesh_export(h, _ptr(xy), _ptr(tri), _ptr(nbr)))
    return xy, tri, nbr


def sl_step(h, probs, n, v_in, v_out, debug=None, stream=None):
    """debug: None or a dict with any of 'feet', 'tri', 'moves', 'flags',
    'feet_lo' (device tensors of 2N float64, N int32, N int32, N uint8, 2N
    float64); the foot the kernel located is feet + feet_lo exactly."""
    dbg = None
    if debug:
        dbg = sl_debug(_ptr(debug.get("feet")), _ptr(debug.get("tri")), _ptr(debug.get("moves")),
                       _ptr(debug.get("flags")), _ptr(debug.get("feet_lo")))
    _check(library().sl_step(h, probs, int(n), _ptr(v_in), _ptr(v_out),
                             ctypes.byref(dbg) if dbg is not None else None, _stream(stream)))


def sl_run(h, probs, n0, n_steps, v, v_scratch, use_graph=True, stream=None, stats=True):
    """Returns the walk statistics as a dict, or None with stats=False (which
    with SL_OPT_ASYNC = 1 returns without synchronising)."""
    st = sl_stats() if stats else None
    _check(library().sl_run(h, probs, int(n0), int(n_steps), _ptr(v), _ptr(v_scratch), 1 if use_graph else 0,
                            ctypes.byref(st) if stats else None, _stream(stream)))
    return st.as_dict() if stats else None


def sl_run_host(h, probs, n0, n_steps, v_host, use_graph=True, stream=None):
    st = sl_stats()
    _check(library().sl_run_host(h, probs, int(n0), int(n_steps), _ptr(v_host), 1 if use_graph else 0,
                                 ctypes.byref(st), _stream(stream)))
    return st.as_dict()


def sl_mesh_get_t0(h, t0_dev, stream=None):
    _check(library().sl_mesh_get_t0(h, _ptr(t0_dev), _stream(stream)))


def sl_mesh_set_t0(h, t0_dev, stream=None):
    _check(library().sl_mesh_set_t0(h, _ptr(t0_dev), _stream(stream)))


def sl_mesh_reset_t0(h, stream=None):
    _check(library().sl_mesh_reset_t0(h, _stream(stream)))


def sl_mesh_status(h, stream=None):
    """Raises SLError for a deferred device condition (e.g. SL_E_WALK_LIMIT)."""
    _check(library().sl_mesh_status(h, _stream(stream)))


def sl_mesh_stats(h, reset=False, stream=None):
    st = sl_stats()
    _check(library().sl_mesh_stats(h, ctypes.byref(st), 1 if reset else 0, _stream(stream)))
    return st.as_dict()


def sl_mesh_set_option(h, option, value):
    _check(library().sl_mesh_set_option(h, int(option), int(value)))


def sl_mesh_get_option(h, option):
    """The option's value (SL_OPT_RECORDS: the walk records' size in bytes)."""
    v = ctypes.c_int64()
    _check(library().sl_mesh_get_option(h, int(option), ctypes.byref(v)))
    return v.value


def sl_mesh_destroy(h):
    if h:
        library().sl_mesh_destroy(h)


def sl_step_noalloc(h, probs, n, v_in, v_out, stream=None):
    """sl_step without any device allocation (FP64 meshes, double tensors);
    its scratch is a fixed static device array of the library (meshes of at
    most SL_NOALLOC_MAX_NODES nodes).  For callers that cannot allocate device
    memory while stepping."""
    _check(library().sl_step_noalloc(h, probs, int(n), _ptr(v_in), _ptr(v_out), _stream(stream)))


def sl_probe_gather(h, v, v_scratch, reps=10, stream=None):
    """Mean time (ms) of a kernel making only the memory accesses of a steady
    step on this mesh (see sl.h); v is read, v_scratch overwritten."""
    ms = ctypes.c_float()
    _check(library().sl_probe_gather(h, _ptr(v), _ptr(v_scratch), int(reps), ctypes.byref(ms), _stream(stream)))
    return float(ms.value)


def _tune_dict(t):
    n = t.n_configs
    d = {"config_first": t.config_first, "config_rest": t.config_rest, "split": t.split,
         "first_ms": [round(float(x), 4) for x in list(t.first_ms)[:n]],
         "rest_ms": [round(float(x), 4) for x in list(t.rest_ms)[:n]],
         "split_ms": [round(float(x), 4) for x in list(t.split_ms)[:n] if x >= 0],
         "records": t.records, "compact_first_ms": round(float(t.compact_first_ms), 4),
         "compact_rest_ms": round(float(t.compact_rest_ms), 4)}
    if t.curve >= 0:
        d["curve"] = {0: "as given", 1: "hilbert", 2: "morton"}[t.curve]
        d["curve_ms"] = {name: round(float(x), 4) for name, x in zip(("as given", "hilbert", "morton"), t.curve_ms)
                         if x >= 0}
    return d


def sl_autotune(h, probs, probe_steps, v, v_scratch, stream=None):
    """Time every launch configuration of the fast kernels on this mesh and
    set the fastest (see sl.h); returns the measurements."""
    t = sl_tune()
    _check(library().sl_autotune(h, probs, int(probe_steps), _ptr(v), _ptr(v_scratch), ctypes.byref(t),
                                 _stream(stream)))
    return _tune_dict(t)


def sl_autotune_layout(h, probs, probe_steps, v, v_scratch, curves=0b111, stream=None):
    """Choose the numbering (curves: bit c = try sl_curve c, SL_CURVE_NONE =
    as given) and then the launch configurations by measurement; v (device
    V^0) is permuted in place.  Returns (node_perm, tri_perm, measurements),
    the permutations new -> old relative to the numbering at the call, local
    to each problem."""
    info = sl_mesh_info(h)
    node_perm = np.empty(info["n_nodes"], dtype=np.int32)
    tri_perm = np.empty(info["n_tri"], dtype=np.int32)
    t = sl_tune()
    _check(library().sl_autotune_layout(h, probs, int(probe_steps), int(curves), _ptr(v), _ptr(v_scratch),
                                        _ptr(node_perm), _ptr(tri_perm), ctypes.byref(t), _stream(stream)))
    return node_perm, tri_perm, _tune_dict(t)
