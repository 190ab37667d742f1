"""CPU oracle for the semi-Lagrangian foot -> clip -> locate -> P1 step.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it; the product package never imports it.  It shares no
code with the CUDA library (its own C source, its own header, its own build).

The arithmetic lives in ``sl_oracle.c`` (plain C, IEEE double, no FMA
contraction, exact orientation signs); this module compiles it with gcc and
wraps it with ctypes.  Paper passages each function follows are cited in the
C source.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sl_oracle.c")
_HDR = os.path.join(_HERE, "sl_oracle.h")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FLAG_CLIPPED = 1
FLAG_DEGENERATE = 2
FLAG_MULTI = 4
FLAG_EXCLUDED = 8


def build(force=False):
    """Compile sl_oracle.c into liboracle.so next to it (gcc, -O2)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            D = ctypes.c_double
            P = ctypes.c_void_p
            I = ctypes.c_int
            I64 = ctypes.c_int64
            L.orc_field.argtypes = [I, P, D, D, D, P, P]
            L.orc_foot.argtypes = [I, P, D, D, D, D, P, P]
            L.orc_foot.restype = I
            L.orc_orient_sign.argtypes = [D] * 6
            L.orc_orient_sign.restype = I
            L.orc_orient_sign2.argtypes = [D] * 8
            L.orc_orient_sign2.restype = I
            L.orc_set_force_exact.argtypes = [I]
            L.orc_exact_calls.restype = ctypes.c_long
            L.orc_mesh_create.argtypes = [I64, I64, P, P]
            L.orc_mesh_create.restype = P
            L.orc_mesh_destroy.argtypes = [P]
            L.orc_mesh_bins.argtypes = [P]
            L.orc_mesh_bins.restype = I
            L.orc_interp.argtypes = [P, ctypes.c_int32, D, D, P]
            L.orc_interp.restype = D
            L.orc_step_range.argtypes = [P, I, P, D, I64, P, P, P, P, P, I64, I64, I]
            L.orc_step_range.restype = I
            L.orc_step_range_x.argtypes = [P, I, P, D, I64, P, P, P, P, P, I64, I64, I, I]
            L.orc_step_range_x.restype = I
            L.orc_step.argtypes = [P, I, P, D, I64, P, P, P, P, P, I]
            L.orc_step.restype = I
            L.orc_run.argtypes = [P, I, P, D, I64, I, P, P, I]
            L.orc_run.restype = I
            L.orc_locate_points.argtypes = [P, I64, P, P, P]
            L.orc_locate_points.restype = I
            L.orc_locate_points2.argtypes = [P, I64, P, P, P, P, I]
            L.orc_locate_points2.restype = I
            L.orc_tri_signs2.argtypes = [P, I64, P, P, P, P, I]
            L.orc_feet.argtypes = [I, P, D, I64, I64, P, P, P]
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data if a is not None else None


def default_threads():
    return max(1, os.cpu_count() or 1)


def orient_sign(a, b, c, force_exact=False):
    L = lib()
    L.orc_set_force_exact(1 if force_exact else 0)
    try:
        return L.orc_orient_sign(float(a[0]), float(a[1]), float(b[0]), float(b[1]), float(c[0]), float(c[1]))
    finally:
        L.orc_set_force_exact(0)


def orient_sign2(a, b, qh, ql, force_exact=False):
    """Exact sign of orient(a, b, q) for the point q = qh + ql (the sum of
    the two doubles of each coordinate, taken exactly)."""
    L = lib()
    L.orc_set_force_exact(1 if force_exact else 0)
    try:
        return L.orc_orient_sign2(float(a[0]), float(a[1]), float(b[0]), float(b[1]),
                                  float(qh[0]), float(qh[1]), float(ql[0]), float(ql[1]))
    finally:
        L.orc_set_force_exact(0)


def field(kind, params, x, y, t):
    p = np.ascontiguousarray(params, dtype=np.float64)
    fx = ctypes.c_double()
    fy = ctypes.c_double()
    lib().orc_field(int(kind), _ptr(p), float(x), float(y), float(t), ctypes.byref(fx), ctypes.byref(fy))
    return fx.value, fy.value


def feet(kind, params, dt, n, xy):
    """Clipped Euler feet of all points in xy for the step n -> n+1."""
    p = np.ascontiguousarray(params, dtype=np.float64)
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    out = np.empty_like(xy)
    clipped = np.empty(xy.shape[0], dtype=np.uint8)
    lib().orc_feet(int(kind), _ptr(p), float(dt), int(n), xy.shape[0], _ptr(xy), _ptr(out), _ptr(clipped))
    return out, clipped


class OracleMesh:
    """A mesh plus its uniform bin grid, owned by the oracle."""

    def __init__(self, xy, tri):
        self.xy = np.ascontiguousarray(xy, dtype=np.float64)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32)
        self.n = self.xy.shape[0]
        self.nt = self.tri.shape[0]
        self._h = lib().orc_mesh_create(self.n, self.nt, _ptr(self.xy), _ptr(self.tri))
        if not self._h:
            raise MemoryError("orc_mesh_create failed")

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def bins(self):
        return lib().orc_mesh_bins(self._h)

    def locate(self, q, q_lo=None, nthreads=None):
        """Exact location of query points: the lowest-index triangle that
        contains each point and its flags (FLAG_DEGENERATE: on an edge line
        of that triangle; FLAG_MULTI: more than one triangle contains it).
        With q_lo the points are q + q_lo, the sum of each coordinate's two
        doubles taken exactly (a double-float foot)."""
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 2)
        ql = None if q_lo is None else np.ascontiguousarray(q_lo, dtype=np.float64).reshape(-1, 2)
        tri = np.empty(q.shape[0], dtype=np.int32)
        flags = np.empty(q.shape[0], dtype=np.uint8)
        err = lib().orc_locate_points2(self._h, q.shape[0], _ptr(q), _ptr(ql), _ptr(tri), _ptr(flags),
                                       int(nthreads or default_threads()))
        if err:
            raise RuntimeError("oracle: a query point lies in no triangle (mesh does not cover it)")
        return tri, flags

    def signs(self, tri, q, q_lo=None, nthreads=None):
        """Exact orientation signs of each point against the three edges of
        the given triangle (opposite vertex 0, 1, 2): int8 (n, 3), -2 for an
        index that is not a triangle.  The point lies in the closed triangle
        iff all three are >= 0."""
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 2)
        ql = None if q_lo is None else np.ascontiguousarray(q_lo, dtype=np.float64).reshape(-1, 2)
        out = np.empty((q.shape[0], 3), dtype=np.int8)
        lib().orc_tri_signs2(self._h, q.shape[0], _ptr(tri), _ptr(q), _ptr(ql), _ptr(out),
                             int(nthreads or default_threads()))
        return out

    def interp(self, j, X, Y, V):
        V = np.ascontiguousarray(V, dtype=np.float64)
        return lib().orc_interp(self._h, int(j), float(X), float(Y), _ptr(V))

    def step(self, kind, params, dt, n, vin, lo=0, hi=None, nthreads=None, want_feet=True, exclude=False):
        """One step n -> n+1 on nodes [lo, hi).  Returns (vout, tri, flags, feet)
        restricted to that range.  exclude: nodes whose Euler foot leaves the
        square keep their value (flag FLAG_EXCLUDED, tri -1) instead of being
        clipped (Sec. 4)."""
        hi = self.n if hi is None else hi
        cnt = hi - lo
        p = np.ascontiguousarray(params, dtype=np.float64)
        vin = np.ascontiguousarray(vin, dtype=np.float64)
        vout = np.zeros(self.n, dtype=np.float64)
        tri = np.full(self.n, -1, dtype=np.int32)
        flags = np.zeros(self.n, dtype=np.uint8)
        ft = np.zeros((self.n, 2), dtype=np.float64) if want_feet else None
        err = lib().orc_step_range_x(self._h, int(kind), _ptr(p), float(dt), int(n), _ptr(vin), _ptr(vout),
                                     _ptr(ft), _ptr(tri), _ptr(flags), int(lo), int(hi),
                                     int(nthreads or default_threads()), 1 if exclude else 0)
        if err:
            raise RuntimeError("oracle: a foot lies in no triangle (mesh does not cover the square)")
        sl = slice(lo, hi)
        return vout[sl], tri[sl], flags[sl], (ft[sl] if want_feet else None)

    def run(self, kind, params, dt, n0, nsteps, v, nthreads=None, record=False, exclude=False):
        """nsteps steps from V^{n0}.  Returns V^{n0+nsteps} (and, with record,
        the list of (V, tri, flags, feet) after every step)."""
        v = np.array(v, dtype=np.float64, copy=True)
        hist = []
        for s in range(nsteps):
            vout, tri, flags, ft = self.step(kind, params, dt, n0 + s, v, nthreads=nthreads, want_feet=record,
                                             exclude=exclude)
            v = vout.copy()
            if record:
                hist.append((v.copy(), tri.copy(), flags.copy(), ft.copy()))
        return (v, hist) if record else v
