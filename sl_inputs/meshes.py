"""Jittered, shorter-diagonal-split triangle meshes of the unit square.

Numbering (0-based; the paper's Sec. 3 uses 1-based lists V, T):
  node (i, j), 0 <= i, j <= M, has index j*(M+1) + i (x runs fastest);
  cell (l, m), 0 <= l, m < M, owns triangles 2*(M*m + l) and 2*(M*m + l) + 1.
With corners a=(l,m), b=(l+1,m), c=(l+1,m+1), d=(l,m+1):
  diagonal a-c (the shorter one, or a tie):  T[2k] = (a, c, d), T[2k+1] = (a, b, c)
  diagonal b-d (strictly shorter):           T[2k] = (a, b, d), T[2k+1] = (b, c, d)
On the un-jittered grid every cell takes diagonal a-c and T[2k] is the
triangle above it, which is the labelling of the paper's structured Courant
grid (Sec. 4, direct location formula).  Every triangle is listed
counter-clockwise.
"""
from dataclasses import dataclass
import numpy as np

from .rng import uniform01


@dataclass
class Mesh:
    M: int                 # cells per side
    xy: np.ndarray         # (N, 2) float64 node coordinates in [0,1]^2
    tri: np.ndarray        # (Nt, 3) int32 vertex indices, CCW
    jitter: float = 0.0    # jitter half-width in units of h
    graded: bool = False
    seed: int = 0

    @property
    def n_nodes(self):
        return self.xy.shape[0]

    @property
    def n_tri(self):
        return self.tri.shape[0]

    @property
    def h(self):
        return 1.0 / self.M


def _graded_map(v):
    # x -> x + 0.3 sin(2 pi x) / (2 pi): monotone, derivative in [0.7, 1.3].
    return v + 0.3 * np.sin(2.0 * np.pi * v) / (2.0 * np.pi)


def grid_mesh(M, jitter=0.25, seed=1, graded=False):
    """M x M cells, (M+1)^2 nodes, 2 M^2 triangles on [0,1]^2.

    Interior nodes move by i.i.d. U[-jitter*h, jitter*h) per axis (stream 0
    for x, 1 for y, counter = node index).  Nodes on the boundary are not
    jittered at all, so they stay exactly on the boundary.  With `graded`,
    the jittered logical coordinates are mapped by x + 0.3 sin(2 pi x)/(2 pi)
    per axis and boundary coordinates are then set back to exactly 0 or 1.
    """
    M = int(M)
    n1 = M + 1
    h = 1.0 / M
    base = np.arange(n1, dtype=np.float64) / M
    X = np.broadcast_to(base[None, :], (n1, n1)).copy()   # X[j, i]
    Y = np.broadcast_to(base[:, None], (n1, n1)).copy()
    if jitter and M >= 2:
        ji = np.arange(1, M, dtype=np.int64)
        idx = (ji[:, None] * n1 + ji[None, :]).ravel()
        ux = uniform01(seed, 0, idx).reshape(M - 1, M - 1)
        uy = uniform01(seed, 1, idx).reshape(M - 1, M - 1)
        X[1:M, 1:M] += jitter * h * (2.0 * ux - 1.0)
        Y[1:M, 1:M] += jitter * h * (2.0 * uy - 1.0)
    if graded:
        X = _graded_map(X)
        Y = _graded_map(Y)
    X[:, 0] = 0.0
    X[:, M] = 1.0
    Y[0, :] = 0.0
    Y[M, :] = 1.0
    xy = np.empty((n1 * n1, 2), dtype=np.float64)
    xy[:, 0] = X.ravel()
    xy[:, 1] = Y.ravel()

    # diagonals of cell (l, m): a=(l,m) c=(l+1,m+1) ; b=(l+1,m) d=(l,m+1)
    ac2 = (X[1:, 1:] - X[:-1, :-1]) ** 2 + (Y[1:, 1:] - Y[:-1, :-1]) ** 2
    bd2 = (X[1:, :-1] - X[:-1, 1:]) ** 2 + (Y[1:, :-1] - Y[:-1, 1:]) ** 2
    use_ac = (ac2 <= bd2).ravel()
    del X, Y, ac2, bd2
    a = (np.arange(M, dtype=np.int32)[:, None] * n1 + np.arange(M, dtype=np.int32)[None, :]).ravel()
    b = a + 1
    c = a + (n1 + 1)
    d = a + n1
    tri = np.empty((2 * M * M, 3), dtype=np.int32)
    even = tri[0::2]
    odd = tri[1::2]
    even[:, 0] = a
    even[:, 1] = np.where(use_ac, c, b)
    even[:, 2] = d
    odd[:, 0] = np.where(use_ac, a, b)
    odd[:, 1] = np.where(use_ac, b, c)
    odd[:, 2] = np.where(use_ac, c, d)
    return Mesh(M=M, xy=xy, tri=tri, jitter=float(jitter), graded=bool(graded), seed=int(seed))


def courant_grid(M):
    """The paper's structured Courant grid (Sec. 4), mapped to [0,1]^2."""
    return grid_mesh(M, jitter=0.0, seed=0, graded=False)


def shuffled(mesh, seed):
    """The same mesh with nodes and triangles renumbered by seeded random
    permutations (an unstructured numbering with no locality), and the
    vertex list of each triangle rotated by a random amount (orientation
    kept)."""
    n, nt = mesh.n_nodes, mesh.n_tri
    pn = np.argsort(uniform01(seed, 10, np.arange(n)), kind="stable")      # new -> old
    pt = np.argsort(uniform01(seed, 11, np.arange(nt)), kind="stable")
    inv_n = np.empty(n, dtype=np.int64)
    inv_n[pn] = np.arange(n)
    xy = mesh.xy[pn]
    tri = inv_n[mesh.tri[pt]]
    rot = (splitmix_small(seed, nt) % 3).astype(np.int64)
    cols = (np.arange(3)[None, :] + rot[:, None]) % 3
    tri = np.take_along_axis(tri, cols, axis=1).astype(np.int32)
    return Mesh(M=mesh.M, xy=xy, tri=tri, jitter=mesh.jitter, graded=mesh.graded, seed=mesh.seed)


def splitmix_small(seed, n):
    from .rng import splitmix64
    return splitmix64(seed, 12, np.arange(n)) >> np.uint64(40)
