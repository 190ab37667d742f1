"""Exact rational helpers used by the tests as an independent yardstick
(Python Fractions; nothing here is shared with the oracle or the library)."""
from fractions import Fraction as F


def orient(a, b, c):
    """Sign of the signed area of (a, b, c) in exact rational arithmetic."""
    ax, ay, bx, by, cx, cy = (F(float(v)) for v in (a[0], a[1], b[0], b[1], c[0], c[1]))
    d = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
    return (d > 0) - (d < 0)


def contains(xy, tri_row, q):
    """Signs of q against the three edges of a CCW triangle (vertex k's
    opposite edge first); q is inside or on the boundary iff all >= 0."""
    p1, p2, p3 = (xy[v] for v in tri_row)
    return (orient(p2, p3, q), orient(p3, p1, q), orient(p1, p2, q))


def orient_pair(a, b, qh, ql):
    """orient(a, b, q) for the point q = qh + ql (coordinate sums exact)."""
    q = (F(float(qh[0])) + F(float(ql[0])), F(float(qh[1])) + F(float(ql[1])))
    ax, ay, bx, by = (F(float(v)) for v in (a[0], a[1], b[0], b[1]))
    d = (bx - ax) * (q[1] - ay) - (by - ay) * (q[0] - ax)
    return (d > 0) - (d < 0)
