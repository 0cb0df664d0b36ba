"""Line solves (oracle; test infrastructure).

Sec. 4: every factor of the direction-split operator is a tridiagonal system
along one grid line, solved directly by the Thomas algorithm (Gaussian
elimination without pivoting, forward elimination then back substitution).
"""
from __future__ import annotations

import numpy as np


def thomas(lo, di, up, b, axis):
    """Solve lo[m] x[m-1] + di[m] x[m] + up[m] x[m+1] = b[m] along ``axis``
    for every line at once (lo of the first row and up of the last row are
    ignored)."""
    lo, di, up, b = (np.moveaxis(np.asarray(a, dtype=np.float64), axis, 0) for a in (lo, di, up, b))
    n = b.shape[0]
    cp = np.empty_like(b)
    dp = np.empty_like(b)
    cp[0] = up[0] / di[0]
    dp[0] = b[0] / di[0]
    for m in range(1, n):
        den = di[m] - lo[m] * cp[m - 1]
        cp[m] = up[m] / den
        dp[m] = (b[m] - lo[m] * dp[m - 1]) / den
    x = np.empty_like(b)
    x[n - 1] = dp[n - 1]
    for m in range(n - 2, -1, -1):
        x[m] = dp[m] - cp[m] * x[m + 1]
    return np.moveaxis(x, 0, axis)


AXIS = {"r": 1, "t": 2, "p": 3}


def solve_factored(factors, order, b):
    """Apply the inverse of the factored operator P = F_1 F_2 F_3 (F_1 the
    first factor of ``order``): solve F_1 y1 = b, F_2 y2 = y1, F_3 x = y2
    (Sec. 4: the leftmost factor is solved first)."""
    y = b
    for d in order:
        lo, di, up = factors[d]
        y = thomas(lo, di, up, y, AXIS[d])
    return y
