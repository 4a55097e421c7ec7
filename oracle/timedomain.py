"""Time-domain ASHRT / AASHRT by hyperbolic summation, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The adjoint follows ch. 6 Eq. ch6_AASHRT_adjoint (and, with tau0 = 0, the
ASHRT row of ch. 3 Table ch3_table_Radon_operators):
    m~(tau, v, x_a, tau0) = sum_{x_r} d(t = tau0 + sqrt(tau^2 + (x_r - x_a)^2 / v^2), x_r)
with d read at the fractional time by linear interpolation between samples.
The forward is the exact transpose of that adjoint (reading of the garbled
inverse traveltime of Eq. ch6_AASHRT_forward: the path is t = tau0 +
sqrt(tau^2 + h^2), i.e. tau = sqrt((t - tau0)^2 - h^2)).  Every trace position
is also an apex position (x_a == x_r == x).  Defined for v > 0 and tau0 >= 0
(the path then starts inside or after the record).  Cost O(nx^2 nt nv nt0)
(ch. 5, cost of the classical ASHRT).
"""
import numpy as np


def _paths(nt, nx, dt, dx, v, t0):
    if not (v > 0.0) or not (t0 >= 0.0):
        raise ValueError("the time-domain pair needs v > 0 and tau0 >= 0")
    tau = np.arange(nt) * dt
    for a in range(nx):
        for r in range(nx):
            h = (r - a) * dx / v
            s = (t0 + np.sqrt(tau * tau + h * h)) / dt
            i0 = np.floor(s).astype(np.int64)
            f = s - i0
            ok0 = i0 < nt
            ok1 = (i0 + 1) < nt
            yield a, r, i0, f, ok0, ok1


def adjoint(nt, nx, dt, dx, velocities, d, t0s=(0.0,)):
    """m~[nt0][nv][nx][nt] from d[nx][nt] (Eq. ch6_AASHRT_adjoint)."""
    v = np.asarray(velocities, dtype=np.float32).astype(np.float64)
    t0 = np.asarray(t0s, dtype=np.float32).astype(np.float64)
    d = np.asarray(d, dtype=np.float64)
    m = np.zeros((len(t0), len(v), nx, nt))
    for j, tj in enumerate(t0):
        for i, vi in enumerate(v):
            for a, r, i0, f, ok0, ok1 in _paths(nt, nx, dt, dx, vi, tj):
                acc = np.zeros(nt)
                acc[ok0] += (1.0 - f[ok0]) * d[r, i0[ok0]]
                acc[ok1] += f[ok1] * d[r, i0[ok1] + 1]
                m[j, i, a] += acc
    return m


def forward(nt, nx, dt, dx, velocities, m, t0s=(0.0,)):
    """d[nx][nt] from m[nt0][nv][nx][nt]: the transpose of ``adjoint``."""
    v = np.asarray(velocities, dtype=np.float32).astype(np.float64)
    t0 = np.asarray(t0s, dtype=np.float32).astype(np.float64)
    m = np.asarray(m, dtype=np.float64).reshape(len(t0), len(v), nx, nt)
    d = np.zeros((nx, nt))
    for j, tj in enumerate(t0):
        for i, vi in enumerate(v):
            for a, r, i0, f, ok0, ok1 in _paths(nt, nx, dt, dx, vi, tj):
                np.add.at(d[r], i0[ok0], (1.0 - f[ok0]) * m[j, i, a][ok0])
                np.add.at(d[r], i0[ok1] + 1, f[ok1] * m[j, i, a][ok1])
    return d
