"""Additive continuous collision detection (oracle, FP64).

Conservative advancement in the form of "additive CCD" (Li, Kaufman & Jiang
2021, Codimensional IPC): with the points of a pair moving linearly,
x(t) = x0 + t p, the mean displacement is removed and
l_p = max |p| over the first primitive + max |p| over the second bounds how
fast the distance can shrink.  Starting from d0 = d(x0), the pair is advanced
by (1 - s) d0 / l_p and then by 0.9 d / l_p at the current distance d; the
loop stops before the step after which the distance falls below s * d0 and
reports the time reached, a lower bound on the time of impact at which the
distance is still at least s * d0 > 0.  s = 0.1 here; a pair that reaches
t_max without stopping is collision-free on [0, t_max].
"""
import numpy as np

from .geometry import distance_sq


def accd(x0, p, kind, s=0.1, t_max=1.0, max_iter=100000):
    """Per-pair conservative TOI for points x0 (n,4,3) moving by p (n,4,3).
    Returns t (n,) with t >= t_max meaning no impact before t_max."""
    n = x0.shape[0]
    out = np.full(n, np.inf)
    if n == 0:
        return out
    p = p - p.mean(axis=1, keepdims=True)
    nrm = np.linalg.norm(p, axis=2)
    if kind == "pt":
        lp = nrm[:, 0] + nrm[:, 1:].max(axis=1)
    else:
        lp = nrm[:, :2].max(axis=1) + nrm[:, 2:].max(axis=1)
    d0 = np.sqrt(distance_sq(x0, kind)[0])
    touching = (lp > 0) & ~(d0 > 0)
    out[touching] = 0.0
    active = (lp > 0) & (d0 > 0)
    g = s * d0
    t = np.zeros(n)
    step = np.where(active, (1.0 - s) * d0 / np.where(active, lp, 1.0), 0.0)
    idx = np.nonzero(active)[0]
    it = 0
    while len(idx) > 0 and it < max_iter:
        it += 1
        tn = t[idx] + step[idx]
        d = np.sqrt(distance_sq(x0[idx] + tn[:, None, None] * p[idx], kind)[0])
        stop = (t[idx] > 0) & (d < g[idx])
        out[idx[stop]] = t[idx[stop]]
        go = ~stop
        t[idx[go]] = tn[go]
        over = go & (tn > t_max)
        # no impact within [0, t_max]
        go &= ~over
        step[idx] = 0.9 * d / lp[idx]
        idx = idx[go]
    if len(idx) > 0:  # iteration cap: report the safe time reached
        out[idx] = t[idx]
    return out
