"""An independently written naive reconstructor for tiny events (pins the oracle).

It shares nothing with the C oracle: the circle comes from the linear system
x^2 + y^2 + E x + F y + G = 0 (numpy.linalg.solve), the sense of motion from the order of
the polar angles about the centre, signed path lengths from the angle swept about the
centre in the sense of motion (negative before the perigee),
the longitudinal line from numpy.polyfit, bin indices from numpy.searchsorted on
numpy.linspace edges, and the enumeration walks every ordered triple of distinct hits,
keeping those whose layers form a listed layer triple.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

K = 0.299792458e-2


def helix(p1, p2, p3, b_tesla):
    """(phi0, q/pT, d0, cot, z0) or None (degenerate)."""
    P = [np.asarray(p, dtype=np.float64) for p in (p1, p2, p3)]
    A = np.array([[p[0], p[1], 1.0] for p in P])
    rhs = -np.array([p[0] ** 2 + p[1] ** 2 for p in P])
    det = np.linalg.det(A)
    if abs(det) < 1e-300 or ((P[1][0] - P[0][0]) * (P[2][1] - P[0][1])
                             == (P[1][1] - P[0][1]) * (P[2][0] - P[0][0])):
        # collinear: the straight line from p1 towards p3
        d = P[2][:2] - P[0][:2]
        if not np.any(d):
            return None
        t = d / np.hypot(*d)
        foot = P[0][:2] - np.dot(P[0][:2], t) * t
        phi0 = math.atan2(t[1], t[0])
        d0 = -foot[0] * math.sin(phi0) + foot[1] * math.cos(phi0)
        # signed distance along the direction of motion
        s = np.array([np.dot(p[:2] - foot, t) for p in P])
        qopt = 0.0
    else:
        E, F, G = np.linalg.solve(A, rhs)
        c = np.array([-E / 2.0, -F / 2.0])
        R = math.sqrt(c @ c - G)
        th = [math.atan2(p[1] - c[1], p[0] - c[0]) for p in P]
        ccw = ((th[1] - th[0]) % (2 * math.pi)) < ((th[2] - th[0]) % (2 * math.pi))
        cn = math.hypot(*c)
        if cn == 0.0:
            return None
        foot = c - R * c / cn
        r = (foot - c) / R
        tan = np.array([-r[1], r[0]]) if ccw else np.array([r[1], -r[0]])
        phi0 = math.atan2(tan[1], tan[0])
        d0 = -foot[0] * math.sin(phi0) + foot[1] * math.cos(phi0)
        qopt = (-1.0 if ccw else 1.0) / (K * b_tesla * R)
        thp = math.atan2(foot[1] - c[1], foot[0] - c[0])
        s = []
        for t_ in th:
            # angle swept from the perigee in the sense of motion, in (-pi, pi]
            dth = (t_ - thp + math.pi) % (2 * math.pi) - math.pi
            s.append(R * (dth if ccw else -dth))
        s = np.array(s)
    z = np.array([p[2] for p in P])
    if np.ptp(s) == 0.0:
        return None
    cot, z0 = np.polyfit(s, z, 1)
    return np.array([phi0, qopt, d0, cot, z0])


def bin_of(par, lo, hi, n, periodic):
    """Row-major bin or None if some parameter is out of range."""
    lin = 0
    for k in range(5):
        p = par[k]
        if periodic[k]:
            p = (p - lo[k]) % (hi[k] - lo[k]) + lo[k]
        edges = np.linspace(lo[k], hi[k], n[k] + 1)
        i = int(np.searchsorted(edges, p, side="right")) - 1
        if i < 0 or i >= n[k] or p >= hi[k]:
            return None
        lin = lin * int(n[k]) + i
    return lin


def enumerate_event(xyz, layer, triples, b_tesla, lo, hi, n, periodic):
    """Accepted triplets of one event: dict (i, j, k) -> (bin, params)."""
    allowed = {tuple(int(v) for v in t) for t in triples}
    N = len(xyz)
    out = {}
    for i, j, k in itertools.permutations(range(N), 3):
        if (int(layer[i]), int(layer[j]), int(layer[k])) not in allowed:
            continue
        par = helix(xyz[i], xyz[j], xyz[k], b_tesla)
        if par is None:
            continue
        b = bin_of(par, lo, hi, n, periodic)
        if b is not None:
            out[(i, j, k)] = (b, par)
    return out
