"""Pins of the oracle's candidate fit (CPU only).

The fit is a stated reading (the paper fits candidates to their hits, Sec. 8 and Fig. 6,
without defining the fit): algebraic circle fit through the normal equations, one hit
per layer (the one closest to the all-hit circle), signed arcs and a least-squares line.
Each pin checks it against something other than itself:
  * exact helix points from the event generator's forward model: parameters recovered;
  * three hits: the circle through them is the triplet circle, so the fit equals the
    oracle's triplet fit (an independent function of the same definition);
  * the circle equals numpy's SVD least-squares solution of the same algebraic problem;
  * the selection drops the off-circle hit of a layer; collinear and two-layer lists are
    degenerate; B scaling and a 90-degree rotation act exactly as they must.
"""
import numpy as np
import pytest

import oracle
from oracle.core import fit_one, fit_track_points
from paper_1305_4855_gb300 import events as ev

K = 0.299792458e-2


def _helix_points(cfg, n_tracks, seed):
    rng = np.random.default_rng(seed)
    tr = ev._tracks(cfg, rng, n_tracks)
    out = []
    for t in range(n_tracks):
        pts, lay = [], []
        for L, r in enumerate(cfg["geometry"]["radius"]):
            if r <= tr["r_start"][t]:
                continue
            s = ev._first_crossing(tr["sx"][t:t + 1], tr["sy"][t:t + 1], tr["psi"][t:t + 1],
                                   tr["kappa"][t:t + 1], r)[0]
            if not np.isfinite(s):
                break
            x, y = ev._position(tr["sx"][t], tr["sy"][t], tr["psi"][t], tr["kappa"][t], s)
            pts.append([x, y, tr["sz"][t] + tr["cot"][t] * s])
            lay.append(L)
        if len(pts) >= 3:
            out.append((np.array(pts), np.array(lay, dtype=np.int32), tr["truth"][t]))
    return out


def _close(par, truth, rel, floor):
    d = np.abs(par - truth)
    d[0] = min(d[0], 2 * np.pi - d[0])
    return bool(np.all(d <= rel * np.maximum(np.abs(truth), floor))), d


@pytest.mark.parametrize("name", ["barrel4_20trk", "barrel10_500trk", "barrel10_2000trk_precision"])
def test_exact_helix_points_recovered(name):
    cfg = ev.load_workload(name)
    B = cfg["geometry"]["b_tesla"]
    n = 0
    for pts, lay, truth in _helix_points(cfg, 150, 5):
        f = fit_track_points(pts, lay, B)
        assert f["status"] == 0
        ok, d = _close(f["par"], truth, rel=1e-7, floor=1e-3)
        assert ok, (f["par"], truth, d)
        assert f["chi2"][0] < 1e-12 * max(1.0, 1.0 / abs(truth[1]) ** 2)
        assert f["chi2"][1] < 1e-12 and f["use"].all()
        n += 1
    assert n > 100


def test_three_hits_equal_the_triplet_fit():
    cfg = ev.load_workload("barrel10_500trk")
    b = ev.make_batch(cfg)
    B = cfg["geometry"]["b_tesla"]
    rng = np.random.default_rng(3)
    n_ok = 0
    for _ in range(3000):
        la = rng.integers(0, 8)
        idx = [rng.choice(np.nonzero(b.layer == L)[0]) for L in (la, la + 1, la + 2)]
        p = b.xyz[idx].astype(np.float64)
        t = fit_one(p[0], p[1], p[2], B)
        f = fit_track_points(p, np.array([la, la + 1, la + 2]), B)
        if t is None or f["status"] != 0 or (f["amb"] & 4):
            continue
        scale = np.array([np.pi, 2.0, 50.0, 5.5, 30.0])
        d = np.abs(f["par"] - t)
        d[0] = min(d[0], 2 * np.pi - d[0])
        # the two evaluate the same circle by different formulas (FP64): agreement to
        # ~1e-9 relative, more for nearly straight triplets where both lose digits
        assert np.all(d <= 1e-6 * np.maximum(np.abs(t), scale)), (f["par"], t, d)
        n_ok += 1
    assert n_ok > 1000


def test_circle_equals_svd_least_squares():
    rng = np.random.default_rng(9)
    for trial in range(200):
        R = 10 ** rng.uniform(1.5, 4)
        cx, cy = rng.uniform(-R - 50, R + 50, 2)
        ang0 = rng.uniform(0, 2 * np.pi)
        n = int(rng.integers(3, 14))
        ang = ang0 + np.sort(rng.uniform(0, min(1.5, 100.0 / R), n))
        x = cx + R * np.cos(ang) + rng.normal(0, 0.01, n)
        y = cy + R * np.sin(ang) + rng.normal(0, 0.01, n)
        z = rng.normal(0, 5, n)
        pts = np.stack([x, y, z], 1)
        f = fit_track_points(pts, np.arange(n), 3.8)
        if f["status"] != 0:
            continue
        # independent: SVD least squares of x^2 + y^2 + a x + b y + c = 0
        A = np.stack([x, y, np.ones(n)], 1)
        sol = np.linalg.lstsq(A, -(x * x + y * y), rcond=None)[0]
        cx_ref, cy_ref = -sol[0] / 2, -sol[1] / 2
        R_ref = np.sqrt(cx_ref ** 2 + cy_ref ** 2 - sol[2])
        phi0, qopt, d0 = f["par"][:3]
        Rf = 1.0 / (K * 3.8 * abs(qopt))
        sgn = -np.sign(qopt)
        nx, ny = -np.sin(phi0), np.cos(phi0)          # left normal of the direction
        ccx = d0 * nx + sgn * Rf * nx
        ccy = d0 * ny + sgn * Rf * ny
        tol = 1e-7 * R_ref
        assert abs(Rf - R_ref) <= tol and abs(ccx - cx_ref) <= tol and abs(ccy - cy_ref) <= tol, \
            (trial, Rf, R_ref, ccx, cx_ref, ccy, cy_ref)


def test_selection_drops_the_off_circle_hit():
    cfg = ev.load_workload("barrel10_500trk")
    B = cfg["geometry"]["b_tesla"]
    pts, lay, truth = _helix_points(cfg, 40, 21)[0]
    k = len(pts) // 2
    extra = pts[k].copy()
    extra[:2] *= 1.0 + 0.5 / np.hypot(*extra[:2])      # 0.5 cm further out on the same layer
    p2 = np.insert(pts, k + 1, extra, axis=0)
    l2 = np.insert(lay, k + 1, lay[k])
    f = fit_track_points(p2, l2, B)
    assert f["status"] == 0 and f["use"].sum() == len(pts) and not f["use"][k + 1]
    ok, d = _close(f["par"], truth, rel=1e-7, floor=1e-3)
    assert ok, d
    # the same hit listed first: still the on-circle one is kept
    p3 = np.insert(pts, k, extra, axis=0)
    l3 = np.insert(lay, k, lay[k])
    f3 = fit_track_points(p3, l3, B)
    assert not f3["use"][k] and f3["use"][k + 1]


def test_degenerate_lists():
    line = np.array([[1.0, 2.0, 0.0], [2.0, 4.0, 1.0], [3.0, 6.0, 2.0], [4.0, 8.0, 3.0]])
    assert fit_track_points(line, [0, 1, 2, 3], 3.8)["status"] == 2
    two = np.array([[5.0, 0.0, 0.0], [7.0, 1.0, 1.0], [7.1, 1.0, 1.0], [11.0, 3.0, 2.0]])
    assert fit_track_points(two, [0, 1, 1, 1], 3.8)["status"] == 1
    assert fit_track_points(two[:2], [0, 1], 3.8)["status"] == 1


def test_b_scaling_and_rotation():
    cfg = ev.load_workload("barrel10_500trk")
    for pts, lay, truth in _helix_points(cfg, 30, 8)[:20]:
        f1 = fit_track_points(pts, lay, 3.8)
        f2 = fit_track_points(pts, lay, 7.6)
        assert f2["par"][1] * 2 == f1["par"][1]
        assert np.array_equal(np.delete(f2["par"], 1), np.delete(f1["par"], 1))
        rot = np.stack([-pts[:, 1], pts[:, 0], pts[:, 2]], 1)       # +90 degrees about z
        fr = fit_track_points(rot, lay, 3.8)
        dphi = (fr["par"][0] - f1["par"][0] - np.pi / 2 + np.pi) % (2 * np.pi) - np.pi
        assert abs(dphi) < 1e-9
        assert np.allclose(fr["par"][1:], f1["par"][1:], rtol=1e-8, atol=1e-9)


def test_fit_tracks_matches_single_fits():
    cfg = ev.load_workload("barrel4_20trk")
    b = ev.make_batch(cfg)
    rng = np.random.default_rng(1)
    lists = [np.sort(rng.choice(b.n_hits, int(rng.integers(3, 9)), replace=False))
             for _ in range(50)]
    r = oracle.fit_tracks(b.xyz, b.layer, lists, cfg["geometry"]["b_tesla"])
    for t, h in enumerate(lists):
        f = fit_track_points(b.xyz[h].astype(np.float64), b.layer[h], cfg["geometry"]["b_tesla"])
        assert r["status"][t] == f["status"]
        if f["status"] == 0:
            assert np.array_equal(r["par"][t], f["par"]) and np.array_equal(r["use"][t], f["use"])


def test_golden_residual_sums():
    # chi2_rphi and chi2_rz on hit lists whose fitted circle and line are known by
    # symmetry or construction (tests/golden/track_fit_chi2.json): a residual that is not
    # squared, or a sum over a dropped hit, changes them
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                    "track_fit_chi2.json")))
    for c in g["cases"]:
        f = fit_track_points(np.array(c["hits"]), np.array(c["layers"], dtype=np.int32),
                             c["b_tesla"])
        assert f["status"] == 0, c["name"]
        assert np.array_equal(f["use"], np.array(c["used"], dtype=bool)), c["name"]
        ok, d = _close(f["par"], np.array(c["expected"]), rel=1e-9, floor=1e-6)
        assert ok, (c["name"], f["par"], c["expected"], d)
        assert np.allclose(f["chi2"], c["chi2"], rtol=1e-9, atol=1e-12), (c["name"], f["chi2"], c["chi2"])
        assert int(f["amb"]) == c["amb"], (c["name"], f["amb"], c["amb_why"])
