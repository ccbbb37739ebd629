"""Pins of the 2-D per-hit Hough oracle (CPU only): straight lines (Sec. 7, Fig. 3) and
curved tracks through the interaction point (Sec. 8, Fig. 5).

  * exact points on a line / on a circle through the origin: at the true column every
    hit's row value equals the true rho / q/pT (closed form), so all of them vote in one bin;
  * the row value of a hit is the independent geometric quantity: the distance of the line
    to the origin for rho, and 1/(K B R) of the circle through the origin, the hit and the
    column's direction (checked against the circle built from its centre);
  * the mirror wrap of the straight case: theta = 0 and pi are the same line with rho
    negated (hand-built histogram), and the curved case wraps phi0;
  * the peak rule on hand-built 2-D histograms, and a brute-force peak check.
"""
import numpy as np
import pytest

from oracle import hough2d as H

K = 0.299792458e-2


def _setup(kind, n_cols=64, n_rows=32, lo=-8.0, hi=8.0, T=3, b=0.0):
    return H.Hough2DSetup(kind=kind, n_cols=n_cols, n_rows=n_rows, lo=lo, hi=hi, threshold=T,
                          b_tesla=b)


def test_column_centres_hand_worked():
    # columns sit at the centres of equal slices of the angle range: two straight columns at
    # 45 and 135 degrees, four at 22.5, 67.5, 112.5, 157.5; four curved (phi0 over a full
    # turn) at -135, -45, 45, 135 degrees
    pi = np.pi
    assert np.allclose(_setup("straight", n_cols=2).columns(), [pi / 4, 3 * pi / 4], atol=1e-15)
    assert np.allclose(_setup("straight", n_cols=4).columns(),
                       [pi / 8, 3 * pi / 8, 5 * pi / 8, 7 * pi / 8], atol=1e-15)
    assert np.allclose(_setup("curved_ip", n_cols=4, b=3.8).columns(),
                       [-3 * pi / 4, -pi / 4, pi / 4, 3 * pi / 4], atol=1e-15)
    # the hit (1, 0) lies on the lines x cos(t) + y sin(t) = rho with rho = cos(t): at 45 and
    # 135 degrees rho = +-sqrt(2)/2, rows 19 and 4 of 24 rows of width 0.1 from -1.2
    s = _setup("straight", n_cols=2, n_rows=24, lo=-1.2, hi=1.2)
    j, _ = H.votes(np.array([[1.0, 0.0]]), s)
    assert j[0].tolist() == [19, 4]


def test_single_column_rows_edges_and_centres():
    # one straight column sits at 90 degrees, where the row value of a hit (0, y) is y
    # itself: rows of width 0.5 over [-1, 1).  y = 0.5 is on the edge between rows 2 and 3
    # (ambiguous), y = 0.3 is inside row 2, y = -1 is the first row, y = 1 is outside.
    s = _setup("straight", n_cols=1, n_rows=4, lo=-1.0, hi=1.0, T=2)
    j, amb = H.votes(np.array([[0.0, 0.5], [0.0, 0.3], [0.0, -1.0], [0.0, 1.0]]), s)
    assert j[:, 0].tolist() == [3, 2, 0, -1]
    assert amb[:, 0].tolist() == [True, False, True, True]
    # three hits on the line y = 0.3 vote in row 2, whose centre is -1 + 2.5 * 0.5 = 0.25
    ev = H.reconstruct(np.array([[0.0, 0.3], [5.0, 0.3], [-5.0, 0.3]]), np.array([0, 3]), s)[0]
    assert ev["cand_bins"].tolist() == [2] and ev["cand_votes"].tolist() == [3]
    assert np.allclose(ev["cand_params"], [[np.pi / 2, 0.25]], atol=1e-15)
    assert ev["cand_hits"][0].tolist() == [0, 1, 2]


def test_vertex_raster_and_centre_hand_worked():
    vs = H.VertexSetup(n_bins=4, range=2.0, threshold=2)
    # the line through the origin at 60 degrees, y = -x / sqrt(3), is rastered along x
    # (|sin| >= |cos|): at the column centres -1.5, -0.5, 0.5, 1.5 it has y = 0.87, 0.29,
    # -0.29, -0.87, rows 2, 2, 1, 1: cells 0*4+2, 1*4+2, 2*4+1, 3*4+1
    cells = [v[0] for v in H.vertex_votes(np.array([[np.pi / 3, 0.0]]), vs)[0]]
    assert cells == [2, 6, 9, 13]
    # the vertical line x = 1.5 and the horizontal line y = -0.5 meet in cell (3, 1), whose
    # centre is (1.5, -0.5)
    r = H.vertex_hough(np.array([[0.0, 1.5], [np.pi / 2, -0.5]]), vs)
    assert r["cells"].tolist() == [13] and r["votes"].tolist() == [2]
    assert np.allclose(r["centres"], [[1.5, -0.5]])
    assert r["tracks"][0].tolist() == [0, 1]


def test_vertex_minimum_votes_is_inclusive():
    # candidates with exactly min_track_votes votes draw their lines; fewer do not
    vs = H.VertexSetup(n_bins=4, range=2.0, threshold=2, min_track_votes=3)
    event = dict(cand_votes=np.array([3, 2, 3]),
                 cand_params=np.array([[0.0, 1.5], [np.pi / 3, 0.0], [np.pi / 2, -0.5]]))
    r = H.event_vertices(event, vs)
    assert r["cells"].tolist() == [13] and r["tracks"][0].tolist() == [0, 2]


def test_vertex_grid_is_half_open():
    # a vertical line x = rho (theta = 0) votes once per y row in the x column of rho; the
    # grid covers [-2, 2) in 5 cells: x = -2 is inside (column 0), x = +2 is outside
    vs = H.VertexSetup(n_bins=5, range=2.0, threshold=2)
    inside, outside = H.vertex_votes(np.array([[0.0, -2.0], [0.0, 2.0]]), vs)
    assert [v[0] for v in inside] == [0, 1, 2, 3, 4]
    assert outside == []


def test_straight_line_points_vote_in_one_bin():
    s = _setup("straight", n_cols=180, n_rows=64, lo=-16.0, hi=16.0)
    rng = np.random.default_rng(1)
    for _ in range(50):
        c = int(rng.integers(0, s.n_cols))
        theta = s.columns()[c]
        rho = rng.uniform(-15, 15)
        t = rng.uniform(-100, 100, 10)
        x = rho * np.cos(theta) - t * np.sin(theta)
        y = rho * np.sin(theta) + t * np.cos(theta)
        v = s.row_values(x, y)[:, c]
        assert np.allclose(v, rho, atol=1e-12)
        j, _ = H.votes(np.stack([x, y], 1), s)
        assert len(set(j[:, c].tolist())) == 1


def test_curved_ip_points_vote_in_one_bin():
    B = 3.8
    s = _setup("curved_ip", n_cols=256, n_rows=64, lo=-1.0, hi=1.0, b=B)
    rng = np.random.default_rng(2)
    for _ in range(50):
        c = int(rng.integers(0, s.n_cols))
        phi0 = s.columns()[c]
        qopt = rng.uniform(-0.9, 0.9)
        R = 1.0 / (K * B * abs(qopt))
        sense = -np.sign(qopt)              # counter-clockwise (+) for negative charge
        # circle through the origin leaving in direction phi0: centre at R along the normal
        cx, cy = -sense * R * np.sin(phi0), sense * R * np.cos(phi0)
        ang = np.arctan2(-cy, -cx) + sense * rng.uniform(0.01, 1.0, 10)
        x, y = cx + R * np.cos(ang), cy + R * np.sin(ang)
        v = s.row_values(x, y)[:, c]
        assert np.allclose(v, qopt, rtol=1e-10, atol=1e-12)


def test_curved_row_value_is_the_circle_through_origin_and_hit():
    B = 2.0
    s = _setup("curved_ip", n_cols=32, lo=-5.0, hi=5.0, b=B)
    rng = np.random.default_rng(3)
    x, y = rng.uniform(-50, 50, 20), rng.uniform(-50, 50, 20)
    v = s.row_values(x, y)
    for k in range(20):
        for c, phi0 in enumerate(s.columns()):
            # independent: centre on the normal to the direction at the origin, equidistant
            # from the origin and the hit: c = t n, |t n - p|^2 = t^2 -> t = |p|^2 / (2 n.p)
            n = np.array([-np.sin(phi0), np.cos(phi0)])
            p = np.array([x[k], y[k]])
            t = p @ p / (2 * (n @ p))
            ccw = t > 0                       # centre on the left: counter-clockwise
            qopt = (-1.0 if ccw else 1.0) / (K * B * abs(t))
            assert np.isclose(v[k, c], qopt, rtol=1e-9)


def test_straight_mirror_wrap_and_peak_rule():
    s = _setup("straight", n_cols=8, n_rows=6, lo=-3.0, hi=3.0, T=2)
    h = np.zeros(48, dtype=np.int64)
    # (0, 1) = 5; its neighbour across the wrap is column 7, rows mirrored: 6-1-(1+dj)
    h[0 * 6 + 1] = 5
    h[7 * 6 + 4] = 5                       # mirror of row 1 in column 7: the same count
    assert sorted(H.neighbours(0, 1, s)) == sorted([6 + 0, 6 + 1, 6 + 2, 0, 2,
                                                    7 * 6 + 5, 7 * 6 + 4, 7 * 6 + 3])
    # the tie goes to the smaller bin number: bin 1 is the peak, bin 46 is not
    assert H.peaks(h, s).tolist() == [1]
    h[7 * 6 + 4] = 6
    assert H.peaks(h, s).tolist() == [46]
    c = _setup("curved_ip", n_cols=8, n_rows=6, lo=-1.0, hi=1.0, T=2, b=1.0)
    assert sorted(H.neighbours(0, 0, c)) == sorted([7 * 6 + 0, 7 * 6 + 1, 1, 6, 7])


def test_peaks_brute_force():
    rng = np.random.default_rng(4)
    for kind in ("straight", "curved_ip"):
        s = _setup(kind, n_cols=12, n_rows=9, lo=-1.0, hi=1.0, T=2, b=1.0)
        for _ in range(100):
            h = rng.integers(0, 5, s.n_cols * s.n_rows)
            got = H.peaks(h, s).tolist()
            want = []
            for b in range(len(h)):
                if h[b] < s.threshold:
                    continue
                c, j = divmod(b, s.n_rows)
                nb = []
                for dc in (-1, 0, 1):
                    for dj in (-1, 0, 1):
                        if dc == dj == 0:
                            continue
                        cc = c + dc
                        jj = j + dj
                        if not 0 <= cc < s.n_cols:
                            cc %= s.n_cols
                            if kind == "straight":
                                jj = s.n_rows - 1 - jj
                        if 0 <= jj < s.n_rows:
                            nb.append(cc * s.n_rows + jj)
                if all(h[b] >= h[n] for n in nb) and all(h[b] > h[n] for n in nb if n < b):
                    want.append(b)
            assert got == want


def test_votes_and_hits_consistent():
    s = _setup("curved_ip", n_cols=128, n_rows=32, lo=-1.0, hi=1.0, T=3, b=3.8)
    rng = np.random.default_rng(5)
    xy = rng.uniform(-100, 100, (300, 2))
    ev = H.reconstruct(xy, np.array([0, 150, 300]), s)
    for e, (a, b) in enumerate([(0, 150), (150, 300)]):
        hh = ev[e]["hist"]
        j, _ = H.votes(xy[a:b], s)
        assert hh.sum() == (j >= 0).sum()
        for bb, hits in zip(ev[e]["cand_bins"], ev[e]["cand_hits"]):
            assert len(hits) == hh[bb] and np.all((hits >= a) & (hits < b))


# ---------------------------------------------------------------------------------------
# the second transform (displaced-jet vertices)
# ---------------------------------------------------------------------------------------

def test_lines_through_a_point_meet_in_its_cell():
    vs = H.VertexSetup(n_bins=64, range=64.0, threshold=3)
    rng = np.random.default_rng(6)
    w = 2 * vs.range / vs.n_bins
    for _ in range(30):
        x0, y0 = rng.uniform(-60, 60, 2)
        thetas = rng.uniform(0, np.pi, 8)
        rhos = x0 * np.cos(thetas) + y0 * np.sin(thetas)
        r = H.vertex_hough(np.stack([thetas, rhos], 1), vs)
        cell = int(np.floor((x0 + vs.range) / w)) * vs.n_bins + int(np.floor((y0 + vs.range) / w))
        # each line passes through the vertex; its raster may take the neighbouring cell of
        # the swept column or row, never farther
        a0, b0 = divmod(cell, vs.n_bins)
        near = [i for i in range(vs.n_bins ** 2)
                if abs(i // vs.n_bins - a0) <= 1 and abs(i % vs.n_bins - b0) <= 1]
        assert r["hist"][near].sum() >= 8
        assert any(abs(c // vs.n_bins - a0) <= 1 and abs(c % vs.n_bins - b0) <= 1
                   for c in r["cells"])


def test_line_raster_one_vote_per_step():
    vs = H.VertexSetup(n_bins=32, range=10.0, threshold=1)
    for theta in (0.1, 0.7, np.pi / 4, 1.2, np.pi / 2, 2.5, 3.0):
        votes = H.vertex_votes(np.array([[theta, 1.5]]), vs)[0]
        by_col = abs(np.sin(theta)) >= abs(np.cos(theta))
        steps = [a for (_, _, bc, a, _) in votes]
        assert len(steps) == len(set(steps)) and all(bc == by_col for (_, _, bc, _, _) in votes)
        # the raster is connected: consecutive steps move at most one cell across
        ks = [k for (*_, k) in votes]
        assert all(abs(k1 - k0) <= 1 for k0, k1 in zip(ks, ks[1:]))
        # every voted cell centre lies within half a diagonal of the line
        w = 2 * vs.range / vs.n_bins
        for cell, *_ in votes:
            a, b = divmod(cell, vs.n_bins)
            xc, yc = -vs.range + (a + 0.5) * w, -vs.range + (b + 0.5) * w
            assert abs(xc * np.cos(theta) + yc * np.sin(theta) - 1.5) <= w * 0.75


def test_vertex_peak_rule_no_wrap():
    vs = H.VertexSetup(n_bins=5, range=5.0, threshold=2)
    assert sorted(H.vertex_neighbours(0, vs)) == [1, 5, 6]
    assert len(H.vertex_neighbours(12, vs)) == 8
