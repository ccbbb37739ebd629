"""Per-hit 2-D Hough transforms, FP64 numpy oracle.  TEST INFRASTRUCTURE ONLY.

Two parameter spaces, each swept one column at a time by every hit (plain definition: no
pruning, no blocking; the histogram, peak rule and hit lists follow directly):

* straight lines (Sec. 7 and Fig. 3: each hit of a straight track traces a sinusoid in the
  parameter space; peaks are tracks).  Reading: the line x cos(theta) + y sin(theta) = rho;
  column c has theta_c = (c + 1/2) pi / n_cols in [0, pi); the row value of a hit is
  rho = x cos(theta_c) + y sin(theta_c).
* curved tracks through the interaction point (Sec. 8 and Fig. 5: the curves are constrained
  to pass through the interaction point, which leaves a 2-D space like the straight case).
  Reading: a circle through the origin leaving it in direction phi0 with signed curvature;
  column c has phi0_c = -pi + (c + 1/2) 2 pi / n_cols; the row value of a hit is the q/pT of
  the circle through the origin and the hit with that direction,
  q/pT = 2 (x sin(phi0_c) - y cos(phi0_c)) / (K B (x^2 + y^2)), with q = -sign of the turn
  (counter-clockwise is negative), K = 0.299792458e-2 GeV/(T cm).

For both: row bin j = floor((v - lo) / ((hi - lo) / n_rows)), a vote iff lo <= v < hi;
histogram h[c][j] per event, linear index c * n_rows + j.  Neighbours of (c, j): the 8 bins
(c + dc, j + dj); rows outside the range are skipped; columns wrap: for curved tracks
c +- n_cols is the same phi0; for straight lines theta and theta + pi are the same line with
rho negated, so column -1 is column n_cols - 1 and column n_cols is column 0, with the row
mirrored (j -> n_rows - 1 - j; the rho range must be symmetric).  Peak rule as for the 5-D
space: h >= T, h >= every neighbour, h > every neighbour with a smaller linear index.
A candidate's hits are the hits whose vote went to its bin, sorted by input index.
Ambiguity: a vote whose value lies within eps = eps_rel * max(|v|, half-range) of a bin
edge or range limit is flagged (its FP32 bin may differ).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

K = 0.299792458e-2


@dataclass
class Hough2DSetup:
    kind: str                 # "straight" or "curved_ip"
    n_cols: int
    n_rows: int
    lo: float                 # row range
    hi: float
    threshold: int
    b_tesla: float = 0.0
    eps_rel: float = 1e-5

    @classmethod
    def from_workload(cls, cfg: dict) -> "Hough2DSetup":
        h = cfg["hough2d"]
        return cls(kind=h["kind"], n_cols=int(h["n_cols"]), n_rows=int(h["n_rows"]),
                   lo=float(h["lo"]), hi=float(h["hi"]), threshold=int(h["threshold"]),
                   b_tesla=float(cfg["geometry"].get("b_tesla", 0.0)))

    def columns(self) -> np.ndarray:
        c = np.arange(self.n_cols, dtype=np.float64) + 0.5
        if self.kind == "straight":
            return c * np.pi / self.n_cols
        return -np.pi + c * 2.0 * np.pi / self.n_cols

    def row_values(self, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        """(n_hits, n_cols) row values of every hit at every column."""
        x = np.asarray(x, dtype=np.float64)[:, None]
        y = np.asarray(y, dtype=np.float64)[:, None]
        a = self.columns()[None, :]
        if self.kind == "straight":
            return x * np.cos(a) + y * np.sin(a)
        return 2.0 * (x * np.sin(a) - y * np.cos(a)) / (K * self.b_tesla * (x * x + y * y))


def votes(xy: np.ndarray, s: Hough2DSetup):
    """Per hit and column: row bin (-1: out of range) and the ambiguity flag."""
    v = s.row_values(xy[:, 0], xy[:, 1])
    w = (s.hi - s.lo) / s.n_rows
    inside = (v >= s.lo) & (v < s.hi)
    j = np.where(inside, np.floor((v - s.lo) / w), -1).astype(np.int64)
    j = np.where(inside, np.minimum(j, s.n_rows - 1), -1)
    eps = s.eps_rel * np.maximum(np.abs(v), 0.5 * (s.hi - s.lo))
    t = (v - s.lo) / w
    near_edge = np.abs(t - np.round(t)) * w <= eps
    near_limit = (np.abs(v - s.lo) <= eps) | (np.abs(v - s.hi) <= eps)
    return j, near_edge | near_limit


def histogram(j: np.ndarray, s: Hough2DSetup) -> np.ndarray:
    h = np.zeros(s.n_cols * s.n_rows, dtype=np.int64)
    cols = np.broadcast_to(np.arange(s.n_cols)[None, :], j.shape)
    ok = j >= 0
    np.add.at(h, cols[ok] * s.n_rows + j[ok], 1)
    return h


def neighbours(c: int, j: int, s: Hough2DSetup):
    """Linear indices of the neighbours of (c, j) (the wrap and mirror rules above)."""
    out = []
    for dc in (-1, 0, 1):
        for dj in (-1, 0, 1):
            if dc == 0 and dj == 0:
                continue
            cc, jj = c + dc, j + dj
            if cc < 0 or cc >= s.n_cols:
                cc %= s.n_cols
                if s.kind == "straight":
                    jj = s.n_rows - 1 - jj
            if jj < 0 or jj >= s.n_rows:
                continue
            nb = cc * s.n_rows + jj
            if nb != c * s.n_rows + j:
                out.append(nb)
    return out


def peaks(h: np.ndarray, s: Hough2DSetup) -> np.ndarray:
    """Candidate bins (sorted) by the peak rule, neighbour by neighbour."""
    out = []
    for b in np.nonzero(h >= s.threshold)[0]:
        c, j = divmod(int(b), s.n_rows)
        ok = True
        for nb in neighbours(c, j, s):
            if h[nb] > h[b] or (nb < b and h[nb] == h[b]):
                ok = False
                break
        if ok:
            out.append(int(b))
    return np.array(out, dtype=np.int64)


def reconstruct(xy: np.ndarray, offsets: np.ndarray, s: Hough2DSetup) -> list:
    """Per event: histogram, candidates (bins, votes, centre parameters), hit lists (global
    input indices), and the ambiguous (hit, column) votes."""
    events = []
    w = (s.hi - s.lo) / s.n_rows
    cols = s.columns()
    for e in range(len(offsets) - 1):
        a, b = int(offsets[e]), int(offsets[e + 1])
        j, amb = votes(xy[a:b], s)
        h = histogram(j, s)
        cb = peaks(h, s)
        hits = []
        for bb in cb:
            c, r = divmod(int(bb), s.n_rows)
            hits.append(a + np.nonzero(j[:, c] == r)[0].astype(np.int64))
        amb_bins = set()
        hh, cc = np.nonzero(amb & (j >= 0))
        for k, c in zip(hh, cc):
            amb_bins.add(int(c * s.n_rows + j[k, c]))
            # the FP32 value may fall in the adjacent bin instead
            for d in (-1, 1):
                jj = j[k, c] + d
                if 0 <= jj < s.n_rows:
                    amb_bins.add(int(c * s.n_rows + jj))
        hh, cc = np.nonzero(amb & (j < 0))
        for k, c in zip(hh, cc):      # just outside the range: the edge row may gain it
            v = s.row_values(xy[a + k:a + k + 1, 0], xy[a + k:a + k + 1, 1])[0, c]
            amb_bins.add(int(c * s.n_rows + (0 if v < s.lo + w else s.n_rows - 1)))
        centres = np.stack([cols[cb // s.n_rows], s.lo + (cb % s.n_rows + 0.5) * w], 1) \
            if len(cb) else np.zeros((0, 2))
        events.append(dict(hist=h, cand_bins=cb, cand_votes=h[cb], cand_params=centres,
                           cand_hits=hits, amb_bins=amb_bins))
    return events


# ---------------------------------------------------------------------------------------
# Second transform: displaced-jet vertices (Sec. 9 and Figs. 7-8: the track peaks of a
# displaced jet lie on one sinusoid of the (theta, rho) space, the sinusoid of the jet's
# vertex, and a second Hough transform over the peaks finds it).
# Reading: a vertex (xv, yv) lies on every track line x cos(theta) + y sin(theta) = rho of
# its jet, so each straight-line candidate votes along its line in a binned (xv, yv)
# space: n_bins x n_bins cells over [-range, range)^2, cell centres g_a = -range + (a + 1/2) w.
# A candidate with |sin theta| >= |cos theta| votes once per x column, in the row of
# y = (rho - g_a cos theta) / sin theta; otherwise once per y row, in the column of
# x = (rho - g_b sin theta) / cos theta (a connected raster of the line).  (theta, rho) are
# the candidate's bin centres.  Cell (a, b) has linear index a * n_bins + b; the peak rule is
# the 2-D one without wrap; a vertex's tracks are the candidates that voted in its cell.
# ---------------------------------------------------------------------------------------

@dataclass
class VertexSetup:
    n_bins: int
    range: float
    threshold: int
    eps_rel: float = 1e-5

    min_track_votes: int = 0

    @classmethod
    def from_workload(cls, cfg: dict) -> "VertexSetup":
        v = cfg["hough2d"]["vertex"]
        return cls(n_bins=int(v["n_bins"]), range=float(v["range"]), threshold=int(v["threshold"]),
                   min_track_votes=int(v.get("min_track_votes", 0)))


def vertex_votes(params: np.ndarray, vs: VertexSetup):
    """Per candidate, the list of (cell, ambiguous) votes of its line."""
    n, V = vs.n_bins, vs.range
    w = 2.0 * V / n
    g = -V + (np.arange(n) + 0.5) * w
    out = []
    for theta, rho in np.asarray(params, dtype=np.float64).reshape(-1, 2):
        c, s = np.cos(theta), np.sin(theta)
        if abs(s) >= abs(c):
            other = (rho - g * c) / s          # y at each x column
            by_col = True
        else:
            other = (rho - g * s) / c          # x at each y row
            by_col = False
        inside = (other >= -V) & (other < V)
        k = np.floor((other + V) / w)
        t = (other + V) / w
        eps = vs.eps_rel * np.maximum(np.abs(other), V)
        amb = (np.abs(t - np.round(t)) * w <= eps)
        votes = []
        for a in np.nonzero(inside)[0]:
            kk = int(min(k[a], n - 1))
            cell = a * n + kk if by_col else kk * n + a
            votes.append((cell, bool(amb[a]), by_col, int(a), kk))
        out.append(votes)
    return out


def vertex_neighbours(cell: int, vs: VertexSetup):
    n = vs.n_bins
    a, b = divmod(cell, n)
    out = []
    for da in (-1, 0, 1):
        for db in (-1, 0, 1):
            if da == 0 and db == 0:
                continue
            aa, bb = a + da, b + db
            if 0 <= aa < n and 0 <= bb < n:
                out.append(aa * n + bb)
    return out


def event_vertices(event: dict, vs: VertexSetup) -> dict:
    """The vertex transform of one event of `reconstruct`: the candidates with at least
    min_track_votes votes draw their lines; track lists are candidate positions within the
    event's (sorted) candidate list."""
    sel = np.nonzero(event["cand_votes"] >= vs.min_track_votes)[0]
    r = vertex_hough(event["cand_params"][sel], vs)
    r["tracks"] = [sel[t] for t in r["tracks"]]
    return r


def vertex_hough(params: np.ndarray, vs: VertexSetup) -> dict:
    """Histogram, vertex cells (sorted), votes, cell centres, track lists (candidate
    positions within the given list) and the cells an FP32 rounding could change."""
    n, V = vs.n_bins, vs.range
    w = 2.0 * V / n
    h = np.zeros(n * n, dtype=np.int64)
    voters = {}
    amb_cells = set()
    for i, votes in enumerate(vertex_votes(params, vs)):
        for cell, amb, by_col, a, kk in votes:
            h[cell] += 1
            voters.setdefault(cell, []).append(i)
            if amb:
                amb_cells.add(cell)
                for d in (-1, 1):
                    k2 = kk + d
                    if 0 <= k2 < n:
                        amb_cells.add(a * n + k2 if by_col else k2 * n + a)
    cells = []
    for cell in np.nonzero(h >= vs.threshold)[0]:
        cell = int(cell)
        ok = all(not (h[nb] > h[cell] or (nb < cell and h[nb] == h[cell]))
                 for nb in vertex_neighbours(cell, vs))
        if ok:
            cells.append(cell)
    cells = np.array(cells, dtype=np.int64)
    centres = np.stack([-V + (cells // n + 0.5) * w, -V + (cells % n + 0.5) * w], 1) \
        if len(cells) else np.zeros((0, 2))
    return dict(hist=h, cells=cells, votes=h[cells] if len(cells) else np.zeros(0, np.int64),
                centres=centres, tracks=[np.array(voters[c], dtype=np.int64) for c in cells],
                amb_cells=amb_cells)
