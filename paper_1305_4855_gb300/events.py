"""Seeded synthetic tracker events (forward model only).

Charged helices in a uniform axial field B along +z are propagated analytically to the
barrel layers (cylinders of given radius and half-length) and their first outgoing
crossings become hits; uniform noise hits are added.  This module is the single input
generator shared by the tests, the benchmark and the oracle-side checks: it draws the
random numbers and produces hits and truth, and contains none of the reconstruction
arithmetic (no triplet fit, no binning, no peak finding).

Conventions (the same physical reading the reconstruction uses):
  * units cm, GeV, T; pT = K * B * R with K = 0.299792458e-2 GeV / (T cm);
  * a positive charge turns clockwise seen from +z (F = q v x B), so the signed
    curvature (counter-clockwise positive) is kappa = -q / R;
  * perigee w.r.t. the origin: direction phi0 at the point of closest approach P,
    d0 = -P_x sin(phi0) + P_y cos(phi0), z0 = z at P, cot(theta) = dz/ds.

Hits are float32 (x, y, z) plus an int32 layer id, 16 bytes per hit, laid out as a
float32 array of shape (N, 4) whose last column holds the layer id's int32 bits.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

K_GEV_PER_T_CM = 0.299792458e-2
WORKLOAD_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "workloads")


def load_workload(name: str) -> dict:
    """Load a workload description (geometry, binning, event recipe, seed) by name."""
    path = name if name.endswith(".json") else os.path.join(WORKLOAD_DIR, name + ".json")
    with open(path) as f:
        return json.load(f)


def list_workloads() -> list[str]:
    return sorted(p[:-5] for p in os.listdir(WORKLOAD_DIR) if p.endswith(".json"))


@dataclass
class Batch:
    """Hits of one or more events, concatenated event after event."""
    xyz: np.ndarray            # (N, 3) float32
    layer: np.ndarray          # (N,) int32
    offsets: np.ndarray        # (n_events + 1,) int64
    track: np.ndarray          # (N,) int32, index into `truth` of the batch, -1 for noise
    truth: np.ndarray          # (n_tracks_total, 6) float64: phi0, q/pT, d0, cot(theta), z0, event
    extra: dict = field(default_factory=dict)

    @property
    def n_events(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_hits(self) -> int:
        return int(self.offsets[-1])

    def packed(self) -> np.ndarray:
        """(N, 4) float32 array: x, y, z and the int32 layer id stored bitwise."""
        out = np.empty((self.n_hits, 4), dtype=np.float32)
        out[:, :3] = self.xyz
        out[:, 3] = self.layer.astype(np.int32).view(np.float32)
        return out

    def event(self, e: int) -> "Batch":
        a, b = int(self.offsets[e]), int(self.offsets[e + 1])
        sel = self.truth[:, 5] == e
        remap = -np.ones(len(self.truth), dtype=np.int64)
        remap[np.nonzero(sel)[0]] = np.arange(int(sel.sum()))
        trk = self.track[a:b]
        trk = np.where(trk >= 0, remap[np.maximum(trk, 0)], -1).astype(np.int32)
        tr = self.truth[sel].copy()
        tr[:, 5] = 0
        return Batch(self.xyz[a:b].copy(), self.layer[a:b].copy(),
                     np.array([0, b - a], dtype=np.int64), trk, tr)


def concat(batches: list[Batch]) -> Batch:
    xyz = np.concatenate([b.xyz for b in batches]) if batches else np.zeros((0, 3), np.float32)
    layer = np.concatenate([b.layer for b in batches]) if batches else np.zeros(0, np.int32)
    offs = [0]
    tracks, truths, verts = [], [], []
    ntr = 0
    ev = 0
    for b in batches:
        if "vertices" in b.extra:
            v = np.asarray(b.extra["vertices"], dtype=np.float64).reshape(-1, b.extra["vertices"].shape[-1])
            if v.shape[1] == 3:               # (x, y, n_tracks) of a single event
                v = np.concatenate([v, np.zeros((len(v), 1))], axis=1)
            v = v.copy()
            v[:, 3] += ev
            verts.append(v)
        for e in range(b.n_events):
            offs.append(offs[-1] + int(b.offsets[e + 1] - b.offsets[e]))
        t = b.track.copy()
        t[t >= 0] += ntr
        tracks.append(t)
        tr = b.truth.copy()
        tr[:, 5] += ev
        truths.append(tr)
        ntr += len(b.truth)
        ev += b.n_events
    extra = {"vertices": np.concatenate(verts)} if verts else {}
    return Batch(xyz, layer, np.array(offs, dtype=np.int64),
                 np.concatenate(tracks) if tracks else np.zeros(0, np.int32),
                 np.concatenate(truths) if truths else np.zeros((0, 6)), extra)


# ---------------------------------------------------------------------------------------
# helix propagation (forward model)
# ---------------------------------------------------------------------------------------

def _line_crossing(sx, sy, psi, r):
    """Path length t > 0 at which the straight line leaving (sx, sy) in direction psi first
    reaches radius r (B = 0); inf where it never does."""
    ux, uy = np.cos(psi), np.sin(psi)
    su = sx * ux + sy * uy
    disc = su * su - (sx * sx + sy * sy) + r * r
    t = -su + np.sqrt(np.maximum(disc, 0.0))
    return np.where((disc >= 0.0) & (t > 1e-9), t, np.inf)


def _first_crossing(sx, sy, psi, kappa, r):
    """Arc length t > 0 at which a circle track leaving (sx, sy) with direction psi and
    signed curvature kappa first reaches radius r; inf where it never does.  kappa = 0 is a
    straight line."""
    if np.all(np.asarray(kappa) == 0.0):
        return _line_crossing(sx, sy, psi, r)
    cx = sx - np.sin(psi) / kappa
    cy = sy + np.cos(psi) / kappa
    rho = 1.0 / np.abs(kappa)
    d = np.hypot(cx, cy)
    ok = (d <= r + rho) & (d >= np.abs(r - rho)) & (d > 0)
    d_safe = np.where(ok, d, 1.0)
    a = (r * r - rho * rho + d_safe * d_safe) / (2.0 * d_safe)
    h = np.sqrt(np.maximum(r * r - a * a, 0.0))
    ux, uy = cx / d_safe, cy / d_safe
    best = np.full(np.shape(sx), np.inf)
    # angle of the start point around the centre, and the rotation sense
    a0 = np.arctan2(sy - cy, sx - cx)
    sense = np.sign(kappa)
    for sgn in (1.0, -1.0):
        px = a * ux - sgn * h * uy
        py = a * uy + sgn * h * ux
        a1 = np.arctan2(py - cy, px - cx)
        dphi = np.mod(sense * (a1 - a0), 2.0 * np.pi)
        t = dphi * rho
        t = np.where(ok & (t > 1e-9), t, np.inf)
        best = np.minimum(best, t)
    return best


def _position(sx, sy, psi, kappa, t):
    if np.all(np.asarray(kappa) == 0.0):
        return sx + t * np.cos(psi), sy + t * np.sin(psi)
    x = sx + (np.sin(psi + kappa * t) - np.sin(psi)) / kappa
    y = sy - (np.cos(psi + kappa * t) - np.cos(psi)) / kappa
    return x, y


def _perigee_from_state(sx, sy, psi, kappa, sz, cot):
    """Truth perigee parameters of the circle track through (sx, sy) with direction psi
    (kappa = 0: the straight line)."""
    if np.all(np.asarray(kappa) == 0.0):
        d0 = -sx * np.sin(psi) + sy * np.cos(psi)
        t_ps = sx * np.cos(psi) + sy * np.sin(psi)      # path length from P to the start
        return np.asarray(psi, dtype=np.float64) + 0.0, d0, sz - cot * t_ps
    cx = sx - np.sin(psi) / kappa
    cy = sy + np.cos(psi) / kappa
    rho = 1.0 / np.abs(kappa)
    cn = np.hypot(cx, cy)
    px = cx * (1.0 - rho / cn)
    py = cy * (1.0 - rho / cn)
    # unit tangent at P in the sense of motion: counter-clockwise = z x (P - C)
    rx, ry = (px - cx) / rho, (py - cy) / rho
    tx, ty = -np.sign(kappa) * ry, np.sign(kappa) * rx
    phi0 = np.arctan2(ty, tx)
    d0 = -px * np.sin(phi0) + py * np.cos(phi0)
    # signed arc length from P to the start point (the start lies on the outgoing
    # branch, less than half a turn after P; a start at P itself gives 0)
    a_p = np.arctan2(py - cy, px - cx)
    a_s = np.arctan2(sy - cy, sx - cx)
    t_ps = (np.mod(np.sign(kappa) * (a_s - a_p) + np.pi, 2.0 * np.pi) - np.pi) * rho
    z0 = sz - cot * t_ps
    return phi0, d0, z0


def _jet_tracks(cfg: dict, rng: np.random.Generator, n_prompt: int):
    """Prompt tracks plus displaced jets: each jet's tracks leave one vertex (radius in
    rprod_range, uniform azimuth) within +-cone of the radial direction."""
    ev = cfg["events"]
    d = ev["displaced"]
    n_jets = int(rng.integers(d["n_jets"][0], d["n_jets"][1] + 1))
    per = [int(rng.integers(d["tracks_per_jet"][0], d["tracks_per_jet"][1] + 1))
           for _ in range(n_jets)]
    rp = rng.uniform(d["rprod_range"][0], d["rprod_range"][1], n_jets)
    phv = rng.uniform(-np.pi, np.pi, n_jets)
    n = n_prompt + sum(per)
    sub = dict(cfg, events=dict(ev, displaced={"kind": "none", "fraction": 0.0}))
    tr = _tracks(sub, rng, n)
    k = n_prompt
    vertices = []
    for j in range(n_jets):
        sl = slice(k, k + per[j])
        vx, vy = rp[j] * np.cos(phv[j]), rp[j] * np.sin(phv[j])
        tr["sx"][sl], tr["sy"][sl] = vx, vy
        tr["psi"][sl] = phv[j] + rng.uniform(-d["cone"], d["cone"], per[j])
        tr["r_start"][sl] = rp[j]
        vertices.append((vx, vy, per[j]))
        k += per[j]
    phi0, d0, z0 = _perigee_from_state(tr["sx"], tr["sy"], tr["psi"], tr["kappa"], tr["sz"],
                                       tr["cot"])
    tr["truth"] = np.stack([phi0, tr["truth"][:, 1], d0, tr["cot"], z0], axis=1)
    tr["vertices"] = np.array(vertices, dtype=np.float64).reshape(-1, 3)
    return tr


def _tracks(cfg: dict, rng: np.random.Generator, n_tracks: int):
    ev = cfg["events"]
    B = cfg["geometry"]["b_tesla"]
    if ev.get("displaced", {}).get("kind") == "jets":
        return _jet_tracks(cfg, rng, n_tracks)
    lo_pt, hi_pt = ev["pt_range"]
    pt = np.exp(rng.uniform(math.log(lo_pt), math.log(hi_pt), n_tracks))
    q = rng.choice(np.array([-1.0, 1.0]), n_tracks)
    eta = rng.uniform(ev["eta_range"][0], ev["eta_range"][1], n_tracks)
    cot = np.sinh(eta)
    phi = rng.uniform(-np.pi, np.pi, n_tracks)
    zpv = rng.normal(0.0, ev["z0_sigma"], n_tracks)
    kappa = -q * K_GEV_PER_T_CM * B / pt
    disp = ev.get("displaced", {"kind": "none", "fraction": 0.0})
    is_disp = rng.uniform(0.0, 1.0, n_tracks) < disp.get("fraction", 0.0)
    if disp["kind"] == "perigee_d0":
        # the start state is the perigee itself: d0 drawn directly
        d0 = np.where(is_disp, rng.uniform(disp["d0_range"][0], disp["d0_range"][1], n_tracks), 0.0)
        sx = -d0 * np.sin(phi)
        sy = d0 * np.cos(phi)
        psi = phi
        sz = zpv
        r_start = np.abs(d0)
    elif disp["kind"] == "vertex":
        # long-lived parent decays at radius rp; daughter leaves within +-pi/2 of radial-out
        rp = rng.uniform(disp["rprod_range"][0], disp["rprod_range"][1], n_tracks)
        phv = rng.uniform(-np.pi, np.pi, n_tracks)
        dpsi = rng.uniform(-0.5 * np.pi, 0.5 * np.pi, n_tracks)
        sx = np.where(is_disp, rp * np.cos(phv), 0.0)
        sy = np.where(is_disp, rp * np.sin(phv), 0.0)
        psi = np.where(is_disp, phv + dpsi, phi)
        sz = zpv
        r_start = np.where(is_disp, rp, 0.0)
    else:
        sx = np.zeros(n_tracks)
        sy = np.zeros(n_tracks)
        psi = phi
        sz = zpv
        r_start = np.zeros(n_tracks)
    phi0, d0, z0 = _perigee_from_state(sx, sy, psi, kappa, sz, cot)
    truth = np.stack([phi0, q / pt, d0, cot, z0], axis=1)
    return dict(sx=sx, sy=sy, psi=psi, kappa=kappa, sz=sz, cot=cot, r_start=r_start, truth=truth)


def make_event(cfg: dict, rng: np.random.Generator, n_tracks: int,
               smear: bool = True, noise: bool = True, shuffle: bool = True) -> Batch:
    """One event of `n_tracks` helices following the workload's recipe."""
    geo = cfg["geometry"]
    ev = cfg["events"]
    radius = np.asarray(geo["radius"], dtype=np.float64)
    zhalf = np.asarray(geo["z_half"], dtype=np.float64)
    tr = _tracks(cfg, rng, n_tracks)
    n_tracks = len(tr["truth"])
    xs, ys, zs, ls, ts = [], [], [], [], []
    alive = np.ones(n_tracks, dtype=bool)
    for L, (r, zh) in enumerate(zip(radius, zhalf)):
        t = _first_crossing(tr["sx"], tr["sy"], tr["psi"], tr["kappa"], r)
        ok = alive & np.isfinite(t) & (r > tr["r_start"])
        x, y = _position(tr["sx"], tr["sy"], tr["psi"], tr["kappa"], np.where(ok, t, 0.0))
        z = tr["sz"] + tr["cot"] * np.where(ok, t, 0.0)
        inside = ok & (np.abs(z) < zh)
        # once a track leaves through the end of the barrel it produces no further hits
        alive &= ~(ok & ~inside)
        idx = np.nonzero(inside)[0]
        x, y, z = x[idx], y[idx], z[idx]
        if smear:
            # r-phi smear along the layer (rotation keeps the hit on the cylinder), z smear
            dphi = rng.normal(0.0, ev["smear_rphi"], len(idx)) / r
            c, s = np.cos(dphi), np.sin(dphi)
            x, y = c * x - s * y, s * x + c * y
            z = z + rng.normal(0.0, ev["smear_z"], len(idx))
        xs.append(x); ys.append(y); zs.append(z)
        ls.append(np.full(len(idx), L, dtype=np.int32)); ts.append(idx.astype(np.int32))
    x = np.concatenate(xs); y = np.concatenate(ys); z = np.concatenate(zs)
    lay = np.concatenate(ls); trk = np.concatenate(ts)
    if noise and ev.get("noise_fraction", 0.0) > 0:
        n_noise = int(round(ev["noise_fraction"] * len(x)))
        nl = rng.integers(0, len(radius), n_noise).astype(np.int32)
        nphi = rng.uniform(-np.pi, np.pi, n_noise)
        nz = rng.uniform(-1.0, 1.0, n_noise) * zhalf[nl]
        x = np.concatenate([x, radius[nl] * np.cos(nphi)])
        y = np.concatenate([y, radius[nl] * np.sin(nphi)])
        z = np.concatenate([z, nz])
        lay = np.concatenate([lay, nl])
        trk = np.concatenate([trk, -np.ones(n_noise, dtype=np.int32)])
    if shuffle:
        perm = rng.permutation(len(x))
        x, y, z, lay, trk = x[perm], y[perm], z[perm], lay[perm], trk[perm]
    xyz = np.stack([x, y, z], axis=1).astype(np.float32)
    truth = np.concatenate([tr["truth"], np.zeros((n_tracks, 1))], axis=1)
    extra = {"vertices": tr["vertices"]} if "vertices" in tr else {}
    return Batch(xyz, lay.astype(np.int32), np.array([0, len(x)], dtype=np.int64),
                 trk.astype(np.int32), truth, extra)


def track_counts(cfg: dict, rng: np.random.Generator, n_events: int) -> np.ndarray:
    nt = cfg["events"]["n_tracks"]
    if isinstance(nt, dict):
        lam = nt["poisson_mean"]
        lo, hi = nt["clip"]
        return np.clip(rng.poisson(lam, n_events), lo, hi).astype(np.int64)
    return np.full(n_events, int(nt), dtype=np.int64)


def make_batch(cfg: dict | str, n_events: int | None = None, seed: int | None = None,
               **kw) -> Batch:
    """All events of a workload (or the first `n_events` of it), seeded."""
    if isinstance(cfg, str):
        cfg = load_workload(cfg)
    n_events = cfg["events"]["n_events"] if n_events is None else n_events
    rng = np.random.default_rng(cfg["seed"] if seed is None else seed)
    counts = track_counts(cfg, rng, n_events)
    return concat([make_event(cfg, rng, int(n), **kw) for n in counts])


def layer_triplet_count(batch: Batch, triples) -> np.ndarray:
    """Per event, the number of hit triplets sum |La||Lb||Lc| over the layer triples."""
    out = np.zeros(batch.n_events, dtype=np.int64)
    for e in range(batch.n_events):
        a, b = int(batch.offsets[e]), int(batch.offsets[e + 1])
        cnt = np.bincount(batch.layer[a:b], minlength=64).astype(np.int64)
        out[e] = sum(int(cnt[t[0]] * cnt[t[1]] * cnt[t[2]]) for t in triples)
    return out
