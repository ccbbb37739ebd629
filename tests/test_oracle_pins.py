"""Pins of the FP64 oracle against things other than itself (CPU only).

  * hand-derived worked triplets (tests/golden/hand_triplets.json);
  * hand-worked acceptance, bins and ambiguity flags (tests/golden/hand_bins.json);
  * a charged particle integrated through F = q v x B with RK4: the oracle must recover
    the starting perigee from three layer crossings (checks the charge sign and the
    phi0 / d0 conventions against the force law, not against a closed form);
  * closed-form helix points from the forward model, prompt and displaced, both charges;
  * exact special cases and symmetries (collinear -> q/pT = 0, circle through the origin
    -> d0 = 0, B scaling, 90-degree rotation, mirrors);
  * an independently written brute-force enumerator on tiny events;
  * invariants (thread count, hit permutation, duplicated events) and the peak rule on
    hand-built histograms (tests/golden/peak_rule.json).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle.core import fit_one
from paper_1305_4855_gb300 import events as ev

import brute_force

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
K = ev.K_GEV_PER_T_CM


def _wrap(a):
    return (a + math.pi) % (2 * math.pi) - math.pi


def _close(par, exp, rel=1e-9, floor=1e-9):
    par = np.asarray(par, dtype=np.float64)
    exp = np.asarray(exp, dtype=np.float64)
    d = np.abs(par - exp)
    d[0] = abs(_wrap(par[0] - exp[0]))
    return np.all(d <= rel * np.maximum(np.abs(exp), 1.0) + floor), d


# ---------------------------------------------------------------------------------------
# worked examples
# ---------------------------------------------------------------------------------------

def test_golden_hand_triplets():
    g = json.load(open(os.path.join(GOLDEN, "hand_triplets.json")))
    for c in g["cases"]:
        h = np.asarray(c["hits"], dtype=np.float64)
        par = fit_one(h[0], h[1], h[2], c["b_tesla"])
        assert par is not None, c["name"]
        ok, d = _close(par, c["expected"], rel=1e-12, floor=1e-12)
        assert ok, (c["name"], par, c["expected"], d)


def test_golden_hand_bins():
    # acceptance, bin numbers and ambiguity bits of triplets with exact parameters
    # (tests/golden/hand_bins.json): the half-open ranges, the phi0 period, row-major strides
    # on a binning with a different count per dimension, eps scaled by the half-range, and the
    # flag of a hit opposite the perigee
    g = json.load(open(os.path.join(GOLDEN, "hand_bins.json")))
    b = g["binning"]
    s = oracle.OracleSetup(b_tesla=g["b_tesla"], n_layers=3,
                           triples=np.array([[0, 1, 2]], np.int32), lo=np.array(b["lo"]),
                           hi=np.array(b["hi"]), n=np.array(b["n"]),
                           periodic=np.array(b["periodic"]), threshold=2)
    for c in g["cases"]:
        f = oracle.fit_list(np.array(c["hits"]), np.array([0, 1, 2], np.int32),
                            np.array([[0, 1, 2]], np.int32), s)
        assert int(f["status"][0]) == c["status"], c["name"]
        if c["idx"] is not None:
            assert int(f["bin"][0]) == int(np.ravel_multi_index(tuple(c["idx"]), tuple(b["n"]))), \
                (c["name"], np.unravel_index(int(f["bin"][0]), tuple(b["n"])))
        assert int(f["amb_bits"][0]) & c["amb_mask"] == c["amb"], (c["name"], f["amb_bits"])


def test_golden_hand_triplets_from_float32_hits():
    # the same examples through float32 storage (how hits reach both implementations)
    g = json.load(open(os.path.join(GOLDEN, "hand_triplets.json")))
    for c in g["cases"]:
        h = np.asarray(c["hits"], dtype=np.float32).astype(np.float64)
        par = fit_one(h[0], h[1], h[2], c["b_tesla"])
        ok, d = _close(par, c["expected"], rel=1e-6, floor=1e-5)
        assert ok, (c["name"], d)


def test_collinear_gives_exact_zero_curvature():
    for pts in ([(3, 4, 0), (6, 8, 1), (9, 12, 2)], [(1, 2, 0), (4, 2, 1), (9, 2, 3)],
                [(0, -5, 1), (0, -7, 2), (0, -30, 4)], [(-1, -1, 0), (-2, -2, 0), (-7, -7, 5)]):
        par = fit_one(*[np.asarray(p, dtype=np.float64) for p in pts], 3.8)
        assert par[1] == 0.0


# ---------------------------------------------------------------------------------------
# physics: Lorentz-force integration
# ---------------------------------------------------------------------------------------

def _rk4_crossings(q, pt, phi0, d0, cot, z0, b_tesla, radii, h=0.002):
    """Integrate dp/dl = q K (p_hat x B), dx/dl = p_hat from the perigee state; return the
    first outward crossing of each radius (linear interpolation between steps)."""
    x = np.array([-d0 * math.sin(phi0), d0 * math.cos(phi0), z0])
    p = pt * np.array([math.cos(phi0), math.sin(phi0), cot])
    Bv = np.array([0.0, 0.0, b_tesla])

    def deriv(state):
        pos, mom = state[:3], state[3:]
        ph = mom / np.linalg.norm(mom)
        return np.concatenate([ph, q * K * np.cross(ph, Bv)])

    st = np.concatenate([x, p])
    out = []
    want = list(radii)
    r_prev = math.hypot(st[0], st[1])
    for _ in range(2_000_000):
        k1 = deriv(st)
        k2 = deriv(st + 0.5 * h * k1)
        k3 = deriv(st + 0.5 * h * k2)
        k4 = deriv(st + h * k3)
        nst = st + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        r_new = math.hypot(nst[0], nst[1])
        if want and r_prev < want[0] <= r_new:
            f = (want[0] - r_prev) / (r_new - r_prev)
            out.append(st[:3] + f * (nst[:3] - st[:3]))
            want.pop(0)
            if not want:
                return out
        st, r_prev = nst, r_new
    raise AssertionError("particle did not reach all radii")


@pytest.mark.parametrize("q,pt,phi0,d0,cot,z0", [
    (+1, 2.0, 0.3, 0.0, 0.4, 1.0),
    (-1, 2.0, 0.3, 0.0, 0.4, 1.0),
    (+1, 1.2, -2.5, 1.5, -0.8, -3.0),
    (-1, 0.9, 2.9, -2.0, 1.1, 4.0),
    (-1, 5.0, -0.7, 3.0, 0.0, 0.0),
])
def test_lorentz_force_rk4(q, pt, phi0, d0, cot, z0):
    B = 3.8
    pts = _rk4_crossings(q, pt, phi0, d0, cot, z0, B, [6.0, 14.0, 26.0])
    par = fit_one(pts[0], pts[1], pts[2], B)
    exp = [phi0, q / pt, d0, cot, z0]
    # the interpolated crossings sit within ~h^2 kappa of the true circle
    ok, d = _close(par, exp, rel=2e-5, floor=2e-5)
    assert ok, (par, exp, d)


# ---------------------------------------------------------------------------------------
# closed form from the forward model, exact double-precision points
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["barrel4_20trk", "barrel10_500trk", "barrel10_2000trk_precision"])
def test_closed_form_recovery(name):
    cfg = ev.load_workload(name)
    rng = np.random.default_rng(11)
    tr = ev._tracks(cfg, rng, 200)
    radius = cfg["geometry"]["radius"]
    B = cfg["geometry"]["b_tesla"]
    n_checked = 0
    for t in range(200):
        pts = []
        for r in radius:
            if r <= tr["r_start"][t]:
                continue
            s = ev._first_crossing(tr["sx"][t:t + 1], tr["sy"][t:t + 1], tr["psi"][t:t + 1],
                                   tr["kappa"][t:t + 1], r)[0]
            if not np.isfinite(s):
                break
            x, y = ev._position(tr["sx"][t], tr["sy"][t], tr["psi"][t], tr["kappa"][t], s)
            pts.append(np.array([x, y, tr["sz"][t] + tr["cot"][t] * s]))
        for a in range(len(pts) - 2):
            par = fit_one(pts[a], pts[a + 1], pts[a + 2], B)
            ok, d = _close(par, tr["truth"][t], rel=1e-8, floor=1e-8)
            assert ok, (t, par, tr["truth"][t], d)
            n_checked += 1
    assert n_checked > 100


# ---------------------------------------------------------------------------------------
# exact special cases and symmetries on a whole event
# ---------------------------------------------------------------------------------------

def _c1():
    cfg = ev.load_workload("barrel4_20trk")
    return cfg, ev.make_batch(cfg), oracle.OracleSetup.from_workload(cfg)


def test_b_field_scaling_is_exact():
    cfg, b, s = _c1()
    e1 = oracle.enumerate_batch(b.xyz, b.layer, b.offsets, s)
    s2 = oracle.OracleSetup.from_workload(cfg, b_tesla=2 * s.b_tesla,
                                          lo=s.lo * np.array([1, 0.5, 1, 1, 1]),
                                          hi=s.hi * np.array([1, 0.5, 1, 1, 1]))
    e2 = oracle.enumerate_batch(b.xyz, b.layer, b.offsets, s2)
    assert np.array_equal(e1["ijk"], e2["ijk"])
    assert np.array_equal(e1["par"][:, 1] * 0.5, e2["par"][:, 1])
    assert np.array_equal(e1["par"][:, [0, 2, 3, 4]], e2["par"][:, [0, 2, 3, 4]])
    assert np.array_equal(e1["bin"], e2["bin"])


def _compare_transformed(e1, e2, map_par, map_bin, tol=1e-9):
    """Triplets accepted on both sides (neither ambiguous) have mapped params and bins."""
    k1 = {tuple(t): i for i, t in enumerate(e1["ijk"])}
    k2 = {tuple(t): i for i, t in enumerate(e2["ijk"])}
    amb1 = {tuple(t) for t, a in zip(e1["ijk"], e1["amb"]) if a}
    amb2 = {tuple(t) for t, a in zip(e2["ijk"], e2["amb"]) if a}
    near = {tuple(t) for t in e1["near_ijk"]} | {tuple(t) for t in e2["near_ijk"]}
    only = (set(k1) ^ set(k2)) - amb1 - amb2 - near
    assert not only, list(only)[:5]
    n = 0
    for t in set(k1) & set(k2):
        p1, p2 = e1["par"][k1[t]], e2["par"][k2[t]]
        ok, d = _close(map_par(p1), p2, rel=tol, floor=tol)
        assert ok, (t, p1, p2, d)
        if t not in amb1 and t not in amb2:
            assert map_bin(e1["bin"][k1[t]]) == e2["bin"][k2[t]]
            n += 1
    assert n > 100


def test_rotation_by_90_degrees():
    cfg, b, s = _c1()
    xyz2 = b.xyz.copy()
    xyz2[:, 0], xyz2[:, 1] = -b.xyz[:, 1], b.xyz[:, 0]
    e1 = oracle.enumerate_batch(b.xyz, b.layer, b.offsets, s)
    e2 = oracle.enumerate_batch(xyz2, b.layer, b.offsets, s)
    dims = tuple(int(x) for x in s.n)
    shift = dims[0] // 4

    def map_par(p):
        q = p.copy()
        q[0] = _wrap(p[0] + math.pi / 2)
        return q

    def map_bin(bn):
        idx = list(np.unravel_index(bn, dims))
        idx[0] = (idx[0] + shift) % dims[0]
        return int(np.ravel_multi_index(idx, dims))
    _compare_transformed(e1, e2, map_par, map_bin)


def test_mirror_y_flips_charge_phi_and_d0():
    cfg, b, s = _c1()
    xyz2 = b.xyz.copy()
    xyz2[:, 1] = -b.xyz[:, 1]
    e1 = oracle.enumerate_batch(b.xyz, b.layer, b.offsets, s)
    e2 = oracle.enumerate_batch(xyz2, b.layer, b.offsets, s)
    dims = tuple(int(x) for x in s.n)

    def map_par(p):
        return np.array([-p[0], -p[1], -p[2], p[3], p[4]])

    def map_bin(bn):
        idx = list(np.unravel_index(bn, dims))
        # phi0 -> -phi0 on [-pi, pi) periodic: bin i -> n-1-i; q/pT, d0 symmetric ranges
        idx[0] = dims[0] - 1 - idx[0]
        idx[1] = dims[1] - 1 - idx[1]
        idx[2] = dims[2] - 1 - idx[2]
        return int(np.ravel_multi_index(idx, dims))
    _compare_transformed(e1, e2, map_par, map_bin)


def test_mirror_z_flips_cot_and_z0():
    cfg, b, s = _c1()
    xyz2 = b.xyz.copy()
    xyz2[:, 2] = -b.xyz[:, 2]
    e1 = oracle.enumerate_batch(b.xyz, b.layer, b.offsets, s)
    e2 = oracle.enumerate_batch(xyz2, b.layer, b.offsets, s)
    dims = tuple(int(x) for x in s.n)

    def map_par(p):
        return np.array([p[0], p[1], p[2], -p[3], -p[4]])

    def map_bin(bn):
        idx = list(np.unravel_index(bn, dims))
        idx[3] = dims[3] - 1 - idx[3]
        idx[4] = dims[4] - 1 - idx[4]
        return int(np.ravel_multi_index(idx, dims))
    _compare_transformed(e1, e2, map_par, map_bin)


def test_prompt_tracks_have_zero_impact_parameter():
    # Sec. 8: the interaction-point-constrained curved Hough is the d0 = 0 special case
    cfg = ev.load_workload("barrel10_500trk")
    cfg["events"]["displaced"]["fraction"] = 0.0
    rng = np.random.default_rng(5)
    tr = ev._tracks(cfg, rng, 100)
    for t in range(100):
        assert abs(tr["truth"][t, 2]) < 1e-12
        pts = []
        for r in (10.0, 30.0, 60.0):
            s_ = ev._first_crossing(tr["sx"][t:t + 1], tr["sy"][t:t + 1], tr["psi"][t:t + 1],
                                    tr["kappa"][t:t + 1], r)[0]
            if not np.isfinite(s_):
                break
            x, y = ev._position(tr["sx"][t], tr["sy"][t], tr["psi"][t], tr["kappa"][t], s_)
            pts.append(np.array([x, y, tr["sz"][t] + tr["cot"][t] * s_]))
        if len(pts) == 3:
            par = fit_one(pts[0], pts[1], pts[2], 3.8)
            assert abs(par[2]) < 1e-9


# ---------------------------------------------------------------------------------------
# brute force on tiny events
# ---------------------------------------------------------------------------------------

def _tiny_event(seed, per_layer=5):
    cfg = ev.load_workload("barrel4_20trk")
    b = ev.make_batch(cfg, seed=seed)
    keep = []
    for L in range(4):
        idx = np.nonzero(b.layer == L)[0][:per_layer]
        keep.extend(idx.tolist())
    keep = np.array(sorted(keep))
    return cfg, b.xyz[keep], b.layer[keep]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_brute_force_agreement(seed):
    cfg, xyz, layer = _tiny_event(seed)
    # a binning wide enough that most combinations vote (stresses the whole range logic)
    # (a different bin count per dimension, so that wrong row-major strides change the bins)
    s = oracle.OracleSetup.from_workload(cfg, lo=np.array([-math.pi, -3.0, -12.0, -4.0, -60.0]),
                                         hi=np.array([math.pi, 3.0, 12.0, 4.0, 60.0]),
                                         n=np.array([16, 12, 10, 8, 6]))
    offs = np.array([0, len(xyz)], dtype=np.int64)
    e = oracle.enumerate_batch(xyz, layer, offs, s)
    bf = brute_force.enumerate_event(xyz.astype(np.float64), layer, s.triples, s.b_tesla,
                                     s.lo, s.hi, s.n, s.periodic)
    orc = {tuple(t): (bn, p, a) for t, bn, p, a in zip(e["ijk"], e["bin"], e["par"], e["amb"])}
    near = {tuple(t) for t in e["near_ijk"]}
    assert len(orc) > 50
    for t in set(orc) | set(bf):
        if t in orc and t in bf:
            ok, d = _close(orc[t][1], bf[t][1], rel=1e-7, floor=1e-7)
            assert ok, (t, orc[t][1], bf[t][1], d)
            if not orc[t][2]:
                assert orc[t][0] == bf[t][0], t
        elif t in orc:
            assert orc[t][2], ("only oracle", t)
        else:
            assert t in near, ("only brute force", t)


# ---------------------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------------------

def test_thread_count_does_not_change_output():
    cfg = ev.load_workload("barrel10_500trk")
    b = ev.make_batch(cfg)
    # two inner layer triples only, to keep the CPU time small
    s = oracle.OracleSetup.from_workload(cfg, triples=np.array([[0, 1, 2], [1, 2, 3]], np.int32))
    sub = np.nonzero(b.layer <= 3)[0][:900]
    xyz, lay = b.xyz[sub], b.layer[sub]
    offs = np.array([0, len(sub)], np.int64)
    e1 = oracle.enumerate_batch(xyz, lay, offs, s, n_threads=1)
    e8 = oracle.enumerate_batch(xyz, lay, offs, s, n_threads=8)
    for k in ("event", "ijk", "bin", "amb", "par", "near_ijk"):
        assert np.array_equal(e1[k], e8[k]), k
    assert e1["n_triplets"] == e8["n_triplets"]


def test_vote_total_equals_accepted_count():
    cfg, b, s = _c1()
    r = oracle.reconstruct(b.xyz, b.layer, b.offsets, s)
    assert int(r["events"][0]["hist_counts"].sum()) == len(r["enum"]["bin"])
    # every accepted triplet's bin is in range and every vote lands in a listed triple
    assert np.all(r["enum"]["bin"] < s.n_bins)
    allowed = {tuple(t) for t in s.triples.tolist()}
    lay = b.layer[r["enum"]["ijk"]]
    assert all(tuple(x) in allowed for x in lay.tolist())


def test_hit_permutation_invariance():
    cfg, b, s = _c1()
    rng = np.random.default_rng(7)
    perm = rng.permutation(b.n_hits)
    r1 = oracle.reconstruct(b.xyz, b.layer, b.offsets, s)
    r2 = oracle.reconstruct(b.xyz[perm], b.layer[perm], b.offsets, s)
    a, c = r1["events"][0], r2["events"][0]
    assert np.array_equal(a["hist_bins"], c["hist_bins"])
    assert np.array_equal(a["hist_counts"], c["hist_counts"])
    assert np.array_equal(a["cand_bins"], c["cand_bins"])
    for h1, h2 in zip(a["cand_hits"], c["cand_hits"]):
        assert np.array_equal(np.sort(perm[h2]), h1)


def test_duplicated_event_in_a_batch():
    cfg, b, s = _c1()
    two = ev.concat([b, b])
    r1 = oracle.reconstruct(b.xyz, b.layer, b.offsets, s)
    r2 = oracle.reconstruct(two.xyz, two.layer, two.offsets, s)
    for e in range(2):
        a, c = r1["events"][0], r2["events"][e]
        assert np.array_equal(a["hist_bins"], c["hist_bins"])
        assert np.array_equal(a["cand_bins"], c["cand_bins"])
        for h1, h2 in zip(a["cand_hits"], c["cand_hits"]):
            assert np.array_equal(h1 + e * b.n_hits, h2)


def test_empty_and_sparse_events():
    cfg, b, s = _c1()
    # an empty event, an event with hits in one layer only, then the real event
    one_layer = np.nonzero(b.layer == 0)[0]
    xyz = np.concatenate([b.xyz[one_layer], b.xyz])
    lay = np.concatenate([b.layer[one_layer], b.layer])
    offs = np.array([0, 0, len(one_layer), len(xyz)], np.int64)
    r = oracle.reconstruct(xyz, lay, offs, s)
    assert len(r["events"][0]["cand_bins"]) == 0 and len(r["events"][1]["cand_bins"]) == 0
    ref = oracle.reconstruct(b.xyz, b.layer, b.offsets, s)
    assert np.array_equal(r["events"][2]["cand_bins"], ref["events"][0]["cand_bins"])


def test_invalid_layer_is_rejected():
    cfg, b, s = _c1()
    lay = b.layer.copy()
    lay[3] = 7
    with pytest.raises(ValueError):
        oracle.enumerate_batch(b.xyz, lay, b.offsets, s)


def test_degenerate_triplets_are_counted():
    # (10,0), (0,10), (-10,0) and (10,0), (0,10), (0,-10) lie on the circle of radius 10 about
    # the origin: a centre on the origin has no perigee, so both triplets are degenerate;
    # (10,0), (0,10), (5,30) is an ordinary circle.  The full and the block-restricted
    # enumerations both count exactly two.
    xyz = np.array([[10.0, 0.0, 0.0], [0.0, 10.0, 1.0], [-10.0, 0.0, 2.0], [0.0, -10.0, 2.0],
                    [5.0, 30.0, 3.0]])
    layer = np.array([0, 1, 2, 2, 2], np.int32)
    s = oracle.OracleSetup(b_tesla=3.8, n_layers=3, triples=np.array([[0, 1, 2]], np.int32),
                           lo=np.array([-math.pi, -2.0, -50.0, -5.5, -30.0]),
                           hi=np.array([math.pi, 2.0, 50.0, 5.5, 30.0]), n=np.array([4, 3, 2, 2, 2]),
                           periodic=np.array([True, False, False, False, False]), threshold=2)
    full = oracle.enumerate_batch(xyz, layer, np.array([0, 5], np.int64), s)
    assert full["n_triplets"] == 3 and full["n_degenerate"] == 2
    blk = oracle.enumerate_blocks(xyz, layer, s, [(0, 0)], [], [])
    assert blk["n_triplets"] == 3 and blk["n_degenerate"] == 2


def test_fit_list_matches_enumeration():
    cfg, b, s = _c1()
    e = oracle.enumerate_batch(b.xyz, b.layer, b.offsets, s)
    f = oracle.fit_list(b.xyz, b.layer, e["ijk"], s)
    assert np.all(f["status"] == 0)
    assert np.array_equal(f["par"], e["par"])
    assert np.array_equal(f["bin"], e["bin"])


# ---------------------------------------------------------------------------------------
# peak rule and hit assignment
# ---------------------------------------------------------------------------------------

def test_golden_peak_rule():
    g = json.load(open(os.path.join(GOLDEN, "peak_rule.json")))
    dims = tuple(g["dims"])
    for c in g["cases"]:
        s = oracle.OracleSetup(b_tesla=3.8, n_layers=1, triples=np.zeros((0, 3), np.int32),
                               lo=np.zeros(5), hi=np.ones(5), n=np.array(dims),
                               periodic=np.array(g["periodic"]), threshold=c["threshold"])
        bins = np.array([np.ravel_multi_index(tuple(h[0]), dims) for h in c["hist"]], np.int64)
        cnts = np.array([h[1] for h in c["hist"]], np.int64)
        o = np.argsort(bins)
        cb, cv = oracle.peaks(bins[o], cnts[o], s)
        exp = sorted(int(np.ravel_multi_index(tuple(x), dims)) for x in c["expected"])
        assert cb.tolist() == exp, c["name"]


def test_peaks_brute_force_on_random_histograms():
    # brute force: compare every bin with every other bin by explicit index distance
    rng = np.random.default_rng(3)
    dims = (5, 4, 3, 4, 3)
    per = np.array([True, False, False, False, False])
    s = oracle.OracleSetup(b_tesla=3.8, n_layers=1, triples=np.zeros((0, 3), np.int32),
                           lo=np.zeros(5), hi=np.ones(5), n=np.array(dims), periodic=per,
                           threshold=2)
    nb = int(np.prod(dims))
    all_idx = np.stack(np.unravel_index(np.arange(nb), dims), axis=1)
    for trial in range(20):
        h = np.where(rng.uniform(size=nb) < 0.2, rng.integers(1, 5, nb), 0)
        ub = np.nonzero(h)[0]
        cb, _ = oracle.peaks(ub.astype(np.int64), h[ub].astype(np.int64), s)
        exp = []
        for b in range(nb):
            if h[b] < 2:
                continue
            d = np.abs(all_idx - all_idx[b])
            d[:, 0] = np.minimum(d[:, 0], dims[0] - d[:, 0])
            nbr = np.all(d <= 1, axis=1)
            nbr[b] = False
            if np.all(h[b] >= h[nbr]) and np.all(h[b] > h[np.nonzero(nbr)[0][np.nonzero(nbr)[0] < b]]):
                exp.append(b)
        assert cb.tolist() == exp


def test_assign_hits_union():
    ijk = np.array([[0, 1, 2], [0, 3, 4], [5, 6, 7], [2, 1, 9]])
    bins = np.array([5, 5, 7, 5])
    out = oracle.assign_hits(ijk, bins, np.array([5, 7]))
    assert out[0].tolist() == [0, 1, 2, 3, 4, 9]
    assert out[1].tolist() == [5, 6, 7]


def test_golden_bin_centres():
    # candidate parameters: hand-worked centres of chosen bins (lowest, highest, next to
    # the phi0 wrap, middle; an odd binning with a single z0 bin)
    g = json.load(open(os.path.join(GOLDEN, "bin_centres.json")))
    for c in g["cases"]:
        b = g["binnings"][c["binning"]]
        setup = oracle.OracleSetup(
            b_tesla=3.8, n_layers=3, triples=np.array([[0, 1, 2]], dtype=np.int32),
            lo=np.array(b["lo"]), hi=np.array(b["hi"]), n=np.array(b["n"]),
            periodic=np.array(b["periodic"]), threshold=1)
        got = oracle.bin_centres(np.array([c["bin"]], dtype=np.int64), setup)[0]
        assert np.allclose(got, c["expected"], rtol=0, atol=1e-12), (c["name"], got, c["expected"])


def _blocks_around(setup, centre_blocks):
    n0, n1 = int(setup.n[0]), int(setup.n[1])
    out = set()
    for i0, i1 in centre_blocks:
        for d0 in (-1, 0, 1):
            for d1 in (-1, 0, 1):
                j1 = i1 + d1
                if 0 <= j1 < n1:
                    out.add(((i0 + d0) % n0, j1))
    return sorted(out)


@pytest.mark.parametrize("periodic", [True, False])
def test_block_enumeration_equals_full_enumeration(periodic):
    # the output-restricted definition must give exactly the full definition's counts,
    # accepted triplets and candidates inside its blocks (blocks at the phi0 wrap included)
    cfg = ev.load_workload("barrel4_20trk")
    setup = oracle.OracleSetup.from_workload(cfg)
    setup.periodic = np.array([periodic] + [False] * 4)
    b = ev.concat([ev.make_batch(cfg, seed=61), ev.make_batch(cfg, seed=62)]).event(0)
    n0, n1 = int(setup.n[0]), int(setup.n[1])
    inner = int(np.prod(setup.n[2:]))
    full = oracle.enumerate_batch(b.xyz, b.layer, b.offsets, setup)
    ub0, cnt0 = np.unique(full["bin"], return_counts=True)
    cand0, _ = oracle.peaks(ub0, cnt0, setup)
    # blocks of some candidates, and blocks on both sides of the phi0 wrap
    keep = sorted({(int(c // inner) // n1, int(c // inner) % n1) for c in cand0[::5]} |
                  {(0, 8), (n0 - 1, 8), (5, 0), (9, n1 - 1)})
    count = _blocks_around(setup, keep)
    if not periodic:
        # without wrap the neighbour rows are the in-range ones; blocks across the wrap are
        # absent and must not be needed
        count = sorted({(i0 + d0, i1 + d1) for i0, i1 in keep for d0 in (-1, 0, 1)
                        for d1 in (-1, 0, 1) if 0 <= i0 + d0 < n0 and 0 <= i1 + d1 < n1})
    flip = _blocks_around(setup, count)
    blk = oracle.enumerate_blocks(b.xyz, b.layer, setup, count, keep, flip)
    assert blk["n_triplets"] == full["n_triplets"]
    assert blk["n_degenerate"] == full["n_degenerate"]
    fb = full["bin"]
    for q, (i0, i1) in enumerate(count):
        sel = fb // inner == i0 * n1 + i1
        dense = np.bincount(fb[sel] % inner, minlength=inner)
        assert np.array_equal(blk["counts"][q], dense), (i0, i1)
    kset = np.isin(fb // inner, [i0 * n1 + i1 for i0, i1 in keep])
    assert np.array_equal(np.sort(parity_keys(blk["keep_ijk"])), np.sort(parity_keys(full["ijk"][kset])))
    # every edge-ambiguous accepted triplet of a flip block, and every near-accepted one, is
    # listed
    fsel = np.isin(fb // inner, [i0 * n1 + i1 for i0, i1 in flip]) & full["amb"]
    listed = set(parity_keys(blk["flip_ijk"]).tolist())
    assert set(parity_keys(full["ijk"][fsel]).tolist()) <= listed
    assert set(parity_keys(full["near_ijk"]).tolist()) <= listed
    # candidates of the keep blocks: the plain C rule over the block counts equals the
    # numpy rule over the whole histogram
    cb, cv = oracle.block_peaks(blk, setup, keep)
    ub, cnt = np.unique(fb, return_counts=True)
    rb, rv = oracle.peaks(ub, cnt, setup)
    rsel = np.isin(rb // inner, [i0 * n1 + i1 for i0, i1 in keep])
    assert len(rb[rsel]) > 0
    assert np.array_equal(cb, rb[rsel]) and np.array_equal(cv, rv[rsel])


def test_block_peaks_on_random_histograms():
    # dense random counts: the C block rule against the numpy rule, wrap and edges included
    rng = np.random.default_rng(7)
    setup = oracle.OracleSetup(b_tesla=3.8, n_layers=3, triples=np.array([[0, 1, 2]], np.int32),
                               lo=np.zeros(5), hi=np.ones(5), n=np.array([5, 4, 3, 4, 3]),
                               periodic=np.array([True, False, False, False, False]),
                               threshold=3)
    n0, n1 = 5, 4
    inner = 3 * 4 * 3
    for trial in range(40):
        # counts up to 5 make plateaus (ties decided by the bin number); counts up to 10^6
        # make strict maxima in every row, so that the neighbours across the phi0 wrap decide
        h = rng.integers(0, 6 if trial % 2 == 0 else 1_000_000, size=n0 * n1 * inner)
        ub = np.nonzero(h)[0]
        keep = [(int(rng.integers(0, n0)), int(rng.integers(0, n1))) for _ in range(3)]
        keep = sorted(set(keep))
        count = _blocks_around(setup, keep)
        counts = np.stack([h[(i0 * n1 + i1) * inner:(i0 * n1 + i1 + 1) * inner] for i0, i1 in count])
        slot = -np.ones(n0 * n1, np.int32)
        for q, (i0, i1) in enumerate(count):
            slot[i0 * n1 + i1] = q
        cb, cv = oracle.block_peaks(dict(slot=slot, counts=counts.astype(np.int32)), setup, keep)
        rb, rv = oracle.peaks(ub.astype(np.int64), h[ub].astype(np.int64), setup)
        rsel = np.isin(rb // inner, [i0 * n1 + i1 for i0, i1 in keep])
        assert np.array_equal(cb, rb[rsel]) and np.array_equal(cv, rv[rsel]), trial


def parity_keys(ijk):
    ijk = np.asarray(ijk, dtype=np.int64).reshape(-1, 3)
    return (ijk[:, 0] << 42) | (ijk[:, 1] << 21) | ijk[:, 2]
