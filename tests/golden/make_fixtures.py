"""Writes the hand-derived fixtures of tests/golden/ (no example is printed in the paper).

Every expected value below follows from the stated geometric construction alone (points
picked on a circle of known centre and radius, or on a line), not from any program under
test: it imports neither the oracle nor the CUDA library.

  hand_triplets.json -- helix-from-triplet worked examples.  Sec. 8 of the paper: a circle
      is fixed by its centre and radius; readings: pT = K B R, K = 0.299792458e-2
      GeV/(T cm), positive charges turn clockwise seen from +z, perigee about the origin,
      z = z0 + s cot(theta) with s the signed path length from the perigee (negative for
      a hit the particle passes before reaching the perigee).
  peak_rule.json -- hand-built 5-D histograms for the local-maximum rule (Sec. 7 and
      Fig. 3 of the paper: candidates are local maxima of the parameter space).
  bin_centres.json -- candidate parameters (bin centres) of chosen bins, worked out by
      hand from the bin widths and the row-major numbering.
  track_fit_chi2.json -- the candidate fit (Sec. 8 and Fig. 6: candidates are fitted to
      their hits) on hit lists whose fitted circle and line are fixed by symmetry or by
      construction, with their residual sums.
  hand_bins.json -- acceptance, bin numbers and ambiguity flags of triplets with exact
      parameters, on a binning with a different count in every dimension.

Run: python tests/golden/make_fixtures.py
"""
import json
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
K = 0.299792458e-2
B = 3.8


def hand_triplets():
    cases = []
    a_p = -math.pi / 2  # angle of the perigee about a centre on the +y axis
    # circle centre (0, 50), radius 50, through the origin; counter-clockwise
    R = 50.0
    ang = [math.atan2(-40, 30), math.atan2(-30, 40), 0.0]
    s = [R * (a - a_p) for a in ang]
    cot, z0 = 0.5, 1.0
    cases.append(dict(
        name="prompt_ccw_circle_through_origin",
        derivation="Circle centre (0,50), radius 50: (30,10), (40,20), (50,50) lie on it (3-4-5 "
                   "triangles). Angles about the centre increase p1->p2->p3: counter-clockwise, "
                   "negative charge. The origin is on the circle: P = (0,0), d0 = 0, tangent +x so "
                   "phi0 = 0. s = 50*(angle + pi/2); z = 1 + 0.5 s.",
        b_tesla=B, hits=[[30.0, 10.0, z0 + cot * s[0]], [40.0, 20.0, z0 + cot * s[1]],
                         [50.0, 50.0, z0 + cot * s[2]]],
        expected=[0.0, -1.0 / (K * B * R), 0.0, cot, z0], arc_lengths=s))
    # circle centre (0, 50), radius 40: perigee (0, 10)
    R = 40.0
    ang = [math.atan2(-32, 24), math.atan2(-24, 32), 0.0]
    s = [R * (a - a_p) for a in ang]
    cot, z0 = -0.25, 3.0
    cases.append(dict(
        name="displaced_ccw",
        derivation="Circle centre (0,50), radius 40: (24,18), (32,26), (40,50) lie on it. "
                   "Counter-clockwise, negative charge. Closest point to the origin P = (0,10), "
                   "tangent +x: phi0 = 0, d0 = -Px sin(phi0) + Py cos(phi0) = +10. z = 3 - 0.25 s.",
        b_tesla=B, hits=[[24.0, 18.0, z0 + cot * s[0]], [32.0, 26.0, z0 + cot * s[1]],
                         [40.0, 50.0, z0 + cot * s[2]]],
        expected=[0.0, -1.0 / (K * B * R), 10.0, cot, z0], arc_lengths=s))
    cases.append(dict(
        name="displaced_cw_mirror",
        derivation="displaced_ccw mirrored x -> -x: clockwise, positive charge; the tangent at "
                   "P = (0,10) is -x so phi0 = pi (binned as -pi); d0 = 10 cos(pi) = -10.",
        b_tesla=B, hits=[[-24.0, 18.0, z0 + cot * s[0]], [-32.0, 26.0, z0 + cot * s[1]],
                         [-40.0, 50.0, z0 + cot * s[2]]],
        expected=[math.pi, 1.0 / (K * B * R), -10.0, cot, z0], arc_lengths=s))
    # hits on both sides of the perigee: circle centre (0, 25), radius 25, through the origin
    R = 25.0
    th1 = 2.0 * math.asin(math.sqrt(50.0) / 50.0)     # |p1 - P| = sqrt(7^2 + 1^2)
    th3 = 2.0 * math.asin(30.0 / 50.0)                # |p3 - P| = sqrt(24^2 + 18^2) = 30
    s = [-R * th1, R * th1, R * th3]
    cot, z0 = 0.5, 2.0
    cases.append(dict(
        name="hits_before_and_after_perigee",
        derivation="Circle centre (0,25), radius 25 through the origin: (-7,1), (7,1), (24,18) lie on "
                   "it. Their angles about the centre increase (-106.3, -73.7, -16.3 degrees): "
                   "counter-clockwise, negative charge, P = (0,0), tangent +x, phi0 = 0, d0 = 0. The "
                   "first hit comes before the perigee: s = -2R asin(sqrt(50)/50), then "
                   "+2R asin(sqrt(50)/50), +2R asin(30/50); z = 2 + 0.5 s.",
        b_tesla=B, hits=[[-7.0, 1.0, z0 + cot * s[0]], [7.0, 1.0, z0 + cot * s[1]],
                         [24.0, 18.0, z0 + cot * s[2]]],
        expected=[0.0, -1.0 / (K * B * R), 0.0, cot, z0], arc_lengths=s))
    cases.append(dict(
        name="straight_through_origin",
        derivation="(3,4), (6,8), (9,12) are exactly collinear (D = 0): q/pT = 0, direction "
                   "atan2(4,3), through the origin so d0 = 0; s = 5, 10, 15, z = -1 + 0.2 s.",
        b_tesla=B, hits=[[3.0, 4.0, 0.0], [6.0, 8.0, 1.0], [9.0, 12.0, 2.0]],
        expected=[math.atan2(4, 3), 0.0, 0.0, 0.2, -1.0], arc_lengths=[5.0, 10.0, 15.0]))
    cases.append(dict(
        name="straight_offset",
        derivation="(1,2), (4,2), (9,2): the line y = 2 travelled towards +x: q/pT = 0, phi0 = 0, "
                   "P = (0,2), d0 = +2; s = 1, 4, 9, z = 0.5 + 0.25 s.",
        b_tesla=B, hits=[[1.0, 2.0, 0.75], [4.0, 2.0, 1.5], [9.0, 2.0, 2.75]],
        expected=[0.0, 0.0, 2.0, 0.25, 0.5], arc_lengths=[1.0, 4.0, 9.0]))
    return dict(source="hand-derived worked examples, see make_fixtures.py", cases=cases)


def peak_rule():
    pk = []

    def case(name, hist, expected, why, threshold=2):
        pk.append(dict(name=name, hist=hist, threshold=threshold, expected=expected, why=why))
    case("isolated_peak", [[[1, 1, 1, 1, 1], 5]], [[1, 1, 1, 1, 1]],
         "one non-empty bin above threshold is a local maximum")
    case("below_threshold", [[[1, 1, 1, 1, 1], 1]], [], "a single vote is below T = 2")
    case("plateau_lower_index_wins", [[[1, 1, 1, 1, 1], 3], [[1, 1, 1, 1, 2], 3]],
         [[1, 1, 1, 1, 1]], "equal neighbours: the smaller row-major index keeps the candidate")
    case("periodic_wrap_larger_neighbour", [[[0, 1, 1, 1, 1], 3], [[3, 1, 1, 1, 1], 4]],
         [[3, 1, 1, 1, 1]], "phi0 is periodic: phi0 bins 0 and 3 are neighbours")
    case("periodic_wrap_plateau", [[[0, 1, 1, 1, 1], 3], [[3, 1, 1, 1, 1], 3]],
         [[0, 1, 1, 1, 1]], "plateau across the phi0 wrap: the smaller row-major index wins")
    case("range_edge", [[[1, 0, 0, 0, 0], 2]], [[1, 0, 0, 0, 0]],
         "neighbours outside a non-periodic range are skipped")
    case("diagonal_neighbour", [[[1, 1, 1, 1, 1], 3], [[2, 2, 2, 2, 2], 4]], [[2, 2, 2, 2, 2]],
         "all 242 neighbours count, diagonals included")
    case("two_separate_peaks", [[[0, 0, 0, 0, 0], 2], [[2, 2, 2, 2, 2], 2], [[1, 1, 1, 1, 0], 1]],
         [[0, 0, 0, 0, 0], [2, 2, 2, 2, 2]],
         "(0,0,0,0,0) and (2,2,2,2,2) are not neighbours; the 1-vote bin is below both")
    case("not_neighbours_across_nonperiodic_edge", [[[1, 0, 1, 1, 1], 3], [[1, 2, 1, 1, 1], 4]],
         [[1, 0, 1, 1, 1], [1, 2, 1, 1, 1]], "q/pT indices 0 and 2 differ by 2: both are peaks")
    case("threshold_four", [[[2, 1, 1, 1, 1], 3], [[0, 0, 0, 0, 0], 4]], [[0, 0, 0, 0, 0]],
         "T = 4: a 3-vote local maximum is not a candidate", threshold=4)
    return dict(source="hand-built histograms, see make_fixtures.py", dims=[4, 3, 3, 3, 3],
                periodic=[True, False, False, False, False], cases=pk)


def bin_centres():
    """Candidate parameters are bin centres, lo + (idx + 1/2)(hi - lo)/n per dimension, with
    the bin number row-major (phi0 slowest).  Each expected value is worked out below from
    the widths, not computed from that expression."""
    pi = math.pi
    # 64 x 64 x 32 x 32 x 16 over (-pi, pi), (-2, 2), (-50, 50), (-5.5, 5.5), (-30, 30):
    # widths pi/32, 1/16, 3.125, 0.34375, 3.75; strides 1048576, 16384, 512, 16, 1
    big = dict(lo=[-pi, -2.0, -50.0, -5.5, -30.0], hi=[pi, 2.0, 50.0, 5.5, 30.0],
               n=[64, 64, 32, 32, 16], periodic=[True, False, False, False, False])
    # 5 x 7 x 3 x 9 x 1 over (-pi, pi), (-1, 1), (-3, 3), (-1.25, 1.25), (-20, 20):
    # widths 2pi/5, 2/7, 2, 5/18, 40; strides 189, 27, 9, 1, 1
    odd = dict(lo=[-pi, -1.0, -3.0, -1.25, -20.0], hi=[pi, 1.0, 3.0, 1.25, 20.0],
               n=[5, 7, 3, 9, 1], periodic=[True, False, False, False, False])
    cases = [
        dict(name="lowest_bin", binning="big", bin=0,
             expected=[-63.0 * pi / 64.0, -1.96875, -48.4375, -5.328125, -28.125],
             why="every index 0: half a width above each lower edge (pi/64, 1/32, 1.5625, "
                 "0.171875, 1.875)"),
        dict(name="highest_bin", binning="big", bin=67108863,
             expected=[63.0 * pi / 64.0, 1.96875, 48.4375, 5.328125, 28.125],
             why="63*1048576 + 63*16384 + 31*512 + 31*16 + 15 = 67108863, the last bin: half a "
                 "width below each upper edge"),
        dict(name="phi0_wrap_row", binning="big", bin=66068495,
             expected=[63.0 * pi / 64.0, -1.96875, 1.5625, -5.328125, 28.125],
             why="63*1048576 + 0 + 16*512 + 0 + 15 = 66068495: the phi0 row next to the wrap, "
                 "d0 index 16 is -50 + 16.5*3.125 = 1.5625"),
        dict(name="middle_bin", binning="big", bin=34087176,
             expected=[pi / 64.0, 0.03125, 1.5625, 0.171875, 1.875],
             why="32*1048576 + 32*16384 + 16*512 + 16*16 + 8 = 34087176: the first bin above "
                 "the middle of every dimension, half a width above zero"),
        dict(name="odd_last_bin", binning="odd", bin=944,
             expected=[0.8 * pi, 6.0 / 7.0, 2.0, 10.0 / 9.0, 0.0],
             why="4*189 + 6*27 + 2*9 + 8 = 944 = 5*7*3*9 - 1: -pi + 4.5*2pi/5 = 0.8 pi, "
                 "-1 + 6.5*2/7 = 6/7, -3 + 2.5*2 = 2, -1.25 + 8.5*5/18 = 10/9, single z0 bin "
                 "centred on 0"),
        dict(name="odd_centre_bin", binning="odd", bin=472,
             expected=[0.0, 0.0, 0.0, 0.0, 0.0],
             why="2*189 + 3*27 + 1*9 + 4 = 472: the middle bin of each odd count, centred on "
                 "zero in every dimension"),
    ]
    return dict(source="hand-worked bin centres, see make_fixtures.py",
                binnings=dict(big=big, odd=odd), cases=cases)


def track_fit_chi2():
    """Candidate-fit residual sums (the fit's stated reading: algebraic circle fit, one hit
    per layer, signed arcs, least-squares line) on hit lists whose fitted circle and line
    are fixed by symmetry or by construction, so that chi2_rphi and chi2_rz are known."""
    cases = []
    # A: centre (0, 50); hits at 0, 90, 180, 270 degrees about it at distances 40.5, 39.5,
    # 40.5, 39.5.  The set is symmetric under the point reflection through the centre, so
    # the algebraic fit's centre is (0, 50) and its R^2 is the mean squared distance,
    # (40.5^2 + 39.5^2)/2 = 1600.25.  Radial residuals 40.5 - R', 39.5 - R'.  z constant:
    # cot = 0, z0 = 3, chi2_rz = 0.
    rp = math.sqrt(1600.25)
    cases.append(dict(
        name="symmetric_radial_residuals",
        derivation="centrally symmetric about (0,50): fitted centre (0,50), R'^2 = 1600.25; "
                   "counter-clockwise in layer order (negative charge); P = (0, 50 - R'), "
                   "phi0 = 0, d0 = 50 - R'; chi2_rphi = 2(40.5 - R')^2 + 2(39.5 - R')^2",
        b_tesla=B, hits=[[0.0, 9.5, 3.0], [39.5, 50.0, 3.0], [0.0, 90.5, 3.0], [-39.5, 50.0, 3.0]],
        layers=[0, 1, 2, 3], used=[1, 1, 1, 1],
        expected=[0.0, -1.0 / (K * B * rp), 50.0 - rp, 0.0, 3.0],
        chi2=[2.0 * (40.5 - rp) ** 2 + 2.0 * (39.5 - rp) ** 2, 0.0],
        amb=4, amb_why="(0, 90.5) lies on the line from the perigee through the centre, "
                       "beyond it: the point opposite the perigee (bit 4); one hit per layer, "
                       "so no selection tie"))
    # B: four hits exactly on the circle centre (0, 50), radius 40 (3-4-5 triangles); the
    # arcs from P = (0, 10) are 40 (theta + pi/2).  z = 1 + 0.5 s + r with
    # r = 0.01 (s3 - s2, s1 - s3, s2 - s1, 0), orthogonal to (1,1,1,1) and to s, so the
    # least-squares line is exactly z = 1 + 0.5 s and chi2_rz = sum r^2.
    R = 40.0
    th = [math.atan2(-32.0, 24.0), math.atan2(-24.0, 32.0), 0.0, math.atan2(32.0, 24.0)]
    s = [R * (t + math.pi / 2.0) for t in th]
    a = 0.01
    r = [a * (s[2] - s[1]), a * (s[0] - s[2]), a * (s[1] - s[0]), 0.0]
    pts = [[24.0, 18.0], [32.0, 26.0], [40.0, 50.0], [24.0, 82.0]]
    hits = [[p[0], p[1], 1.0 + 0.5 * sk + rk] for p, sk, rk in zip(pts, s, r)]
    chi2_rz = sum(x * x for x in r)
    cases.append(dict(
        name="z_residuals_orthogonal_to_the_line",
        derivation="hits on the circle centre (0,50), R = 40; P = (0,10), phi0 = 0, d0 = 10; "
                   "z residuals orthogonal to 1 and s: the line is z = 1 + 0.5 s; "
                   "chi2_rz = sum r_k^2, chi2_rphi = 0",
        b_tesla=B, hits=hits, layers=[0, 1, 2, 3], used=[1, 1, 1, 1],
        expected=[0.0, -1.0 / (K * B * R), 10.0, 0.5, 1.0], chi2=[0.0, chi2_rz],
        amb=0, amb_why="angles from the perigee at most 143 degrees; one hit per layer"))
    # C: B plus a second layer-1 hit far off the circle; it is dropped, and the sums run
    # over the kept hits only, so chi2 equals B's.
    hits_c = hits[:2] + [[32.0, 35.0, 0.0]] + hits[2:]
    cases.append(dict(
        name="dropped_duplicate_not_summed",
        derivation="B with an extra layer-1 hit (32, 35), 4.7 cm inside the circle: the "
                   "per-layer choice keeps (32, 26); the refit and both sums equal B's",
        b_tesla=B, hits=hits_c, layers=[0, 1, 1, 2, 3], used=[1, 1, 0, 1, 1],
        expected=[0.0, -1.0 / (K * B * R), 10.0, 0.5, 1.0], chi2=[0.0, chi2_rz],
        amb=0, amb_why="the layer-1 residuals differ by about 4.7 cm: no tie"))
    # D: a list symmetric under x -> -x.  Layers 0 and 3 hold one hit each on the y axis,
    # (0, 5) and (0, 55); layers 1 and 2 hold mirror pairs, (+-20, 15) and (+-15, 50).  All six
    # lie on the circle centre (0, 30), radius 25 (15-20-25 triangles), and the mirror symmetry
    # puts the all-hit circle's centre on the y axis, so the two hits of a pair are equally far
    # from it: a tie, which keeps the earlier hit of the list (+20, then +15).  The refit on the
    # four kept hits is the same circle.  Angles about the centre in layer order: -90, -36.9,
    # 53.1, 90 degrees, counter-clockwise (negative charge); P = (0, 5), tangent +x: phi0 = 0,
    # d0 = 5.  z = 0 everywhere: cot = 0, z0 = 0, both sums 0.  amb bit 0: a layer's two
    # smallest residuals are equal; bit 4: (0, 55) is the point opposite the perigee.
    cases.append(dict(
        name="tie_keeps_the_earlier_hit",
        derivation="mirror-symmetric list on the circle centre (0,30), R = 25: equal residuals "
                   "within each pair, the earlier hit of each pair is kept; phi0 = 0, d0 = 5",
        b_tesla=B,
        hits=[[0.0, 5.0, 0.0], [20.0, 15.0, 0.0], [-20.0, 15.0, 0.0], [15.0, 50.0, 0.0],
              [-15.0, 50.0, 0.0], [0.0, 55.0, 0.0]],
        layers=[0, 1, 1, 2, 2, 3], used=[1, 1, 0, 1, 0, 1],
        expected=[0.0, -1.0 / (K * B * 25.0), 5.0, 0.0, 0.0], chi2=[0.0, 0.0], amb=5,
        amb_why="equal residuals in layers 1 and 2 (bit 1); (0, 55) opposite the perigee (bit 4)"))
    return dict(source="hand-derived candidate-fit sums, see make_fixtures.py", cases=cases)


def hand_bins():
    """Acceptance, bin numbers and ambiguity flags of triplets whose parameters are exact.

    The hits lie on straight lines parallel to an axis (B = 3.8 T, D = 0 exactly, so q/pT = 0),
    or on a circle through points of 3-4-5 triangles.  The binning has a different count in
    every dimension, so a bin number written with the wrong strides differs from the one
    expected.  Each index below is worked out by hand: the count of whole widths between the
    lower edge and the value.  Ranges: phi0 [-pi, pi) periodic, q/pT [-1, 1), d0 [-3, 3),
    cot [-1.25, 1.25), z0 [-20, 20); counts 7, 5, 12, 4, 6; widths 2pi/7, 0.4, 0.5, 0.625,
    20/3.  Bits of `amb`: 1 a parameter within eps of a bin edge or range limit
    (eps = 1e-5 max(|p|, half-range)), 2 rejected only by parameters within eps outside
    their range, 4 a hit at the point of the circle opposite the perigee.
    """
    binning = dict(lo=[-math.pi, -1.0, -3.0, -1.25, -20.0], hi=[math.pi, 1.0, 3.0, 1.25, 20.0],
                   n=[7, 5, 12, 4, 6], periodic=[True, False, False, False, False])
    # the longitudinal part of every straight case: arcs s = 1, 2, 4 from the perigee and
    # z = 2 + 0.25 s, so cot = 0.25 (index 2: 1.5/0.625 = 2.4) and z0 = 2 (index 3: 22/(20/3)
    # = 3.3); phi0 = 0 has index 3 (pi/(2pi/7) = 3.5) and q/pT = 0 index 2 (1/0.4 = 2.5)
    z = [2.25, 2.5, 3.0]
    cases = []

    def line(y, sign):
        return [[sign * 1.0, y, z[0]], [sign * 2.0, y, z[1]], [sign * 4.0, y, z[2]]]
    cases.append(dict(
        name="d0_on_its_lower_limit", hits=line(-3.0, 1.0), status=0, idx=[3, 2, 0, 2, 3],
        amb=1, amb_mask=7,
        why="moving along +x at y = -3: perigee (0,-3), phi0 = 0, d0 = -3 = lo: accepted in d0 "
            "bin 0 (the lower limit is inside), and on an edge"))
    cases.append(dict(
        name="d0_on_its_upper_limit", hits=line(3.0, 1.0), status=1, idx=None, amb=3,
        amb_mask=7,
        why="moving along +x at y = +3: d0 = +3 = hi is outside [lo, hi): rejected, and only by "
            "a value on its limit"))
    cases.append(dict(
        name="phi0_equal_to_pi_wraps", hits=line(1.2, -1.0), status=0, idx=[0, 2, 3, 2, 3],
        amb=1, amb_mask=7,
        why="moving along -x at y = 1.2: phi0 = atan2(0, -3) = pi, which the period maps to "
            "-pi (bin 0); perigee (0, 1.2), d0 = 1.2 cos(pi) = -1.2 (index 3: 1.8/0.5 = 3.6)"))
    cases.append(dict(
        name="d0_just_above_the_edge_at_zero", hits=line(1e-6, 1.0), status=0,
        idx=[3, 2, 6, 2, 3], amb=1, amb_mask=7,
        why="y = 1e-6: d0 = 1e-6 (index 6), 1e-6 above the edge at 0; eps is 1e-5 times the "
            "half-range 3, not times |d0|, so the triplet is edge-ambiguous"))
    cases.append(dict(
        name="interior", hits=line(-2.2, 1.0), status=0, idx=[3, 2, 1, 2, 3], amb=0,
        amb_mask=7,
        why="y = -2.2: d0 = -2.2 (index 1: 0.8/0.5 = 1.6); every value at least 0.1 width "
            "from an edge: not ambiguous"))
    cases.append(dict(
        name="hit_opposite_the_perigee",
        hits=[[240.0, 81.0, 0.0], [400.0, 401.0, 0.0], [0.0, 801.0, 0.0]], status=0, idx=None,
        amb=4, amb_mask=4,
        why="circle centre (0,401), R = 400 through (240,81), (400,401), (0,801); perigee "
            "(0,1); the third hit is the point opposite it (half-angle asin(1) = pi/2)"))
    cases.append(dict(
        name="no_hit_opposite_the_perigee",
        hits=[[240.0, 81.0, 0.0], [400.0, 401.0, 0.0], [320.0, 641.0, 0.0]], status=0,
        idx=None, amb=0, amb_mask=4,
        why="the same circle with the third hit at (320,641), 126.9 degrees from the perigee"))
    return dict(source="hand-worked binning cases, see make_fixtures.py", b_tesla=B,
                binning=binning, cases=cases)


if __name__ == "__main__":
    with open(os.path.join(HERE, "hand_triplets.json"), "w") as f:
        json.dump(hand_triplets(), f, indent=1)
    with open(os.path.join(HERE, "peak_rule.json"), "w") as f:
        json.dump(peak_rule(), f, indent=1)
    with open(os.path.join(HERE, "bin_centres.json"), "w") as f:
        json.dump(bin_centres(), f, indent=1)
    with open(os.path.join(HERE, "track_fit_chi2.json"), "w") as f:
        json.dump(track_fit_chi2(), f, indent=1)
    with open(os.path.join(HERE, "hand_bins.json"), "w") as f:
        json.dump(hand_bins(), f, indent=1)
    print("wrote hand_triplets.json, peak_rule.json, bin_centres.json, track_fit_chi2.json, "
          "hand_bins.json")
