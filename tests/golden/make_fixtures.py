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


if __name__ == "__main__":
    with open(os.path.join(HERE, "hand_triplets.json"), "w") as f:
        json.dump(hand_triplets(), f, indent=1)
    with open(os.path.join(HERE, "peak_rule.json"), "w") as f:
        json.dump(peak_rule(), f, indent=1)
    print("wrote hand_triplets.json, peak_rule.json")
