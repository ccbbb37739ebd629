"""The GPU-vs-oracle comparison helpers (tests/parity.py) catch what they are meant to catch
(CPU only): every kind of disagreement planted in small hand-made inputs is reported, and
the explained exceptions (edge-ambiguous and near-accepted triplets) are not."""
import numpy as np

import parity

DIMS = (4, 3, 3, 3, 3)
PER = (True, False, False, False, False)


def _trip(*rows):
    return np.asarray(rows, dtype=np.int64).reshape(-1, 3)


def test_triplets_agree():
    ijk = _trip([0, 1, 2], [0, 1, 3])
    rep, flips = parity.compare_triplets(ijk, [5, 7], ijk, [5, 7], [False, False], _trip())
    assert rep["ok"] and rep["n_both"] == 2 and not flips


def test_triplet_in_another_bin_is_bad_unless_ambiguous():
    ijk = _trip([0, 1, 2], [0, 1, 3])
    rep, _ = parity.compare_triplets(ijk, [5, 8], ijk, [5, 7], [False, False], _trip())
    assert not rep["ok"] and rep["n_bad_bin"] == 1
    rep, flips = parity.compare_triplets(ijk, [5, 8], ijk, [5, 7], [False, True], _trip())
    assert rep["ok"] and rep["n_bin_flips"] == 1 and flips == {7, 8}


def test_gpu_only_triplet_must_be_near_accepted():
    g = _trip([0, 1, 2], [4, 5, 6])
    o = _trip([0, 1, 2])
    rep, _ = parity.compare_triplets(g, [5, 9], o, [5], [False], _trip())
    assert not rep["ok"] and rep["n_gpu_only_unexplained"] == 1
    rep, flips = parity.compare_triplets(g, [5, 9], o, [5], [False], _trip([4, 5, 6]))
    assert rep["ok"] and 9 in flips


def test_oracle_only_triplet_must_be_ambiguous():
    g = _trip([0, 1, 2])
    o = _trip([0, 1, 2], [4, 5, 6])
    rep, _ = parity.compare_triplets(g, [5], o, [5, 9], [False, False], _trip())
    assert not rep["ok"] and rep["n_oracle_only_unexplained"] == 1
    rep, flips = parity.compare_triplets(g, [5], o, [5, 9], [False, True], _trip())
    assert rep["ok"] and 9 in flips


def test_duplicate_gpu_vote_is_an_error():
    g = _trip([0, 1, 2], [0, 1, 2])
    try:
        parity.compare_triplets(g, [5, 5], _trip([0, 1, 2]), [5], [False], _trip())
    except AssertionError:
        return
    raise AssertionError("a triplet voted twice was not reported")


def test_dilate_wraps_phi0_only():
    b = int(np.ravel_multi_index((0, 0, 1, 1, 1), DIMS))
    d = parity.dilate({b}, DIMS, PER)
    # 3 phi0 rows (3, 0, 1) x 2 q/pT rows (0, 1) x 3 x 3 x 3
    assert len(d) == 3 * 2 * 27
    assert int(np.ravel_multi_index((3, 1, 0, 0, 0), DIMS)) in d
    assert int(np.ravel_multi_index((2, 0, 1, 1, 1), DIMS)) not in d


def test_candidates_compared_outside_the_affected_bins():
    h = [np.array([1, 4, 9]), np.array([2, 3])]
    rep = parity.compare_candidates([10, 20], [5, 4], h, [10, 20], [5, 4], h, set())
    assert rep["ok"] and rep["n_compared"] == 2
    # a missing candidate, other votes, other hits, unsorted hits: each reported
    assert not parity.compare_candidates([10], [5], h[:1], [10, 20], [5, 4], h, set())["ok"]
    assert not parity.compare_candidates([10, 20], [5, 3], h, [10, 20], [5, 4], h, set())["ok"]
    bad_hits = [np.array([1, 4, 8]), h[1]]
    assert not parity.compare_candidates([10, 20], [5, 4], bad_hits, [10, 20], [5, 4], h, set())["ok"]
    unsorted = [np.array([4, 1, 9]), h[1]]
    assert not parity.compare_candidates([10, 20], [5, 4], unsorted, [10, 20], [5, 4], h, set())["ok"]
    # the same disagreements inside the affected set are skipped
    rep = parity.compare_candidates([10], [5], h[:1], [10, 20], [5, 4], h, {20})
    assert rep["ok"] and rep["n_compared"] == 1


def test_param_errors_wrap_phi0():
    p32 = np.array([[np.float32(3.1415925), 1.0, 0, 0, 0]], dtype=np.float32)
    p64 = np.array([[-3.14159265, 1.0, 0, 0, 0]])
    assert parity.param_errors(p32, p64)[0, 0] < 1e-6
    tol = parity.param_tolerance(np.array([[0.0, 1e-9, 40.0, 0.0, 0.0]]),
                                 [-np.pi, -2, -50, -5.5, -30], [np.pi, 2, 50, 5.5, 30])
    assert np.allclose(tol[0], [1e-5 * np.pi, 2e-5, 5e-4, 5.5e-5, 3e-4])


def test_plateau_count_hand_built():
    h = np.zeros(DIMS, np.int64)
    h[2, 2, 2, 2, 2] = 5              # strict maximum: not a plateau
    h[3, 0, 0, 0, 0] = 4              # plateau of two, across the phi0 wrap
    h[0, 0, 0, 0, 1] = 4
    h[1, 2, 0, 2, 0] = 1              # below the threshold
    assert parity.plateau_count(h.ravel(), DIMS, PER, threshold=2) == 2
    h[0, 0, 0, 0, 1] = 3              # now (3,0,0,0,0) is a strict maximum
    assert parity.plateau_count(h.ravel(), DIMS, PER, threshold=2) == 0
