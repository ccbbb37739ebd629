"""Candidate fit (one helix through each candidate's hits) through the C ABI vs the FP64
oracle's fit of the oracle's own candidates (GPU only).

Both sides fit in FP64 (algebraic circle fit, one hit per layer, signed arcs, least-squares
line); the GPU sums in a different order and rounds its outputs to FP32, so the parameters
must agree within 1e-6 * max(|p|, half-range): FP32 rounding (6e-8) plus summation-order
differences amplified by the circle fit's conditioning.  Kept-hit flags must be equal
unless the oracle flags the layer choice as ambiguous.  Candidates are matched by
(event, bin) and compared when both sides assigned them the same hits.
"""
import numpy as np
import pytest

import oracle
from paper_1305_4855_gb300 import events as ev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module")
def trk():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1305_4855_gb300 import build
    build.build()
    from paper_1305_4855_gb300 import trk as t
    t.load_library()
    return t


def _gpu(trk, cfg, batch, host=False):
    rec = trk.Reconstructor(cfg, max_events=max(batch.n_events, 1), max_hits=max(batch.n_hits, 1),
                            vote_capacity=1 << 26, cand_capacity=1 << 20, assign_capacity=1 << 24,
                            fit_candidates=1)
    if host:
        rc = rec.reconstruct_host(batch.packed(), batch.offsets.astype(np.int64))
        res = rec.result(rc, from_host=True)
    else:
        rc = rec.reconstruct_device(torch.from_numpy(batch.packed()).cuda(),
                                    torch.from_numpy(batch.offsets).cuda())
        res = rec.result(rc)
    assert res.rc == 0, rec.error()
    rec.close()
    return res


def _compare(cfg, batch, res):
    setup = oracle.OracleSetup.from_workload(cfg)
    ref = oracle.reconstruct(batch.xyz, batch.layer, batch.offsets, setup)
    B = cfg["geometry"]["b_tesla"]
    scale = 0.5 * (setup.hi - setup.lo)
    n_cmp = n_same_hits = n_ok = 0
    worst = np.zeros(5)
    for e in range(batch.n_events):
        cand, hl = res.event(e)
        tracks, used = res.event_fits(e)
        oe = ref["events"][e]
        fo = oracle.fit_tracks(batch.xyz, batch.layer, oe["cand_hits"], B)
        opos = {int(b): i for i, b in enumerate(oe["cand_bins"])}
        for g, c in enumerate(cand):
            i = opos.get(int(c["bin"]))
            if i is None:
                continue
            n_cmp += 1
            if not np.array_equal(hl[g], oe["cand_hits"][i]):
                continue
            n_same_hits += 1
            t = tracks[g]
            assert t["event"] == e
            assert t["status"] == fo["status"][i], (e, c["bin"], t, fo["status"][i])
            if not (fo["amb"][i] & 1):
                assert np.array_equal(used[g], fo["use"][i]), (e, c["bin"])
            if t["status"] != 0 or (fo["amb"][i] & 1):
                continue
            assert t["n_used"] == int(fo["use"][i].sum())
            lay = batch.layer[hl[g][used[g]]]
            assert int(t["layers"]) == int(np.bitwise_or.reduce(np.left_shift(1, lay.astype(np.int64))))
            p = fo["par"][i]
            d = np.abs(t["params"].astype(np.float64) - p)
            d[0] = min(d[0], 2 * np.pi - d[0])
            rel = d / np.maximum(np.abs(p), scale)
            worst = np.maximum(worst, rel)
            assert np.all(rel <= TOL), (e, int(c["bin"]), t["params"], p, rel)
            for k, name in enumerate(("chi2_rphi", "chi2_rz")):
                ref_c = fo["chi2"][i, k]
                assert abs(float(t[name]) - ref_c) <= 1e-5 * ref_c + 1e-9, (name, t[name], ref_c)
            n_ok += 1
    return dict(compared=n_cmp, same_hits=n_same_hits, fitted=n_ok, worst_rel=worst.tolist())


def test_fit_parity_barrel4(trk):
    cfg = ev.load_workload("barrel4_20trk")
    b = ev.make_batch(cfg)
    rep = _compare(cfg, b, _gpu(trk, cfg, b))
    print("FIT barrel4", rep)
    assert rep["fitted"] >= 10 and rep["same_hits"] >= 0.95 * rep["compared"]


@pytest.mark.parametrize("n_tracks,seed", [(40, 3), (80, 17)])
def test_fit_parity_barrel10_reduced(trk, n_tracks, seed):
    cfg = ev.load_workload("barrel10_500trk")
    rng = np.random.default_rng(seed)
    b = ev.concat([ev.make_event(cfg, rng, n_tracks), ev.make_event(cfg, rng, n_tracks // 2)])
    rep = _compare(cfg, b, _gpu(trk, cfg, b))
    print("FIT barrel10", n_tracks, rep)
    assert rep["fitted"] >= 50 and rep["same_hits"] >= 0.95 * rep["compared"]


def test_fit_host_path_equals_device_path(trk):
    cfg = ev.load_workload("barrel10_500trk")
    b = ev.make_event(cfg, np.random.default_rng(5), 60)
    r1, r2 = _gpu(trk, cfg, b), _gpu(trk, cfg, b, host=True)
    assert np.array_equal(r1.tracks.view(np.uint8), r2.tracks.view(np.uint8))
    assert np.array_equal(r1.hit_used, r2.hit_used)


def test_fit_full_event_properties(trk):
    """The 500-track event: properties that hold at any size (one kept hit per layer, the
    layer mask and counts consistent, finite parameters).  How many fits land near their
    candidate's bin is printed as a statistic only: most of the 124 k candidates are
    combinatorial, and their hits do not lie on one helix."""
    cfg = ev.load_workload("barrel10_500trk")
    b = ev.make_batch(cfg)
    rec = trk.Reconstructor(cfg, max_events=1, max_hits=b.n_hits, vote_capacity=1 << 28,
                            cand_capacity=1 << 21, assign_capacity=1 << 25, fit_candidates=1)
    rc = rec.reconstruct_device(torch.from_numpy(b.packed()).cuda(), torch.from_numpy(b.offsets).cuda())
    res = rec.result(rc)
    st = rec.stage_ms()
    rec.close()
    assert res.rc == 0
    cand, hl = res.event(0)
    tracks, used = res.event_fits(0)
    assert len(tracks) == len(cand) > 1000
    ok = tracks["status"] == 0
    assert ok.mean() > 0.99, np.bincount(tracks["status"])
    for t, h, u in zip(tracks[:5000], hl[:5000], used[:5000]):
        lay = b.layer[h[u]]
        assert len(np.unique(lay)) == len(lay) == t["n_used"]
        if t["status"] == 0:
            assert int(t["layers"]) == int(np.bitwise_or.reduce(np.left_shift(1, lay.astype(np.int64))))
            assert np.all(np.isfinite(t["params"])) and t["chi2_rphi"] >= 0 and t["chi2_rz"] >= 0
    # fitted parameters lie near the candidate's bin for most candidates (sanity)
    w = (np.array(cfg["binning"]["hi"]) - np.array(cfg["binning"]["lo"])) / np.array(cfg["binning"]["n"])
    d = np.abs(tracks["params"][ok] - cand["params"][ok])
    d[:, 0] = np.minimum(d[:, 0], 2 * np.pi - d[:, 0])
    near = np.all(d <= 2.0 * w[None, :], axis=1)
    strong = cand["votes"][ok] >= 6
    print("FITFULL", dict(n=len(tracks), ok=float(ok.mean()), near=float(near.mean()),
                          near_votes_ge_6=float(near[strong].mean()) if strong.any() else None,
                          fit_ms=st["fit"]))
