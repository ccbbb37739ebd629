"""2-D per-hit Hough transforms through the C ABI vs the FP64 oracle (GPU only).

Histograms must be equal except in bins the oracle flags (a vote whose FP64 row value lies
within 1e-5 * max(|v|, half-range) of a bin edge, so that the FP32 row may differ);
candidates, their votes and hit lists must be equal except next to such bins; candidate
parameters are the bin centres (FP64 expression rounded to FP32) and must be equal.
"""
import numpy as np
import pytest

from oracle import hough2d as H
from paper_1305_4855_gb300 import events as ev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trk():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1305_4855_gb300 import build
    build.build()
    from paper_1305_4855_gb300 import trk as t
    t.load_library()
    return t


def _affected(bins, s):
    out = set()
    for b in bins:
        c, j = divmod(int(b), s.n_rows)
        out.add(int(b))
        out.update(H.neighbours(c, j, s))
    return out


def _compare(trk, cfg, batch):
    s = H.Hough2DSetup.from_workload(cfg)
    h2 = trk.Hough2D(cfg, max_events=max(batch.n_events, 1), max_hits=max(batch.n_hits, 1))
    hits = torch.from_numpy(batch.packed()).cuda()
    offs = torch.from_numpy(batch.offsets).cuda()
    rc = h2.reconstruct_device(hits, offs)
    assert rc == 0, h2.error()
    cand, hit_ids, cand_off = h2.result(rc)
    ref = H.reconstruct(batch.xyz[:, :2].astype(np.float64), batch.offsets, s)
    n_cmp = n_diff = 0
    for e in range(batch.n_events):
        gh = h2.histogram(e).cpu().numpy().astype(np.int64)
        oe = ref[e]
        diff = set(np.nonzero(gh != oe["hist"])[0].tolist())
        assert diff <= oe["amb_bins"], (e, len(diff - oe["amb_bins"]))
        n_diff += len(diff)
        aff = _affected(diff, s)
        gc = cand[int(cand_off[e]):int(cand_off[e + 1])]
        assert np.all(np.diff(gc["bin"].astype(np.int64)) > 0) and np.all(gc["event"] == e)
        gmap = {int(c["bin"]): c for c in gc}
        omap = {int(b): i for i, b in enumerate(oe["cand_bins"])}
        for b in set(gmap) ^ set(omap):
            assert b in aff, (e, b)
        for b in set(gmap) & set(omap):
            if b in aff:
                continue
            c, i = gmap[b], omap[b]
            assert c["votes"] == oe["cand_votes"][i]
            got = hit_ids[int(c["hit_off"]):int(c["hit_off"]) + int(c["votes"])]
            assert np.array_equal(got, oe["cand_hits"][i]), (e, b)
            assert np.array_equal(c["params"], oe["cand_params"][i].astype(np.float32))
            n_cmp += 1
    ms = h2.last_ms()
    h2.close()
    return dict(compared=n_cmp, hist_diff=n_diff, n_cand=len(cand), ms=ms)


def test_straight_toy_parity(trk):
    cfg = ev.load_workload("sht_toy50")
    b = ev.make_batch(cfg, n_events=8)
    rep = _compare(trk, cfg, b)
    print("H2 straight", rep)
    assert rep["compared"] > 0.95 * rep["n_cand"] and rep["n_cand"] > 100


def test_curved_ip_parity(trk):
    cfg = ev.load_workload("curved_ip200")
    b = ev.make_batch(cfg, n_events=3)
    rep = _compare(trk, cfg, b)
    print("H2 curved", rep)
    assert rep["compared"] > 0.95 * rep["n_cand"] and rep["n_cand"] > 100


def test_edge_events(trk):
    """An empty event, a one-hit event and a normal one in one call."""
    cfg = ev.load_workload("sht_toy50")
    full = ev.make_batch(cfg, n_events=1)
    one = ev.make_batch(cfg, n_events=1, seed=99).event(0)
    one = ev.Batch(one.xyz[:1], one.layer[:1], np.array([0, 1]), one.track[:1], one.truth)
    empty = ev.Batch(np.zeros((0, 3), np.float32), np.zeros(0, np.int32), np.array([0, 0]),
                     np.zeros(0, np.int32), np.zeros((0, 6)))
    b = ev.concat([empty, one, full])
    rep = _compare(trk, cfg, b)
    assert rep["n_cand"] > 0


def test_rejects_bad_configs(trk):
    cfg = ev.load_workload("sht_toy50")
    bad = dict(cfg, hough2d=dict(cfg["hough2d"], lo=-10.0, hi=16.0))
    with pytest.raises(trk.TrkError):
        trk.Hough2D(bad, max_events=1, max_hits=10)
    bad = dict(cfg, hough2d=dict(cfg["hough2d"], n_cols=2))
    with pytest.raises(trk.TrkError):
        trk.Hough2D(bad, max_events=1, max_hits=10)
