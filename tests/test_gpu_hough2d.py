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


def test_vertex_transform_parity(trk):
    """Displaced jets: the second transform over the oracle's own straight-line candidates
    (fed to trk2d_find_vertices) against the oracle's vertex transform of the same
    candidates: vertices, votes and track lists equal away from oracle-flagged cells."""
    cfg = ev.load_workload("sht_jets")
    b = ev.make_batch(cfg, n_events=6)
    s = H.Hough2DSetup.from_workload(cfg)
    vs = H.VertexSetup.from_workload(cfg)
    ref = H.reconstruct(b.xyz[:, :2].astype(np.float64), b.offsets, s)
    cand = np.zeros(sum(len(e["cand_bins"]) for e in ref), dtype=trk.CAND2D_DTYPE)
    off = np.zeros(b.n_events + 1, dtype=np.int64)
    k = 0
    for e, oe in enumerate(ref):
        n = len(oe["cand_bins"])
        cand["bin"][k:k + n] = oe["cand_bins"]
        cand["event"][k:k + n] = e
        cand["votes"][k:k + n] = oe["cand_votes"]
        k += n
        off[e + 1] = k
    h2 = trk.Hough2D(cfg, max_events=b.n_events, max_hits=b.n_hits)
    rc = h2.find_vertices(cand, off)
    assert rc == 0, h2.error()
    verts, voff, vtracks, over = h2.vertices()
    h2.close()
    assert over == 0
    n_vtx = n_skip = found = 0
    for e, oe in enumerate(ref):
        ge = verts[int(voff[e]):int(voff[e + 1])]
        assert np.all(np.diff(ge["cell"].astype(np.int64)) > 0) and np.all(ge["event"] == e)
        ov = H.event_vertices(oe, vs)
        aff = set()
        for c in ov["amb_cells"]:
            aff.add(c)
            aff.update(H.vertex_neighbours(c, vs))
        gmap = {int(v["cell"]): i for i, v in enumerate(ge)}
        omap = {int(c): i for i, c in enumerate(ov["cells"])}
        for c in set(gmap) ^ set(omap):
            assert c in aff, (e, c)
        for c in set(gmap) & set(omap):
            if c in aff:
                n_skip += 1
                continue
            g, o = ge[gmap[c]], omap[c]
            assert g["votes"] == ov["votes"][o]
            gt = vtracks[int(voff[e]) + gmap[c]] - int(off[e])
            assert np.array_equal(gt, ov["tracks"][o][:64]), (e, c)
            assert np.array_equal(g["xy"], ov["centres"][o].astype(np.float32))
            n_vtx += 1
        tv = b.extra["vertices"][b.extra["vertices"][:, 3] == e]
        for x, y, *_ in tv:
            if len(ge):
                found += np.hypot(ge["xy"][:, 0] - x, ge["xy"][:, 1] - y).min() < 2.5
    print("VTX", dict(vertices_compared=n_vtx, skipped_flagged=n_skip, true_found=int(found),
                      true=len(b.extra["vertices"])))
    assert n_vtx > 100


def test_vertex_end_to_end_properties(trk):
    """The whole chain (first transform, candidates, second transform) in one call:
    vertices sorted per event, votes above the threshold, track lists ascending and made of
    candidates with enough votes."""
    cfg = ev.load_workload("sht_jets")
    b = ev.make_batch(cfg, n_events=16)
    vs = H.VertexSetup.from_workload(cfg)
    h2 = trk.Hough2D(cfg, max_events=b.n_events, max_hits=b.n_hits)
    rc = h2.reconstruct_device(torch.from_numpy(b.packed()).cuda(), torch.from_numpy(b.offsets).cuda())
    assert rc == 0, h2.error()
    cand, hit_ids, cand_off = h2.result(rc)
    verts, voff, vtracks, over = h2.vertices()
    h2.close()
    assert len(verts) > 0 and voff[-1] == len(verts)
    for e in range(b.n_events):
        ge = verts[int(voff[e]):int(voff[e + 1])]
        assert np.all(np.diff(ge["cell"].astype(np.int64)) > 0)
        assert np.all(ge["votes"] >= vs.threshold)
    for v, t in zip(verts, vtracks):
        assert len(t) == min(int(v["votes"]), 64) and np.all(np.diff(t) > 0)
        assert np.all(cand["votes"][t] >= vs.min_track_votes) and np.all(cand["event"][t] == v["event"])
