"""CUDA path vs the FP64 oracle, through the C ABI (GPU only).

Integer outputs (votes, histograms, candidates, hit lists) must match bit for bit except
where an FP32 parameter lies within eps = 1e-5 * max(|p|, half-range) of a bin edge or
range limit (tests/parity.py explains each difference by such an oracle-flagged
triplet).  Helix parameters must agree within the same relative tolerance.
"""
import numpy as np
import pytest

import oracle
import parity
from paper_1305_4855_gb300 import events as ev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS_REL = 1e-5


@pytest.fixture(scope="module")
def trk():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1305_4855_gb300 import build
    build.build()
    from paper_1305_4855_gb300 import trk as t
    t.load_library()
    return t


def _run(trk, cfg, batch, max_hits=None, **opts):
    kw = dict(vote_capacity=1 << 24, cand_capacity=1 << 20, assign_capacity=1 << 24)
    kw.update(opts)
    rec = trk.Reconstructor(cfg, max_events=max(batch.n_events, 1),
                            max_hits=max_hits or max(batch.n_hits, 1), **kw)
    hits = torch.from_numpy(batch.packed()).cuda()
    offs = torch.from_numpy(batch.offsets).cuda()
    rc = rec.reconstruct_device(hits, offs)
    return rec, rec.result(rc), hits


def _full_compare(trk, cfg, batch, threads=0, check_plateaus=False, **opts):
    """Triplets, histograms and candidates of every event of `batch`; with
    check_plateaus, also the count of plateau bins the peak passes listed."""
    plateaus = 0
    rec, res, hits = _run(trk, cfg, batch, **opts)
    assert res.rc == 0, rec.error()
    setup = oracle.OracleSetup.from_workload(cfg)
    ref = oracle.reconstruct(batch.xyz, batch.layer, batch.offsets, setup, n_threads=threads)
    en = ref["enum"]
    gv, gb = rec.votes()
    gv = gv.cpu().numpy()
    gb = gb.cpu().numpy().view(np.uint32).astype(np.int64)
    dims = tuple(int(x) for x in setup.n)
    reports = []
    st = rec.stats()
    assert st["n_triplets"] == en["n_triplets"]
    assert st["n_votes"] == len(gv)
    for e in range(batch.n_events):
        gs = gv[:, 0] == e
        os_ = en["event"] == e
        ns = en["near_event"] == e
        rep, flips = parity.compare_triplets(gv[gs, 1:], gb[gs], en["ijk"][os_], en["bin"][os_],
                                             en["amb"][os_], en["near_ijk"][ns])
        assert rep["ok"], rep
        gh = rec.histogram(e).cpu().numpy().astype(np.int64)
        oh = parity.dense_oracle_hist(en["bin"][os_], setup.n_bins)
        diff = np.nonzero(gh != oh)[0]
        assert set(diff.tolist()) <= flips, (len(diff), len(flips))
        affected = parity.dilate(set(diff.tolist()), dims, setup.periodic)
        cand, hits_l = res.event(e)
        oe = ref["events"][e]
        crep = parity.compare_candidates(cand["bin"], cand["votes"], hits_l, oe["cand_bins"],
                                         oe["cand_votes"], oe["cand_hits"], affected)
        assert crep["ok"], crep
        # candidate parameters are bin centres: identical FP64 expression, rounded to FP32
        if len(cand) and len(oe["cand_bins"]):
            common, gi, oi = np.intersect1d(cand["bin"].astype(np.int64), oe["cand_bins"],
                                            return_indices=True)
            assert np.array_equal(cand["params"][gi], oe["cand_params"][oi].astype(np.float32))
        rep.update(n_hist_diff=len(diff), cand=crep["n_compared"])
        reports.append(rep)
        if check_plateaus:
            plateaus += parity.plateau_count(gh, dims, setup.periodic, setup.threshold)
    # the votes in candidate bins, and the plateau bins the tie pass checked
    assert st["n_cand_votes"] == int(res.cand["votes"].sum())
    if check_plateaus:
        assert st["n_plateau"] == plateaus, (st["n_plateau"], plateaus)
    rec.close()
    return reports


def test_smoke_barrel4_20trk(trk):
    cfg = ev.load_workload("barrel4_20trk")
    reps = _full_compare(trk, cfg, ev.make_batch(cfg), check_plateaus=True)
    assert reps[0]["n_both"] > 1000


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_barrel4_other_seeds(trk, seed):
    cfg = ev.load_workload("barrel4_20trk")
    _full_compare(trk, cfg, ev.make_batch(cfg, seed=seed))


def test_barrel10_reduced_event(trk):
    # the 10-layer geometry and binning with 60 tracks: several tiles per layer triple and
    # ragged tile tails, small enough for the oracle
    cfg = ev.load_workload("barrel10_500trk")
    cfg["events"]["n_tracks"] = 60
    reps = _full_compare(trk, cfg, ev.make_batch(cfg, seed=21))
    assert reps[0]["n_both"] > 10000


@pytest.mark.parametrize("dims", [(15, 13, 9, 7, 5), (17, 32, 16, 16, 16)])
def test_odd_binnings(trk, dims):
    """Bin counts whose inner block (d0 x cot x z0) is odd and not a multiple of 4 (the
    scalar peak pass), and a non-power-of-two phi0 count, on the reduced 10-layer event."""
    cfg = ev.load_workload("barrel10_500trk")
    cfg["events"]["n_tracks"] = 40
    cfg["binning"]["n"] = list(dims)
    cfg["binning"]["threshold"] = 3
    reps = _full_compare(trk, cfg, ev.make_batch(cfg, seed=23), check_plateaus=True)
    assert reps[0]["n_both"] > 5000


def test_batch_of_uneven_events(trk):
    cfg = ev.load_workload("barrel10_500trk")
    rng = np.random.default_rng(5)
    evs = [ev.make_event(cfg, rng, n) for n in (3, 40, 0, 25, 1, 60)]
    batch = ev.concat(evs)
    _full_compare(trk, cfg, batch)


@pytest.mark.parametrize("tile", [(16, 16), (8, 16), (16, 8), (8, 8), (4, 16), (8, 4), (4, 8)])
def test_tile_shapes_agree(trk, tile):
    cfg = ev.load_workload("barrel10_500trk")
    cfg["events"]["n_tracks"] = 30
    batch = ev.make_batch(cfg, seed=31)
    r0, res0, _ = _run(trk, cfg, batch)
    h0 = r0.histogram(0).cpu().numpy()
    r1, res1, _ = _run(trk, cfg, batch, tile_i=tile[0], tile_j=tile[1])
    h1 = r1.histogram(0).cpu().numpy()
    assert np.array_equal(h0, h1)
    assert np.array_equal(res0.cand, res1.cand)
    assert np.array_equal(res0.hit_ids, res1.hit_ids)
    r0.close()
    r1.close()


def test_alone_equals_in_batch(trk):
    cfg = ev.load_workload("barrel10_500trk")
    rng = np.random.default_rng(8)
    evs = [ev.make_event(cfg, rng, n) for n in (20, 35, 10)]
    batch = ev.concat(evs)
    rb, resb, _ = _run(trk, cfg, batch)
    for e, one in enumerate(evs):
        ra, resa, _ = _run(trk, cfg, one)
        ca, ha = resa.event(0)
        cb, hb = resb.event(e)
        assert np.array_equal(ca["bin"], cb["bin"])
        assert np.array_equal(ca["votes"], cb["votes"])
        off = int(batch.offsets[e])
        for x, y in zip(ha, hb):
            assert np.array_equal(x + off, y)
        assert np.array_equal(ra.histogram(0).cpu().numpy(), rb.histogram(e).cpu().numpy())
        ra.close()
    rb.close()


def test_graph_and_eager_agree(trk):
    cfg = ev.load_workload("barrel4_20trk")
    batch = ev.make_batch(cfg, seed=4)
    r0, res0, _ = _run(trk, cfg, batch, max_hits=4096, use_graph=1)
    r1, res1, _ = _run(trk, cfg, batch, max_hits=4096, use_graph=0)
    assert np.array_equal(res0.cand, res1.cand) and np.array_equal(res0.hit_ids, res1.hit_ids)
    # replaying the captured graph on new inputs
    b2 = ev.make_batch(cfg, seed=5)
    hits = torch.from_numpy(b2.packed()).cuda()
    offs = torch.from_numpy(b2.offsets).cuda()
    res0b = r0.result(r0.reconstruct_device(hits, offs))
    res1b = r1.result(r1.reconstruct_device(hits, offs))
    assert np.array_equal(res0b.cand, res1b.cand) and np.array_equal(res0b.hit_ids, res1b.hit_ids)
    r0.close()
    r1.close()


def test_host_path_equals_device_path(trk):
    cfg = ev.load_workload("barrel4_20trk")
    batch = ev.make_batch(cfg, seed=6)
    rec, resd, _ = _run(trk, cfg, batch)
    hp = batch.packed()
    rc = rec.reconstruct_host(hp, batch.offsets.astype(np.int64))
    resh = rec.result(rc, from_host=True)
    assert np.array_equal(resd.cand, resh.cand)
    assert np.array_equal(resd.hit_ids, resh.hit_ids)
    rec.close()


def test_edge_cases(trk):
    cfg = ev.load_workload("barrel4_20trk")
    b = ev.make_batch(cfg, seed=7)
    one_layer = np.nonzero(b.layer == 2)[0]
    bad = b.event(0)
    bad.layer = bad.layer.copy()
    bad.layer[5] = 9                       # layer id out of range
    parts = [ev.Batch(np.zeros((0, 3), np.float32), np.zeros(0, np.int32), np.array([0, 0]),
                      np.zeros(0, np.int32), np.zeros((0, 6))),
             ev.Batch(b.xyz[one_layer], b.layer[one_layer], np.array([0, len(one_layer)]),
                      b.track[one_layer], np.zeros((0, 6))),
             bad, b]
    batch = ev.concat(parts)
    rec, res, _ = _run(trk, cfg, batch)
    assert res.status.tolist() == [0, 0, trk.TRK_EV_BAD_HIT, 0]
    assert res.cand_off[1] - res.cand_off[0] == 0
    assert res.cand_off[2] - res.cand_off[1] == 0
    assert res.cand_off[3] - res.cand_off[2] == 0
    ra, resa, _ = _run(trk, cfg, b)
    c3, h3 = res.event(3)
    ca, ha = resa.event(0)
    assert np.array_equal(c3["bin"], ca["bin"])
    off = int(batch.offsets[3])
    for x, y in zip(ha, h3):
        assert np.array_equal(x + off, y)
    rec.close()
    ra.close()


def test_capacity_overflow_is_reported(trk):
    cfg = ev.load_workload("barrel4_20trk")
    b = ev.make_batch(cfg)
    rec, res, _ = _run(trk, cfg, b, vote_capacity=64)
    assert res.rc == trk.TRK_ERR_CAPACITY
    assert res.status[0] & trk.TRK_EV_VOTE_OVERFLOW
    assert res.cand_off[1] == res.cand_off[0]
    rec.close()


def test_fit_triplets_precision_sample(trk):
    """FP32 parameters of random triplets vs FP64 within 1e-5 * max(|p|, half-range)."""
    for name in ("barrel10_500trk", "barrel10_2000trk_precision"):
        cfg = ev.load_workload(name)
        b = ev.make_batch(cfg)
        setup = oracle.OracleSetup.from_workload(cfg)
        rng = np.random.default_rng(1)
        rows = []
        for (la, lb, lc) in setup.triples:
            A = np.nonzero(b.layer == la)[0]
            B = np.nonzero(b.layer == lb)[0]
            Cc = np.nonzero(b.layer == lc)[0]
            n = 40000
            rows.append(np.stack([rng.choice(A, n), rng.choice(B, n), rng.choice(Cc, n)], 1))
        ijk = np.concatenate(rows).astype(np.int32)
        ref = oracle.fit_list(b.xyz, b.layer, ijk, setup)
        rec = trk.Reconstructor(cfg, max_events=1, max_hits=b.n_hits)
        hits = torch.from_numpy(b.packed()).cuda()
        par, bins, flags = rec.fit_triplets(hits, torch.from_numpy(ijk).cuda())
        par = par.cpu().numpy()
        bins = bins.cpu().numpy().view(np.uint32).astype(np.int64)
        flags = flags.cpu().numpy()
        # the tolerance applies to the triplets that can vote: accepted by the oracle, or
        # rejected only by a parameter within eps of its range limit
        # (a hit at the point opposite the perigee has an undefined path-length sign: the
        # oracle flags it, bit 2, and its parameters may legitimately differ)
        relevant = ((ref["status"] == 0) | ((ref["status"] == 1) & ref["amb"])) & \
            ((ref["amb_bits"] & 4) == 0)
        err = parity.param_errors(par[relevant], ref["par"][relevant])
        tol = parity.param_tolerance(ref["par"][relevant], setup.lo, setup.hi, EPS_REL)
        worst = (err / tol).max(axis=0)
        assert relevant.sum() > 1000
        assert np.all(worst <= 1.0), (name, worst)
        acc_o = ref["status"] == 0
        acc_g = (flags & 1) != 0
        mismatch = (acc_o != acc_g) & ~ref["amb"]
        assert not mismatch.any(), (name, int(mismatch.sum()))
        both = acc_o & acc_g & ~ref["amb"]
        assert np.array_equal(bins[both], ref["bin"][both])
        rec.close()


def test_autotune_keeps_results(trk):
    cfg = ev.load_workload("barrel10_500trk")
    cfg["events"]["n_tracks"] = 40
    batch = ev.make_batch(cfg, seed=17)
    rec, res0, hits = _run(trk, cfg, batch)
    offs = torch.from_numpy(batch.offsets).cuda()
    best = rec.autotune(hits, offs, reps=1)
    assert (best["tile_i"], best["tile_j"]) in [(16, 16), (8, 16), (16, 8), (8, 8), (4, 16),
                                                (8, 4), (4, 8)]
    assert best["vote_level"] in (2, 3, 4) and best["vote_ms"] > 0
    res1 = rec.result(rec.reconstruct_device(hits, offs))
    assert np.array_equal(res0.cand, res1.cand)
    assert np.array_equal(res0.hit_ids, res1.hit_ids)
    rec.close()


@pytest.mark.parametrize("level", [2, 3, 4])
def test_vote_levels_agree(trk, level):
    cfg = ev.load_workload("barrel10_500trk")
    cfg["events"]["n_tracks"] = 30
    batch = ev.make_batch(cfg, seed=33)
    r0, res0, _ = _run(trk, cfg, batch)
    r1, res1, _ = _run(trk, cfg, batch, vote_level=level)
    assert np.array_equal(r0.histogram(0).cpu().numpy(), r1.histogram(0).cpu().numpy())
    assert np.array_equal(res0.cand, res1.cand)
    assert np.array_equal(res0.hit_ids, res1.hit_ids)
    r0.close()
    r1.close()
