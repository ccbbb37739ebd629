"""Full-size parity of the batched launch configuration (GPU only).

The benchmark's batched figure runs the 256-event mix (tracks ~ Poisson(400)) in calls of
32 events on a handle with its own capacities.  This test runs the first of those calls
in the same configuration and checks:
  * for two seeded events of the call, against the FP64 oracle run on the event alone:
    the dense histogram, where every differing bin must be explained by an edge-ambiguous
    triplet (its GPU bin taken from trk_fit_triplets, which evaluates the vote kernel's
    arithmetic), and the candidates with their hit lists in seeded phi0 slabs (an exact
    sample: the oracle's peak test of a bin reads only its neighbours), away from the
    differing bins;
  * for one of them, that the event run alone through the one-event handle of the plain
    benchmark gives the same histogram, candidates and hit lists as inside the batch;
  * for all 32 events, that the histograms add up to the call's vote count.
"""
import numpy as np
import pytest

import oracle
import parity
from paper_1305_4855_gb300 import events as ev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SUB = 32


@pytest.fixture(scope="module")
def trk():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1305_4855_gb300 import build
    build.build()
    from paper_1305_4855_gb300 import trk as t
    t.load_library()
    return t


def _gpu_bins_of(rec, hits_dev, ijk):
    """Bins the vote kernel gives explicit triplets (accepted ones only)."""
    if len(ijk) == 0:
        return set()
    _, bins, flags = rec.fit_triplets(hits_dev, torch.from_numpy(ijk.astype(np.int32)).cuda())
    bins = bins.cpu().numpy().view(np.uint32).astype(np.int64)
    acc = (flags.cpu().numpy() & 1) != 0
    return set(bins[acc].tolist())


def test_batch256_first_call_sampled_events(trk):
    cfg = ev.load_workload("barrel10_batch256")
    full = ev.make_batch(cfg)
    sub = ev.concat([full.event(e) for e in range(SUB)])
    per_event_max = int(np.diff(full.offsets).max())
    setup = oracle.OracleSetup.from_workload(cfg)
    dims = tuple(int(x) for x in setup.n)
    stride0 = int(np.prod(dims[1:]))

    # the benchmark's batched handle
    rec = trk.Reconstructor(cfg, max_events=SUB, max_hits=SUB * per_event_max,
                            vote_capacity=1 << 32, cand_capacity=1 << 23,
                            assign_capacity=1 << 28, peak_scratch_bytes=8 << 30)
    hits = torch.from_numpy(sub.packed()).cuda()
    offs = torch.from_numpy(sub.offsets).cuda()
    rc = rec.reconstruct_device(hits, offs)
    res = rec.result(rc)
    assert rc == 0 and np.all(res.status == 0), rec.error()
    st = rec.stats()
    tot = 0
    for e in range(SUB):
        tot += int(rec.histogram(e).sum().item())
    assert tot == st["n_votes"]

    rng = np.random.default_rng(77)
    picks = sorted(rng.choice(SUB, 2, replace=False).tolist())
    for e in picks:
        one = sub.event(e)
        a = int(sub.offsets[e])
        en = oracle.enumerate_batch(one.xyz, one.layer, one.offsets, setup)
        oh = parity.dense_oracle_hist(en["bin"], setup.n_bins)
        gh = rec.histogram(e).cpu().numpy().astype(np.int64)
        diff = np.nonzero(gh != oh)[0]
        # differing bins must be those of edge-ambiguous triplets, on either side
        hits_e = torch.from_numpy(one.packed()).cuda()
        amb_ijk = en["ijk"][en["amb"]]
        flips = set(en["bin"][en["amb"]].tolist())
        flips |= _gpu_bins_of(rec, hits_e, amb_ijk)
        flips |= _gpu_bins_of(rec, hits_e, en["near_ijk"])
        assert set(diff.tolist()) <= flips, (e, len(diff), len(flips))
        affected = parity.dilate(set(diff.tolist()), dims, setup.periodic)

        slabs = {0, dims[0] - 1} | set(rng.choice(np.arange(1, dims[0] - 1), 3,
                                                  replace=False).tolist())
        ub = np.nonzero(oh)[0].astype(np.int64)
        cb, cv = oracle.peaks(ub, oh[ub], setup, only_phi0=slabs)
        ch = oracle.assign_hits(en["ijk"], en["bin"], cb)
        cand, hl = res.event(e)
        sel = np.isin(cand["bin"].astype(np.int64) // stride0, list(slabs))
        g_hits = [np.asarray(h, np.int64) - a for h, k in zip(hl, sel) if k]
        crep = parity.compare_candidates(cand["bin"][sel], cand["votes"][sel], g_hits,
                                         cb, cv, ch, affected)
        print("event", e, "hist diffs", len(diff), crep)
        assert crep["ok"], crep
        assert crep["n_compared"] > 500

    # the first sampled event alone, through the plain benchmark's handle
    e = picks[0]
    one = sub.event(e)
    a = int(sub.offsets[e])
    batch_hist = rec.histogram(e).cpu().numpy()
    cand_b, hl_b = res.event(e)
    cand_b = cand_b.copy()
    hl_b = [np.asarray(h, np.int64) - a for h in hl_b]
    rec.close()
    alone = trk.Reconstructor(cfg, max_events=1, max_hits=per_event_max,
                              vote_capacity=1 << 29, cand_capacity=1 << 21,
                              assign_capacity=1 << 25)
    rc = alone.reconstruct_device(torch.from_numpy(one.packed()).cuda(),
                                  torch.from_numpy(one.offsets).cuda())
    r1 = alone.result(rc)
    assert rc == 0 and r1.status[0] == 0, alone.error()
    assert np.array_equal(alone.histogram(0).cpu().numpy(), batch_hist)
    cand_a, hl_a = r1.event(0)
    assert np.array_equal(cand_a["bin"], cand_b["bin"])
    assert np.array_equal(cand_a["votes"], cand_b["votes"])
    assert len(hl_a) == len(hl_b)
    assert all(np.array_equal(np.asarray(x, np.int64), y) for x, y in zip(hl_a, hl_b))
    alone.close()
