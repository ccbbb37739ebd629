"""Serving (continuous batching) through the C ABI (GPU only).

Events of the batch workload's multiplicity mix (scaled down so the suite stays quick)
arrive with random gaps, including bursts; each event's candidates and hit lists from the
server must equal those of the same event reconstructed alone, whatever batch it shared.
The server batches by backlog (one more event per 24 waiting), so a burst of 60 events
makes it run multi-event batches and the gaps after it make it run single events.
"""
import ctypes
import time

import numpy as np
import pytest

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


def _events(n, seed):
    cfg = ev.load_workload("barrel10_batch256")
    rng = np.random.default_rng(seed)
    counts = np.clip(rng.poisson(40, n), 5, 120)
    return cfg, [ev.make_event(cfg, rng, int(c)) for c in counts]


def _alone(trk, cfg, e):
    rec = trk.Reconstructor(cfg, max_events=1, max_hits=max(e.n_hits, 1), vote_capacity=1 << 24,
                            cand_capacity=1 << 18, assign_capacity=1 << 22)
    hits = torch.from_numpy(e.packed()).cuda()
    offs = torch.from_numpy(e.offsets).cuda()
    res = rec.result(rec.reconstruct_device(hits, offs))
    rec.close()
    assert res.rc == 0
    return res.event(0)


def test_served_results_equal_alone(trk):
    n_burst = 60
    cfg, evs = _events(n_burst + 14, seed=91)
    srv = trk.Server(cfg, lane_events=4, lane_hits=8192, n_lanes=2, vote_capacity=1 << 25,
                     cand_capacity=1 << 19, assign_capacity=1 << 23)
    rng = np.random.default_rng(3)
    tickets = []
    for i, e in enumerate(evs):
        tickets.append(srv.submit(e.packed()))
        if i < n_burst or i % 5 != 4:       # one long burst, then bursts of five and pauses
            continue
        time.sleep(float(rng.uniform(0.0, 0.05)))
    batch_sizes = []
    for t, e in zip(tickets, evs):
        info = srv.wait(t, timeout_s=120.0)
        assert info is not None and info["status"] == 0, info
        batch_sizes.append(info["batch_events"])
        cand, hits = srv.take(t, info)
        ca, ha = _alone(trk, cfg, e)
        assert np.array_equal(cand["bin"], ca["bin"])
        assert np.array_equal(cand["votes"], ca["votes"])
        assert np.array_equal(cand["params"], ca["params"])
        for x, y in zip(hits, ha):
            assert np.array_equal(x, y)
    c = srv.counts()
    assert c["events"] == len(evs) and c["failed"] == 0 and c["queued"] == 0
    assert max(batch_sizes) > 1, batch_sizes        # some events shared a batch
    assert batch_sizes[-1] == 1, batch_sizes        # a short queue runs one event per call
    srv.close()


def test_server_rejects_oversized_event(trk):
    cfg, evs = _events(1, seed=5)
    srv = trk.Server(cfg, lane_events=2, lane_hits=64, n_lanes=1, vote_capacity=1 << 20,
                     cand_capacity=1 << 16, assign_capacity=1 << 20)
    big = max(evs, key=lambda e: e.n_hits)
    assert big.n_hits > 64
    with pytest.raises(trk.TrkError) as ex:
        srv.submit(big.packed())
    assert ex.value.code == trk.TRK_ERR_CAPACITY
    srv.close()


def test_handles_created_and_destroyed_while_the_server_runs(trk):
    # handles with graph capture are created, used and destroyed in this thread while the
    # server's lanes reconstruct in theirs: destruction waits for the handle's own work
    # only, so neither side fails
    cfg, evs = _events(12, seed=17)
    srv = trk.Server(cfg, lane_events=4, lane_hits=8192, n_lanes=2, vote_capacity=1 << 25,
                     cand_capacity=1 << 19, assign_capacity=1 << 23)
    tickets = [srv.submit(e.packed()) for e in evs]
    alone = []
    for e in evs[:6]:
        rec = trk.Reconstructor(cfg, max_events=1, max_hits=max(e.n_hits, 1),
                                vote_capacity=1 << 24, cand_capacity=1 << 18,
                                assign_capacity=1 << 22, use_graph=1)
        hits = torch.from_numpy(e.packed()).cuda()
        offs = torch.from_numpy(e.offsets).cuda()
        res = rec.result(rec.reconstruct_device(hits, offs))
        assert res.rc == 0, rec.error()
        h = torch.empty(rec.lib.trk_histogram_size(rec.h), dtype=torch.int32, device="cuda")
        # an asynchronous copy left pending when the handle is destroyed
        assert rec.lib.trk_get_histogram(rec.h, 0, ctypes.c_void_p(h.data_ptr()),
                                         ctypes.c_void_p(0)) == 0
        alone.append(res.event(0))
        rec.close()
    for i, (t, e) in enumerate(zip(tickets, evs)):
        info = srv.wait(t, timeout_s=120.0)
        assert info is not None and info["status"] == 0 and info["rc"] == 0, info
        cand, hits = srv.take(t, info)
        if i < len(alone):
            ca, ha = alone[i]
            assert np.array_equal(cand["bin"], ca["bin"])
            for x, y in zip(hits, ha):
                assert np.array_equal(x, y)
    assert srv.counts()["failed"] == 0
    srv.close()
