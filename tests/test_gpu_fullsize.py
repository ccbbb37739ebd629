"""Full-size parity on the 500-track 10-layer event (1.1e9 triplets), in the launch
configuration the benchmark times (GPU only).

Every accepted triplet and every histogram bin is compared with the FP64 oracle; the
candidates and their hit lists are compared in seeded phi0 slabs (the oracle's peak test
of each bin is independent of the others, so a slab is an exact sample), including the
phi0 wrap-around slabs.
"""
import time

import numpy as np
import pytest

import oracle
import parity
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


def test_barrel10_500trk_full(trk):
    cfg = ev.load_workload("barrel10_500trk")
    batch = ev.make_batch(cfg)
    setup = oracle.OracleSetup.from_workload(cfg)
    dims = tuple(int(x) for x in setup.n)
    # the benchmark's handle configuration
    rec = trk.Reconstructor(cfg, max_events=1, max_hits=batch.n_hits, vote_capacity=1 << 28,
                            cand_capacity=1 << 21, assign_capacity=1 << 25)
    hits = torch.from_numpy(batch.packed()).cuda()
    offs = torch.from_numpy(batch.offsets).cuda()
    rc = rec.reconstruct_device(hits, offs)
    res = rec.result(rc)
    assert rc == 0 and res.status[0] == 0, rec.error()
    st = rec.stats()
    gv, gb = rec.votes()
    gv = gv.cpu().numpy()
    gb = gb.cpu().numpy().view(np.uint32).astype(np.int64)
    gh = rec.histogram(0).cpu().numpy().astype(np.int64)

    t0 = time.time()
    en = oracle.enumerate_batch(batch.xyz, batch.layer, batch.offsets, setup)
    print("oracle enumeration %.1f s, %d accepted" % (time.time() - t0, len(en["bin"])))
    assert st["n_triplets"] == en["n_triplets"]
    rep, flips = parity.compare_triplets(gv[:, 1:], gb, en["ijk"], en["bin"], en["amb"],
                                         en["near_ijk"])
    print(rep)
    assert rep["ok"], rep
    oh = parity.dense_oracle_hist(en["bin"], setup.n_bins)
    diff = np.nonzero(gh != oh)[0]
    assert set(diff.tolist()) <= flips, (len(diff), len(flips))
    affected = parity.dilate(set(diff.tolist()), dims, setup.periodic)

    rng = np.random.default_rng(2024)
    slabs = {0, dims[0] - 1} | set(rng.choice(np.arange(1, dims[0] - 1), 3, replace=False).tolist())
    ub = np.nonzero(oh)[0].astype(np.int64)
    cb, cv = oracle.peaks(ub, oh[ub], setup, only_phi0=slabs)
    ch = oracle.assign_hits(en["ijk"], en["bin"], cb)
    stride0 = int(np.prod(dims[1:]))
    cand, hl = res.event(0)
    sel = np.isin(cand["bin"].astype(np.int64) // stride0, list(slabs))
    crep = parity.compare_candidates(cand["bin"][sel], cand["votes"][sel],
                                     [h for h, k in zip(hl, sel) if k], cb, cv, ch, affected)
    print(crep, "hist diffs", len(diff), "candidates total", len(cand))
    assert crep["ok"], crep
    assert crep["n_compared"] > 1000
    rec.close()
