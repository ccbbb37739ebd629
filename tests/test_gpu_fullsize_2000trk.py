"""Candidate parity on the 2000-track precision event at full size (128 x 128 x 64 x 32 x 32
bins, 5.2e10 triplets), in blocks of the parameter space (GPU only).

The FP64 oracle fits and bins every triplet of the event (its output restricted to chosen
(phi0 row, q/pT row) blocks, trk_oracle.c orc_run_blocks), on all host cores: this test
takes about ten minutes of CPU time.  Five slabs of eight q/pT rows are compared: the two
phi0 rows at the wrap and three seeded rows.  Inside them:
  * every histogram bin of the slabs and their neighbour blocks that differs between the
    GPU and the oracle must be the oracle bin or the GPU bin of a triplet whose parameters
    lie within eps of a bin edge or range limit, and whose two sides bin it differently
    (the GPU's bin of such a triplet comes from trk_fit_triplets, the vote kernel's own
    arithmetic);
  * every candidate whose 3^5 neighbourhood holds no differing bin must be a candidate on
    both sides or neither, with equal votes and hit lists.
"""
import os
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


def _around(blocks, n0, n1):
    out = set()
    for i0, i1 in blocks:
        for d0 in (-1, 0, 1):
            for d1 in (-1, 0, 1):
                if 0 <= i1 + d1 < n1:
                    out.add(((i0 + d0) % n0, i1 + d1))
    return sorted(out)


def test_barrel10_2000trk_candidates_in_slabs(trk):
    cfg = ev.load_workload("barrel10_2000trk_precision")
    b = ev.make_batch(cfg)
    setup = oracle.OracleSetup.from_workload(cfg)
    dims = tuple(int(x) for x in setup.n)
    n0, n1 = dims[0], dims[1]
    inner = int(np.prod(dims[2:]))
    rng = np.random.default_rng(2025)
    rows = [0, n0 - 1] + sorted(rng.choice(np.arange(1, n0 - 1), 3, replace=False).tolist())
    q0s = rng.integers(n1 // 2 - 24, n1 // 2 + 16, size=len(rows))
    keep = sorted({(int(r), int(q)) for r, q0 in zip(rows, q0s) for q in range(q0, q0 + 8)})
    count = _around(keep, n0, n1)
    flip = _around(count, n0, n1)

    # the whole event through the CUDA path, as the precision study's full-event test runs it
    rec = trk.Reconstructor(cfg, max_events=1, max_hits=b.n_hits, vote_capacity=1 << 34,
                            cand_capacity=1 << 23, assign_capacity=1 << 28,
                            peak_scratch_bytes=8 << 30)
    hits = torch.from_numpy(b.packed()).cuda()
    offs = torch.from_numpy(b.offsets).cuda()
    rc = rec.reconstruct_device(hits, offs)
    res = rec.result(rc)
    assert rc == 0 and res.status[0] == 0, rec.error()
    h = rec.histogram(0)
    g_counts = torch.stack([h[(i0 * n1 + i1) * inner:(i0 * n1 + i1 + 1) * inner]
                            for i0, i1 in count]).cpu().numpy().astype(np.int64)
    del h
    cand = res.cand[res.cand_off[0]:res.cand_off[1]]
    cblk = cand["bin"].astype(np.int64) // inner
    ksel = np.isin(cblk, [i0 * n1 + i1 for i0, i1 in keep])
    g_bins = cand["bin"][ksel].astype(np.int64)
    g_votes = cand["votes"][ksel]
    g_hits = [res.hit_ids[int(r["hit_off"]):int(r["hit_off"]) + int(r["n_hits"])] for r in cand[ksel]]

    t0 = time.time()
    blk = oracle.enumerate_blocks(b.xyz, b.layer, setup, count, keep, flip)
    print("oracle over %d triplets in %.0f s on %d threads" % (blk["n_triplets"], time.time() - t0,
                                                              oracle.max_threads()))
    assert blk["n_triplets"] == int(ev.layer_triplet_count(b, cfg["geometry"]["triples"]).sum())

    # explained flips: the listed triplets binned by the vote kernel's own arithmetic
    fl = blk["flip_ijk"]
    par, fbins, flags = rec.fit_triplets(hits, torch.from_numpy(fl.astype(np.int32)).cuda())
    fbins = fbins.cpu().numpy().view(np.uint32).astype(np.int64)
    gacc = (flags.cpu().numpy() & 1) != 0
    oacc = blk["flip_acc"]
    moved = (gacc != oacc) | (gacc & oacc & (fbins != blk["flip_bin"]))
    flips = set(blk["flip_bin"][moved & oacc].tolist()) | set(fbins[moved & gacc].tolist())
    o_counts = blk["counts"].astype(np.int64)
    diff_rows, diff_r = np.nonzero(g_counts != o_counts)
    diff = set((np.array([count[q][0] * n1 + count[q][1] for q in diff_rows], np.int64) * inner
                + diff_r).tolist())
    assert diff <= flips, (len(diff), len(diff - flips), sorted(diff - flips)[:5])
    affected = parity.dilate(diff, dims, setup.periodic)

    cb, cv = oracle.block_peaks(blk, setup, keep)
    ch = oracle.assign_hits(blk["keep_ijk"], blk["keep_bin"], cb)
    crep = parity.compare_candidates(g_bins, g_votes, g_hits, cb, cv, ch, affected)
    print("2000trk slabs:", crep, "differing bins", len(diff), "listed flips", int(moved.sum()),
          "candidates in slabs", len(g_bins), len(cb))
    assert crep["ok"], crep
    assert crep["n_compared"] >= 1000
    rec.close()
