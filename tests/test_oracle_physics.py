"""Physics sanity of the oracle, not parity (CPU only).

On the 4-layer, 20-track event (10 seeds): every generated track that leaves a hit on each
layer of at least one listed layer triple, and whose true parameters lie inside the
binning, should have its true bin, or a neighbour of it, among the candidates.  This checks
the whole chain (fit conventions, binning, votes, peak rule) against the generator's truth
rather than against another implementation of the same formulas.  The fraction found is a
sanity figure, printed with -s; the paper's 80-86 % efficiencies (Sec. 8) belong to other
algorithms and workloads and are not a target.
"""
import numpy as np

import oracle
from paper_1305_4855_gb300 import events as ev


def _truth_bin(p, s):
    """5-D bin of true parameters p (phi0 wrapped into [lo, hi)), or None if out of range."""
    idx = []
    for k in range(5):
        v = float(p[k])
        if s.periodic[k]:
            period = s.hi[k] - s.lo[k]
            v = s.lo[k] + (v - s.lo[k]) % period
        if not (s.lo[k] <= v < s.hi[k]):
            return None
        w = (s.hi[k] - s.lo[k]) / s.n[k]
        idx.append(min(int(np.floor((v - s.lo[k]) / w)), int(s.n[k]) - 1))
    return np.array(idx)


def _near(a, b, n, periodic):
    d = np.abs(a - b)
    for k in range(5):
        if periodic[k]:
            d[k] = min(d[k], n[k] - d[k])
    return bool(np.all(d <= 1))


def test_truth_bins_are_found_barrel4():
    cfg = ev.load_workload("barrel4_20trk")
    s = oracle.OracleSetup.from_workload(cfg)
    n = np.asarray(s.n, dtype=np.int64)
    found = findable = 0
    for seed in range(1, 11):
        b = ev.make_batch(cfg, seed=seed)
        r = oracle.reconstruct(b.xyz, b.layer, b.offsets, s)
        cb = np.asarray(r["events"][0]["cand_bins"], dtype=np.int64)
        cand = np.stack(np.unravel_index(cb, tuple(n)), axis=1) if len(cb) else np.zeros((0, 5))
        for t in range(len(b.truth)):
            layers = set(b.layer[b.track == t].tolist())
            if not any(all(int(l) in layers for l in tri) for tri in s.triples):
                continue
            tb = _truth_bin(b.truth[t, :5], s)
            if tb is None:
                continue
            findable += 1
            if any(_near(tb, c, n, s.periodic) for c in cand):
                found += 1
    eff = found / findable
    print(f"truth bins found: {found} of {findable} findable tracks ({eff:.3f})")
    assert findable >= 150
    assert eff >= 0.9
