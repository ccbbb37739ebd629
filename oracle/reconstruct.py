"""Votes, peaks and hit assignment of the oracle (numpy).  Test infrastructure only.

Paper: Sec. 7 and Fig. 3 -- votes of all hit combinations accumulate in the parameter
space and candidate tracks are its local maxima; Sec. 8 -- candidates are then handed,
with their hits, to a fit.  The paper gives no tie rule, threshold or hit assignment;
the readings are:
  * peak rule: bin b is a candidate iff h[b] >= T, h[b] >= h[m] for every one of the
    3^5 - 1 neighbours m (periodic dimensions wrap, neighbours outside a non-periodic
    range are skipped, a neighbour equal to b itself is skipped), and h[b] > h[m] for
    every neighbour m with a smaller row-major index (deterministic plateau rule);
  * candidate hits: the sorted, de-duplicated union of the hits of every accepted
    triplet that voted into the candidate's bin;
  * candidate parameters: the centre of its bin, lo + (idx + 1/2) (hi - lo) / n.
"""
from __future__ import annotations

import itertools

import numpy as np

from .core import OracleSetup, enumerate_batch


def neighbour_offsets() -> np.ndarray:
    """The 3^5 - 1 offsets of the 5-D neighbourhood, shape (242, 5)."""
    offs = [o for o in itertools.product((-1, 0, 1), repeat=5) if any(o)]
    return np.asarray(offs, dtype=np.int64)


def histogram(event: np.ndarray, bins: np.ndarray, n_events: int):
    """Per event: (sorted non-empty bins, their vote counts)."""
    out = []
    for e in range(n_events):
        b = bins[event == e]
        ub, cnt = np.unique(b, return_counts=True)
        out.append((ub.astype(np.int64), cnt.astype(np.int64)))
    return out


def peaks(ubins: np.ndarray, counts: np.ndarray, setup: OracleSetup, chunk: int = 65536,
          only_phi0=None):
    """Candidates of one event's histogram given as sorted non-empty bins and counts.
    Returns (candidate bins ascending, their votes).  Bins above threshold are examined
    in chunks only to bound memory; each bin's test is independent of the others, so
    `only_phi0` (a set of phi0 bin indices) restricts the answer to those slabs without
    changing it there."""
    T = setup.threshold
    sel = counts >= T
    if only_phi0 is not None:
        stride0 = int(np.prod(setup.n[1:]))
        sel &= np.isin(ubins // stride0, np.asarray(sorted(only_phi0), dtype=np.int64))
    over_all, hv_all = ubins[sel], counts[sel]
    if len(over_all) == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    dims = tuple(int(x) for x in setup.n)
    offs = neighbour_offsets()                                      # (242, 5)
    keep_all = np.zeros(len(over_all), dtype=bool)
    for c0 in range(0, len(over_all), chunk):
        over, hv = over_all[c0:c0 + chunk], hv_all[c0:c0 + chunk]
        idx = np.stack(np.unravel_index(over, dims), axis=1)          # (m, 5)
        nidx = idx[:, None, :] + offs[None, :, :]                       # (m, 242, 5)
        valid = np.ones(nidx.shape[:2], dtype=bool)
        for k in range(5):
            if setup.periodic[k]:
                nidx[:, :, k] %= dims[k]
            else:
                valid &= (nidx[:, :, k] >= 0) & (nidx[:, :, k] < dims[k])
        nidx = np.where(valid[:, :, None], nidx, 0)
        nbin = np.ravel_multi_index(tuple(nidx[:, :, k] for k in range(5)), dims)
        valid &= nbin != over[:, None]
        pos = np.searchsorted(ubins, nbin)
        pos_c = np.minimum(pos, len(ubins) - 1)
        present = ubins[pos_c] == nbin
        ncnt = np.where(present, counts[pos_c], 0)
        ge = np.all(~valid | (hv[:, None] >= ncnt), axis=1)
        gt_lower = np.all(~valid | (nbin > over[:, None]) | (hv[:, None] > ncnt), axis=1)
        keep_all[c0:c0 + chunk] = ge & gt_lower
    return over_all[keep_all], hv_all[keep_all]


def bin_centres(cand_bins: np.ndarray, setup: OracleSetup) -> np.ndarray:
    dims = tuple(int(x) for x in setup.n)
    idx = np.stack(np.unravel_index(cand_bins, dims), axis=1).astype(np.float64)
    w = (setup.hi - setup.lo) / setup.n
    return setup.lo[None, :] + (idx + 0.5) * w[None, :]


def assign_hits(ijk: np.ndarray, bins: np.ndarray, cand_bins: np.ndarray):
    """For each candidate bin, the sorted unique hit ids of the triplets voting there."""
    order = np.argsort(bins, kind="stable")
    sb = bins[order]
    out = []
    for b in cand_bins:
        lo = np.searchsorted(sb, b, side="left")
        hi = np.searchsorted(sb, b, side="right")
        out.append(np.unique(ijk[order[lo:hi]].ravel()).astype(np.int64))
    return out


def reconstruct(xyz, layer, offsets, setup: OracleSetup, n_threads: int = 0, enum=None) -> dict:
    """Whole oracle: enumeration, per-event histogram, candidates and their hits."""
    if enum is None:
        enum = enumerate_batch(xyz, layer, offsets, setup, n_threads=n_threads)
    n_events = len(offsets) - 1
    hists = histogram(enum["event"], enum["bin"], n_events)
    events = []
    for e in range(n_events):
        ub, cnt = hists[e]
        cb, cv = peaks(ub, cnt, setup)
        sel = enum["event"] == e
        hits = assign_hits(enum["ijk"][sel], enum["bin"][sel], cb)
        events.append(dict(hist_bins=ub, hist_counts=cnt, cand_bins=cb, cand_votes=cv,
                           cand_params=bin_centres(cb, setup), cand_hits=hits))
    return dict(enum=enum, events=events)
