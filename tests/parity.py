"""GPU-vs-oracle comparison helpers (test infrastructure).

The CUDA path must reproduce the oracle exactly on integer outputs, except where an FP32
parameter sits within eps of a bin edge (the oracle flags such triplets as ambiguous, or
as near-accepted when they fall just outside a range).  The checks, stage by stage:

  triplets   -- a triplet accepted by both sides has the same bin unless ambiguous; one
                accepted by the GPU only must be near-accepted in the oracle; one accepted
                by the oracle only must be ambiguous;
  histogram  -- every bin whose count differs must be touched by such an explained flip;
  candidates -- every bin whose 3^5 neighbourhood contains no differing bin must be a
                candidate on both sides or on neither, with equal votes and hit lists.

Nothing computed here is fed back into the oracle: the oracle runs on the generated
inputs alone and the GPU outputs are only compared with its results.
"""
from __future__ import annotations

import itertools

import numpy as np

SHIFT = 21


def triplet_keys(ijk: np.ndarray) -> np.ndarray:
    ijk = np.asarray(ijk, dtype=np.int64)
    return (ijk[:, 0] << (2 * SHIFT)) | (ijk[:, 1] << SHIFT) | ijk[:, 2]


def compare_triplets(gpu_ijk, gpu_bin, orc_ijk, orc_bin, orc_amb, orc_near_ijk):
    """Returns (report dict, set of bins touched by explained flips)."""
    gk = triplet_keys(gpu_ijk)
    ok_ = triplet_keys(orc_ijk)
    nk = triplet_keys(orc_near_ijk) if len(orc_near_ijk) else np.zeros(0, np.int64)
    go = np.argsort(gk)
    gk, gb = gk[go], np.asarray(gpu_bin, np.int64)[go]
    oo = np.argsort(ok_)
    ok_, ob, oa = ok_[oo], np.asarray(orc_bin, np.int64)[oo], np.asarray(orc_amb, bool)[oo]
    assert len(np.unique(gk)) == len(gk), "GPU voted a triplet twice"
    both, gi, oi = np.intersect1d(gk, ok_, assume_unique=True, return_indices=True)
    diff_bin = gb[gi] != ob[oi]
    bad_bin = diff_bin & ~oa[oi]
    g_only = np.setdiff1d(gk, ok_, assume_unique=True)
    o_only_mask = np.ones(len(ok_), bool)
    o_only_mask[oi] = False
    o_only_amb = oa[o_only_mask]
    g_only_near = np.isin(g_only, nk)
    flip_bins = set(gb[gi][diff_bin].tolist()) | set(ob[oi][diff_bin].tolist())
    flip_bins |= set(ob[o_only_mask].tolist())
    gmask = np.isin(gk, g_only)
    flip_bins |= set(gb[gmask].tolist())
    rep = dict(n_gpu=len(gk), n_oracle=len(ok_), n_both=len(both),
               n_bin_flips=int(diff_bin.sum()), n_bad_bin=int(bad_bin.sum()),
               n_gpu_only=len(g_only), n_gpu_only_unexplained=int((~g_only_near).sum()),
               n_oracle_only=int(o_only_mask.sum()),
               n_oracle_only_unexplained=int((~o_only_amb).sum()))
    rep["ok"] = (rep["n_bad_bin"] == 0 and rep["n_gpu_only_unexplained"] == 0
                 and rep["n_oracle_only_unexplained"] == 0)
    return rep, flip_bins


def dense_oracle_hist(bins: np.ndarray, nbins: int) -> np.ndarray:
    return np.bincount(np.asarray(bins, np.int64), minlength=nbins).astype(np.int64)


def dilate(bins, dims, periodic):
    """Bins within the 3^5 box of any of `bins` (phi0 wraps when periodic)."""
    if len(bins) == 0:
        return set()
    idx = np.stack(np.unravel_index(np.asarray(sorted(bins), np.int64), dims), axis=1)
    out = set()
    for off in itertools.product((-1, 0, 1), repeat=5):
        n = idx + np.asarray(off)
        ok = np.ones(len(n), bool)
        for k in range(5):
            if periodic[k]:
                n[:, k] %= dims[k]
            else:
                ok &= (n[:, k] >= 0) & (n[:, k] < dims[k])
        n = n[ok]
        out.update(np.ravel_multi_index(tuple(n[:, k] for k in range(5)), dims).tolist())
    return out


def compare_candidates(gpu_bins, gpu_votes, gpu_hits, orc_bins, orc_votes, orc_hits, affected):
    """Candidates outside `affected` must agree exactly (bins, votes, hit lists)."""
    g = {int(b): (int(v), np.asarray(h)) for b, v, h in zip(gpu_bins, gpu_votes, gpu_hits)}
    o = {int(b): (int(v), np.asarray(h)) for b, v, h in zip(orc_bins, orc_votes, orc_hits)}
    bad = []
    n_cmp = 0
    for b in set(g) | set(o):
        if b in affected:
            continue
        n_cmp += 1
        if b not in g or b not in o:
            bad.append(("missing", b, b in g, b in o))
            continue
        if g[b][0] != o[b][0]:
            bad.append(("votes", b, g[b][0], o[b][0]))
        elif not np.array_equal(np.sort(g[b][1]), o[b][1]) or not np.all(np.diff(g[b][1]) > 0):
            bad.append(("hits", b, g[b][1][:10].tolist(), o[b][1][:10].tolist()))
    return dict(n_compared=n_cmp, n_gpu=len(g), n_oracle=len(o), n_bad=len(bad),
                bad=bad[:10], ok=not bad)


def param_tolerance(par64: np.ndarray, lo, hi, rel=1e-5) -> np.ndarray:
    """|p32 - p64| allowed: rel * max(|p64|, half-range) per parameter."""
    half = 0.5 * (np.asarray(hi) - np.asarray(lo))
    return rel * np.maximum(np.abs(par64), half[None, :])


def param_errors(par32: np.ndarray, par64: np.ndarray):
    d = np.abs(par32.astype(np.float64) - par64)
    d[:, 0] = np.abs((par32[:, 0].astype(np.float64) - par64[:, 0] + np.pi) % (2 * np.pi) - np.pi)
    return d


def plateau_count(hist: np.ndarray, dims, periodic, threshold: int) -> int:
    """Bins at or above the threshold that equal the maximum of their 3^5 box while some
    other bin of the box has the same count: the bins the peak passes hand to the tie pass.
    Brute force over the 243 offsets (small histograms only); axis k wraps when
    periodic[k], and a wrapping axis needs at least three bins for the box to hold
    distinct bins."""
    h = np.asarray(hist, dtype=np.int64).reshape(dims)
    p = h
    for k in range(5):
        width = [(0, 0)] * 5
        width[k] = (1, 1)
        if periodic[k]:
            assert dims[k] >= 3
            p = np.pad(p, width, mode="wrap")
        else:
            p = np.pad(p, width, mode="constant", constant_values=-1)
    box = np.full(h.shape, -1, np.int64)
    views = []
    for off in itertools.product((0, 1, 2), repeat=5):
        sl = tuple(slice(o, o + n) for o, n in zip(off, h.shape))
        v = p[sl]
        views.append(v)
        np.maximum(box, v, out=box)
    eq = np.zeros(h.shape, np.int64)
    for v in views:
        eq += (v == box)
    return int(np.count_nonzero((h >= threshold) & (h == box) & (eq > 1)))
