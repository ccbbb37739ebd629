"""The synthetic inputs follow the stated recipe (CPU only).

The generator (paper_1305_4855_gb300/events.py) stands in for the paper's standalone
Monte Carlo, which is not available; these checks pin what its workload files promise:
hits on their layer cylinders inside the barrel, the noise share, the truth ranges, the
displaced fraction, per-event shuffling, and determinism under the seed.
"""
import math

import numpy as np
import pytest

from paper_1305_4855_gb300 import events as ev


def _radii(b):
    return np.hypot(b.xyz[:, 0].astype(np.float64), b.xyz[:, 1].astype(np.float64))


@pytest.mark.parametrize("name", ["barrel4_20trk", "barrel10_500trk"])
def test_hits_on_their_layers(name):
    cfg = ev.load_workload(name)
    b = ev.make_batch(cfg)
    radius = np.asarray(cfg["geometry"]["radius"])
    zhalf = np.asarray(cfg["geometry"]["z_half"])
    r = _radii(b)
    # the r-phi smear is a rotation on the cylinder: the radius only carries float32
    # rounding
    assert np.all(np.abs(r - radius[b.layer]) <= 1e-5 * radius[b.layer] + 1e-6)
    # z smear (50 um) may push a hit just past the end of the barrel
    assert np.all(np.abs(b.xyz[:, 2]) <= zhalf[b.layer] + 5 * cfg["events"]["smear_z"])
    assert b.layer.min() >= 0 and b.layer.max() < len(radius)


def test_noise_share_and_shuffle():
    cfg = ev.load_workload("barrel10_500trk")
    b = ev.make_batch(cfg)
    n_noise = int((b.track < 0).sum())
    n_true = b.n_hits - n_noise
    assert n_noise == int(round(cfg["events"]["noise_fraction"] * n_true))
    # hits are shuffled within the event: neither layers nor tracks come in runs
    assert np.count_nonzero(np.diff(b.layer) != 0) > b.n_hits // 2
    assert np.count_nonzero(np.diff(b.track) != 0) > b.n_hits // 2


def test_truth_ranges_barrel10():
    cfg = ev.load_workload("barrel10_500trk")
    e = cfg["events"]
    b = ev.make_batch(cfg)
    t = b.truth
    assert len(t) == e["n_tracks"]
    pt = 1.0 / np.abs(t[:, 1])
    assert pt.min() >= e["pt_range"][0] * (1 - 1e-9) and pt.max() <= e["pt_range"][1] * (1 + 1e-9)
    eta = np.arcsinh(t[:, 3])
    assert eta.min() >= e["eta_range"][0] - 1e-9 and eta.max() <= e["eta_range"][1] + 1e-9
    assert np.all((t[:, 0] >= -math.pi) & (t[:, 0] < math.pi))
    # long-lived daughters: about the stated fraction have a sizeable impact parameter;
    # prompt tracks have d0 = 0 up to rounding
    frac = e["displaced"]["fraction"]
    displaced = np.abs(t[:, 2]) > 1e-6
    assert abs(displaced.mean() - frac) < 4 * math.sqrt(frac * (1 - frac) / len(t)) + 0.01
    # z0 of prompt tracks ~ N(0, sigma)
    z0 = t[~displaced, 4]
    assert abs(z0.std() - e["z0_sigma"]) < 0.15 * e["z0_sigma"]


def test_batch_multiplicities():
    cfg = ev.load_workload("barrel10_batch256")
    nt = cfg["events"]["n_tracks"]
    counts = ev.track_counts(cfg, np.random.default_rng(cfg["seed"]), cfg["events"]["n_events"])
    assert counts.min() >= nt["clip"][0] and counts.max() <= nt["clip"][1]
    assert abs(counts.mean() - nt["poisson_mean"]) < 4 * math.sqrt(nt["poisson_mean"] / len(counts))


def test_seeded_and_deterministic():
    cfg = ev.load_workload("barrel4_20trk")
    a, b = ev.make_batch(cfg), ev.make_batch(cfg)
    assert np.array_equal(a.xyz, b.xyz) and np.array_equal(a.layer, b.layer)
    assert np.array_equal(a.truth, b.truth)
    c = ev.make_batch(cfg, seed=cfg["seed"] + 1)
    assert not np.array_equal(a.xyz, c.xyz)
