"""The arcsine and arctangent polynomials of the FP32 fit (CPU only).

The coefficients written in trk_common.cuh must be the ones gen_minimax.py computes (Lawson's
near-minimax fit), rounded to float32, and their float32 evaluation (fused multiply-adds,
the kernels' order) must stay within the stated error of numpy's float64 functions.  The
atan2 octant logic is checked against numpy on points of every octant and the axes.
"""
import importlib.util
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1305_4855_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_minimax", os.path.join(CSRC, "gen_minimax.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _header_coeffs(fn):
    src = open(os.path.join(CSRC, "trk_common.cuh")).read()
    body = src[src.index(fn):]
    body = body[:body.index("\n}\n")]
    vals = [float(v) for v in re.findall(r"(-?\d\.\d+e[-+]\d+)f", body)]
    return vals


def test_header_coefficients_match_generator():
    g = _gen()
    for fn, coef in (("V asin_poly(V x)", g.ASIN), ("float atan_poly(float x)", g.ATAN)):
        got = _header_coeffs(fn)
        # Horner order in the source: highest degree first
        want = [float(np.float32(c)) for c in coef[1:]][::-1]
        assert len(got) == len(want) == 8
        assert np.array_equal(np.float32(got), np.float32(want)), (fn, got, want)
        assert abs(coef[0] - 1.0) < 3e-8          # the evaluation assumes c0 = 1


def _ulp_err(r, ref):
    return np.abs(r.astype(np.float64) - ref) / np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)


def test_float32_error_bounds():
    g = _gen()
    x = np.linspace(0.0, 0.75, 300001).astype(np.float32)[1:]
    assert _ulp_err(g.evaluate32(g.ASIN, x), np.arcsin(x.astype(np.float64))).max() < 1.0
    x = np.linspace(0.0, 1.0, 300001).astype(np.float32)[1:]
    assert _ulp_err(g.evaluate32(g.ATAN, x), np.arctan(x.astype(np.float64))).max() < 1.5
    # the known expansions: asin x = x + x^3/6 + ..., atan x = x - x^3/3 + ...
    assert abs(g.ASIN[1] - 1 / 6) < 1e-5 and abs(g.ATAN[1] + 1 / 3) < 1e-5


def _atan2_emulated(g, y, x):
    """The octant logic of atan2_poly, in float32 (reciprocal correctly rounded here; the
    device's approximate reciprocal adds at most 1 ulp to the ratio)."""
    f32 = np.float32
    y = np.asarray(y, f32)
    x = np.asarray(x, f32)
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    a = g.evaluate32(g.ATAN, (mn * (f32(1) / np.maximum(mx, f32(1e-30)))).astype(f32))
    r = np.where(ay > ax, (f32(1.57079637) - a) + f32(-4.37113883e-08), a).astype(f32)
    r = np.where(x < 0, (f32(3.14159274) - r) + f32(-8.74227766e-08), r).astype(f32)
    return np.copysign(r, y)


def test_atan2_octants():
    g = _gen()
    rng = np.random.default_rng(4)
    th = rng.uniform(-np.pi, np.pi, 200000)
    rad = 10.0 ** rng.uniform(-3, 4, th.size)
    x = (rad * np.cos(th)).astype(np.float32)
    y = (rad * np.sin(th)).astype(np.float32)
    got = _atan2_emulated(g, y, x)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    assert np.abs(got - ref).max() < 4e-7
    axes_y = np.float32([0, 1, 0, -1, 0, 1, -1, 1, -1])
    axes_x = np.float32([1, 0, -1, 0, 0, 1, 1, -1, -1])
    assert np.abs(_atan2_emulated(g, axes_y, axes_x) - np.arctan2(axes_y, axes_x)).max() < 4e-7
