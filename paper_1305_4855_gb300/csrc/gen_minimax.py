"""Coefficients of the arcsine and arctangent polynomials in trk_common.cuh.

Both are near-minimax fits of the relative error, by Lawson's algorithm (C. L. Lawson,
"Contributions to the theory of linear least maximum approximation", 1961): weighted least
squares on Chebyshev nodes, each weight multiplied by the point's current absolute error
until the error levels out.  The fitted functions are even in x, so they are fitted in
t = x^2:

* asin(x) / x on x in [0, 0.75] (t in [0, 0.5625]), degree 8 in t;
* atan(x) / x on x in [0, 1] (t in [0, 1]), degree 8 in t.

The kernels evaluate x + x t (c1 + c2 t + ... + c8 t^7) (the fitted c0 is 1 within 2e-8).
Run this file to print the coefficients rounded to float32 and the worst error of that
evaluation in float32 with fused multiply-adds, measured against numpy's float64 functions
on 2,000,001 points.
"""
import numpy as np


def lawson(f, a, b, deg, n=6000, iters=300):
    k = np.arange(n)
    t = 0.5 * (a + b) + 0.5 * (b - a) * np.cos(np.pi * (k + 0.5) / n)
    y = f(t)
    w = np.ones(n) / n
    V = np.vander(t, deg + 1, increasing=True)
    for _ in range(iters):
        sw = np.sqrt(w) / np.abs(y)
        c, *_ = np.linalg.lstsq(V * sw[:, None], y * sw, rcond=None)
        e = (V @ c - y) / y
        w = w * np.abs(e)
        w /= w.sum()
    return c


def _even(g):
    return lambda t: np.where(t > 0, g(np.sqrt(t)) / np.sqrt(np.maximum(t, 1e-300)), 1.0)


def _fma32(a, b, c):
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def evaluate32(coef, x):
    """x + x t (c1 + c2 t + ...), every step rounded to float32 (fused multiply-adds)."""
    f32 = np.float32
    x = np.asarray(x, dtype=f32)
    t = (x * x).astype(f32)
    c = [f32(v) for v in coef[1:]]
    r = np.full_like(t, c[-1])
    for v in reversed(c[:-1]):
        r = _fma32(r, t, v)
    return _fma32((x * t).astype(f32), r, x)


ASIN = lawson(_even(np.arcsin), 0.0, 0.5625, 8)
ATAN = lawson(_even(np.arctan), 0.0, 1.0, 8)

if __name__ == "__main__":
    for name, coef, hi, g in (("asin", ASIN, 0.75, np.arcsin), ("atan", ATAN, 1.0, np.arctan)):
        x = np.linspace(0.0, hi, 2000001).astype(np.float32)
        ref = g(x.astype(np.float64))
        r = evaluate32(coef, x)
        ulp = np.abs(r - ref)[1:] / np.spacing(ref[1:].astype(np.float32)).astype(np.float64)
        print("%s: c0 = %.10f, worst error %.2f ulp" % (name, coef[0], ulp.max()))
        print("  " + ", ".join("%.9ef" % np.float32(v) for v in coef[1:]))
