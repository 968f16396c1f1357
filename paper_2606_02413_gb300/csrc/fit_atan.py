"""Fits the odd polynomial used for arctan in the field evaluation.

atan(a) ~ a * P(a^2) on [0, 1], P of degree 7 in a^2: a weighted least-squares
fit on Chebyshev nodes followed by a few Lawson iterations (iteratively
re-weighted least squares, which converges toward the minimax fit).  Prints
the coefficients (highest power first) and the maximum absolute error in
double precision; the kernel evaluates the same polynomial in FP32 by
Horner's rule.  Arguments outside [0, 1] are reduced with
atan(a) = pi/2 - atan(1/a) and the quadrant of (x, y).
"""
import numpy as np


def fit(deg=7, n=4000, iters=60):
    k = np.arange(n)
    a = 0.5 + 0.5 * np.cos(np.pi * (k + 0.5) / n)  # Chebyshev nodes on [0, 1]
    s = a * a
    A = np.stack([a * s ** j for j in range(deg + 1)], 1)
    y = np.arctan(a)
    w = np.ones(n)
    for _ in range(iters):
        c, *_ = np.linalg.lstsq(A * np.sqrt(w)[:, None], y * np.sqrt(w), rcond=None)
        e = np.abs(A @ c - y)
        w *= e / e.max() + 1e-3
        w /= w.sum()
    aa = np.linspace(0, 1, 200001)
    err = np.abs(np.stack([aa * (aa * aa) ** j for j in range(deg + 1)], 1) @ c - np.arctan(aa)).max()
    return c[::-1], err


if __name__ == "__main__":
    c, err = fit()
    print("coefficients (a^14 ... a^0 of P):", ", ".join(f"{v:.9e}f" for v in c))
    print("max |error| =", err)
