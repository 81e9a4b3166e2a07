"""Derive the constants of the rollout's sine and cosine (sbs_device.cuh, sincos_v).

    python -m paper_2403_11383_b300.sincos_coefficients

Method: Cody-Waite argument reduction (W. J. Cody and W. Waite, Software Manual
for the Elementary Functions, 1980): x = j pi/2 + r with j = rint(2 x / pi) and
|r| <= pi/4, pi/2 split into three single-precision parts P1 + P2 + P3 (each the
single-precision rounding of what the previous parts leave), subtracted from x
one fused multiply-add at a time.  On the reduced range,

    sin r = r + r^3 (s1 + s2 r^2 + s3 r^4)
    cos r = 1 + r^2 (c1 + c2 r^2 + c3 r^4 + c4 r^6)

with coefficients fitted here by least squares in double precision on Chebyshev
nodes of u = r^2 in (0, (pi/4)^2] (the remainders (sin r - r) / r^3 and
(cos r - 1) / r^2 as polynomials in u), then rounded to single precision.  The
fit's error is checked against math.sin / math.cos on a dense grid.
"""
import math

import numpy as np

SIN_DEGREE = 2   # s1..s3: a polynomial of degree 2 in u = r^2
COS_DEGREE = 3   # c1..c4


def f32(v):
    return float(np.float32(v))


def pio2_parts():
    """pi/2 = P1 + P2 + P3 + (a remainder below 2^-73), each part the
    single-precision rounding of what the previous ones leave (50-digit pi)."""
    import mpmath
    mpmath.mp.dps = 50
    rest = mpmath.pi / 2
    parts = []
    for _ in range(3):
        p = f32(float(rest))
        parts.append(p)
        rest = rest - mpmath.mpf(p)
    return tuple(parts)


def _fit(g, degree, nodes=400):
    umax = (math.pi / 4) ** 2
    k = np.arange(nodes)
    u = 0.5 * umax * (1.0 - np.cos(math.pi * (k + 0.5) / nodes))  # Chebyshev nodes on (0, umax)
    A = np.vander(u, degree + 1, increasing=True)
    coef, *_ = np.linalg.lstsq(A, g(u), rcond=None)
    return [f32(c) for c in coef]


def coefficients():
    sin_c = _fit(lambda u: (np.sin(np.sqrt(u)) - np.sqrt(u)) / u ** 1.5, SIN_DEGREE)
    cos_c = _fit(lambda u: (np.cos(np.sqrt(u)) - 1.0) / u, COS_DEGREE)
    return {"two_over_pi": f32(2.0 / math.pi), "pio2": pio2_parts(), "sin": sin_c, "cos": cos_c}


def max_error(c, n=200001):
    """Largest relative error of the two polynomials (double-precision evaluation
    of the single-precision coefficients) on [-pi/4, pi/4]."""
    r = np.linspace(-math.pi / 4, math.pi / 4, n)
    r = r[r != 0.0]
    u = r * r
    s1, s2, s3 = c["sin"]
    c1, c2, c3, c4 = c["cos"]
    sp = r + r * u * (s1 + u * (s2 + u * s3))
    cp = 1.0 + u * (c1 + u * (c2 + u * (c3 + u * c4)))
    return float(np.max(np.abs(sp - np.sin(r)) / np.abs(np.sin(r)))), float(np.max(np.abs(cp - np.cos(r))))


if __name__ == "__main__":
    c = coefficients()
    for k, v in c.items():
        print(k, [float(x).hex() for x in (v if isinstance(v, (list, tuple)) else [v])], v)
    print("max relative error sin, max error cos:", max_error(c))
