"""The constants of the model step's sine and cosine (sbs_device.cuh, sincos_v)
are those paper_2403_11383_b300/sincos_coefficients.py derives, and the fitted
polynomials meet their error bound on the reduced range."""
import os
import re

import numpy as np

from paper_2403_11383_b300 import sincos_coefficients as SC

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _hexf(v):
    return float(v).hex().replace("0x", "").rstrip("0").rstrip(".")


def test_header_constants_match_derivation():
    src = open(os.path.join(ROOT, "paper_2403_11383_b300", "csrc", "sbs_device.cuh")).read()
    body = src[src.index("__device__ __forceinline__ void sincos_v"):]
    body = body[:body.index("#pragma unroll")]
    got = [float.fromhex(h[:-1]) for h in re.findall(r"-?0x[0-9a-f.]+p[-+]?\d+f", body)]
    c = SC.coefficients()
    p1, p2, p3 = c["pio2"]
    s1, s2, s3 = c["sin"]
    c1, c2, c3, c4 = c["cos"]
    want = [c["two_over_pi"], -p1, -p2, -p3, s3, s2, s1, c4, c3, c2]
    assert got == want, (got, want)
    assert c1 == -0.5  # written as -0.5f
    # every constant is a single-precision value
    assert all(np.float32(v) == v for v in want)


def test_fit_error_bound():
    es, ec = SC.max_error(SC.coefficients())
    assert es < 2e-8 and ec < 1e-9, (es, ec)


def test_pio2_split():
    import mpmath
    mpmath.mp.dps = 50
    p1, p2, p3 = SC.pio2_parts()
    assert abs(mpmath.pi / 2 - (mpmath.mpf(p1) + p2 + p3)) < mpmath.mpf(2) ** -72
