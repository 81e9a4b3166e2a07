"""The model step's own sine and cosine of the attitude angles against double
precision and against the library's sincosf: at most 2 ulp from the correctly
rounded value within |x| <= 65536 (dense sweep, points near multiples of pi/2,
tiny arguments), the hardware approximation beyond and for non-finite x, and the
packed two-sample form bit-identical to the one-sample form."""
import math

import numpy as np
import pytest

from paper_2403_11383_b300 import sbs as S

pytestmark = pytest.mark.gpu


def _ulp_err(got, ref):
    """Error of float32 results in units of the float32 ulp of the reference."""
    ref32 = ref.astype(np.float32)
    ulp = np.spacing(np.abs(ref32)).astype(np.float64)
    return np.abs(got.astype(np.float64) - ref) / np.maximum(ulp, np.float64(np.spacing(np.float32(1e-30))))


def test_sincos_error_and_forms():
    import torch
    rng = np.random.default_rng(0)
    xs = [np.linspace(-65536.0, 65536.0, 2_000_003), rng.uniform(-4.0, 4.0, 500_000),
          np.ldexp(rng.uniform(0.5, 1.0, 20_000), rng.integers(-40, 0, 20_000)) * rng.choice([-1, 1], 20_000)]
    k = np.arange(-41000, 41001)
    near = (k * (math.pi / 2)).astype(np.float32)
    xs += [near, np.nextafter(near, np.float32(np.inf)), np.nextafter(near, np.float32(-np.inf))]
    x = np.concatenate([a.astype(np.float32) for a in xs])
    outs = [o.cpu().numpy() for o in S.sincos(torch.tensor(x, device="cuda"))]
    s, c, s2, c2, sl, cl, _, _ = outs
    np.testing.assert_array_equal(s, s2)
    np.testing.assert_array_equal(c, c2)
    xd = x.astype(np.float64)
    es, ec = _ulp_err(s, np.sin(xd)), _ulp_err(c, np.cos(xd))
    print(f"max ulp error: sin {es.max():.3f}, cos {ec.max():.3f}; library: sin {_ulp_err(sl, np.sin(xd)).max():.3f}, "
          f"cos {_ulp_err(cl, np.cos(xd)).max():.3f}")
    assert es.max() <= 2.0 and ec.max() <= 2.0


def test_sincos_beyond_range_and_nonfinite():
    import torch
    x = np.array([65536.01, -70000.0, 1e5, -3.3e7, 1e30, np.inf, -np.inf, np.nan], dtype=np.float32)
    s, c, s2, c2, _, _, sh, ch = [o.cpu().numpy() for o in S.sincos(torch.tensor(x, device="cuda"))]
    np.testing.assert_array_equal(s, sh)
    np.testing.assert_array_equal(c, ch)
    np.testing.assert_array_equal(s2, sh)
    np.testing.assert_array_equal(c2, ch)
