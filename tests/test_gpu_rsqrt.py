"""The block loop's reciprocal square root (a binary32 seed refined by one third-order
Newton-Householder step) against 1/sqrt(y) evaluated in extended precision: within 2 ulp of the
correctly rounded value over the whole exponent range, subnormals included."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_2511_03598_gb300 import build
    build.build()
    from paper_2511_03598_gb300 import binding
    assert torch.cuda.is_available()
    return binding


def test_rsqrt_within_two_ulp(B):
    rng = np.random.default_rng(12)
    mant = rng.uniform(1.0, 2.0, 200_000)
    expo = rng.integers(-1070, 1020, 200_000)
    y = np.ldexp(mant, expo)                                   # includes subnormals (exponent < -1022)
    y = np.concatenate([y, [1.0, 2.0, 4.0, 0.25, 3.0, np.nextafter(4.0, 0.0), 5e-324, 1.7976931348623157e308]])
    y = y[(y > 0) & np.isfinite(y)]
    got = B.selftest_rsqrt(torch.from_numpy(y).cuda()).cpu().numpy()
    ld = np.longdouble
    if np.finfo(ld).nmant <= 52:
        pytest.skip("no extended-precision long double on this host")
    ref = (ld(1) / np.sqrt(y.astype(ld))).astype(np.float64)   # correctly rounded to ~1/2 ulp
    ulp = np.spacing(np.abs(ref))
    err = np.abs(got - ref) / ulp
    assert np.all(np.isfinite(got))
    assert err.max() <= 2.0, (err.max(), y[np.argmax(err)])
