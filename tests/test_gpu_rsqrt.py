"""The block loop's reciprocal square root (a binary32 seed refined by one third-order
Newton-Householder step) against 1/sqrt(y) evaluated in extended precision: within 2 ulp of the
correctly rounded value over the whole exponent range, subnormals included.  The one-sided Jacobi
rotation built on it against the textbook formula."""
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


def _rotation_reference(A2, B2, G):
    """The textbook one-sided Jacobi rotation (Hestenes; Golub and Van Loan, Sec. 8.5) in extended
    precision: zeta = (B2 - A2) / (2 G), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
    cs = 1 / sqrt(1 + t^2), sn = cs t."""
    ld = np.longdouble
    A2, B2, G = A2.astype(ld), B2.astype(ld), G.astype(ld)
    zeta = (B2 - A2) / (ld(2) * G)
    t = np.where(zeta >= 0, ld(1), ld(-1)) / (np.abs(zeta) + np.sqrt(ld(1) + zeta * zeta))
    cs = ld(1) / np.sqrt(ld(1) + t * t)
    return cs.astype(np.float64), (cs * t).astype(np.float64)


def test_jacobi_rotation_against_the_textbook_formula(B):
    """The rotation the Jacobi SVD kernels use (square roots and reciprocals from the reciprocal
    square root above) against the textbook formula in extended precision: relative errors of cs
    within 8 eps and of sn within 24 eps (eps = 2^-52; a rounding model with every reciprocal square
    root 2 ulp off gives at most 3 and 11), cs^2 + sn^2 = 1 to 1e-15, across pair correlations from 1e-12 to
    nearly 1, norm ratios up to 1e200 (|zeta| beyond 2^500 included) and inputs whose products leave
    the normal range; exactly (1, 0) for G = 0, for pairs already orthogonal to 1e-15 and for pairs
    below `tiny`."""
    if np.finfo(np.longdouble).nmant <= 52:
        pytest.skip("no extended-precision long double on this host")
    rng = np.random.default_rng(7)
    n = 100_000
    A2 = np.exp(rng.uniform(-60, 60, n))
    B2 = A2 * np.exp(rng.uniform(-30, 30, n))
    rho = np.sign(rng.standard_normal(n)) * np.exp(rng.uniform(np.log(1e-12), np.log(0.999999), n))
    G = rho * np.sqrt(A2) * np.sqrt(B2)
    # |zeta| beyond 2^500 (norm ratios up to 1e400, correlations above the 1e-15 cut)
    big = np.array([[1e200, 1e-200, 1e-14], [1e-200, 1e200, -1e-14], [3e180, 2e-150, 5e10]])
    # products below or above the normal range (library square root and division)
    edge = np.array([[1e-200, 2e-200, 1e-200], [1e200, 3e200, -1.5e200], [1e-160, 1e-160, 5e-161],
                     [1e170, 4e170, 1.5e170]])
    abg = np.concatenate([np.stack([A2, B2, G], axis=1), big, edge])
    got = B.selftest_jacobi_rotation(torch.from_numpy(abg).cuda()).cpu().numpy()
    cs_ref, sn_ref = _rotation_reference(abg[:, 0], abg[:, 1], abg[:, 2])
    cs, sn = got[:, 0], got[:, 1]
    eps = np.finfo(np.float64).eps
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(cs - cs_ref) / cs_ref) <= 8 * eps
    assert np.max(np.abs(sn - sn_ref) / np.abs(sn_ref)) <= 24 * eps
    assert np.max(np.abs(cs * cs + sn * sn - 1.0)) <= 1e-15
    # no rotation: G = 0, pairs orthogonal to below 1e-15 of sqrt(A2 B2), pairs below tiny
    none = np.array([[1.0, 2.0, 0.0], [4.0, 9.0, 1e-16], [1e-30, 1e-31, 1e-31], [1e300, 1e-300, 0.0]])
    got = B.selftest_jacobi_rotation(torch.from_numpy(none).cuda(), tiny=1e-20).cpu().numpy()
    assert np.array_equal(got, np.tile([1.0, 0.0], (len(none), 1)))
