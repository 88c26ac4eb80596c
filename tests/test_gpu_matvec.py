"""GPU parity of the rounding of an operator-applied TT vector y = A x without forming y (the
operator application of TT-GMRES, Sec. 4.3): the fused right-to-left partial contractions against
the oracle's Algorithm 3 on the formed product (1e-12 of max|W_k| in FP64, the sliced form's stated
bar at 8 slices), and the whole rounding against the oracle's Algorithm 6 on y formed by its
definition (identical ranks, represented tensors within 1e-10 in FP64, the tolerance met)."""
import numpy as np
import pytest

import workloads as WL
from oracle import rounding as R
from oracle import tt as T

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_2511_03598_gb300 import build
    build.build()
    from paper_2511_03598_gb300 import binding
    assert torch.cuda.is_available()
    return binding


def dev(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).to("cuda") for c in cores]


def c3_parts(d=16, n=64, r=30, seed=3):
    """The operator-applied workload's factors: the Laplacian TT operator and the vector x."""
    return WL.c3_factors(seed, d, n, r)


def random_op(rng, d, n, m, p):
    pk = [1] + [p] * (d - 1) + [1]
    return [rng.standard_normal((pk[k], n[k], m[k], pk[k + 1])) / np.sqrt(m[k] * p) for k in range(d)]


CASES = [("c3_small", lambda: c3_parts(d=6, n=16, r=10), 0, 40),
         ("rect", lambda: (lambda rng: (random_op(rng, 5, [4, 3, 5, 2, 3], [3, 4, 2, 5, 2], 3),
                                        WL.random_tt(rng, 5, [3, 4, 2, 5, 2], 4)))(np.random.default_rng(6)), 3, 30),
         ("c3", lambda: c3_parts(), 0, 70)]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,make,c0,c1", CASES)
def test_fused_partial_contractions(B, prec, name, make, c0, c1):
    op, x = make()
    y = T.tt_matvec(op, x)
    ref = R.partial_contractions_rl(y, 21, c0, c1)
    got = B.partial_contractions_matvec(dev(op), dev(x), 21, c0, c1, precision=prec, slices=8)
    for k, Wk in ref.items():
        g = got[k].cpu().numpy()
        assert g.shape == Wk.shape
        assert np.abs(g - Wk).max() <= 1e-12 * np.abs(Wk).max(), (k, np.abs(g - Wk).max() / np.abs(Wk).max())


@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_matvec_c3_full_size(B, prec):
    """The operator-applied workload (d = 16, n = 64, rank-2 Laplacian operator, rank-30 x; y of
    formal rank 60) at tol 1e-8 with the estimator reading R16, as the formed-y test of the same
    configuration; in sliced form at the slice count chosen for 1e-8 the bar is that form's 1e-9."""
    op, x = c3_parts()
    y = T.tt_matvec(op, x)
    nrm = T.tt_norm(y)
    ref, info = R.tt_round_adaptive_matvec(op, x, 1e-8, seed=3, nrmx=nrm, est_min=10, est_safety=10.0)
    with B.round_adaptive_matvec(dev(op), dev(x), 1e-8, 0, 3,
                                 B.options(precision=prec, nrmx=nrm, est_min=10, est_safety=10.0)) as yr:
        assert yr.ranks == info["ranks"]
        got = yr.to_numpy()
    assert T.tt_dist(got, ref) <= (1e-10 if prec == 0 else 1e-9) * T.tt_norm(ref)
    assert T.tt_dist(got, y) <= 1e-8 * nrm


@pytest.mark.parametrize("name,make,tol,block", [("c3_small", lambda: c3_parts(d=6, n=16, r=10), 1e-8, 0),
                                                 ("rect", lambda: (lambda rng: (random_op(rng, 5, [4, 3, 5, 2, 3], [3, 4, 2, 5, 2], 3),
                                                                                WL.random_tt(rng, 5, [3, 4, 2, 5, 2], 4)))(np.random.default_rng(6)), 1e-6, 2)])
def test_adaptive_matvec_parity(B, name, make, tol, block):
    op, x = make()
    y = T.tt_matvec(op, x)
    nrm = T.tt_norm(y)
    ref, info = R.tt_round_adaptive_matvec(op, x, tol, seed=9, block=block)       # norm estimated (Eq. (3.6))
    with B.round_adaptive_matvec(dev(op), dev(x), tol, block, 9) as yr:
        assert yr.ranks == info["ranks"]
        assert abs(yr.info["nrmx"] - info["nrmx"]) <= 1e-12 * info["nrmx"]
        got = yr.to_numpy()
    assert T.tt_dist(got, ref) <= 1e-10 * T.tt_norm(ref)
    assert nrm > 0


def test_adaptive_matvec_rejects_bad_shapes(B):
    op, x = c3_parts(d=4, n=8, r=3)
    with pytest.raises(ValueError):
        B.round_adaptive_matvec(dev(op[:3]), dev(x), 1e-6, 2, 1)
    bad = [torch.zeros((1, 8, 7, 2), dtype=torch.float64, device="cuda")] + dev(op[1:])
    with pytest.raises(ValueError):                     # input size 7 against x's mode size 8
        B.round_adaptive_matvec(bad, dev(x), 1e-6, 2, 1)
    with pytest.raises(B.TTRoundError):                 # outer operator rank 2 (checked by the library)
        B.round_adaptive_matvec([torch.zeros((2, 8, 8, 2), dtype=torch.float64, device="cuda")] + dev(op[1:]),
                                dev(x), 1e-6, 2, 1)
