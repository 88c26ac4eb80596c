"""The TF32 and BF16 sketch forms (TTR_PREC_TF32_SKETCH, TTR_PREC_BF16_SKETCH): reduced-precision
operands with FP32 accumulation in the W chain and the sketch only, everything else FP64-accurate.

Stated error, from the arithmetic: a product with operands rounded to u_low (2^-11 TF32, 2^-8 BF16
relative) and FP32 accumulation errs by about u_low sum |a||b|; along the right-to-left chain of d - 1
such products the partial contractions W_k err by a few u_low of max|W_k| (measured against the
FP64 oracle: TF32 2.7e-4..1.9e-3, BF16 2.1e-3..1.7e-2 on the 6-, 16- and 20-core workloads).  The
sketched subspace is then that of X plus a perturbation of about u_low kappa ||X|| (kappa the copy
coefficients' cancellation), which no later FP64 step removes: the rounding error is floored near
that level (measured 9e-4 and 9e-3 relative for TF32, 7e-3 and 7e-2 for BF16 on the 6- and 20-core
workloads), so these forms serve tolerances above it.  Bars here: the partial contractions within
12 u_low of max|W_k|; at tol 1e-1 (TF32) and 1e-1 / 2e-1 (BF16) the roundings meet the tolerance, keep the FP64 oracle's
ranks, and the represented tensor lies within tol / 2 of the oracle's."""
import numpy as np
import pytest

import workloads as WL
from oracle import rounding as R
from oracle import tt as T

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ULOW = {2: 2.0 ** -11, 3: 2.0 ** -8}        # TTR_PREC_TF32_SKETCH, TTR_PREC_BF16_SKETCH


@pytest.fixture(scope="module")
def B():
    from paper_2511_03598_gb300 import build
    build.build()
    from paper_2511_03598_gb300 import binding
    assert torch.cuda.is_available()
    return binding


def dev(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).to("cuda") for c in cores]


@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("name,make,w", [("c1", lambda: WL.c1().cores, 13), ("c3s", lambda: WL.c3(d=6, n=16, r=10).cores, 40),
                                         ("c2", lambda: WL.c2().cores, 70)])
def test_reduced_partial_contractions(B, prec, name, make, w):
    cores = make()
    ref = R.partial_contractions_rl(cores, 77, 0, w)
    got = B.partial_contractions(dev(cores), 77, 0, w, precision=prec)
    for k, Wk in ref.items():
        err = np.abs(got[k].cpu().numpy() - Wk).max() / np.abs(Wk).max()
        assert err <= 12 * ULOW[prec], (k, err)


@pytest.mark.parametrize("name,make,block,prec,tol", [("c1", lambda: WL.c1(), 2, 2, 1e-1), ("c1", lambda: WL.c1(), 2, 3, 1e-1),
                                                      ("c2", lambda: WL.c2(), 10, 2, 1e-1), ("c2", lambda: WL.c2(), 10, 3, 2e-1)])
def test_reduced_rounding_at_a_tolerance_above_its_floor(B, name, make, block, prec, tol):
    """Tolerances whose thresholds sit far above each form's floor and whose oracle estimates stay at
    least 25 % away from tau (the reduced sketch moves an estimate by about u_low kappa of it), so the
    rank decisions are the oracle's."""
    x = make()
    ref, info = R.tt_round_adaptive(x.cores, tol, seed=5, block=block, nrmx=x.norm)
    with B.round_adaptive(dev(x.cores), tol, block, 5, B.options(precision=prec, nrmx=x.norm)) as y:
        assert y.ranks == info["ranks"], (y.ranks, info["ranks"])
        got = y.to_numpy()
    assert T.tt_dist(got, x.cores) <= tol * x.norm
    assert T.tt_dist(got, ref) <= 0.5 * tol * T.tt_norm(ref)


@pytest.mark.parametrize("prec", [2, 3])
def test_reduced_rounding_operator_applied_vector_meets_tol(B, prec):
    """The small operator-applied vector (d = 6, n = 16, rank 20; the paper's fractions give b_inc = 1)
    with the estimator reading R16, at tol 1e-1: the tolerance is met (its spectrum decays steadily,
    so estimates sit near the threshold and the ranks may differ from the oracle's by a block)."""
    x = WL.c3(d=6, n=16, r=10)
    with B.round_adaptive(dev(x.cores), 1e-1, 0, 9, B.options(precision=prec, nrmx=x.norm, est_min=10,
                                                              est_safety=10.0)) as y:
        got = y.to_numpy()
    assert T.tt_dist(got, x.cores) <= 1e-1 * x.norm
