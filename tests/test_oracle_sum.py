"""Pins for the oracle's rounding of a sum of TTs (Remark 3.3, Appendix D), each against
something other than the sum code itself.

* Stacked per-summand partial contractions equal Algorithm 3 on the explicit block-diagonal
  formal sum (the identity the method rests on: the sketch of a sum is the sum of sketches).
* In block mode the whole rounding equals the oracle's Algorithm 6 on the formal sum, built by
  ``oracle.tt.tt_sum`` (a separate, plain construction): same ranks, estimates, tau and
  represented tensor.  A wrong block offset, a transposed M block or a missing sum at the last
  core breaks this.
* The relative error against the dense sum of the summands' full tensors is <= tol.
* Block sizes in fraction mode follow the appendix (b_init = max summand rank).
* Planted mistakes (summand blocks stacked in the wrong order, a summand's projected block
  attached to the wrong directions of Q, the last core taken from one summand instead of summed)
  must fail the identity pin.
"""
import math

import numpy as np
import pytest

import workloads as WL
from oracle import rounding as R
from oracle import tt as T


def summands_of(seed, d, n, ranks, coef=None):
    rng = np.random.default_rng(seed)
    xs = [WL.random_tt(rng, d, n, r) for r in ranks]
    if coef is not None:
        for x, c in zip(xs, coef):
            x[0] = x[0] * c
    return xs


def formal_sum(xs):
    out = xs[0]
    for x in xs[1:]:
        out = T.tt_sum(out, x)
    return out


def dense(xs):
    return sum(T.full(x) for x in xs)


def low_rank_sum(seed, d=5, n=4, r=3, copies=3, noise_rank=2, eta=1e-6):
    """copies scaled copies of one rank-r TT plus a small rank-noise_rank TT: numerical rank ~r."""
    rng = np.random.default_rng(seed)
    base = WL.random_tt(rng, d, n, r)
    xs = []
    for c in rng.standard_normal(copies) + 0.5:
        x = [b.copy() for b in base]
        x[0] = x[0] * c
        xs.append(x)
    noise = WL.random_tt(rng, d, n, noise_rank)
    noise[0] = noise[0] * (eta * T.tt_norm(formal_sum(xs)) / T.tt_norm(noise))
    return xs + [noise]


@pytest.mark.parametrize("d,n,ranks", [(4, 3, [2, 3]), (5, 2, [1, 2, 2]), (4, [2, 3, 4, 2], [[2, 3, 1], [1, 2, 2]])])
def test_stacked_partial_contractions_equal_formal_sum(d, n, ranks):
    xs = summands_of(30 + d, d, n, ranks)
    seed = 99
    Ws = R.partial_contractions_rl_sum(xs, seed, 0, 7)
    Wf = R.partial_contractions_rl(formal_sum(xs), seed, 0, 7)
    assert set(Ws) == set(Wf)
    for k in Wf:
        np.testing.assert_allclose(Ws[k], Wf[k], rtol=0, atol=1e-14 * max(1.0, np.abs(Wf[k]).max()))


@pytest.mark.parametrize("case", [
    dict(d=5, n=4, ranks=[3, 2, 4], block=2, tol=1e-2),
    dict(d=4, n=5, ranks=[2, 2], block=1, tol=1e-3),
    dict(d=6, n=3, ranks=[2, 3, 1, 2], block=3, tol=1e-1),
    dict(d=5, n=4, ranks=[3, 2, 4], block=2, tol=1e-3, est_min=5, est_safety=4.0),   # reading R16
])
@pytest.mark.parametrize("given_norm", [False, True])
def test_block_mode_equals_adaptive_on_formal_sum(case, given_norm):
    xs = summands_of(7, case["d"], case["n"], case["ranks"], coef=[1.0, -0.7, 0.4, 1.3][:len(case["ranks"])])
    xf = formal_sum(xs)
    nrmx = T.tt_norm(xf) if given_norm else None
    est = dict(est_min=case.get("est_min", 0), est_safety=case.get("est_safety", 1.0))
    Ys, infs = R.tt_round_adaptive_sum(xs, case["tol"], 5, block=case["block"], nrmx=nrmx, **est)
    Yf, inff = R.tt_round_adaptive(xf, case["tol"], 5, block=case["block"], nrmx=nrmx, **est)
    assert infs["ranks"] == inff["ranks"]
    assert infs["formal_ranks"] == T.ranks(xf)
    assert math.isclose(infs["tau"], inff["tau"], rel_tol=1e-12)
    for es, ef in zip(infs["estimates"], inff["estimates"]):
        np.testing.assert_allclose(es, ef, rtol=1e-9, atol=1e-14 * inff["nrmx"])
    assert T.tt_dist(Ys, Yf) <= 1e-11 * T.tt_norm(Yf)


def test_single_summand_is_algorithm_6():
    xs = summands_of(3, 5, 4, [3])
    Ys, infs = R.tt_round_adaptive_sum(xs, 1e-2, 11, block=2)
    Yf, inff = R.tt_round_adaptive(xs[0], 1e-2, 11, block=2)
    assert infs["ranks"] == inff["ranks"]
    assert T.tt_dist(Ys, Yf) <= 1e-13 * T.tt_norm(Yf)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("block", [1, 0])
def test_error_against_dense_sum(seed, block):
    xs = low_rank_sum(seed)
    X = dense(xs)
    tol = 1e-3
    Y, info = R.tt_round_adaptive_sum(xs, tol, 100 + seed, block=block, nrmx=float(np.linalg.norm(X)))
    err = np.linalg.norm(T.full(Y) - X) / np.linalg.norm(X)
    assert err <= tol
    # numerical rank 3 (+ noise far below tol): the adaptive ranks cover it, no more than the formal ones
    assert all(3 <= r <= fr for r, fr in zip(info["ranks"][1:-1], info["formal_ranks"][1:-1]))
    assert T.left_orth_defect(Y) <= 1e-12


def test_fraction_mode_block_sizes_follow_appendix():
    xs = summands_of(5, 5, 4, [[2, 3, 2, 4], [3, 1, 2, 2]])
    Y, info = R.tt_round_adaptive_sum(xs, 1e-1, 3, block=0, f_inc=0.2)
    n = T.modes(xs[0])
    rprev = 1
    for k in range(1, 5):
        rbar = min(rprev * n[k - 1], info["formal_ranks"][k])
        assert info["b_init"][k - 1] == min(rbar, max(T.ranks(x)[k] for x in xs))
        rprev = info["ranks"][k]
    assert info["w0"] == 4


def test_summands_must_share_modes():
    a = summands_of(1, 4, 3, [2])[0]
    b = summands_of(2, 4, 4, [2])[0]
    with pytest.raises(ValueError):
        R.tt_round_adaptive_sum([a, b], 1e-2, 1, block=1)


def test_planted_stacking_mistake_is_caught(monkeypatch):
    xs = summands_of(7, 5, 4, [3, 2, 4], coef=[1.0, -0.7, 0.4])
    xf = formal_sum(xs)
    nrmx = T.tt_norm(xf)
    Yf, _ = R.tt_round_adaptive(xf, 1e-2, 5, block=2, nrmx=nrmx)
    good = R.partial_contractions_rl_sum

    def reversed_stack(summands, seed, col0, col1, t=2):
        return good(list(reversed(summands)), seed, col0, col1, t)

    monkeypatch.setattr(R, "partial_contractions_rl_sum", reversed_stack)
    Yb, _ = R.tt_round_adaptive_sum(xs, 1e-2, 5, block=2, nrmx=nrmx)
    assert T.tt_dist(Yb, Yf) > 1e-6 * T.tt_norm(Yf)


def test_workload_summands_form_the_same_sum():
    x = WL.c1()
    f = formal_sum(x.summands)
    assert T.ranks(f) == x.ranks
    for a, b in zip(f, x.cores):
        np.testing.assert_array_equal(a, b)


def test_c1_sum_equals_formal_sum_rounding():
    x = WL.c1()
    Ys, infs = R.tt_round_adaptive_sum(x.summands, 1e-6, 2024, block=2, nrmx=x.norm)
    Yf, inff = R.tt_round_adaptive(x.cores, 1e-6, 2024, block=2, nrmx=x.norm)
    assert infs["ranks"] == inff["ranks"]
    assert T.tt_dist(Ys, Yf) <= 1e-11 * x.norm


def _identity_gap(xs, nrmx, Yf):
    Yb, _ = R.tt_round_adaptive_sum(xs, 1e-2, 5, block=2, nrmx=nrmx)
    return T.tt_dist(Yb, Yf) / T.tt_norm(Yf)


def test_planted_projection_and_last_core_mistakes_are_caught(monkeypatch):
    xs = summands_of(7, 5, 4, [3, 2, 4], coef=[1.0, -0.7, 0.4])
    xf = formal_sum(xs)
    nrmx = T.tt_norm(xf)
    Yf, _ = R.tt_round_adaptive(xf, 1e-2, 5, block=2, nrmx=nrmx)
    assert _identity_gap(xs, nrmx, Yf) <= 1e-11
    good_project, good_next = R.project_summands, R.next_core_of_sum
    with monkeypatch.context() as m:
        # each summand's projected rows in reverse order: attached to the wrong directions of Q
        m.setattr(R, "project_summands",
                  lambda Mq, summands, off, k: [b[::-1] if b.shape[0] > 1 else b for b in good_project(Mq, summands, off, k)])
        assert _identity_gap(xs, nrmx, Yf) > 1e-6
    with monkeypatch.context() as m:
        m.setattr(R, "next_core_of_sum",
                  lambda parts, lk, n_next, rr, last: good_next(parts[:1] if last else parts, lk, n_next, rr, last))
        assert _identity_gap(xs, nrmx, Yf) > 1e-6


def test_first_block_wider_than_the_last_unfolding():
    """Reading R14: with the appendix's b_init = max_i r_k^(i) = 6 and n_d = 4, the last core's
    unfolding has rank at most 4; rbar_k is clamped to it, so no sketch block is wider than the
    rank it can have, and the result is still within tol of the dense sum."""
    xs = summands_of(13, 5, 4, [6, 5], coef=[1.0, 0.8])
    X = dense(xs)
    Y, info = R.tt_round_adaptive_sum(xs, 1e-10, 3, block=0, nrmx=float(np.linalg.norm(X)))
    assert info["ranks"][4] <= 4 and info["b_init"][3] <= 4
    assert np.linalg.norm(T.full(Y) - X) <= 1e-10 * np.linalg.norm(X)


def test_zero_tensor_rounds_to_the_zero_tt():
    """Reading R15: ||X|| = 0 (estimated here) gives the zero TT of ranks 1, for one TT and a sum."""
    x = [np.zeros_like(c) for c in WL.random_tt(np.random.default_rng(1), 4, 5, 3)]
    for Y, info in (R.tt_round_adaptive(x, 1e-6, 3, block=2), R.tt_round_adaptive_sum([x, x], 1e-6, 3, block=0)):
        assert info["ranks"] == [1, 1, 1, 1, 1] and info["nrmx"] == 0.0
        assert T.tt_norm(Y) == 0.0 and T.modes(Y) == T.modes(x)


def test_two_cores():
    """d = 2: no partial-contraction step, one sketched core; the sum equals the formal-sum rounding."""
    xs = summands_of(17, 2, [9, 7], [3, 4], coef=[1.0, 0.5])
    xf = formal_sum(xs)
    Ys, infs = R.tt_round_adaptive_sum(xs, 1e-12, 2, block=2)
    Yf, inff = R.tt_round_adaptive(xf, 1e-12, 2, block=2)
    assert infs["ranks"] == inff["ranks"] == [1, 7, 1]
    assert T.tt_dist(Ys, xf) <= 1e-12 * T.tt_norm(xf)


def test_serving_stream_summands_form_its_sums():
    """The serving stream's requests as summands reproduce their formal sums (small requests)."""
    for q in WL.c4_stream(count=200, max_bytes=40e6):
        f = formal_sum(q.tt.summands)
        assert T.ranks(f) == T.ranks(q.tt.cores)
        for a, b in zip(f, q.tt.cores):
            np.testing.assert_array_equal(a, b)
        assert len(q.tt.summands) == q.tt.meta["s"]
        break
    else:
        pytest.skip("no small request in the first 200")
