"""GPU parity of the rounding of a sum of TTs (tt_round_adaptive_sum, Remark 3.3 / Appendix D)
against the oracle's sum algorithm on the same seeded inputs.

Bars as for the single-TT adaptive rounding: FP64 form identical ranks, represented tensors within
1e-10 relative, estimates within 1e-8 relative; sliced form identical ranks and the stated
contraction-error bounds of the full-size test in test_gpu_parity.py.  Summands that share core
arrays on the host share device buffers too, as a caller holding scaled copies would pass them.
"""
import math

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


def dev_summands(summands):
    cache = {}
    out = []
    for x in summands:
        cs = []
        for c in x:
            if id(c) not in cache:
                cache[id(c)] = torch.from_numpy(np.ascontiguousarray(c)).to("cuda")
            cs.append(cache[id(c)])
        out.append(cs)
    return out


def rel(a, b):
    return T.tt_dist(a, b) / max(T.tt_norm(b), 1e-300)


def mixed_summands(seed):
    rng = np.random.default_rng(seed)
    n = [3, 4, 5, 4, 3]
    xs = [WL.random_tt(rng, 5, n, r) for r in ([2, 3, 4, 2], [1, 2, 2, 3], [3, 3, 1, 2])]
    for x, c in zip(xs, (1.0, -0.6, 0.3)):
        x[0] = x[0] * c
    return xs


@pytest.mark.parametrize("block", [2, 0])
def test_sum_c1_fp64(B, block):
    x = WL.c1()
    ref, info = R.tt_round_adaptive_sum(x.summands, 1e-6, 2024, block=block, nrmx=x.norm)
    with B.round_adaptive_sum(dev_summands(x.summands), 1e-6, block, 2024, B.options(nrmx=x.norm)) as y:
        yi = y.info
        got = y.to_numpy()
    assert yi["ranks"] == info["ranks"]
    flat = [e for es in info["estimates"] for e in es]
    np.testing.assert_allclose(yi["estimates"], flat, rtol=1e-8, atol=1e-14 * x.norm)
    assert rel(got, ref) <= 1e-10


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("given_norm", [True, False])
def test_sum_mixed_ranks(B, prec, given_norm):
    xs = mixed_summands(8)
    nrmx = T.tt_norm(WL.block_sum([(1.0, x) for x in xs])) if given_norm else None
    ref, info = R.tt_round_adaptive_sum(xs, 1e-3, 17, block=0, f_inc=0.2, nrmx=nrmx)
    opts = B.options(precision=prec, slices=8, f_inc=0.2, nrmx=nrmx or 0.0)
    with B.round_adaptive_sum(dev_summands(xs), 1e-3, 0, 17, opts) as y:
        yi = y.info
        got = y.to_numpy()
    assert yi["ranks"] == info["ranks"]
    assert math.isclose(yi["tau"], info["tau"], rel_tol=1e-10 if prec == 0 else 1e-9)
    assert rel(got, ref) <= (1e-10 if prec == 0 else 1e-9)


def test_sum_single_summand_equals_adaptive(B):
    x = WL.random_tt(np.random.default_rng(5), 6, 7, 9)
    opts = B.options(nrmx=T.tt_norm(x))
    with B.round_adaptive_sum(dev_summands([x]), 1e-2, 3, 9, opts) as y:
        ys = y.to_numpy()
        rs = y.info["ranks"]
    with B.round_adaptive([torch.from_numpy(c).to("cuda") for c in x], 1e-2, 3, 9, opts) as y:
        yf = y.to_numpy()
        rf = y.info["ranks"]
    assert rs == rf
    assert rel(ys, yf) <= 1e-12


@pytest.mark.parametrize("prec", [0, 1])
def test_sum_c2_full_size(B, prec):
    """The d=20, n=50 workload as its 5 summands (4 scaled copies of a rank-50 TT sharing their
    cores after the first, and the rank-10 noise TT), tol 1e-6, block 10: the same ranks as the
    oracle's sum algorithm and as the formal-sum rounding on the GPU; tensors within the bars of
    the formal-sum tests (FP64 1e-10, sliced 1e-8)."""
    x = WL.c2()
    ref, info = R.tt_round_adaptive_sum(x.summands, 1e-6, 2024, block=10, nrmx=x.norm)
    opts = B.options(precision=prec, nrmx=x.norm)
    with B.round_adaptive_sum(dev_summands(x.summands), 1e-6, 10, 2024, opts) as y:
        yi = y.info
        got = y.to_numpy()
    assert yi["ranks"] == info["ranks"]
    assert rel(got, ref) <= (1e-10 if prec == 0 else 1e-8)
    assert T.tt_dist(got, x.cores) <= 1e-6 * x.norm
    with B.round_adaptive([torch.from_numpy(c).to("cuda") for c in x.cores], 1e-6, 10, 2024, opts) as y:
        assert y.info["ranks"] == yi["ranks"]


def test_sum_argument_errors(B):
    xs = mixed_summands(1)
    with pytest.raises(ValueError):
        B.round_adaptive_sum([], 1e-3, 1, 1)
    bad = [xs[0], xs[1][:4]]
    with pytest.raises(ValueError):
        B.round_adaptive_sum(dev_summands(bad), 1e-3, 1, 1)


@pytest.mark.parametrize("prec", [0, 1])
def test_sum_more_summands_than_one_launch(B, prec):
    """10 summands: the grouped launches take 8 and then 2."""
    rng = np.random.default_rng(21)
    n = [6, 5, 7, 4, 6, 5]
    xs = [WL.random_tt(rng, 6, n, int(r)) for r in rng.integers(1, 6, size=10)]
    for x, c in zip(xs, rng.standard_normal(10)):
        x[0] = x[0] * c
    ref, info = R.tt_round_adaptive_sum(xs, 1e-4, 5, block=3)
    with B.round_adaptive_sum(dev_summands(xs), 1e-4, 3, 5, B.options(precision=prec, slices=8)) as y:
        yi = y.info
        got = y.to_numpy()
    assert yi["ranks"] == info["ranks"]
    assert rel(got, ref) <= (1e-10 if prec == 0 else 1e-9)


@pytest.mark.parametrize("prec", [0, 1])
def test_sum_first_block_wider_than_the_last_unfolding(B, prec):
    """b_init = max summand rank (6) exceeds the rank of the last unfolding (n_d = 4): reading R14
    clamps it, and the CholeskyQR of the first block sees a full-rank sketch."""
    rng = np.random.default_rng(13)
    xs = [WL.random_tt(rng, 5, 4, r) for r in (6, 5)]
    xs[1][0] = xs[1][0] * 0.8
    ref, info = R.tt_round_adaptive_sum(xs, 1e-8, 3, block=0)
    with B.round_adaptive_sum(dev_summands(xs), 1e-8, 0, 3, B.options(precision=prec, slices=8)) as y:
        assert y.info["ranks"] == info["ranks"]
        assert rel(y.to_numpy(), ref) <= (1e-10 if prec == 0 else 1e-9)


@pytest.mark.parametrize("prec", [0, 1])
def test_host_driven_block_loop(B, prec, monkeypatch):
    """The host-driven block loop (used where a block or the sketch is too wide for the persistent
    kernel), forced here: C1's summands, and a full-rank sum (formal rank 120, rows up to 6000,
    blocks of 30) whose block projections take the tensor-core branch in sliced form.  The slice
    count follows the tolerance (5 slices at 1e-4, each product exact to ~5 * 2^-31 = 2e-9 of the
    operand scales), so the sliced bar is 1e-3 * tol, at least 1e-8."""
    monkeypatch.setenv("TTR_HOST_LOOP", "1")
    rng = np.random.default_rng(77)
    wide = [WL.random_tt(rng, 6, 50, r) for r in (40, 40, 40)]
    for x, c in zip(wide, (1.0, -0.5, 0.7)):
        x[0] = x[0] * c
    x1 = WL.c1()
    for xs, tol, block, nrmx, em, beta in ((x1.summands, 1e-6, 2, x1.norm, 0, 1.0), (wide, 1e-4, 30, None, 0, 1.0),
                                           (x1.summands, 1e-6, 2, x1.norm, 6, 4.0)):   # the last: reading R16
        ref, info = R.tt_round_adaptive_sum(xs, tol, 5, block=block, nrmx=nrmx, est_min=em, est_safety=beta)
        with B.round_adaptive_sum(dev_summands(xs), tol, block, 5,
                                  B.options(precision=prec, nrmx=nrmx or 0.0, est_min=em, est_safety=beta)) as y:
            assert y.info["ranks"] == info["ranks"]
            assert rel(y.to_numpy(), ref) <= (1e-10 if prec == 0 else max(1e-8, 1e-3 * tol))


@pytest.mark.parametrize("prec", [0, 1])
def test_wide_ranks_device_block_loop(B, prec):
    """A full-rank sum whose block loop rows do not fit in shared memory (three summands of rank 60,
    n = 40: rows up to 180 x 40 = 7200, sketch widths near 200) and whose first block (the appendix's
    b_init = 60) is wider than the device loop factors: the first block is factored on the host side,
    the rest of the loop runs on the device with its rows in global memory.  Against the oracle."""
    rng = np.random.default_rng(91)
    xs = [WL.random_tt(rng, 6, 40, 60) for _ in range(3)]
    for x, c in zip(xs, (1.0, -0.6, 0.8)):
        x[0] = x[0] * c
    ref, info = R.tt_round_adaptive_sum(xs, 1e-6, 7, block=0)
    assert max(info["ranks"]) == 180
    with B.round_adaptive_sum(dev_summands(xs), 1e-6, 0, 7, B.options(precision=prec, slices=8)) as y:
        assert y.info["ranks"] == info["ranks"]
        assert rel(y.to_numpy(), ref) <= (1e-10 if prec == 0 else 1e-9)
