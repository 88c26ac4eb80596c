"""Degenerate inputs and the largest single-GPU workload on the GPU path.

* A zero tensor rounds to the zero TT of ranks 1 (reading R15), for one TT and for a sum.
* d = 2 (no partial-contraction step): fixed, adaptive and sum entry points against the oracle.
* The d=50, n=100 workload (4 scaled copies of a rank-200 TT + rank-10 noise at 1e-8; formal rank
  810, 25 GB as a formal sum) at full size through the sum entry point, whose inputs are only the
  summands (1.6 GB).  The oracle cannot round it in test time, so properties that hold at any
  size are checked: cores 1..d-1 left-orthonormal, ranks between the true rank 200 and
  b_init + b_inc, and ||X - Y|| <= tol ||X|| with ||X - Y||^2 = ||X||^2 + ||Y||^2 - 2 <X, Y>
  computed in FP64 from the summands (resolution ~1e-8 ||X||, tol = 1e-6).
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


def dev(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).to("cuda") for c in cores]


def dev_summands(summands):
    cache = {}
    return [[cache.setdefault(id(c), torch.from_numpy(np.ascontiguousarray(c)).to("cuda")) for c in x] for x in summands]


def rel(a, b):
    return T.tt_dist(a, b) / max(T.tt_norm(b), 1e-300)


@pytest.mark.parametrize("prec", [0, 1])
def test_zero_tensor(B, prec):
    x = [np.zeros_like(c) for c in WL.random_tt(np.random.default_rng(1), 4, 5, 3)]
    opts = B.options(precision=prec, slices=8)
    with B.round_adaptive(dev(x), 1e-6, 2, 3, opts) as y:
        assert y.ranks == [1, 1, 1, 1, 1] and y.info["nrmx"] == 0.0
        assert all(np.count_nonzero(c) == 0 for c in y.to_numpy())
    with B.round_adaptive_sum(dev_summands([x, x]), 1e-6, 0, 3, opts) as y:
        assert y.ranks == [1, 1, 1, 1, 1]


@pytest.mark.parametrize("prec", [0, 1])
def test_two_cores(B, prec):
    rng = np.random.default_rng(17)
    xs = [WL.random_tt(rng, 2, [9, 7], r) for r in (3, 4)]
    xs[1][0] = xs[1][0] * 0.5
    xf = WL.block_sum([(1.0, x) for x in xs])
    opts = B.options(precision=prec, slices=8)
    bar = 1e-10 if prec == 0 else 1e-9
    ref, info = R.tt_round_fixed(xf, 5, seed=4)
    with B.round_fixed(dev(xf), 5, 4, opts=opts) as y:
        assert y.ranks == info["ranks"]
        assert rel(y.to_numpy(), ref) <= bar
    ref, info = R.tt_round_adaptive(xf, 1e-12, 2, block=2)
    with B.round_adaptive(dev(xf), 1e-12, 2, 2, opts) as y:
        assert y.ranks == info["ranks"] == [1, 7, 1]
        assert rel(y.to_numpy(), ref) <= bar
    ref, info = R.tt_round_adaptive_sum(xs, 1e-12, 2, block=0)
    with B.round_adaptive_sum(dev_summands(xs), 1e-12, 0, 2, opts) as y:
        assert y.ranks == info["ranks"]
        assert rel(y.to_numpy(), ref) <= bar


def _inner(xs, ys):
    """<X, Y> of TTs given as lists of CUDA tensors, by left-to-right contraction in FP64."""
    g = torch.ones((1, 1), dtype=torch.float64, device="cuda")
    for a, b in zip(xs, ys):
        t = torch.tensordot(g, a, dims=([0], [0]))                # (r_y, n, r_x')
        g = torch.tensordot(t, b, dims=([0, 1], [0, 1]))          # (r_x', r_y')
    return float(g.reshape(-1)[0])


def test_c5_full_size_properties(B):
    x = WL.c5(formal=False)
    summ = dev_summands(x.summands)
    tol = 1e-6
    opts = B.options(precision=B.TTR_PREC_SLICED, nrmx=x.norm)
    with B.round_adaptive_sum(summ, tol, 0, 2024, opts) as y:
        ranks = y.ranks
        Y = y.to_torch()
    d = len(Y)
    assert ranks[1] <= 100 and ranks[d - 1] <= 100
    assert all(200 <= r <= 241 for r in ranks[2:d - 1]), ranks
    for k in range(d - 1):
        v = Y[k].reshape(-1, Y[k].shape[2])
        eye = torch.eye(v.shape[1], dtype=torch.float64, device="cuda")
        assert float((v.T @ v - eye).abs().max()) <= 1e-9, k
    ny2 = _inner(Y, Y)
    nxy = sum(_inner(part, Y) for part in summ)
    err2 = x.norm ** 2 + ny2 - 2.0 * nxy
    assert math.sqrt(max(err2, 0.0)) <= tol * x.norm, (err2, x.norm)
