"""GPU parity of the per-core-parallel partial contractions (the Conclusion's observation, Sec. 5):
all G_k(:, :, j) = sum_i X_k(:, i, :) Omega_k(i, j) in one launch, then the column-wise chain
W_k(:, j) = G_k(:, :, j) W_{k+1}(:, j).  Against the oracle's Algorithm 3 element by element
(1e-12 of max|W_k|, the FP64 bar of the chain form), and inside the roundings against the oracle's
Algorithm 6 (FP64 bars)."""
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


CASES = [("c1", lambda: WL.c1().cores, 0, 13, 2), ("ragged", lambda: WL.random_tt(np.random.default_rng(3), 5, [3, 7, 1, 5, 4], [4, 9, 2, 6]), 3, 24, 2),
         ("c3s", lambda: WL.c3(d=6, n=16, r=10).cores, 5, 45, 3),
         ("wide_cols", lambda: WL.random_tt(np.random.default_rng(9), 4, [6, 5, 7, 4], [9, 70, 11]), 0, 150, 2),
         ("c3", lambda: WL.c3().cores, 0, 70, 2)]


@pytest.mark.parametrize("name,make,c0,c1,t", CASES)
def test_percore_equals_algorithm_3(B, name, make, c0, c1, t):
    cores = make()
    got = B.partial_contractions_percore(dev(cores), 77, c0, c1, t)
    ref = R.partial_contractions_rl(cores, 77, c0, c1, t)
    for k, Wk in ref.items():
        g = got[k].cpu().numpy()
        assert g.shape == Wk.shape
        assert np.abs(g - Wk).max() <= 1e-12 * np.abs(Wk).max(), (k, np.abs(g - Wk).max() / np.abs(Wk).max())


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name,make,tol,block", [("c1", lambda: WL.c1(), 1e-6, 2),
                                                 ("c3_small", lambda: WL.c3(d=6, n=16, r=10), 1e-8, 0),
                                                 ("width_growth", lambda: WL.c1(), 1e-7, 2)])
def test_adaptive_with_percore_contractions(B, prec, name, make, tol, block):
    x = make()
    ref, info = R.tt_round_adaptive(x.cores, tol, seed=5, block=block, nrmx=x.norm)
    hint = 2 if name == "width_growth" else 0      # forces Algorithm 5 to append columns repeatedly
    with B.round_adaptive(dev(x.cores), tol, block, 5,
                          B.options(precision=prec, slices=8, nrmx=x.norm, rl_percore=1, width_hint=hint)) as y:
        assert y.ranks == info["ranks"]
        got = y.to_numpy()
        if name == "width_growth":
            assert y.info["extensions"] > 0
    assert T.tt_dist(got, ref) <= 1e-10 * T.tt_norm(ref)


def test_sum_with_percore_contractions(B):
    x = WL.c1()
    ref, info = R.tt_round_adaptive_sum(x.summands, 1e-6, 5, block=2, nrmx=x.norm)
    sdev = [dev(p) for p in x.summands]
    with B.round_adaptive_sum(sdev, 1e-6, 2, 5, B.options(nrmx=x.norm, rl_percore=1)) as y:
        assert y.ranks == info["ranks"]
        assert T.tt_dist(y.to_numpy(), ref) <= 1e-10 * T.tt_norm(ref)


def test_fixed_with_percore_contractions(B):
    x = WL.c1()
    ref, info = R.tt_round_fixed(x.cores, 13, seed=31)
    with B.round_fixed(dev(x.cores), 13, 31, opts=B.options(rl_percore=2)) as y:
        assert y.ranks == info["ranks"]
        assert T.tt_dist(y.to_numpy(), ref) <= 1e-10 * T.tt_norm(ref)
