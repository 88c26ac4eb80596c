"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

Tolerances (FP64 mode): Omega bit for bit; partial contractions 1e-12 relative (max-norm);
rounded tensors 1e-10 relative Frobenius distance of the represented tensors (the QR bases
themselves are not unique), identical ranks, residual estimates 1e-8 relative.
"""
import math

import numpy as np
import pytest

import workloads as WL
from oracle import philox as OP
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


def rel_tensor_diff(a, b):
    return T.tt_dist(a, b) / max(T.tt_norm(b), 1e-300)


# ------------------------------------------------------------------ Omega
@pytest.mark.parametrize("seed,k,n,c0,c1", [(1, 2, 50, 0, 64), (2**63 + 12345, 7, 3, 5, 77), (0, 20, 128, 100, 101),
                                             (987654321, 3, 1, 0, 300)])
def test_omega_bitwise(B, seed, k, n, c0, c1):
    got = B.sketch_omega(seed, k, n, c0, c1).cpu().numpy()
    ref = OP.omega(seed, k, n, c0, c1)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))


# ------------------------------------------------------------------ Algorithm 3
CASES_RL = [("c1", lambda: WL.c1().cores, 13), ("ragged", lambda: WL.random_tt(np.random.default_rng(3), 5, [3, 7, 1, 5, 4], [4, 9, 2, 6]), 21),
            ("c3s", lambda: WL.c3(d=6, n=16, r=10).cores, 40),
            # one wide bond (r_2 = 600): the tensor-core step for core 2 splits its K = 600 over CTAs
            ("wide", lambda: WL.random_tt(np.random.default_rng(4), 4, [5, 8, 6, 3], [4, 600, 7]), 80)]


@pytest.mark.parametrize("name,make,w", CASES_RL)
@pytest.mark.parametrize("prec", [0, 1])
def test_partial_contractions(B, name, make, w, prec):
    cores = make()
    got = B.partial_contractions(dev(cores), 77, 3, 3 + w, precision=prec, slices=8)
    ref = R.partial_contractions_rl(cores, 77, 3, 3 + w)
    for k, Wk in ref.items():
        g = got[k].cpu().numpy()
        assert g.shape == Wk.shape
        scale = np.abs(Wk).max()
        assert np.abs(g - Wk).max() <= 1e-12 * scale, (k, np.abs(g - Wk).max() / scale)


def test_partial_contractions_c2_full_size(B):
    x = WL.c2()
    got = B.partial_contractions(dev(x.cores), 5, 0, 70)
    ref = R.partial_contractions_rl(x.cores, 5, 0, 70)
    for k in (2, 11, 20):
        g = got[k].cpu().numpy()
        assert np.abs(g - ref[k]).max() <= 1e-12 * np.abs(ref[k]).max()


# ------------------------------------------------------------------ Algorithm 4
def test_fixed_c1(B):
    x = WL.c1()
    ref, info = R.tt_round_fixed(x.cores, 13, seed=31)
    with B.round_fixed(dev(x.cores), 13, 31) as y:
        assert y.ranks == info["ranks"]
        got = y.to_numpy()
    assert rel_tensor_diff(got, ref) <= 1e-10
    assert T.left_orth_defect(got) <= 1e-12


def test_fixed_c1_orthonormal_every_time(B):
    """Rank 13 exceeds C1's true rank 10, so every sketch block is numerically rank-deficient and
    the QR completes it from rounding noise, which varies from run to run (the FP64 products that
    form M_k sum with atomics).  The completing directions must still be orthonormal, every run."""
    x = WL.c1()
    cores = dev(x.cores)
    for _ in range(12):
        with B.round_fixed(cores, 13, 31) as y:
            got = y.to_numpy()
        assert T.left_orth_defect(got) <= 1e-12
        assert T.tt_dist(got, x.cores) <= 1e-10 * x.norm


def test_fixed_c1_target(B):
    x = WL.c1()
    Y, _ = R.tt_round_fixed(x.cores, 13, seed=31)
    ref = R.svd_pass_rl(Y, max_rank=8)
    with B.round_fixed(dev(x.cores), 13, 31, target=8) as y:
        assert y.ranks == [1, 8, 8, 8, 8, 8, 1]
        got = y.to_numpy()
    assert rel_tensor_diff(got, ref) <= 1e-10


# ------------------------------------------------------------------ Algorithm 6
CASES_AD = [
    ("c1_blk2", lambda: WL.c1(), 1e-6, 2),
    ("c1_frac", lambda: WL.c1(), 1e-3, 0),
    ("c3_small", lambda: WL.c3(d=6, n=16, r=10), 1e-8, 0),
    ("ragged", lambda: WL.copies_plus_noise(8, 5, 7, 5, 3, 2, 1e-6, "ragged"), 1e-5, 3),
]


@pytest.mark.parametrize("name,make,tol,block", CASES_AD)
@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_parity(B, name, make, tol, block, prec):
    x = make()
    ref, info = R.tt_round_adaptive(x.cores, tol, seed=5, block=block, nrmx=x.norm)
    with B.round_adaptive(dev(x.cores), tol, block, 5, B.options(precision=prec, slices=8, nrmx=x.norm)) as y:
        yi = y.info
        got = y.to_numpy()
    assert yi["ranks"] == info["ranks"]
    flat = [e for es in info["estimates"] for e in es]
    assert len(flat) == len(yi["estimates"])
    assert np.allclose(yi["estimates"], flat, rtol=1e-8, atol=1e-13 * x.norm)
    assert rel_tensor_diff(got, ref) <= 1e-10
    assert T.tt_dist(got, x.cores) <= tol * x.norm * (1 + 1e-9)


def test_adaptive_norm_estimate(B):
    x = WL.c1()
    ref, info = R.tt_round_adaptive(x.cores, 1e-6, seed=9, block=2)
    with B.round_adaptive(dev(x.cores), 1e-6, 2, 9) as y:
        assert math.isclose(y.info["nrmx"], info["nrmx"], rel_tol=1e-12)
        assert y.ranks == info["ranks"]
        assert rel_tensor_diff(y.to_numpy(), ref) <= 1e-10


def test_adaptive_width_hint_does_not_change_result(B):
    x = WL.c1()
    outs = []
    for hint in (2, 9, 40):          # width 2 forces Algorithm 5 to append columns repeatedly
        with B.round_adaptive(dev(x.cores), 1e-7, 2, 3, B.options(nrmx=x.norm, width_hint=hint)) as y:
            outs.append((y.ranks, y.to_numpy(), y.info["extensions"]))
    for ranks, cores, _ in outs[1:]:
        assert ranks == outs[0][0]
        assert rel_tensor_diff(cores, outs[0][1]) <= 1e-12
    assert outs[2][2] < outs[0][2] and outs[0][2] > 0


def test_adaptive_adap_r(B):
    x = WL.c1()
    ref, info = R.tt_round_adaptive(x.cores, 1e-6, seed=5, block=2, nrmx=x.norm, adap_r=True)
    with B.round_adaptive(dev(x.cores), 1e-6, 2, 5, B.options(nrmx=x.norm, adap_r=True)) as y:
        assert y.ranks == info["ranks"]
        assert rel_tensor_diff(y.to_numpy(), ref) <= 1e-10


def test_adaptive_c2_full_size(B):
    """The bench workload: d=20, n=50, formal rank 210, tol 1e-6, block 10."""
    x = WL.c2()
    ref, info = R.tt_round_adaptive(x.cores, 1e-6, seed=2024, block=10, nrmx=x.norm)
    with B.round_adaptive(dev(x.cores), 1e-6, 10, 2024, B.options(nrmx=x.norm)) as y:
        yi = y.info
        got = y.to_numpy()
    assert yi["ranks"] == info["ranks"]
    flat = [e for es in info["estimates"] for e in es]
    assert np.allclose(yi["estimates"], flat, rtol=1e-8, atol=1e-14 * x.norm)
    assert rel_tensor_diff(got, ref) <= 1e-10


@pytest.mark.parametrize("max_sms", [0, 50])
def test_adaptive_c2_full_size_sliced_default(B, max_sms):
    """The bench configuration: sliced precision with the slice count chosen for tol 1e-6 (6 slices,
    contraction error ~6 * 2^-41 of the operand scales), against the FP64 oracle.

    Stated bound for this form: each sliced contraction is exact to ~6 * 2^-41 = 2.7e-12 of
    sum_c |a_rc| |b_cj|.  The input is a formal sum of copies whose coefficients c_i partly cancel,
    so sum |a||b| exceeds |sum a b| by up to kappa = sum |c_i| / |sum c_i| (about 20 here); a
    residual estimate (||S||_F / sqrt(b) over a rows x b block) then moves by about
    kappa * 2.7e-12 * sqrt(rows) ||X|| ~ 3e-9 ||X|| for rows = 3000.  The same perturbation turns
    the sketched subspaces in the directions near the truncation level (singular values ~1e-7
    ||X||) and moves each core's projection by ~kappa * 2.7e-12 ||X||; over d - 1 = 19 cores the
    stated bound for the rounded tensor is 1e-8 relative (1 % of tol).  Ranks must be identical.
    With max_sms = 50 (a third of the SMs, as each rounding has with three in flight) the block loop
    runs on 50 CTAs and the K-split tensor-core launches are sized for 50 SMs: other K segments,
    the same bound."""
    x = WL.c2()
    ref, info = R.tt_round_adaptive(x.cores, 1e-6, seed=2024, block=10, nrmx=x.norm)
    opts = B.options(precision=B.TTR_PREC_SLICED, nrmx=x.norm, max_sms=max_sms)
    with B.round_adaptive(dev(x.cores), 1e-6, 10, 2024, opts) as y:
        yi = y.info
        got = y.to_numpy()
    assert yi["ranks"] == info["ranks"]
    flat = [e for es in info["estimates"] for e in es]
    coef = np.asarray(x.meta["coef"])
    kappa = np.abs(coef).sum() / abs(coef.sum())
    bound = kappa * 2.7e-12 * math.sqrt(3000)
    dev_est = np.abs(np.asarray(yi["estimates"]) - np.asarray(flat)).max() / x.norm
    diff = rel_tensor_diff(got, ref)
    print(f"max estimate deviation {dev_est:.3e} ||X|| (bound {bound:.1e}), tensor difference {diff:.3e}")
    assert dev_est <= bound
    assert diff <= 1e-8
    assert T.tt_dist(got, x.cores) <= 1e-6 * x.norm


@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_c3_full_size(B, prec):
    """The operator-applied TT vector (d=16, n=64, y = A x, formal rank 60) at tol 1e-8 with the
    paper's block fractions (b_init = 6, b_inc = 3) and the estimator reading R16 (10 estimator
    columns, stop at tau / 10), which keeps the result within tol (Algorithm 6 as printed stops at
    ~7 tol on this input, in the oracle and here alike).  FP64 form: FP64 bars.  Sliced form with the
    slice count chosen for 1e-8 (7 slices, contraction error ~7 * 2^-48 of the operand scales):
    identical ranks, tensor within 1e-9 of the FP64 oracle.  Both forms meet the tolerance."""
    x = WL.c3()
    ref, info = R.tt_round_adaptive(x.cores, 1e-8, seed=3, block=0, nrmx=x.norm, est_min=10, est_safety=10.0)
    assert T.tt_dist(ref, x.cores) <= 1e-8 * x.norm
    with B.round_adaptive(dev(x.cores), 1e-8, 0, 3,
                          B.options(precision=prec, nrmx=x.norm, est_min=10, est_safety=10.0)) as y:
        yi = y.info
        got = y.to_numpy()
    assert yi["ranks"] == info["ranks"]
    flat = [e for es in info["estimates"] for e in es]
    if prec == 0:
        assert np.allclose(yi["estimates"], flat, rtol=1e-8, atol=1e-14 * x.norm)
        assert rel_tensor_diff(got, ref) <= 1e-10
    else:
        assert np.allclose(yi["estimates"], flat, rtol=1e-6, atol=1e-12 * x.norm)
        assert rel_tensor_diff(got, ref) <= 1e-9
    assert T.tt_dist(got, x.cores) <= 1e-8 * x.norm


@pytest.mark.parametrize("name,make,tol,block,est_min,beta", [
    ("c1_blk2", lambda: WL.c1(), 1e-6, 2, 6, 4.0),
    ("ragged", lambda: WL.copies_plus_noise(8, 5, 7, 5, 3, 2, 1e-6, "ragged"), 1e-5, 3, 10, 10.0),
    ("c3_small", lambda: WL.c3(d=6, n=16, r=10), 1e-7, 0, 10, 10.0),
])
def test_adaptive_estimator_reading_parity(B, name, make, tol, block, est_min, beta):
    """Reading R16 on the device loop: residual sketches wider than the appended block and the stop
    at tau / beta, against the oracle with the same settings (FP64 bars).  The estimate of a block
    whose residual vanishes exactly (the rank of the unfolding is used up) is rounding noise of
    order u ||X|| times the entries summed, whose value depends on the summation order (the device
    reductions add in no fixed order): estimates are compared to 1e-13 ||X|| absolute."""
    x = make()
    ref, info = R.tt_round_adaptive(x.cores, tol, seed=5, block=block, nrmx=x.norm, est_min=est_min, est_safety=beta)
    with B.round_adaptive(dev(x.cores), tol, block, 5, B.options(nrmx=x.norm, est_min=est_min, est_safety=beta)) as y:
        yi = y.info
        got = y.to_numpy()
    assert yi["ranks"] == info["ranks"]
    flat = [e for es in info["estimates"] for e in es]
    assert len(flat) == len(yi["estimates"])
    assert np.allclose(yi["estimates"], flat, rtol=1e-8, atol=1e-13 * x.norm)
    assert rel_tensor_diff(got, ref) <= 1e-10
    assert T.tt_dist(got, x.cores) <= tol * x.norm * (1 + 1e-9)


# ------------------------------------------------------------------ Algorithm 1
@pytest.mark.parametrize("name,make,tol", [("c1", lambda: WL.c1(), 1e-2), ("c1", lambda: WL.c1(), 1e-6),
                                           ("c1", lambda: WL.c1(), 1e-9),
                                           ("c3", lambda: WL.c3(), 1e-8), ("c2", lambda: WL.c2(), 1e-6),
                                           ("ragged", lambda: WL.copies_plus_noise(8, 5, 7, 5, 3, 2, 1e-6, "r"), 1e-5)])
def test_deterministic_fp64(B, name, make, tol):
    """Algorithm 1 in FP64 against the oracle's LAPACK QR/SVD form: identical ranks, the represented
    tensors within 1e-10, the tolerance met.  The formal sums (c1, c2, ragged) have numerically
    rank-deficient unfoldings; the operator-applied vector (c3) is truncated at 1e-8, where a Gram
    matrix could not resolve the discarded singular values."""
    x = make()
    ref, info = R.tt_round_deterministic(x.cores, tol)
    with B.round_deterministic(dev(x.cores), tol) as y:
        assert y.ranks == info["ranks"], (y.ranks, info["ranks"])
        got = y.to_numpy()
        assert math.isclose(y.info["tau"], info["tau"], rel_tol=1e-10)
    assert T.tt_dist(got, x.cores) <= tol * x.norm * (1 + 1e-9)
    assert rel_tensor_diff(got, ref) <= 1e-10


# ------------------------------------------------------------------ edge cases and errors
def test_rank_one_and_n_one(B):
    cores = WL.random_tt(np.random.default_rng(1), 4, [1, 5, 1, 3], [1, 3, 2])
    ref, info = R.tt_round_adaptive(cores, 1e-9, seed=1, block=1, nrmx=T.tt_norm(cores))
    with B.round_adaptive(dev(cores), 1e-9, 1, 1, B.options(nrmx=T.tt_norm(cores))) as y:
        assert y.ranks == info["ranks"]
        assert rel_tensor_diff(y.to_numpy(), ref) <= 1e-10


def test_bad_arguments_raise(B):
    x = WL.c1()
    with pytest.raises(B.TTRoundError):
        B.round_adaptive(dev(x.cores), 0.0, 2, 1)
    with pytest.raises(B.TTRoundError):
        B.round_fixed(dev(x.cores), 0, 1)


@pytest.mark.parametrize("slices", [3, 4, 5, 6, 7, 8])
def test_partial_contractions_every_slice_count(B, slices):
    """The tensor-core issue loop is compiled per slice count; each one against the oracle, within
    the sliced form's stated error s * 2^(1-7s) of sum |a||b| (sum |a||b| <= 50 max|W| here, with a
    margin of 10), and at the FP64 floor for the counts that reach it."""
    cores = WL.random_tt(np.random.default_rng(8), 5, [6, 9, 4, 7, 5], [12, 40, 9, 30])
    got = B.partial_contractions(dev(cores), 21, 0, 80, precision=1, slices=slices)
    ref = R.partial_contractions_rl(cores, 21, 0, 80)
    bound = max(500.0 * slices * 2.0 ** (1 - 7 * slices), 1e-13)
    for k, Wk in ref.items():
        err = np.abs(got[k].cpu().numpy() - Wk).max() / np.abs(Wk).max()
        assert err <= bound, (slices, k, err, bound)


@pytest.mark.parametrize("tol", [1e-3, 1e-4])
def test_adaptive_sliced_at_the_tolerance_chosen_slice_count(B, tol):
    """The bench workload (d=20, n=50, formal rank 210, block 10) in sliced form with the slice count
    the tolerance chooses: 4 slices at 1e-3 (each product exact to ~4 * 2^-27 = 3e-8 of sum |a||b|)
    and 5 at 1e-4 (~3e-10), with the double-float block loop.  A product error e (times the copy
    coefficients' cancellation kappa ~ 20) turns the sketched subspace by about kappa e ||X|| / sigma_r,
    sigma_r the smallest kept singular value (~1e-2 ||X|| here), and moves the projected tensor by as
    much: ~6e-5 at 4 slices, ~5e-7 at 5 (the 6-slice default measures 2.9e-9; each slice is 2^7).
    The slice rule (12 bits beyond -log2 tol) keeps that below tol / 10.  Stated bar for these forms:
    ranks identical to the FP64 oracle's, the represented tensor within tol / 10 of the oracle's, and
    the tolerance met."""
    x = WL.c2()
    ref, info = R.tt_round_adaptive(x.cores, tol, seed=2024, block=10, nrmx=x.norm)
    with B.round_adaptive(dev(x.cores), tol, 10, 2024, B.options(precision=B.TTR_PREC_SLICED, nrmx=x.norm)) as y:
        assert y.ranks == info["ranks"]
        got = y.to_numpy()
    assert rel_tensor_diff(got, ref) <= 0.1 * tol
    assert T.tt_dist(got, x.cores) <= tol * x.norm


def test_adaptive_sliced_default_with_double_float_block_loop(B):
    """The bench configuration (6 slices at tol 1e-6) with the block loop's per-CTA arithmetic in
    double-float (block_loop_df, about 2^-48 relative): the same bars as the default sliced form."""
    x = WL.c2()
    ref, info = R.tt_round_adaptive(x.cores, 1e-6, seed=2024, block=10, nrmx=x.norm)
    with B.round_adaptive(dev(x.cores), 1e-6, 10, 2024,
                          B.options(precision=B.TTR_PREC_SLICED, nrmx=x.norm, block_loop_df=True)) as y:
        assert y.ranks == info["ranks"]
        got = y.to_numpy()
    assert rel_tensor_diff(got, ref) <= 1e-8
    assert T.tt_dist(got, x.cores) <= 1e-6 * x.norm


@pytest.mark.parametrize("name,make,tol,block,slices,bar", [
    ("c2", lambda: WL.c2(), 1e-6, 10, 0, 1e-8),
    ("c3_small", lambda: WL.c3(d=6, n=16, r=10), 1e-7, 0, 8, 1e-10),
    ("ragged", lambda: WL.copies_plus_noise(8, 5, 7, 5, 3, 2, 1e-6, "ragged"), 1e-5, 3, 8, 1e-10),
])
def test_adaptive_block_loop_tensor_core_products(B, name, make, tol, block, slices, bar):
    """The block loop's per-row products on the tensor cores (block_loop_tc, 8-slice products with
    the error bound of FP64 products): the oracle's ranks, and the tensor within the bar of the
    sliced form at that slice count (tolerance-chosen for the bench workload, 8 otherwise)."""
    x = make()
    ref, info = R.tt_round_adaptive(x.cores, tol, seed=2024, block=block, nrmx=x.norm)
    with B.round_adaptive(dev(x.cores), tol, block, 2024,
                          B.options(precision=B.TTR_PREC_SLICED, slices=slices, nrmx=x.norm, block_loop_tc=True)) as y:
        assert y.ranks == info["ranks"]
        got = y.to_numpy()
    assert rel_tensor_diff(got, ref) <= bar
    assert T.tt_dist(got, x.cores) <= tol * x.norm


def test_adaptive_sliced_autotuned(B):
    """The bench configuration with the tile-shape autotuner on (each new shape times its candidate
    launches once per process): the oracle's ranks and the sliced form's bars, on the call that tunes
    and on a later call that reads the table."""
    x = WL.c2()
    ref, info = R.tt_round_adaptive(x.cores, 1e-6, seed=2024, block=10, nrmx=x.norm)
    for _ in range(2):
        with B.round_adaptive(dev(x.cores), 1e-6, 10, 2024,
                              B.options(precision=B.TTR_PREC_SLICED, nrmx=x.norm, autotune=True)) as y:
            assert y.ranks == info["ranks"]
            got = y.to_numpy()
        assert rel_tensor_diff(got, ref) <= 1e-8
        assert T.tt_dist(got, x.cores) <= 1e-6 * x.norm


def test_adaptive_adap_r_sliced(B):
    """The Remark 3.2 pass after the sliced rounding (8 slices): ranks and tensor as the oracle's."""
    x = WL.c1()
    ref, info = R.tt_round_adaptive(x.cores, 1e-6, seed=5, block=2, nrmx=x.norm, adap_r=True)
    with B.round_adaptive(dev(x.cores), 1e-6, 2, 5, B.options(precision=B.TTR_PREC_SLICED, slices=8, nrmx=x.norm,
                                                               adap_r=True)) as y:
        assert y.ranks == info["ranks"]
        assert rel_tensor_diff(y.to_numpy(), ref) <= 1e-10
