"""Pins for the oracle's rounding algorithms, each against something other than itself.

* Algorithm 3 (partial contractions) vs Eq. (3.1) evaluated by brute force: the explicit
  right part H(X_{k:d}) times explicitly formed Khatri-Rao (Kronecker) columns, and an
  einsum over all mode indices.
* Algorithm 4 / 6 vs dense re-implementations on the explicit full tensor: sketches formed
  as X_(1:k) times explicit KRP columns, projections by explicit orthonormal bases.
* Algorithm 1 vs TT-SVD of the full tensor (numpy SVD of sequential unfoldings), which it
  equals in exact arithmetic (Sec. 2.3); Remark 3.2's pass vs right-to-left TT-SVD.
* Invariants: exact reconstruction when l_k >= rank, left-orthonormal cores, rank bounds,
  relative error <= tol, and the per-core error budget of Sec. 3.3.
* Planted mistakes (in the oracle, on the CPU) must make the matching pin fail.
"""
import math

import numpy as np
import pytest

import workloads as WL
from oracle import rounding as R
from oracle import tt as T
from oracle.philox import omega


def tiny_tt(seed, d, n, r):
    rng = np.random.default_rng(seed)
    return WL.random_tt(rng, d, n, r)


def right_part(cores, k):
    """Full right part as an array R[a, i_k, ..., i_d] (1-based k)."""
    t = cores[k - 1]
    for c in cores[k:]:
        t = np.tensordot(t, c, axes=([t.ndim - 1], [0]))
    return t[..., 0]


def krp_columns(seed, ks, n, col0, col1, fastest_last=True):
    """Explicit Khatri-Rao columns kron(omega_{ks[0]}(:,j), ..., omega_{ks[-1]}(:,j))."""
    oms = [omega(seed, k, n[k - 1], col0, col1) for k in ks]
    cols = []
    for j in range(col1 - col0):
        v = np.ones(1)
        for om in oms:
            v = np.kron(v, om[:, j])
        cols.append(v)
    return np.stack(cols, axis=1)


# ------------------------------------------------------------------ Algorithm 3, Eq. (3.1)
@pytest.mark.parametrize("d,n,r", [(3, 3, 2), (4, 2, 3), (5, 3, 2), (4, [2, 3, 4, 2], [2, 3, 1])])
def test_partial_contractions_equal_definition(d, n, r):
    cores = tiny_tt(10 + d, d, n, r)
    nn = T.modes(cores)
    seed, w = 77, 6
    W = R.partial_contractions_rl(cores, seed, 0, w)
    for k in range(2, d + 1):
        Rk = right_part(cores, k)                               # (r_{k-1}, n_k, ..., n_d)
        # paper's column order for H(X_{k:d}) and Omega_d (KRP) ... (KRP) Omega_k: i_k fastest
        Hk = Rk.transpose([0] + list(range(Rk.ndim - 1, 0, -1))).reshape(Rk.shape[0], -1)
        K = krp_columns(seed, list(range(d, k - 1, -1)), nn, 0, w)
        ref = Hk @ K
        assert np.allclose(W[k], ref, rtol=0, atol=1e-13 * np.abs(ref).max())
        # the same by summing over every mode index explicitly
        letters = "ijklmnop"[: Rk.ndim - 1]
        ops = [omega(seed, m, nn[m - 1], 0, w) for m in range(k, d + 1)]
        expr = "a" + letters + "," + ",".join(f"{c}z" for c in letters) + "->az"
        ref2 = np.einsum(expr, Rk, *ops)
        assert np.allclose(W[k], ref2, rtol=0, atol=1e-13 * np.abs(ref2).max())


def test_partial_contractions_column_chunks_append():
    cores = tiny_tt(3, 5, 4, 3)
    full = R.partial_contractions_rl(cores, 5, 0, 9)
    a = R.partial_contractions_rl(cores, 5, 0, 4)
    b = R.partial_contractions_rl(cores, 5, 4, 9, t=3)
    for k in range(3, 6):
        assert np.allclose(full[k], np.concatenate([a[k], b[k]], axis=1), rtol=0, atol=1e-15)


@pytest.mark.parametrize("d,n,r", [(4, 3, 2), (5, [2, 3, 4, 2, 3], 3), (3, 4, [2, 5])])
def test_percore_contractions_equal_definition(d, n, r):
    """The per-core form (Conclusion, Sec. 5) gives Algorithm 3's W_k: against the explicit
    H(X_{k:d}) times the explicit Kronecker columns, and against the chain itself."""
    cores = tiny_tt(10 + d, d, n, r)
    nn = T.modes(cores)
    W = R.partial_contractions_percore(cores, 31, 2, 9)
    Wc = R.partial_contractions_rl(cores, 31, 2, 9)
    for k in range(2, d + 1):
        Rk = right_part(cores, k)                                       # C order: i_d fastest
        ref = Rk.reshape(Rk.shape[0], -1) @ krp_columns(31, list(range(k, d + 1)), nn, 2, 9)
        assert np.allclose(W[k], ref, rtol=0, atol=1e-13 * np.abs(ref).max())
        assert np.allclose(W[k], Wc[k], rtol=0, atol=1e-13 * np.abs(ref).max())
    Wt = R.partial_contractions_percore(cores, 31, 5, 9, t=3)          # column chunk and t > 2
    for k in range(3, d + 1):
        assert np.allclose(Wt[k], W[k][:, 3:], rtol=0, atol=1e-14 * np.abs(W[k]).max())


def test_planted_percore_transpose_mistake_is_caught(monkeypatch):
    """G_k(:, :, j) applied transposed (a plausible index slip) no longer matches the definition."""
    cores = tiny_tt(14, 4, 3, 3)
    real = np.einsum

    def wrong(spec, *ops, **kw):
        return real("jca,cj->aj" if spec == "jac,cj->aj" else spec, *ops, **kw)

    monkeypatch.setattr(R.np, "einsum", wrong)
    W = R.partial_contractions_percore(cores, 31, 0, 6)
    monkeypatch.setattr(R.np, "einsum", real)
    ref = R.partial_contractions_rl(cores, 31, 0, 6)
    assert not np.allclose(W[2], ref[2], rtol=0, atol=1e-10 * np.abs(ref[2]).max())


def test_planted_krp_order_mistake_is_caught(monkeypatch):
    cores = tiny_tt(4, 4, 3, 2)
    nn = T.modes(cores)

    def wrong(cores, seed, col0, col1, t=2):
        d = len(cores)
        W = {d: T.H(cores[d - 1]) @ omega(seed, d, nn[d - 1], col0, col1)}
        for k in range(d - 1, t - 1, -1):
            om = omega(seed, k, nn[k - 1], col0, col1)
            wn = W[k + 1]
            krp = (wn[:, None, :] * om[None, :, :]).reshape(-1, wn.shape[1])   # (c, i) order: wrong
            W[k] = T.H(cores[k - 1]) @ krp
        return W

    monkeypatch.setattr(R, "partial_contractions_rl", wrong)
    W = R.partial_contractions_rl(cores, 8, 0, 5)
    Rk = right_part(cores, 2)
    Hk = Rk.transpose([0, 3, 2, 1]).reshape(Rk.shape[0], -1)
    ref = Hk @ krp_columns(8, [4, 3, 2], nn, 0, 5)
    assert not np.allclose(W[2], ref, rtol=0, atol=1e-13 * np.abs(ref).max())


# ------------------------------------------------------------------ dense re-implementations
def dense_fixed(cores, ell, seed):
    """Algorithm 4 on the explicit tensor: U_k = (U_{k-1} (x) I) orth((U_{k-1} (x) I)^T X_(1:k) Omega)."""
    X = T.full(cores)
    n = X.shape
    d = len(n)
    r = T.ranks(cores)
    U = np.ones((1, 1))
    ranks = [1]
    for k in range(1, d):
        Xk = X.reshape(int(np.prod(n[:k])), -1)
        B = np.kron(U, np.eye(n[k - 1]))
        lk = min(ell, B.shape[1], r[k], int(np.prod(n[k:])))
        S = B.T @ Xk @ krp_columns(seed, list(range(k + 1, d + 1)), list(n), 0, lk)
        Q, _ = np.linalg.qr(S)
        U = B @ Q
        ranks.append(lk)
    Xk = X.reshape(U.shape[0], -1)
    return (U @ (U.T @ Xk)).reshape(n), ranks + [1]


def dense_adaptive(cores, tol, seed, block, nrmx, f_init=0.1, f_inc=0.05, est_min=0, est_safety=1.0):
    """Algorithm 6 on the explicit tensor (same Omega stream, same block and stopping rules; the
    estimator width max(b_inc, est_min) and the stop at tau / est_safety of reading R16)."""
    X = T.full(cores)
    n = X.shape
    d = len(n)
    tau = tol * nrmx / math.sqrt(d - 1)
    U = np.ones((1, 1))
    ranks, ests = [1], []
    for k in range(1, d):
        Xk = X.reshape(int(np.prod(n[:k])), -1)
        B = np.kron(U, np.eye(n[k - 1]))
        A = B.T @ Xk                                      # = V(Y_k) H(X_{k+1:d}) up to column order
        rbar = min(B.shape[1], T.ranks(cores)[k], int(np.prod(n[k:])))    # readings R4, R14
        om = lambda c0, c1: krp_columns(seed, list(range(k + 1, d + 1)), list(n), c0, c1)
        b0 = R.block_size(rbar, block, f_init)
        Q, _ = np.linalg.qr(A @ om(0, b0))
        bi = R.block_size(rbar, block, f_inc)
        be = max(bi, est_min)
        ek = []
        while Q.shape[1] < rbar:
            c = Q.shape[1]
            S = A @ om(c, c + be)
            S = S - Q @ (Q.T @ S)
            est = np.linalg.norm(S) / math.sqrt(be)
            ek.append(est)
            if not est * est_safety > tau:
                break
            bb = min(bi, rbar - c)
            Qn, _ = np.linalg.qr(S[:, :bb])
            Qn, _ = np.linalg.qr(Qn - Q @ (Q.T @ Qn))
            Q = np.concatenate([Q, Qn], axis=1)
        U = B @ Q
        ranks.append(Q.shape[1])
        ests.append(ek)
    Xk = X.reshape(U.shape[0], -1)
    return (U @ (U.T @ Xk)).reshape(n), ranks + [1], ests


@pytest.mark.parametrize("d,n,r,ell", [(4, 3, 3, 2), (5, 3, 4, 3), (4, 4, 5, 4), (5, [3, 2, 4, 3, 2], 4, 3)])
def test_fixed_equals_dense_definition(d, n, r, ell):
    cores = tiny_tt(20 + d, d, n, r)
    Y, info = R.tt_round_fixed(cores, ell, seed=123)
    ref, ranks = dense_fixed(cores, ell, 123)
    assert info["ranks"] == ranks == T.ranks(Y)
    assert np.allclose(T.full(Y), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert T.left_orth_defect(Y) < 1e-13


def test_fixed_exact_when_sketch_covers_rank():
    x = WL.random_tt(np.random.default_rng(5), 6, 5, 3)
    sumx = WL.block_sum([(0.7, x), (-1.9, x)])           # formal rank 6, true rank 3
    Y, info = R.tt_round_fixed(sumx, 4, seed=9)
    assert T.tt_dist(Y, sumx) <= 1e-13 * T.tt_norm(sumx)
    assert max(info["ranks"]) == 4


def test_fixed_c1_target_rank():
    """C1: fixed rank l = 13 then truncation to 8 (Remark 3.2 pass with rank targets)."""
    x = WL.c1()
    Y, info = R.tt_round_fixed(x.cores, 13, seed=31)
    assert info["ranks"] == [1, 10, 13, 13, 13, 10, 1]         # clamped by l_{k-1} n_k and prod n_j
    assert T.tt_dist(Y, x.cores) <= 1e-13 * x.norm
    Y8 = R.svd_pass_rl(Y, max_rank=8)
    err = T.tt_dist(Y8, x.cores) / x.norm
    # the rank-8 part is exact; the error is the rank-2 noise at 1e-8 ||T||, relative to ||X||
    assert T.ranks(Y8) == [1, 8, 8, 8, 8, 8, 1]
    assert err < 1e-7


@pytest.mark.parametrize("case", [(4, 3, 4, 1e-2, 2, 0, 1.0), (5, 3, 4, 1e-3, 1, 0, 1.0), (5, 4, 5, 1e-6, 2, 0, 1.0),
                                  (4, 3, 6, 1e-8, 0, 0, 1.0), (5, 3, 4, 1e-3, 1, 4, 1.0), (5, 4, 5, 1e-6, 2, 3, 10.0),
                                  (4, 3, 6, 1e-5, 0, 5, 4.0)])
def test_adaptive_equals_dense_definition(case):
    d, n, r, tol, block, est_min, est_safety = case
    rng = np.random.default_rng(40 + d)
    base = WL.random_tt(rng, d, n, max(1, r // 2))
    noise = WL.random_tt(rng, d, n, 2)
    noise[0] = noise[0] * 1e-3
    cores = WL.block_sum([(1.3, base), (0.4, base), (1.0, noise)])
    nrmx = T.tt_norm(cores)
    Y, info = R.tt_round_adaptive(cores, tol, seed=99, block=block, nrmx=nrmx, est_min=est_min, est_safety=est_safety)
    ref, ranks, ests = dense_adaptive(cores, tol, 99, block, nrmx, est_min=est_min, est_safety=est_safety)
    assert info["ranks"] == ranks
    for a, b in zip(info["estimates"], ests):
        # an exactly vanishing residual leaves rounding noise of ~u ||X|| sqrt(entries) on both sides
        assert np.allclose(a, b, rtol=1e-9, atol=1e-14 * nrmx)
    assert np.allclose(T.full(Y), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert T.left_orth_defect(Y) < 1e-13


def test_planted_residual_sign_mistake_is_caught(monkeypatch):
    d, n, r = 4, 3, 4
    rng = np.random.default_rng(44)
    base = WL.random_tt(rng, d, n, 2)
    cores = WL.block_sum([(1.3, base), (0.4, base), (1.0, WL.random_tt(rng, d, n, 2))])
    nrmx = T.tt_norm(cores)

    def wrong(sk, Z, Q, k, b):
        c = Q.shape[1]
        sk.ensure(k, c + b)
        S = Z @ sk.W[k + 1][:, c:c + b]
        return S + Q @ (Q.T @ S)                                # sign error in Eq. (3.5)

    monkeypatch.setattr(R, "residual_sketch", wrong)
    _, info = R.tt_round_adaptive(cores, 1e-3, seed=99, block=1, nrmx=nrmx)
    _, _, ests = dense_adaptive(cores, 1e-3, 99, 1, nrmx)
    same = all(len(a) == len(b) and np.allclose(a, b, rtol=1e-9) for a, b in zip(info["estimates"], ests))
    assert not same


# ------------------------------------------------------------------ Algorithm 1 and Remark 3.2
def tt_svd_lr(X, tau):
    n = X.shape
    cores, C, rp = [], X.reshape(n[0], -1), 1
    for k in range(len(n) - 1):
        C = C.reshape(rp * n[k], -1)
        U, s, Vt = np.linalg.svd(C, full_matrices=False)
        r_new = T.truncation_rank(s, tau)
        cores.append(U[:, :r_new].reshape(rp, n[k], r_new))
        C = s[:r_new, None] * Vt[:r_new]
        rp = r_new
    cores.append(C.reshape(rp, n[-1], 1))
    return cores


def tt_svd_rl(X, tau):
    n = X.shape
    d = len(n)
    cores = [None] * d
    C, rp = X.reshape(-1, n[-1]), 1
    for k in range(d - 1, 0, -1):
        C = C.reshape(-1, n[k] * rp)
        U, s, Vt = np.linalg.svd(C, full_matrices=False)
        r_new = T.truncation_rank(s, tau)
        cores[k] = Vt[:r_new].reshape(r_new, n[k], rp)
        C = U[:, :r_new] * s[:r_new]
        rp = r_new
    cores[0] = C.reshape(1, n[0], rp)
    return cores


@pytest.mark.parametrize("tol", [1e-2, 1e-6, 1e-9])
def test_deterministic_equals_tt_svd_c1(tol):
    x = WL.c1()
    X = T.full(x.cores)
    Y, info = R.tt_round_deterministic(x.cores, tol)
    tau = np.linalg.norm(X) * tol / math.sqrt(x.d - 1)
    ref = tt_svd_lr(X, tau)
    assert info["ranks"] == T.ranks(ref)
    assert abs(info["tau"] - tau) <= 1e-13 * tau
    YF = T.full(Y)
    assert np.linalg.norm(YF - T.full(ref)) <= 1e-12 * np.linalg.norm(X)
    assert np.linalg.norm(YF - X) <= tol * np.linalg.norm(X) * (1 + 1e-10)


def test_svd_pass_rl_equals_rl_tt_svd():
    x = WL.c1()
    Y, _ = R.tt_round_fixed(x.cores, 13, seed=31)          # left-orthonormal, excess rank
    for tau in (1e-3 * x.norm, 1e-9 * x.norm):
        Z = R.svd_pass_rl(Y, tau)
        ref = tt_svd_rl(T.full(Y), tau)
        assert T.ranks(Z) == T.ranks(ref)
        assert np.linalg.norm(T.full(Z) - T.full(ref)) <= 1e-12 * x.norm


def test_truncation_rank_closed_forms():
    s = np.array([4.0, 3.0, 2.0, 1.0])
    assert T.truncation_rank(s, 0.0) == 4
    assert T.truncation_rank(s, 1.0) == 3                 # tail {1} has norm 1 <= 1
    assert T.truncation_rank(s, math.sqrt(5.0)) == 2      # tail {2,1}
    assert T.truncation_rank(s, 5.4) == 1                 # tail {3,2,1} = sqrt(14) = 3.74
    assert T.truncation_rank(s, 100.0) == 1               # never below rank 1
    assert T.truncation_rank(np.array([1.0, 0.0]), 0.0) == 1


# ------------------------------------------------------------------ adaptive invariants
def exact_core_residuals(cores, Y):
    """||(I - Q_k Q_k^T) V(Ytilde_k) H(X_{k+1:d})||_F for each k, explicitly (tiny inputs)."""
    X = T.full(cores)
    n = X.shape
    res = []
    U = np.ones((1, 1))
    for k in range(1, len(n)):
        Xk = X.reshape(int(np.prod(n[:k])), -1)
        B = np.kron(U, np.eye(n[k - 1]))
        A = B.T @ Xk
        Q = T.V(Y[k - 1])
        res.append(np.linalg.norm(A - Q @ (Q.T @ A)))
        U = B @ Q
    return np.array(res)


@pytest.mark.parametrize("tol", [1e-2, 1e-4, 1e-7])
def test_adaptive_error_budget_and_tolerance(tol):
    x = WL.c1(seed=11)
    Y, info = R.tt_round_adaptive(x.cores, tol, seed=5, block=2, nrmx=x.norm)
    res = exact_core_residuals(x.cores, Y)
    err = T.tt_dist(Y, x.cores)
    assert err <= math.sqrt(np.sum(res ** 2)) * (1 + 1e-8) + 1e-15      # Pythagoras over left-orthogonal projections
    assert err <= tol * x.norm                                           # the tolerance, exact norm given
    det, dinfo = R.tt_round_deterministic(x.cores, tol)
    for a, b, rb in zip(info["ranks"], dinfo["ranks"], T.ranks(x.cores)):
        assert b <= a <= rb                                              # never below the optimal ranks
    Z = R.svd_pass_rl(Y, info["tau"] / math.sqrt(2.0))
    assert T.tt_dist(Z, x.cores) <= tol * x.norm


def test_estimator_reading_r16_meets_tol_on_the_operator_applied_vector():
    """Reading R16 on the full operator-applied vector (d = 16, n = 64, formal rank 60, tol 1e-8, the
    paper's block fractions: b_init = 6, b_inc = 3).  Algorithm 6 as printed stops early on every
    seed tried here: its 3-column KRP estimate over up to 15 remaining modes is far below the
    residual (Theorem 3.3 asks for a sample count growing like ln^(d-k)(2/delta)).  Ten estimator
    columns and the stop at tau / 10 keep the exact error within tol; the exact per-core residuals
    (from the right Gram matrices) stay below tau, and the sum-of-squares bound of the error holds."""
    x = WL.c3()
    G = right_grams(x.cores)
    for seed in (3, 7, 11):
        Y0, i0 = R.tt_round_adaptive(x.cores, 1e-8, seed=seed, nrmx=x.norm)
        assert T.tt_dist(Y0, x.cores) > 1e-8 * x.norm                       # the printed rule falls short
        Y, info = R.tt_round_adaptive(x.cores, 1e-8, seed=seed, nrmx=x.norm, est_min=10, est_safety=10.0)
        err = T.tt_dist(Y, x.cores)
        res = core_residuals_via_grams(x.cores, Y, G)
        assert err <= 1e-8 * x.norm
        assert res.max() <= info["tau"]
        assert err <= math.sqrt(np.sum(res ** 2)) * (1 + 1e-6) + 1e-30
        assert all(a >= b for a, b in zip(info["ranks"], i0["ranks"]))        # a later stop, never an earlier one


def right_grams(cores):
    """G_k = H(X_{k:d}) H(X_{k:d})^T (r_{k-1} x r_{k-1}) by right-to-left contraction; G_{d+1} = 1."""
    d = len(cores)
    G = {d + 1: np.ones((1, 1))}
    for k in range(d, 0, -1):
        c = cores[k - 1]
        G[k] = np.einsum("aic,cd,bid->ab", c, G[k + 1], c, optimize=True)
    return G


def core_residuals_via_grams(cores, Y, G):
    """||(I - Q_k Q_k^T) V(Ytilde_k) H(X_{k+1:d})||_F for each k without forming H(X_{k+1:d}):
    with P = (I - Q Q^T) V(Ytilde_k), the squared norm is trace(P G_{k+1} P^T).  Ytilde_k is the
    partially projected core Q_{k-1}^T V(Ytilde_{k-1}) H(X_k)."""
    res = []
    Z = T.V(cores[0])
    for k in range(1, len(cores)):
        Q = T.V(Y[k - 1])
        P = Z - Q @ (Q.T @ Z)
        res.append(math.sqrt(max(float(np.einsum("ij,jk,ik->", P, G[k + 1], P)), 0.0)))
        r1, n1, r2 = cores[k].shape
        Z = ((Q.T @ Z) @ T.H(cores[k])).reshape(Q.shape[1] * n1, r2)
    return np.array(res)


def test_core_residuals_via_grams_equal_the_explicit_ones():
    x = WL.c1(seed=11)
    Y, _ = R.tt_round_adaptive(x.cores, 1e-4, seed=5, block=2, nrmx=x.norm)
    a = core_residuals_via_grams(x.cores, Y, right_grams(x.cores))
    b = exact_core_residuals(x.cores, Y)
    assert np.allclose(a, b, rtol=1e-6, atol=1e-14 * x.norm)


def test_adaptive_c3_operator_applied_vector():
    x = WL.c3(d=6, n=16, r=10)
    Y, info = R.tt_round_adaptive(x.cores, 1e-6, seed=3, nrmx=x.norm)
    assert T.tt_dist(Y, x.cores) <= 1e-6 * x.norm
    assert T.left_orth_defect(Y) < 1e-12
    assert max(info["ranks"]) <= 20


# ------------------------------------------------------------------ estimator theory (Sec. 3.4)
def test_norm_estimate_matches_explicit_krp():
    cores = tiny_tt(8, 4, 3, 3)
    W = R.partial_contractions_rl(cores, 17, 0, 7)
    X1 = T.full(cores).reshape(3, -1)                      # C-order mode-1 unfolding
    K = krp_columns(17, [2, 3, 4], T.modes(cores), 0, 7)   # matching C-order Kronecker columns
    assert math.isclose(R.norm_estimate(cores[0], W[2]), np.linalg.norm(X1 @ K) / math.sqrt(7), rel_tol=1e-12)


@pytest.mark.parametrize("d", [3, 5])
def test_norm_estimator_unbiased(d):
    """Thm 3.3: E[||A Omega||_F^2 / l] = ||A||_F^2 for KRP Gaussian Omega."""
    cores = tiny_tt(60 + d, d, 4, 3)
    nrm2 = T.tt_norm(cores) ** 2
    vals = np.array([R.norm_estimate(cores[0], R.partial_contractions_rl(cores, s, 0, 4)[2]) ** 2
                     for s in range(3000)])
    se = vals.std() / math.sqrt(len(vals))
    assert abs(vals.mean() - nrm2) < 4.5 * se


def test_norm_estimator_spread_grows_with_d():
    """Sec. 3.4 / Fig. 3.2: the spread of the estimate grows with the number of modes."""
    spreads = []
    for d in (3, 6, 9):
        cores = tiny_tt(90 + d, d, 3, 2)
        nrm = T.tt_norm(cores)
        v = np.array([R.norm_estimate(cores[0], R.partial_contractions_rl(cores, s, 0, 8)[2]) / nrm
                      for s in range(400)])
        spreads.append(np.std(np.log(v)))
    assert spreads[0] < spreads[1] < spreads[2]


def test_adaptive_rank_bounded_by_the_right_part():
    """Reading R14: with n_d = 2 and formal rank 6, the last unfolding has rank <= 2, so the last
    rank stays <= 2 even with blocks of 3, and the error is still within tol of the full tensor."""
    rng = np.random.default_rng(12)
    base = WL.random_tt(rng, 4, [4, 3, 3, 2], 3)
    noise = WL.random_tt(rng, 4, [4, 3, 3, 2], 3)
    cores = WL.block_sum([(1.0, base), (0.5, noise)])
    assert T.ranks(cores) == [1, 6, 6, 6, 1]
    X = T.full(cores)
    Y, info = R.tt_round_adaptive(cores, 1e-10, seed=4, block=3, nrmx=float(np.linalg.norm(X)))
    assert info["ranks"][3] <= 2
    assert np.linalg.norm(T.full(Y) - X) <= 1e-10 * np.linalg.norm(X)


# ------------------------------------------------------------------ operator application (Sec. 4.3)
def test_tt_matvec_equals_the_dense_product():
    rng = np.random.default_rng(21)
    d, n = 4, [3, 2, 4, 3]
    p = [1, 2, 3, 2, 1]
    op = [rng.standard_normal((p[k], n[k], n[k], p[k + 1])) for k in range(d)]
    x = WL.random_tt(rng, d, n, 3)
    y = T.tt_matvec(op, x)
    assert T.ranks(y) == [1, 6, 9, 6, 1]
    dense = T.full_operator(op) @ T.full(x).reshape(-1)
    assert np.allclose(T.full(y).reshape(-1), dense, rtol=0, atol=1e-13 * np.abs(dense).max())


def test_laplacian_operator_is_the_kronecker_sum():
    """The rank-2 TT operator of the operator-applied workload is sum_m I x .. x L x .. x I with
    L = tridiag(-1, 2, -1): its dense matrix built term by term with numpy.kron."""
    d, n = 4, 5
    op = WL.laplace_tt_operator(d, n)
    L = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    ref = np.zeros((n ** d, n ** d))
    for m in range(d):
        term = np.ones((1, 1))
        for k in range(d):
            term = np.kron(term, L if k == m else np.eye(n))
        ref += term
    assert np.array_equal(T.full_operator(op), ref)


def test_adaptive_matvec_rounds_the_product():
    op = WL.laplace_tt_operator(5, 6)              # y = A x, formal rank 8
    rng = np.random.default_rng(4)
    xv = WL.random_tt(rng, 5, 6, 4)
    Y, info = R.tt_round_adaptive_matvec(op, xv, 1e-10, seed=3, block=2)
    dense = T.full_operator(op) @ T.full(xv).reshape(-1)
    assert np.linalg.norm(T.full(Y).reshape(-1) - dense) <= 1e-10 * np.linalg.norm(dense) * (1 + 1e-9)
