"""TT-rounding algorithms of the paper, written step by step in FP64 (numpy / LAPACK).

TEST INFRASTRUCTURE ONLY: this is the CPU oracle the CUDA path is checked against.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.
It shares no code with the CUDA path; both sides only share the seeded input generators.

Contents (paper sections / algorithms):
* ``partial_contractions_rl``  - Algorithm 3 (KRP-PartialContractionsRL), Eqs. (3.1)-(3.3)
* ``partial_contractions_percore`` - the same W_k through the per-core contractions with Omega that
                                 the Conclusion (Sec. 5) notes can be done in parallel over the cores
* ``tt_round_fixed``           - Algorithm 4 (fixed-rank Rand-Orth with KRP), Sec. 3.2
* ``residual_sketch``          - Algorithm 5 (GenerateResidualSketch), Eqs. (3.4)-(3.5)
* ``tt_round_adaptive``        - Algorithm 6 (adaptive-rank Rand-Orth with KRP), Sec. 3.3
* ``norm_estimate``            - Remark 3.1, Eq. (3.6)
* ``svd_pass_rl``              - Remark 3.2 (the "Adap-R" compression pass, right to left)
* ``partial_contractions_rl_sum`` / ``tt_round_adaptive_sum``
                               - Remark 3.3 and Appendix D (the algorithms for a sum of TT
                                 tensors): every summand sketched with the shared Omega, the
                                 sum never formed
* ``tt_round_deterministic``   - Algorithm 1 (TT-Rounding, Oseledets)
* ``tt_round_adaptive_matvec`` - Algorithm 6 applied to y = A x (the operator application of
                                 TT-GMRES, Sec. 4.3), from its definition: y formed explicitly

Library primitives used as single steps: matrix product, Householder QR (numpy.linalg.qr)
and the SVD (numpy.linalg.svd).  Readings of points where the paper is silent or garbled:
  R1  W_k(a, j) = sum_{i,c} X_k(a,i,c) W_{k+1}(c,j) Omega_k(i,j): the KRP rows are ordered
      (i, c) with c fastest, matching the columns of H(X_k) (Eq. (3.3) read by index).
  R2  Omega_k(i, j) depends only on (seed, k, i, j) for a global column index j; extending W
      (Algorithm 5) appends columns col(W)..col(Q)+b-1 of that one stream (the printed size
      "n_j x (b - col(W_{k+1}))" is read as col(Q) + b - col(W_{k+1}) columns).
  R3  Block sizes: block > 0 gives b_init = b_inc = block; otherwise b = ceil(f * rbar_k)
      with f_init, f_inc as in Sec. 3.3 (a 1e-9 guard makes ceil exact for products like
      30*0.1); every block is clamped to [1, rbar_k].
  R4  The adaptive loop also stops once col(Q_k) = rbar_k (stated in the text of Sec. 3.3,
      missing from the while condition of Algorithm 6); the last block is clamped to
      rbar_k - col(Q_k).
  R5  Initial sketch width w0 = ceil(f_init * max_k r_k) (Algorithm 6, first line), or
      ``block`` in block mode; Eq. (3.6) divides by w0.
  R6  Fixed rank: l_k is clamped to min(l_k, l_{k-1} n_k, r_k, prod_{j>k} n_j) so that the
      sketch has no more columns than the rank it can have.
  R7  The tau-truncated SVD keeps the smallest rank whose discarded tail is <= tau (see
      ``oracle.tt.truncation_rank``); the Adap-R pass reuses tau (Remark 3.2) unless
      ``adap_r_tau`` is given.
  R12 Sum of TTs, block sizes: block > 0 gives b_init = b_inc = block as in R3; otherwise the
      appendix's b_init = max_i r_k^(i) (clamped to rbar_k) and b_inc = ceil(f_inc * rbar_k).
      The norm estimate uses the first w0 columns of the stacked W_2, w0 = block in block mode,
      else the appendix's sketch width max_{i,k} r_k^(i).
  R14 The largest rank of core k, rbar_k, is also bounded by the right part: V(Y_k) H(X_{k+1:d})
      has rank at most prod_{j>k} n_j, so rbar_k = min(rows, cols of V(Y_k), prod_{j>k} n_j) (the
      adaptive counterpart of R6).  Without it an initial block wider than that rank (possible
      with the appendix's b_init = max_i r_k^(i) at the last cores) would sketch an exactly
      rank-deficient matrix.
  R15 A zero tensor: when ||X|| (given, or estimated by Eq. (3.6)) is 0, the rounding is the zero
      TT of ranks 1 (there is no subspace to sketch; tau would be 0).  The estimate is 0 only for
      X = 0, with probability one.
  R16 Estimator width and safety factor (Sec. 3.4, Theorem 3.3 and its Corollary): the residual
      estimate of Algorithm 6 may use more KRP columns than the block it appends, and the stop may
      compare it with tau / beta.  With ``est_min`` = p the residual sketch has max(b_inc, p) columns
      (Eqs. (3.4)-(3.5)) and est = ||S||_F / sqrt(max(b_inc, p)); the new directions still come from
      its first min(b_inc, rbar - col(Q)) columns, and the next residual sketch starts after them.
      With ``est_safety`` = beta the loop stops when est <= tau / beta.  The Corollary bounds the
      estimate from below by ||A_k||_F / sqrt(zeta) with a sample count growing like ln^(d-k)(2/delta):
      few columns and many remaining modes (the operator-applied vector, d = 16, b_inc = 3) leave the
      estimate far below the residual, and the oracle then ends above tol.  Defaults p = 0, beta = 1
      are Algorithm 6 as printed.
  R13 Sum of TTs, the last core: the appendix writes H(Y_{k+1}) = [Y^(1) ... Y^(s)] for every k.
      For k + 1 = d the summands' last cores share the right bond 1 (the formal sum stacks them
      vertically), so H(Y_d) = sum_i M^(i) H(X_d^(i)); for k + 1 < d the blocks sit side by side
      in the concatenated right bond, ordered by summand.
"""
from __future__ import annotations

import math

import numpy as np

from .philox import omega
from .tt import H, V, modes, orthogonalize_rl, ranks, truncation_rank, tt_matvec


def block_size(rbar: int, block: int, frac: float) -> int:
    """Reading R3: block > 0 wins, else ceil(frac * rbar); clamped to [1, rbar]."""
    b = block if block > 0 else int(math.ceil(rbar * frac - 1e-9))
    return max(1, min(rbar, b))


def partial_contractions_rl(cores, seed: int, col0: int, col1: int, t: int = 2):
    """Algorithm 3 on sketch columns [col0, col1): {W_k(:, col0:col1)} for k = d..t (1-based k).

    W_d = H(X_d) Omega_d and W_k = H(X_k) [W_{k+1} (KRP) Omega_k]   (Eqs. (3.1)-(3.3), R1).
    """
    d = len(cores)
    n = modes(cores)
    W = {}
    W[d] = H(cores[d - 1]) @ omega(seed, d, n[d - 1], col0, col1)
    for k in range(d - 1, t - 1, -1):
        om = omega(seed, k, n[k - 1], col0, col1)                 # n_k x w
        wn = W[k + 1]                                              # r_k x w
        krp = (om[:, None, :] * wn[None, :, :]).reshape(-1, wn.shape[1])   # rows (i, c), c fastest
        W[k] = H(cores[k - 1]) @ krp
    return W


def partial_contractions_percore(cores, seed: int, col0: int, col1: int, t: int = 2):
    """Algorithm 3's W_k on sketch columns [col0, col1) for k = d..t, from per-core pieces.

    Each core is contracted with its own Gaussian block first, independently of the others (the
    parallelism over cores noted in the Conclusion, Sec. 5):
        G_k(:, :, j) = sum_i X_k(:, i, :) Omega_k(i, j)            (r_{k-1} x r_k for each column j)
    and the right-to-left dependency is left to one small matrix-vector product per core and column:
        W_d(:, j) = G_d(:, 0, j),   W_k(:, j) = G_k(:, :, j) W_{k+1}(:, j).
    By Eq. (3.3) read by index (R1), W_k(a, j) = sum_c [sum_i X_k(a,i,c) Omega_k(i,j)] W_{k+1}(c, j).
    """
    d = len(cores)
    n = modes(cores)
    G = {k: np.einsum("aic,ij->jac", cores[k - 1], omega(seed, k, n[k - 1], col0, col1))
         for k in range(t, d + 1)}                                 # G[k][j] = G_k(:, :, j)
    W = {d: G[d][:, :, 0].T.copy()}                                # r_d = 1
    for k in range(d - 1, t - 1, -1):
        W[k] = np.einsum("jac,cj->aj", G[k], W[k + 1])
    return W


def norm_estimate(core1: np.ndarray, W2: np.ndarray) -> float:
    """Remark 3.1, Eq. (3.6): ||X|| ~ ||V(X_1) W_2||_F / sqrt(#columns of W_2)."""
    return float(np.linalg.norm(V(core1) @ W2) / math.sqrt(W2.shape[1]))


def tt_round_fixed(cores, ell, seed: int):
    """Algorithm 4: fixed-rank randomize-then-orthogonalize with KRP sketches.

    ``ell`` is one target rank or a list (l_1..l_{d-1}).  Returns (Y cores, info).
    """
    d = len(cores)
    r, n = ranks(cores), modes(cores)
    ell_k = [int(ell)] * (d - 1) if np.isscalar(ell) else [int(v) for v in ell]
    lmax = max(ell_k)
    W = partial_contractions_rl(cores, seed, 0, lmax)              # line: {W_k} = KRP-PartialContractionsRL
    Y = [None] * d
    Yk = cores[0].copy()                                           # Y_1 = X_1
    out_ranks = [1]
    for k in range(1, d):                                          # paper k = 1..d-1
        Z = V(Yk)                                                  # (l_{k-1} n_k) x r_k
        right = int(np.prod(n[k:]))
        lk = min(ell_k[k - 1], Z.shape[0], Z.shape[1], right)      # R6
        S = Z @ W[k + 1][:, :lk]                                   # S_k = V(Y_k) W_{k+1}(:, 1:l_k)
        Q, _ = np.linalg.qr(S)                                     # thin QR
        M = Q.T @ Z                                                # M_k = Q_k^T V(Y_k)
        Y[k - 1] = Q.reshape(out_ranks[-1], n[k - 1], lk)          # V(Y_k) = Q_k
        Yk = (M @ H(cores[k])).reshape(lk, n[k], r[k + 1])         # H(Y_{k+1}) = M_k H(X_{k+1})
        out_ranks.append(lk)
    Y[d - 1] = Yk
    out_ranks.append(1)
    return Y, {"ranks": out_ranks, "width": lmax}


class _Sketches:
    """The growing partial contractions W_{k+1..d} of Algorithm 6 (all share one width).

    ``rl`` computes them for columns [c0, c1): Algorithm 3 for one TT, or its per-summand form
    for a sum of TTs (``cores`` is then the list of summands).
    """

    def __init__(self, cores, seed: int, w0: int, rl=None):
        self.cores, self.seed = cores, seed
        self.rl = partial_contractions_rl if rl is None else rl
        self.W = self.rl(cores, seed, 0, w0)
        self.width = w0
        self.extensions = 0

    def ensure(self, k: int, need: int):
        """Algorithm 5, first branch: if col(W_{k+1}) < need, append columns for j = k+1..d (R2)."""
        if self.width >= need:
            return
        new = self.rl(self.cores, self.seed, self.width, need, t=k + 1)
        for j, wj in new.items():
            self.W[j] = np.concatenate([self.W[j], wj], axis=1)
        self.width = need
        self.extensions += 1


def residual_sketch(sk: _Sketches, Z: np.ndarray, Q: np.ndarray, k: int, b: int) -> np.ndarray:
    """Algorithm 5 (GenerateResidualSketch): S = Z W_{k+1}(:, col(Q)+1 : col(Q)+b), then S - Q(Q^T S)."""
    c = Q.shape[1]
    sk.ensure(k, c + b)
    S = Z @ sk.W[k + 1][:, c:c + b]                                # Eq. (3.4)
    return S - Q @ (Q.T @ S)                                       # Eq. (3.5)


def _zero_tt(n) -> list:
    """The zero TT of ranks 1 with mode sizes n (reading R15)."""
    return [np.zeros((1, int(v), 1)) for v in n]


def _zero_result(n, nrmx, w0, width, extensions):
    d = len(n)
    return _zero_tt(n), {"ranks": [1] * (d + 1), "tau": 0.0, "nrmx": nrmx, "estimates": [[] for _ in range(d - 1)],
                         "width": width, "extensions": extensions, "w0": w0}


def right_bound(n, k: int) -> int:
    """prod_{j>k} n_j (1-based k), capped well above any rank (reading R14)."""
    p = 1
    for v in n[k:]:
        p = min(p * int(v), 1 << 62)
    return p


def tt_round_adaptive(cores, tol: float, seed: int, block: int = 0, f_init: float = 0.1,
                      f_inc: float = 0.05, nrmx: float | None = None, adap_r: bool = False,
                      adap_r_tau: float | None = None, est_min: int = 0, est_safety: float = 1.0):
    """Algorithm 6: adaptive-rank randomize-then-orthogonalize with KRP sketches.

    ``nrmx`` is ||X|| if known; otherwise Eq. (3.6) estimates it (Remark 3.1).  ``adap_r``
    appends the right-to-left compression pass of Remark 3.2.  ``est_min`` and ``est_safety``
    are the estimator width and safety factor of reading R16.  Returns (Y cores, info).
    """
    d = len(cores)
    r, n = ranks(cores), modes(cores)
    w0 = block if block > 0 else int(math.ceil(max(r[1:d]) * f_init - 1e-9))   # R5
    w0 = max(1, w0)
    sk = _Sketches(cores, seed, w0)                                # Omega_2..Omega_d, W_2..W_d
    if nrmx is None:
        nrmx = norm_estimate(cores[0], sk.W[2][:, :w0])
    if nrmx == 0.0:                                                # R15
        return _zero_result(n, nrmx, w0, sk.width, sk.extensions)
    tau = tol * nrmx / math.sqrt(d - 1)
    Y = [None] * d
    Yk = cores[0].copy()                                           # Y_1 = X_1
    out_ranks, ests = [1], []
    for k in range(1, d):
        Z = V(Yk)
        rbar = min(min(Z.shape), right_bound(n, k))                # R4, R14
        b_init = block_size(rbar, block, f_init)
        sk.ensure(k, b_init)
        S = Z @ sk.W[k + 1][:, :b_init]                            # phase 1 sketch
        Q, _ = np.linalg.qr(S)
        Hn = (Q.T @ Z) @ H(cores[k])                               # H(Y_{k+1}) = M_k H(X_{k+1})
        b_inc = block_size(rbar, block, f_inc)
        b_est = max(b_inc, est_min)                                # R16: estimator columns
        est_k = []
        while Q.shape[1] < rbar:                                   # R4
            S = residual_sketch(sk, Z, Q, k, b_est)
            est = float(np.linalg.norm(S) / math.sqrt(b_est))
            est_k.append(est)
            if not est > tau / est_safety:                         # R16: tau / beta
                break
            bb = min(b_inc, rbar - Q.shape[1])                     # R4: last block clamped
            Qn, _ = np.linalg.qr(S[:, :bb])
            Qn, _ = np.linalg.qr(Qn - Q @ (Q.T @ Qn))              # re-orthogonalization
            Q = np.concatenate([Q, Qn], axis=1)
            Hn = np.concatenate([Hn, (Qn.T @ Z) @ H(cores[k])], axis=0)   # append rows
        lk = Q.shape[1]
        Y[k - 1] = Q.reshape(out_ranks[-1], n[k - 1], lk)          # V(Y_k) = Q_k
        Yk = Hn.reshape(lk, n[k], r[k + 1])
        out_ranks.append(lk)
        ests.append(est_k)
    Y[d - 1] = Yk
    out_ranks.append(1)
    info = {"ranks": out_ranks, "tau": tau, "nrmx": nrmx, "estimates": ests,
            "width": sk.width, "extensions": sk.extensions, "w0": w0}
    if adap_r:
        Y = svd_pass_rl(Y, tau if adap_r_tau is None else adap_r_tau)
        info["ranks_before_adap_r"] = out_ranks
        info["ranks"] = ranks(Y)
    return Y, info


def _check_summands(summands):
    if len(summands) < 1:
        raise ValueError("at least one summand")
    d = len(summands[0])
    n = modes(summands[0])
    for x in summands:
        if len(x) != d or modes(x) != n:
            raise ValueError("summands must share d and the mode sizes")
        r = ranks(x)
        if r[0] != 1 or r[d] != 1:
            raise ValueError("summand boundary ranks must be 1")
    return d, n


def partial_contractions_rl_sum(summands, seed: int, col0: int, col1: int, t: int = 2):
    """Algorithm 3 on every summand with the same Omega, stacked by rows (Remark 3.3).

    W_k = [W_k^(1); ...; W_k^(s)]: the sketch of the sum is the sum of the summands' sketches, and
    stacked, these are the partial contractions of the block-diagonal formal sum.
    """
    parts = [partial_contractions_rl(x, seed, col0, col1, t) for x in summands]
    return {k: np.concatenate([p[k] for p in parts], axis=0) for k in parts[0]}


def project_summands(Mq: np.ndarray, summands, off, k: int) -> list:
    """Rows of H(Y_{k+1}) for the directions Mq = Q^T V(Y_k), one block per summand (Appendix D):
    [M^(1) ... M^(s)] = Mq split at the bond-k offsets, block i = M^(i) H(X_{k+1}^(i))."""
    return [Mq[:, off[k][i]:off[k][i + 1]] @ H(x[k]) for i, x in enumerate(summands)]


def next_core_of_sum(parts, lk: int, n_next: int, right_ranks, last: bool) -> np.ndarray:
    """H(Y_{k+1}) from the summands' blocks: side by side in the concatenated right bond, or at the
    last core (shared right bond 1) their sum (reading R13)."""
    if last:
        return sum(parts).reshape(lk, n_next, 1)
    return np.concatenate([p.reshape(lk, n_next, rr) for p, rr in zip(parts, right_ranks)], axis=2)


def tt_round_adaptive_sum(summands, tol: float, seed: int, block: int = 0, f_init: float = 0.1,
                          f_inc: float = 0.05, nrmx: float | None = None, adap_r: bool = False,
                          adap_r_tau: float | None = None, est_min: int = 0, est_safety: float = 1.0):
    """Adaptive-rank rounding of X = X^(1) + ... + X^(s) without forming the formal sum
    (Appendix D: the sum forms of Algorithms 5 and 6; readings R12, R13).

    Y_1 = [X_1^(1) ... X_1^(s)] (first cores side by side); at core k the sketch is
    V(Y_k) [W_{k+1}^(1); ...; W_{k+1}^(s)], and the next core is projected summand by summand,
    M^(i) H(X_{k+1}^(i)) with [M^(1) ... M^(s)] = Q_k^T V(Y_k).  ``f_init`` is unused (R12);
    ``est_min`` and ``est_safety`` as in ``tt_round_adaptive`` (R16).  Returns (Y cores, info).
    """
    d, n = _check_summands(summands)
    rs = [ranks(x) for x in summands]
    off = [np.cumsum([0] + [r[k] for r in rs]).tolist() for k in range(d + 1)]   # bond-k block offsets
    rmax_part = max(max(r[1:d]) for r in rs)
    w0 = block if block > 0 else rmax_part                         # R12
    w0 = max(1, w0)
    sk = _Sketches(summands, seed, w0, rl=partial_contractions_rl_sum)
    Yk = np.concatenate([x[0] for x in summands], axis=2)          # Y_1 = [X_1^(1) ... X_1^(s)]
    if nrmx is None:
        nrmx = norm_estimate(Yk, sk.W[2][:, :w0])
    if nrmx == 0.0:                                                # R15
        Y, info = _zero_result(n, nrmx, w0, sk.width, sk.extensions)
        info.update({"b_init": [], "formal_ranks": [1] + [off[k][-1] for k in range(1, d)] + [1]})
        return Y, info
    tau = tol * nrmx / math.sqrt(d - 1)
    Y = [None] * d
    out_ranks, ests, b_inits = [1], [], []

    for k in range(1, d):
        Z = V(Yk)                                                  # (l_{k-1} n_k) x (sum_i r_k^(i))
        rbar = min(min(Z.shape), right_bound(n, k))                # R4, R14
        b_init = block_size(rbar, block, f_init) if block > 0 else min(rbar, max(r[k] for r in rs))
        b_inits.append(b_init)
        sk.ensure(k, b_init)
        S = Z @ sk.W[k + 1][:, :b_init]
        Q, _ = np.linalg.qr(S)
        parts = project_summands(Q.T @ Z, summands, off, k)
        b_inc = block_size(rbar, block, f_inc)
        b_est = max(b_inc, est_min)                                # R16
        est_k = []
        while Q.shape[1] < rbar:                                   # R4
            S = residual_sketch(sk, Z, Q, k, b_est)                # stacked W: the sum form of Alg. 5
            est = float(np.linalg.norm(S) / math.sqrt(b_est))
            est_k.append(est)
            if not est > tau / est_safety:                         # R16
                break
            bb = min(b_inc, rbar - Q.shape[1])
            Qn, _ = np.linalg.qr(S[:, :bb])
            Qn, _ = np.linalg.qr(Qn - Q @ (Q.T @ Qn))              # re-orthogonalization
            Q = np.concatenate([Q, Qn], axis=1)
            parts = [np.concatenate([p, q], axis=0) for p, q in zip(parts, project_summands(Qn.T @ Z, summands, off, k))]
        lk = Q.shape[1]
        Y[k - 1] = Q.reshape(out_ranks[-1], n[k - 1], lk)
        Yk = next_core_of_sum(parts, lk, n[k], [r[k + 1] for r in rs], last=(k + 1 == d))
        out_ranks.append(lk)
        ests.append(est_k)
    Y[d - 1] = Yk
    out_ranks.append(1)
    info = {"ranks": out_ranks, "tau": tau, "nrmx": nrmx, "estimates": ests, "width": sk.width,
            "extensions": sk.extensions, "w0": w0, "b_init": b_inits,
            "formal_ranks": [1] + [off[k][-1] for k in range(1, d)] + [1]}
    if adap_r:
        Y = svd_pass_rl(Y, tau if adap_r_tau is None else adap_r_tau)
        info["ranks_before_adap_r"] = out_ranks
        info["ranks"] = ranks(Y)
    return Y, info


def svd_pass_rl(cores, tau: float | None = None, max_rank=None):
    """Remark 3.2: right-to-left truncation of a left-orthonormal TT (k = d..2).

    For each k: [Q, R] = QR(H(Y_k)^T); [U, s, Vt] = SVD(R^T) truncated at ``tau`` (R7) and/or
    at ``max_rank``; H(Y_k) = Vt Q^T (orthonormal rows); V(Y_{k-1}) = V(Y_{k-1}) U diag(s).
    """
    Y = [c.copy() for c in cores]
    d = len(Y)
    for k in range(d - 1, 0, -1):
        r0, nk, r1 = Y[k].shape
        Q, R = np.linalg.qr(H(Y[k]).T)                             # (n r1) x m, m x r0
        U, s, Vt = np.linalg.svd(R.T, full_matrices=False)        # r0 x p, p, p x m
        rp = len(s) if tau is None else truncation_rank(s, tau)
        if max_rank is not None:
            mr = max_rank if np.isscalar(max_rank) else max_rank[k - 1]
            rp = min(rp, int(mr))
        Y[k] = (Vt[:rp] @ Q.T).reshape(rp, nk, r1)
        p0, pn, _ = Y[k - 1].shape
        Y[k - 1] = (V(Y[k - 1]) @ (U[:, :rp] * s[:rp])).reshape(p0, pn, rp)
    return Y


def tt_round_deterministic(cores, tol: float):
    """Algorithm 1 (TT-Rounding): orthogonalize right to left, then tau-truncated SVDs left to right."""
    d = len(cores)
    Y = orthogonalize_rl(cores)                                    # OrthogonalizeRL
    tau = float(np.linalg.norm(Y[0])) * tol / math.sqrt(d - 1)     # tau = ||Y_1|| eps / sqrt(d-1)
    for k in range(d - 1):
        r0, nk, r1 = Y[k].shape
        Q, R = np.linalg.qr(V(Y[k]))                               # [V(Y_k), R] = QR(V(Y_k))
        U, s, Vt = np.linalg.svd(R, full_matrices=False)
        rp = truncation_rank(s, tau)
        Y[k] = (Q @ U[:, :rp]).reshape(r0, nk, rp)                 # V(Y_k) = V(Y_k) U
        q0, qn, q1 = Y[k + 1].shape
        Y[k + 1] = ((s[:rp, None] * Vt[:rp]) @ H(Y[k + 1])).reshape(rp, qn, q1)   # H(Y_{k+1}) = S V^T H(Y_{k+1})
    return Y, {"ranks": ranks(Y), "tau": tau}


def tt_round_adaptive_matvec(op, x, tol: float, seed: int, **kw):
    """Algorithm 6 on y = A x (Sec. 4.3: the rounding after an operator application in TT-GMRES):
    the product formed by its definition (``oracle.tt.tt_matvec``), then ``tt_round_adaptive`` with
    the same arguments.  The fused GPU form, which never forms y's cores in its right-to-left
    pass, must agree with this up to rounding."""
    return tt_round_adaptive(tt_matvec(op, x), tol, seed, **kw)
