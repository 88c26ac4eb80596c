"""Tensor-train utilities for the CPU oracle (FP64, numpy).

TEST INFRASTRUCTURE ONLY: part of the oracle; only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may use it.

A TT tensor is a list of cores X_k in R^{r_{k-1} x n_k x r_k}, r_0 = r_d = 1 (Sec. 2.2,
Eq. (2.1)).  The unfoldings follow Sec. 2.2: the horizontal unfolding H(X_k) is
r_{k-1} x (n_k r_k) and the vertical unfolding V(X_k) is (r_{k-1} n_k) x r_k.  With cores
stored row-major as [a][i][c], both are plain reshapes: V has rows (a, i) with i fastest,
H has columns (i, c) with c fastest.
"""
from __future__ import annotations

import numpy as np


def V(core: np.ndarray) -> np.ndarray:
    """Vertical unfolding V(X_k) in R^{(r_{k-1} n_k) x r_k} (Sec. 2.2)."""
    r0, n, r1 = core.shape
    return core.reshape(r0 * n, r1)


def H(core: np.ndarray) -> np.ndarray:
    """Horizontal unfolding H(X_k) in R^{r_{k-1} x (n_k r_k)} (Sec. 2.2)."""
    r0, n, r1 = core.shape
    return core.reshape(r0, n * r1)


def ranks(cores) -> list[int]:
    return [cores[0].shape[0]] + [c.shape[2] for c in cores]


def modes(cores) -> list[int]:
    return [c.shape[1] for c in cores]


def full(cores) -> np.ndarray:
    """The full tensor X(i_1..i_d) = X_1(i_1,:) X_2(:,i_2,:) ... X_d(:,i_d) (Eq. (2.1)); small inputs only."""
    t = cores[0].reshape(cores[0].shape[1], cores[0].shape[2])
    shape = [cores[0].shape[1]]
    for c in cores[1:]:
        r0, n, r1 = c.shape
        t = t.reshape(-1, r0) @ c.reshape(r0, n * r1)
        shape.append(n)
    return t.reshape(shape)


def tt_sum(x, y, alpha: float = 1.0, beta: float = 1.0):
    """Formal sum alpha*x + beta*y: ranks add, middle cores block-diagonal (Sec. 4.3, App. D)."""
    d = len(x)
    out = []
    for k in range(d):
        a, b = x[k], y[k]
        if d == 1:
            out.append(alpha * a + beta * b)
        elif k == 0:
            out.append(np.concatenate([alpha * a, beta * b], axis=2))
        elif k == d - 1:
            out.append(np.concatenate([a, b], axis=0))
        else:
            r0 = a.shape[0] + b.shape[0]
            r1 = a.shape[2] + b.shape[2]
            c = np.zeros((r0, a.shape[1], r1))
            c[: a.shape[0], :, : a.shape[2]] = a
            c[a.shape[0]:, :, a.shape[2]:] = b
            out.append(c)
    return out


def orthogonalize_rl(cores):
    """Right-to-left orthogonalization (Sec. 2.3): QR of H(X_k)^T, R^T pushed into core k-1.

    Returns an equivalent TT whose cores 2..d have orthonormal rows in H(.).  Rank is kept
    (min with the QR's column count), so the represented tensor is unchanged.
    """
    cores = [c.copy() for c in cores]
    for k in range(len(cores) - 1, 0, -1):
        r0, n, r1 = cores[k].shape
        q, r = np.linalg.qr(H(cores[k]).T)           # (n r1) x m, m x r0
        m = q.shape[1]
        cores[k] = q.T.reshape(m, n, r1)
        p0, pn, _ = cores[k - 1].shape
        cores[k - 1] = (V(cores[k - 1]) @ r.T).reshape(p0, pn, m)
    return cores


def tt_norm(cores) -> float:
    """||X|| computed stably: orthogonalize right to left, then the Frobenius norm of core 1."""
    return float(np.linalg.norm(orthogonalize_rl(cores)[0]))


def tt_dist(x, y) -> float:
    """||x - y|| through the formal difference, computed stably (no inner-product cancellation)."""
    return tt_norm(tt_sum(x, y, 1.0, -1.0))


def tt_inner(x, y) -> float:
    """<x, y> by the left-to-right Gram contraction (used only where cancellation is harmless)."""
    g = np.ones((1, 1))
    for a, b in zip(x, y):
        # g_{c,c'} = sum_{a,a',i} g_{a,a'} x(a,i,c) y(a',i,c')
        t = np.einsum("ab,aic->bic", g, a)
        g = np.einsum("bic,bid->cd", t, b)
    return float(g[0, 0])


def tt_matvec(op, x):
    """y = A x for a TT operator A and a TT vector x (the operator application of TT-GMRES,
    Sec. 4.3; the MPO-MPS product of the Introduction and Conclusion).

    Operator cores are A_k in R^{p_{k-1} x n_k x n_k x p_k}, [a][i][j][g] with i the output and
    j the input index, so that A(i_1..i_d; j_1..j_d) = A_1(i_1, j_1) ... A_d(i_d, j_d).  The
    product's cores are y_k((a, b), i, (g, c)) = sum_j A_k(a, i, j, g) x_k(b, j, c), with the
    operator's bond index the slower one in each bond of y (ranks p_k r_k).
    """
    out = []
    for A, X in zip(op, x):
        p0, n, m, p1 = A.shape
        r0, m2, r1 = X.shape
        if m != m2:
            raise ValueError("operator input size must match the vector's mode size")
        y = np.einsum("aijg,bjc->abigc", A, X).reshape(p0 * r0, n, p1 * r1)
        out.append(np.ascontiguousarray(y))
    return out


def full_operator(op) -> np.ndarray:
    """The N x N matrix of a TT operator (N = prod n_k), rows (i_1..i_d) and columns (j_1..j_d) in
    C order; small operators only."""
    M = np.ones((1, 1, 1))                    # (rows, cols, bond)
    for A in op:
        p0, n, m, p1 = A.shape
        M = np.einsum("rca,aijg->ricjg", M, A).reshape(M.shape[0] * n, M.shape[1] * m, p1)
    return M[:, :, 0]


def truncation_rank(sigma: np.ndarray, tau: float) -> int:
    """Smallest r' >= 1 whose discarded tail sqrt(sum_{i>r'} sigma_i^2) is <= tau.

    This is the rank rule of the tau-truncated SVD in Algorithm 1 (line "SVD(R, tau)"): a
    Frobenius-norm tail bound per core.  A tail exactly equal to tau is accepted.
    """
    s2 = np.asarray(sigma, dtype=np.float64) ** 2
    tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])   # tail[j] = sum_{i>=j} s_i^2
    for rp in range(1, len(s2) + 1):
        if np.sqrt(tail[rp]) <= tau:
            return rp
    return len(s2)


def left_orth_defect(cores) -> float:
    """max_k ||V(Y_k)^T V(Y_k) - I||_max over k < d (0 for an exactly left-orthogonal TT)."""
    worst = 0.0
    for c in cores[:-1]:
        v = V(c)
        worst = max(worst, float(np.abs(v.T @ v - np.eye(v.shape[1])).max()))
    return worst
