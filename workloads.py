"""Seeded synthetic TT inputs shaped like the paper's workloads.

This module only builds inputs.  It holds none of the rounding method's arithmetic, imports
neither the oracle nor the CUDA package, and is the one piece of code both sides share.

Workloads (the paper's Sec. 4.1 synthetic construction X = sum of scaled random TTs plus a
small random perturbation, and an operator-applied TT vector as in the TT-GMRES experiments
of Sec. 4.3):

* ``c1`` - 3 scaled copies of one random TT (d=6, n=10, rank 8) + rank-2 noise at 1e-8: formal rank 26.
* ``c2`` - 4 scaled copies of one random TT (d=20, n=50, rank 50) + rank-10 noise at 1e-7: formal rank 210.
* ``c3`` - y = A x, A the rank-2 TT operator of sum_m I x..x L x..x I with L = tridiag(-1, 2, -1)
           (d=16, n=64), x a rank-30 TT with bond weights 2^{-(i-1)}: formal rank 60.
* ``c4`` - a stream of random formal sums (sizes, ranks and tolerances drawn from a seed).
* ``c5`` - 4 scaled copies of a random TT (d=50, n=100, rank 200) + rank-10 noise at 1e-8: formal rank 810.

The sums (c1, c2, c5) also come as their list of summands (``TTInput.summands``: the scaled
copies, whose cores after the first are the same arrays, and the noise TT), the input of the
sum-of-TTs rounding that never forms the block-diagonal formal sum.

Core entries of random TTs are iid N(0, 1) / sqrt(n * r).  Copy coefficients are N(0, 1),
redrawn while |sum c| < 0.1 so the sum is not nearly cancelled.  The noise TT is scaled so
that ||noise|| = eta * ||T||.  Every generator also returns the exact input norm ||X||
(from TT inner products of the small summands), which the adaptive algorithm may take as
``nrmx``.  Cores are float64, C-contiguous, shape (r_{k-1}, n_k, r_k).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class TTInput:
    name: str
    cores: list
    norm: float                    # exact ||X||
    meta: dict = field(default_factory=dict)
    summands: list | None = None   # the same X as a list of TTs (cores of each), when it is a sum

    @property
    def d(self) -> int:
        return len(self.cores)

    @property
    def ranks(self) -> list:
        return [self.cores[0].shape[0]] + [c.shape[2] for c in self.cores]

    @property
    def modes(self) -> list:
        return [c.shape[1] for c in self.cores]

    @property
    def nbytes(self) -> int:
        return sum(c.nbytes for c in self.cores)


def random_tt(rng: np.random.Generator, d: int, n, r) -> list:
    """Random TT with iid N(0,1)/sqrt(n r) core entries; ranks (1, r, ..., r, 1)."""
    n = [n] * d if np.isscalar(n) else list(n)
    rk = [1] + ([r] * (d - 1) if np.isscalar(r) else list(r)) + [1]
    nominal = r if np.isscalar(r) else max(r)
    return [rng.standard_normal((rk[k], n[k], rk[k + 1])) / math.sqrt(n[k] * nominal) for k in range(d)]


def _gram_inner(x, y) -> float:
    # <x, y> by a left-to-right contraction of the (small) summands
    g = np.ones((1, 1))
    for a, b in zip(x, y):
        g = np.einsum("ab,aic,bid->cd", g, a, b, optimize=True)
    return float(g[0, 0])


def block_sum(terms) -> list:
    """Formal sum of TTs given as [(coef, cores), ...]: first core concatenated, others block-diagonal."""
    d = len(terms[0][1])
    out = []
    for k in range(d):
        blocks = [(c if k == 0 else 1.0) * t[k] for c, t in terms]
        if k == 0:
            out.append(np.ascontiguousarray(np.concatenate(blocks, axis=2)))
        elif k == d - 1:
            out.append(np.ascontiguousarray(np.concatenate(blocks, axis=0)))
        else:
            r0 = sum(b.shape[0] for b in blocks)
            r1 = sum(b.shape[2] for b in blocks)
            core = np.zeros((r0, blocks[0].shape[1], r1))
            a = c = 0
            for b in blocks:
                core[a:a + b.shape[0], :, c:c + b.shape[2]] = b
                a += b.shape[0]
                c += b.shape[2]
            out.append(core)
    return out


def copies_plus_noise(seed: int, d: int, n: int, r: int, copies: int, noise_rank: int, eta: float,
                      name: str, formal: bool = True) -> TTInput:
    """Scaled copies of one random TT plus a small random TT.  ``formal=False`` leaves out the
    block-diagonal formal sum (``cores`` empty) and keeps only the summands, for inputs whose
    formal sum is too large to build on the host (c5: 25 GB)."""
    rng = np.random.default_rng(seed)
    T = random_tt(rng, d, n, r)
    while True:
        c = rng.standard_normal(copies)
        if abs(c.sum()) >= 0.1:
            break
    N = random_tt(rng, d, n, noise_rank)
    nT2, nN2 = _gram_inner(T, T), _gram_inner(N, N)
    N[0] = N[0] * (eta * math.sqrt(nT2) / math.sqrt(nN2))
    terms = [(float(ci), T) for ci in c] + [(1.0, N)]
    s = float(c.sum())
    norm2 = s * s * nT2 + 2.0 * s * _gram_inner(T, N) + _gram_inner(N, N)
    meta = {"seed": seed, "d": d, "n": n, "r": r, "copies": copies, "noise_rank": noise_rank,
            "eta": eta, "coef": c.tolist(), "true_rank": r + noise_rank}
    summands = [[ci * T[0]] + T[1:] for ci, T in ((float(c_), T) for c_ in c)] + [N]
    return TTInput(name, block_sum(terms) if formal else [], math.sqrt(norm2), meta, summands)


def c1(seed: int = 1) -> TTInput:
    return copies_plus_noise(seed, 6, 10, 8, 3, 2, 1e-8, "c1_d6_n10_r8x3+2")


def c2(seed: int = 2) -> TTInput:
    return copies_plus_noise(seed, 20, 50, 50, 4, 10, 1e-7, "c2_d20_n50_r50x4+10")


def c5(seed: int = 5, formal: bool = True) -> TTInput:
    return copies_plus_noise(seed, 50, 100, 200, 4, 10, 1e-8, "c5_d50_n100_r200x4+10", formal)


def laplace_tt_operator(d: int, n: int) -> list:
    """Rank-2 TT operator of sum_m I (x) .. (x) L (x) .. (x) I, L = tridiag(-1, 2, -1); cores (a, i, j, g)."""
    L = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    I = np.eye(n)
    first = np.zeros((1, n, n, 2)); first[0, :, :, 0] = L; first[0, :, :, 1] = I
    mid = np.zeros((2, n, n, 2)); mid[0, :, :, 0] = I; mid[1, :, :, 0] = L; mid[1, :, :, 1] = I
    last = np.zeros((2, n, n, 1)); last[0, :, :, 0] = I; last[1, :, :, 0] = L
    return [first] + [mid.copy() for _ in range(d - 2)] + [last]


def tt_matvec(op, x) -> list:
    """y = A x for a TT operator A (cores (a, i, j, g)) and TT vector x: y_k = sum_j A_k(., i, j, .) x_k(., j, .)."""
    out = []
    for A, X in zip(op, x):
        a0, n, _, a1 = A.shape
        r0, _, r1 = X.shape
        y = np.einsum("aijg,bjc->abigc", A, X).reshape(a0 * r0, n, a1 * r1)
        out.append(np.ascontiguousarray(y))
    return out


def c3_factors(seed: int = 3, d: int = 16, n: int = 64, r: int = 30):
    """The factors of the operator-applied vector: (the Laplacian TT operator, the rank-r TT x)."""
    rng = np.random.default_rng(seed)
    w = 2.0 ** -np.arange(r)
    x = []
    rk = [1] + [r] * (d - 1) + [1]
    for k in range(d):
        g = rng.standard_normal((rk[k] * n, rk[k + 1]))
        if k < d - 1:
            q, _ = np.linalg.qr(g)                      # left-orthonormal core
            x.append((q * w[None, :]).reshape(rk[k], n, rk[k + 1]))
        else:
            x.append(g.reshape(rk[k], n, 1) / math.sqrt(n * r))
    return laplace_tt_operator(d, n), x


def c3(seed: int = 3, d: int = 16, n: int = 64, r: int = 30) -> TTInput:
    op, x = c3_factors(seed, d, n, r)
    y = tt_matvec(op, x)
    norm = math.sqrt(max(_gram_inner(y, y), 0.0))
    return TTInput(f"c3_d{d}_n{n}_Ax_r{r}x2", y, norm, {"seed": seed, "d": d, "n": n, "r": r})


@dataclass
class Request:
    rid: int
    arrival_ms: float
    tol: float
    tt: TTInput


def c4_specs(seed: int = 4, count: int = 512, mean_gap_ms: float = 2.0, max_bytes: float | None = None):
    """The serving stream's request parameters in arrival order (cheap; no tensor data): Poisson
    arrivals; each request a sum of s in [2, 6] random TTs with d in [8, 32], n in [16, 128],
    component ranks in [20, 100] (all bonds of a summand equal) and tol in {1e-4, 1e-6, 1e-8}.
    ``max_bytes`` skips requests whose formal sum is larger."""
    rng = np.random.default_rng(seed)
    t = 0.0
    for rid in range(count):
        t += float(rng.exponential(mean_gap_ms))
        s = int(rng.integers(2, 7))
        d = int(rng.integers(8, 33))
        n = int(rng.integers(16, 129))
        comp = [int(rng.integers(20, 101)) for _ in range(s)]
        tol = float([1e-4, 1e-6, 1e-8][int(rng.integers(0, 3))])
        R = sum(comp)
        nb = 8 * (2 * n * R + (d - 2) * n * R * R)
        if max_bytes is not None and nb > max_bytes:
            continue
        yield {"rid": rid, "arrival_ms": t, "tol": tol, "s": s, "d": d, "n": n, "ranks": comp, "formal_bytes": nb}


def c4_request(spec: dict, seed: int = 4, formal: bool = True) -> Request:
    """The request of one spec of ``c4_specs``: coefficients N(0, 1) on the first cores of its random
    summands, drawn from a generator of its own (so requests can be made in any order or in
    parallel).  With ``formal`` it also carries the block-diagonal formal sum as ``cores``."""
    rid, d, n, comp = spec["rid"], spec["d"], spec["n"], spec["ranks"]
    sub = np.random.default_rng([seed, rid])
    terms = [(float(sub.standard_normal()), random_tt(sub, d, n, rc)) for rc in comp]
    summands = [[c * x[0]] + x[1:] for c, x in terms]
    cores = block_sum(terms) if formal else []
    meta = {"s": spec["s"], "d": d, "n": n, "ranks": comp, "formal_bytes": spec["formal_bytes"]}
    return Request(rid, spec["arrival_ms"], spec["tol"], TTInput(f"c4_req{rid}", cores, float("nan"), meta, summands))


def c4_stream(seed: int = 4, count: int = 512, mean_gap_ms: float = 2.0, max_bytes: float | None = None,
              formal: bool = True):
    """Serving stream: the requests of ``c4_specs`` in arrival order, made lazily (the whole stream
    is larger than host or device memory).  Each request carries its summands; with ``formal`` it
    also carries the block-diagonal formal sum as ``cores`` (costly for large requests), else
    ``cores`` is empty."""
    for spec in c4_specs(seed, count, mean_gap_ms, max_bytes):
        yield c4_request(spec, seed, formal)
