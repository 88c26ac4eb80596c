"""Counter-based Gaussian sketch entries for the KRP sketch (oracle side).

TEST INFRASTRUCTURE ONLY: this module belongs to the CPU oracle.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.

What it computes
----------------
The Khatri-Rao sketch of Sec. 3.1 (Eq. (3.1), Algorithm 3) needs Gaussian matrices
Omega_k in R^{n_k x l}, k = 2..d, with iid N(0,1) entries.  Here entry Omega_k(i, j) is a
pure function of (seed, k, i, j), so any prefix of columns is the same no matter how the
columns are drawn or in which chunks (this is what lets the adaptive algorithm of Sec. 3.3
append columns, Algorithm 4, without changing earlier ones).

* Uniform bits: Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
  numbers: as easy as 1, 2, 3", SC'11), key = (seed mod 2^32, seed div 2^32), counter =
  (j, i, k, 0).  Written here from that paper's definition of the round function.
* Gaussian: Box-Muller, first output of the pair:
  g = sqrt(-2 ln u1) * cos(2 pi u2), u1 in (0,1], u2 in [0,1), both with 53 random bits.
* ln and cos are computed by this project from their series (atanh series for ln after an
  exact binary exponent split; Taylor series for sin/cos after exact octant reduction),
  using only correctly rounded IEEE-754 double +, -, *, / and sqrt, in a fixed order.  The
  CUDA side evaluates the same operation sequence with explicitly rounded intrinsics, so the
  two agree bit for bit.
* The sketch entry is the Gaussian rounded to the fixed-point grid 2^-20 (round half to
  even): Omega = rint(g * 2^20) * 2^-20, so |Omega| * 2^20 is an integer below 2^24.  The
  CUDA partial-contraction kernel multiplies by these entries and sums over the mode index
  in exact integer arithmetic, which needs a common scale; the grid changes E[Omega^2] by
  2^-40/12 and leaves the Gaussian sketch properties of Sec. 3.4 intact.

Everything is vectorised over numpy arrays; numpy float64 ufuncs are IEEE-correct per
element and never fuse a multiply with an add.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 block function on uint64 arrays holding 32-bit words.

    One round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (full 64-bit products), then
    (c0, c1, c2, c3) <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is advanced by the
    Weyl constants (W0, W1) between rounds (SC'11, Sec. 4.1 / Table 2).
    """
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _MASK32 for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK32
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK32
            k1 = (k1 + _W1) & _MASK32
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK32
        hi1, lo1 = p1 >> _S32, p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK32, lo1, (hi0 ^ c3 ^ k1) & _MASK32, lo0
    return c0, c1, c2, c3


# ---------------------------------------------------------------------------------------
# ln(u) for u in (0, 1]:  u = m * 2^e exactly, m in [sqrt(1/2), sqrt(2)),
# ln u = e*ln2 + 2*atanh(s),  s = (m-1)/(m+1),  |s| <= 0.1716,
# atanh(s) = s + s^3/3 + s^5/5 + ...  (terms through s^27 leave a remainder < 1e-21 |s|).
# ln2 is carried as hi + lo so that e*ln2_hi is exact for |e| <= 1075.
# ---------------------------------------------------------------------------------------
# ln2_hi = floor(ln 2 * 2^32) / 2^32 (so e*ln2_hi is exact), ln2_lo = ln 2 - ln2_hi rounded;
# both computed once from a 60-digit value of ln 2.
_LN2_HI = float.fromhex("0x1.62e42fee00000p-1")
_LN2_LO = float.fromhex("0x1.a39ef35793c76p-33")
_SQRT_HALF = float.fromhex("0x1.6a09e667f3bcdp-1")   # split point; any fixed value works
_ATANH_TERMS = 14                          # odd powers s^1 .. s^27


def own_log(u: np.ndarray) -> np.ndarray:
    """Natural log on (0, 1] from the atanh series (exact exponent split, fixed op order)."""
    u = np.asarray(u, dtype=np.float64)
    m, e = np.frexp(u)                      # exact: u = m * 2^e, m in [0.5, 1)
    small = m < _SQRT_HALF
    m = np.where(small, m * 2.0, m)         # exact scaling by 2
    e = np.where(small, e - 1, e).astype(np.float64)
    s = (m - 1.0) / (m + 1.0)
    s2 = s * s
    # Horner on the odd series, innermost coefficient first: 1/27, 1/25, ..., 1/3, 1
    p = np.full_like(s, 1.0 / (2 * _ATANH_TERMS - 1))
    for t in range(_ATANH_TERMS - 2, -1, -1):
        p = p * s2
        p = p + 1.0 / (2 * t + 1)
    logm = (s + s) * p
    return e * _LN2_HI + (e * _LN2_LO + logm)


# ---------------------------------------------------------------------------------------
# cos(2*pi*t) for t in [0, 1): exact reductions t -> |t - round(t)| in [0, 1/2] -> [0, 1/4]
# (sign flip) -> [0, 1/8] (cos/sin swap), then x = 2*pi*t' in [0, pi/4] and Taylor series.
# ---------------------------------------------------------------------------------------
_TWO_PI_HI = float.fromhex("0x1.921fb54442d18p+2")   # nearest double to 2*pi
_TWO_PI_LO = float.fromhex("0x1.1a62633145c07p-52")  # 2*pi - _TWO_PI_HI, from a 60-digit pi
_TAYLOR_TERMS = 11                         # x^0 .. x^20 (cos) / x^1 .. x^21 (sin)


def _cos_poly(x2):
    # cos x = sum_k (-1)^k x^{2k}/(2k)!  in Horner form on x^2
    p = np.full_like(x2, _inv_fact(2 * (_TAYLOR_TERMS - 1)) * (-1.0) ** (_TAYLOR_TERMS - 1))
    for k in range(_TAYLOR_TERMS - 2, -1, -1):
        p = p * x2
        p = p + _inv_fact(2 * k) * (-1.0) ** k
    return p


def _sin_poly(x, x2):
    # sin x = x * sum_k (-1)^k x^{2k}/(2k+1)!
    p = np.full_like(x2, _inv_fact(2 * (_TAYLOR_TERMS - 1) + 1) * (-1.0) ** (_TAYLOR_TERMS - 1))
    for k in range(_TAYLOR_TERMS - 2, -1, -1):
        p = p * x2
        p = p + _inv_fact(2 * k + 1) * (-1.0) ** k
    return x * p


def _inv_fact(n: int) -> float:
    """1/n! rounded once to the nearest double (exact rational first; n! > 2^53 for n > 18)."""
    return float(Fraction(1, math.factorial(n)))


def own_cos2pi(t: np.ndarray) -> np.ndarray:
    """cos(2*pi*t) for t in [0, 1) with exact argument reduction and series evaluation."""
    t = np.asarray(t, dtype=np.float64)
    t = np.abs(t - np.rint(t))              # exact; t in [0, 1/2]
    neg = t > 0.25
    t = np.where(neg, 0.5 - t, t)           # exact (Sterbenz); cos(2pi t) = -cos(2pi(1/2 - t))
    swap = t > 0.125
    t = np.where(swap, 0.25 - t, t)         # exact (Sterbenz); cos(2pi t) = sin(2pi(1/4 - t))
    x = t * _TWO_PI_HI + t * _TWO_PI_LO
    x2 = x * x
    c = _cos_poly(x2)
    s = _sin_poly(x, x2)
    r = np.where(swap, s, c)
    return np.where(neg, -r, r)


_TWO_M53 = 2.0 ** -53


def uniforms_from_words(x0, x1, x2, x3):
    """Two 53-bit uniforms per Philox block: u1 in (0, 1] from (x0, x1), u2 in [0, 1) from (x2, x3)."""
    m1 = (np.asarray(x0, np.uint64) << np.uint64(21)) | (np.asarray(x1, np.uint64) >> np.uint64(11))
    m2 = (np.asarray(x2, np.uint64) << np.uint64(21)) | (np.asarray(x3, np.uint64) >> np.uint64(11))
    u1 = (m1 + np.uint64(1)).astype(np.float64) * _TWO_M53     # exact: integer < 2^53 + 1 ... <= 2^53
    u2 = m2.astype(np.float64) * _TWO_M53
    return u1, u2


def gaussian_f64(seed: int, k, i, j) -> np.ndarray:
    """Box-Muller Gaussian (binary64) for counter (j, i, k, 0) and key from ``seed``."""
    k, i, j = np.broadcast_arrays(np.asarray(k, np.uint64), np.asarray(i, np.uint64), np.asarray(j, np.uint64))
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    x0, x1, x2, x3 = philox4x32_10(j, i, k, np.zeros_like(j), seed & 0xFFFFFFFF, seed >> 32)
    u1, u2 = uniforms_from_words(x0, x1, x2, x3)
    return np.sqrt(-2.0 * own_log(u1)) * own_cos2pi(u2)


def omega(seed: int, k: int, n_k: int, col0: int, col1: int) -> np.ndarray:
    """Sketch block Omega_k(:, col0:col1) in R^{n_k x (col1-col0)} (values on the 2^-20 grid, float64).

    ``k`` is the 1-based core index of Sec. 3.1 (Omega_2 .. Omega_d are used); columns use the
    global column index j so that a column never depends on how many columns were drawn.
    """
    i = np.arange(n_k, dtype=np.uint64)[:, None]
    j = np.arange(col0, col1, dtype=np.uint64)[None, :]
    g = gaussian_f64(seed, np.uint64(k), i, j)
    return np.rint(g * OMEGA_SCALE) / OMEGA_SCALE


OMEGA_SCALE = 2.0 ** 20     # sketch entries live on the grid 2^-20 (see module docstring)
