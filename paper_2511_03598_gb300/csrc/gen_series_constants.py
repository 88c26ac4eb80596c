"""Writes series_constants.cuh: the constants of the device-side ln/cos used by the Gaussian
sketch generator, each the double nearest to its exact value (rounded once).

    python paper_2511_03598_gb300/csrc/gen_series_constants.py

ln(2) and pi come from 60-digit decimal series (ln 2 = sum 1/(k 2^k); pi by Machin's
formula), so the script needs nothing beyond the standard library.
"""
import os
from decimal import Decimal, getcontext
from fractions import Fraction
from math import factorial

getcontext().prec = 70


def ln2() -> Decimal:
    s, k, p = Decimal(0), 1, Decimal(2)
    while k < 260:
        s += Decimal(1) / (k * p)
        k += 1
        p *= 2
    return s


def arctan_inv(x: int) -> Decimal:
    s, t, k, x2 = Decimal(0), Decimal(1) / x, 0, x * x
    while t > Decimal(10) ** -68:
        s += t / (2 * k + 1) * (-1) ** k
        t /= x2
        k += 1
    return s


def nearest(q) -> str:
    return float(Fraction(q)).hex()


def main():
    L = ln2()
    hi = Fraction(int(L * 2 ** 32), 2 ** 32)                 # 32 significant bits: e*hi exact
    lo = Fraction(L) - hi
    pi = 16 * arctan_inv(5) - 4 * arctan_inv(239)
    two_pi = 2 * Fraction(pi)
    tp_hi = Fraction(float(two_pi))
    lines = ["// Generated by gen_series_constants.py; do not edit.",
             "#pragma once",
             f"#define TTR_LN2_HI {nearest(hi)}",
             f"#define TTR_LN2_LO {nearest(lo)}",
             f"#define TTR_SQRT_HALF {nearest(Fraction(Decimal(0.5).sqrt()))}",
             f"#define TTR_TWO_PI_HI {nearest(tp_hi)}",
             f"#define TTR_TWO_PI_LO {nearest(two_pi - tp_hi)}",
             "// 1/(2t+1), t = 0..13 (atanh series)",
             "__device__ __constant__ double kTtrAtanh[14] = {" +
             ", ".join(nearest(Fraction(1, 2 * t + 1)) for t in range(14)) + "};",
             "// (-1)^k/(2k)!, k = 0..10 (cos series)",
             "__device__ __constant__ double kTtrCos[11] = {" +
             ", ".join(nearest(Fraction((-1) ** k, factorial(2 * k))) for k in range(11)) + "};",
             "// (-1)^k/(2k+1)!, k = 0..10 (sin series)",
             "__device__ __constant__ double kTtrSin[11] = {" +
             ", ".join(nearest(Fraction((-1) ** k, factorial(2 * k + 1))) for k in range(11)) + "};"]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "series_constants.cuh")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
