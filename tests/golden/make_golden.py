"""Writes the stored expected values under tests/golden/ by calling only ``oracle/``.

Usage: python tests/golden/make_golden.py   (from the repository root)
The files are regression fixtures: they freeze the oracle's Gaussian sketch stream so that a
later change to its arithmetic shows up as a failing test and has to be justified.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import philox  # noqa: E402


def main():
    seed = 20251103
    pts = [(k, i, j) for k in (2, 3, 20) for i in (0, 1, 49) for j in (0, 1, 63, 1000)]
    with open(os.path.join(HERE, f"omega_seed{seed}.txt"), "w") as f:
        f.write("# seed k i j gaussian_f64(hex); Box-Muller of Philox4x32-10 counter (j, i, k, 0)\n")
        for k, i, j in pts:
            g = float(philox.gaussian_f64(seed, k, i, j))
            f.write(f"{seed} {k} {i} {j} {g.hex()}\n")


if __name__ == "__main__":
    main()
