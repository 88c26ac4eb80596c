"""CPU oracle for adaptive randomized TT-rounding with Khatri-Rao sketches (FP64, numpy).

TEST INFRASTRUCTURE.  This package is the plain, slow reference that the CUDA path is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it; the product package never does,
and this package never imports the product package.  The two share only the seeded input
generators in ``workloads.py``.

Modules:
* ``philox``   - counter-based Gaussian sketch entries (Philox4x32-10 + Box-Muller with
                 series-evaluated ln/cos), reproduced bit for bit by the CUDA side.
* ``tt``       - TT unfoldings, formal sums, stable norms and distances, truncation rank.
* ``rounding`` - Algorithms 1, 3, 4, 5, 6 and Remarks 3.1, 3.2 of the paper, step by step.

Pins (``tests/test_oracle_*.py``) tie each function to something other than itself: brute
force on explicit full tensors, library routines (numpy SVD/log/cos), closed forms, exact
reconstruction, orthogonality invariants and the estimator theorems of Sec. 3.4.
"""
from . import philox, rounding, tt  # noqa: F401
