"""FP64 CPU oracle for the OEM penalized least-squares path (TEST INFRASTRUCTURE).

This package is a plain, slow, obviously-correct restatement of what the
method computes, written in numpy float64 from the paper (Huling & Qian,
"Fast penalized regression and cross validation for tall data with the oem
package", arXiv 1801.09661). It exists only to check the CUDA path: only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it. The product (``paper_1801_09661_gb300``) never imports it, and it
never imports the product; they share no code except the seeded input
generators in ``synthgen``.

Every function cites the passage it follows. Readings taken where the paper
is silent or garbled are stated where they are used (scaling of the
objective, the lambda grid, the stopping rule, d as an upper bound of the top
eigenvalue, the CV error definition).

Parity pins: every function here is pinned by the ``-m "not gpu"`` tests
(closed forms, textbook special cases, KKT conditions, brute force on tiny
problems, eigvalsh, fold-sum identity). No function is parity-unpinned.
"""
from .oem import *  # noqa: F401,F403
