"""Plain FP64 CPU oracle of the QTraj 1.0 quantum-trajectory method (arXiv:2107.06147).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers.  Nothing in ``paper_2107_06147_gb300`` imports this package,
and this package imports nothing from it.

``qtraj_oracle.c`` holds the method (own radix-2 FFT, own Philox4x32-10, the Strang step, the
waiting-time jumps, the observables); ``core.py`` is its ctypes wrapper; ``lindblad.py`` is a
brute-force density-matrix integrator used only to pin the oracle's unravelling; ``eigen.py``
diagonalises the dense discretised vacuum Hamiltonian for the numerical eigenstates.
"""
from .core import *  # noqa: F401,F403
