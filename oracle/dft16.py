"""The 16-point DFT blocks of the sine transforms' FFT as a plain matrix product (test infrastructure
only, for the tensor-core study of the radix-16 pass).

Sec. 3.3 evaluates the kinetic half of the split step in the sine basis; the fused kernel computes
the sine transforms with radix-16 FFT passes, whose blocks are 16-point DFTs
    y[m'] = sum_m exp(-2 pi i m' m / 16) x[m].
`passes(x, p)` applies that matrix p times to every 16-point column of x (shape (..., 16)), in FP64,
written as the definition: the matrix is built entry by entry and applied with a matmul.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(n: int = 16) -> np.ndarray:
    """F[m', m] = exp(-2 pi i m' m / n)."""
    F = np.empty((n, n), dtype=np.complex128)
    for a in range(n):
        for b in range(n):
            ang = -2.0 * np.pi * ((a * b) % n) / n
            F[a, b] = complex(np.cos(ang), np.sin(ang))
    return F


def passes(x: np.ndarray, p: int) -> np.ndarray:
    """F^p applied to the last axis of x (length 16)."""
    F = dft_matrix(16)
    y = np.asarray(x, dtype=np.complex128)
    for _ in range(p):
        y = y @ F.T
    return y
