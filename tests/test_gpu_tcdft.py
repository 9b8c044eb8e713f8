"""The radix-16 DFT blocks on the CUDA cores and on the tensor cores (qtraj_dft16_study) against the
FP64 oracle of the definition y = F x (oracle/dft16.py; the study applies F/4), on the FP32-rounded
input.

Bounds, as the relative 2-norm error of a column after one pass (|y| = |x|):
- FP32 CUDA cores: radix 4 x 4 in FP32, about log2(16) roundings of 2^-24 on each path: 1e-6;
- BF16X3: two BF16 parts carry 16 bits and the dropped product lo.lo is 2^-18 of the terms:
  the representation error ~2^-17 per term, bound 6e-5;
- BF16X9, FP16X3, FP16X5: the parts carry 22 bits or more; each real output collects up to 18 MMAs,
  each rounding at most 2^-24 of sum |F/4||x| <= 4 max|x| <= 4 |x|: worst case 72 x 2^-24 = 4.3e-6,
  bound 5e-6.
"""
import numpy as np
import pytest

from oracle import dft16 as odft

pytestmark = pytest.mark.gpu

BOUNDS = {0: 1e-6, 1: 6e-5, 2: 5e-6, 3: 5e-6, 4: 5e-6}


def _x(batches, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    x = scale * (rng.standard_normal((batches, 256, 16)) + 1j * rng.standard_normal((batches, 256, 16)))
    return x.astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("method", [0, 1, 2, 3, 4])
def test_one_pass_against_oracle(method):
    from paper_2107_06147_gb300 import qtraj
    x = _x(5, 11 + method)
    y, ms = qtraj.dft16_study(method, x, 1)
    ref = odft.passes(x, 1) / 4
    rel = np.linalg.norm(y - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    assert rel.max() < BOUNDS[method], (method, rel.max())
    assert ms > 0


@pytest.mark.parametrize("method", [0, 1, 2, 3, 4])
def test_repeated_passes_and_identity(method):
    from paper_2107_06147_gb300 import qtraj
    x = _x(3, 5)
    y0, _ = qtraj.dft16_study(method, x, 0)
    assert np.array_equal(y0, x)   # zero passes: the FP32 input back
    y4, _ = qtraj.dft16_study(method, x, 4)   # (F/4)^4 = I
    rel = np.linalg.norm(y4 - x, axis=-1) / np.linalg.norm(x, axis=-1)
    assert rel.max() < 4 * BOUNDS[method], (method, rel.max())


@pytest.mark.parametrize("method", [3, 4])
def test_fp16_scaling_over_magnitudes(method):
    """The FP16 forms scale every column to [2^14, 2^15) before splitting: columns of 1e-20 and 1e20
    keep the same relative error."""
    from paper_2107_06147_gb300 import qtraj
    x = _x(2, 3)
    x[0] *= 1e-20
    x[1] *= 1e20
    x = x.astype(np.complex64).astype(np.complex128)
    y, _ = qtraj.dft16_study(method, x, 1)
    ref = odft.passes(x, 1) / 4
    rel = np.linalg.norm(y - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    assert rel.max() < BOUNDS[method], (method, rel.max())


def test_arguments():
    from paper_2107_06147_gb300 import qtraj
    x = _x(1, 1)
    for m, p in ((5, 1), (-1, 1), (0, -1)):
        with pytest.raises(qtraj.QtrajError):
            qtraj.dft16_study(m, x, p)
