"""The device generator against the oracle's, bit for bit (no tolerance: integer work).

The trajectory kernels draw their waiting-time thresholds and jump choices from Philox4x32-10
(Salmon et al., SC'11).  The device code (qtraj_device.cuh, reached through qtraj_philox4x32_10 and
qtraj_period_draws) and the oracle's C code were written separately.  Checked here: the
published known-answer vectors (tests/golden/philox4x32_10_kat.txt), all four output words for
10^6 random (counter, key) pairs, and the three uniforms (r, u_l, u_c) of 10^6 random (seed, k)
pairs -- k up to 2^32 - 1, seeds over the whole 64-bit range.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2107_06147_gb300 import build, qtraj
    build.build()
    qtraj.load()
    return qtraj


def _dev_u32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _words(q, ctr, key):
    import torch
    out = q.philox4x32_10(_dev_u32(ctr), _dev_u32(key))
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32)


def test_device_philox_known_answers(q):
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([int(t, 16) for t in line.split()])
    v = np.array(rows, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(_words(q, v[:, 0:4], v[:, 4:6]), v[:, 6:10])


def test_device_philox_words_match_oracle_on_1e6_pairs(q):
    import oracle as o
    rng = np.random.Generator(np.random.PCG64(2024))
    n = 1_000_000
    ctr = rng.integers(0, 2**32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[: n // 2, 1:] = 0                   # half of them in the kernels' (k, 0, 0, 0) form
    got = _words(q, ctr, key)
    ref = o.philox_many(ctr, key)
    assert np.array_equal(got, ref), np.argwhere(got != ref)[:5]


def test_device_period_draws_match_oracle_on_1e6_pairs(q):
    import torch
    import oracle as o
    rng = np.random.Generator(np.random.PCG64(7))
    n = 1_000_000
    seeds = rng.integers(0, 2**64, n, dtype=np.uint64)
    seeds[:1000] = np.arange(1000, dtype=np.uint64)          # small ids, as the workloads use
    k = rng.integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    k[: n // 2] = rng.integers(0, 200, n // 2).astype(np.uint32)   # the periods trajectories reach
    d_seed = torch.from_numpy(seeds.view(np.int64)).cuda()
    d_k = _dev_u32(k)
    got = q.period_draws(d_seed, d_k)
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    ref = o.draws_many(seeds, k)
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    assert (got > 0).all() and (got < 1).all()
