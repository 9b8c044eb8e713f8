"""Tensor-core forms of the radix-16 DFT blocks against the CUDA-core form (qtraj_dft16_study).

Each form applies y = (F/4) x (F the 16-point DFT matrix; (F/4)^4 = I) `passes` times to batches of
256 columns held in shared memory, one CTA per batch.  Reported per form:
- the time of one pass over the whole GPU, as the difference of a launch of 2P passes and one of P
  passes (the load, store and set-up of a launch cancel), in ns per column and columns per second;
- the ceiling that rate puts on a step that did nothing but its sine transforms: a trajectory-step
  of the N-point split step runs 2 transforms x log16(N) passes x N/16 columns (N = 4096: 1536);
- the error of one pass against numpy's FFT in FP64 on the FP32-rounded input, and of 2P passes
  against the input itself ((F/4)^(2P) = I for 2P a multiple of 4), where a coherent error of the
  matrix grows as the pass count and rounding noise as its square root: the largest and the RMS of
  |y - y_exact|_2 / |y_exact|_2 over the columns.
Run: python -m paper_2107_06147_gb300.tcstudy [--batches B] [--passes P] [--seed S]
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import qtraj

FORMS = {0: "fp32_cuda_cores", 1: "tc_bf16x3", 2: "tc_bf16x9", 3: "tc_fp16x3", 4: "tc_fp16x5"}


def columns_per_traj_step(N: int) -> int:
    return 2 * round(math.log(N, 16)) * (N // 16)


def _rel(y, ref):
    r = np.linalg.norm(y - ref, axis=-1) / np.linalg.norm(ref, axis=-1)
    return float(f"{r.max():.3g}"), float(f"{np.sqrt((r ** 2).mean()):.3g}")


def run(batches: int = 1824, passes: int = 32, seed: int = 7, N: int = 4096, reps: int = 3) -> dict:
    if passes % 2:
        raise ValueError("passes must be even (2 x passes a multiple of 4)")
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal((batches, 256, 16)) + 1j * rng.standard_normal((batches, 256, 16)))
    x = x.astype(np.complex64).astype(np.complex128)
    exact1 = np.fft.fft(x, axis=-1) / 4
    cols = columns_per_traj_step(N)
    out = {"batches": batches, "passes": [passes, 2 * passes], "columns_per_traj_step": cols, "N": N, "forms": {}}
    for m, name in FORMS.items():
        y1, _ = qtraj.dft16_study(m, x, 1)
        t1 = min(qtraj.dft16_study(m, x, passes)[1] for _ in range(reps))
        t2s = []
        for _ in range(reps):
            y2, t = qtraj.dft16_study(m, x, 2 * passes)
            t2s.append(t)
        per_pass_ms = (min(t2s) - t1) / passes
        rate = batches * 256 / (per_pass_ms / 1e3)
        e1 = _rel(y1, exact1)
        e2 = _rel(y2, x)
        out["forms"][name] = {"ms_per_pass": round(per_pass_ms, 5), "ns_per_column": float(f"{1e9 / rate:.4g}"),
                              "columns_per_s": float(f"{rate:.4g}"),
                              "transform_only_traj_steps_per_s_ceiling": float(f"{rate / cols:.4g}"),
                              "rel_err_1pass_max": e1[0], "rel_err_1pass_rms": e1[1],
                              f"rel_err_{2 * passes}pass_max": e2[0], f"rel_err_{2 * passes}pass_rms": e2[1]}
    return out


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--batches", type=int, default=1824)
    ap.add_argument("--passes", type=int, default=32)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args()
    print(json.dumps(run(a.batches, a.passes, a.seed, reps=a.reps)))


if __name__ == "__main__":
    main()
