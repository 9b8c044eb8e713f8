"""In-project autotuner for the fused kernel's launch variant.

For a grid size N and precision, every variant the library offers (512 or 640 resident threads
per SM at the size's own radix -- 8 up to N = 2048, 16 above -- and radix 8 with 768 or 1024) is
timed on one full wave of trajectories of
the benchmark medium through its first `steps` steps, and the fastest is recorded, with all measured
rates and the kernel geometry, in a JSON cache (`_lib/autotune.json` in the package, or the path in
QTRAJ_AUTOTUNE_CACHE).  `best_variant` reads the cache and falls back to variant 0.
"""
from __future__ import annotations

import json
import os

from . import qtraj

_HERE = os.path.dirname(os.path.abspath(__file__))
VARIANTS = (0, 1, 2, 3)


def cache_path() -> str:
    return os.environ.get("QTRAJ_AUTOTUNE_CACHE", os.path.join(_HERE, "_lib", "autotune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _key(N, precision) -> str:
    return f"N={N},precision={'fp32' if precision == qtraj.FP32 else 'fp64'}"


def best_variant(N: int, precision=qtraj.FP32) -> int:
    return int(_load().get(_key(N, precision), {}).get("variant", 0))


def measure(N: int, precision, variant: int, steps: int = 300, dr: float = 5.0 / 512, dt: float = 0.001,
            timer=None) -> dict:
    """Trajectory-steps/s of one variant on one full wave (rMin off, so every trajectory runs)."""
    import numpy as np
    import torch
    eng = qtraj.Engine(qtraj.Config(N=N, L=N * dr, dt=dt, precision=precision, use_rmin=0, variant=variant))
    ki = eng.kernel_info()
    B = ki.sm_count * ki.ctas_per_sm
    tau_end = 0.6 + steps * dt * 0.1973269804
    med = qtraj.medium(0.425, 0.6, 0.425 * (0.6 / tau_end) ** (1 / 3) * (1 + 1e-9), 5.0, -1.0)
    eng.init([qtraj.init_spec("gauss", 0.2, 1, 0, 0)], B)
    seeds = np.arange(B, dtype=np.uint64)
    eng.evolve([med], seeds)            # warm-up
    eng.evolve([med], seeds)
    torch.cuda.synchronize()
    s = eng.stats()
    eng.close()
    rate = s.steps_executed / (s.ms_main / 1e3) if timer is None else timer(variant)
    return {"variant": variant, "rate": rate, "regs": ki.regs_per_thread, "ctas_per_sm": ki.ctas_per_sm,
            "threads_per_traj": ki.threads_per_traj, "radix": ki.radix}


def tune(N: int, precision=qtraj.FP32, variants=VARIANTS, steps: int = 300, measure_fn=None) -> dict:
    """Times every variant, stores the fastest in the cache and returns the record."""
    measure_fn = measure_fn or (lambda v: measure(N, precision, v, steps))
    rows = [measure_fn(v) for v in variants]
    best = max(rows, key=lambda r: r["rate"])
    rec = {"variant": best["variant"], "candidates": rows, "steps": steps}
    cache = _load()
    cache[_key(N, precision)] = rec
    os.makedirs(os.path.dirname(cache_path()), exist_ok=True)
    with open(cache_path(), "w") as f:
        json.dump(cache, f, indent=1)
    return rec
