"""Paired precision study of the arithmetic forms.

The same trajectories (same initial states, media and Philox seeds) run in every form, and each form
is compared with the FP64 fused form trajectory by trajectory.  The FP64 form follows the FP64 oracle
to ~1e-10 per wavefunction with identical jump steps, so it stands in for the exact result here at a
size the oracle would take hours for.  Pairing matters: two independent ensembles of n trajectories
differ by ~0.5/sqrt(n) in their survival means, far above the rounding effects being measured.

Reported per form:
- per observable, the absolute error of the ensemble mean and, beside it, the standard error of the
  FP64 mean (the statistical resolution of a run of this size);
- the largest per-trajectory survival error, over all trajectories and over those whose jump
  sequences are identical;
- the fraction of trajectories whose jump sequence differs (jump digests: some jump at another step
  or with another outcome -- a jump whose threshold lies within a form's rounding of the norm moves
  by a step or two);
- the largest per-trajectory error on identical jump sequences over the FP32 error model
  5.5e-8 sqrt(N n_steps) (relative to max(1, S)), n_steps the steps behind the final state (the
  whole medium for a trajectory that took the rMin shortcut);
- the form's throughput on this run.
"""
from __future__ import annotations

import time

import numpy as np

from . import qtraj

FORM_NAMES = {qtraj.FP64: "fp64", qtraj.FP32: "fp32"}
BASIS = ("1S", "2S", "1P", "3S", "2P", "1D")


def _run(w, precision, use_rmin):
    import torch
    eng = qtraj.Engine(qtraj.Config(N=w.grid.N, L=w.grid.L, dt=w.grid.dt, precision=precision, use_rmin=use_rmin))
    eng.init([qtraj.init_spec(s.kind, s.width, s.n, s.l, s.color) for s in w.inits], w.n_traj, w.init_idx)
    t0 = time.perf_counter()
    eng.evolve([qtraj.medium(m.T0, m.tau0, m.Tf, m.kappa_hat, m.gamma_hat) for m in w.media], w.seeds, w.medium_idx)
    obs = eng.observables(check_finite=False)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    s = eng.stats()
    eng.close()
    ms = s.ms_main + s.ms_nojump
    return obs, {"traj_steps": int(s.steps_executed), "ms": round(ms, 1), "wall_s": round(wall, 2),
                 "traj_steps_per_s": round(s.steps_executed / max(ms / 1e3, 1e-9), 1)}


def medium_step_count(T0, tau0, Tf, dt):
    """Steps of a Bjorken medium from T0 at tau0 down to Tf: ceil((tau_f - tau0) / (hbar c dt)),
    tau_f = tau0 (T0/Tf)^3 (Sec. 3.4, Table 1)."""
    return int(np.ceil((tau0 * (T0 / Tf) ** 3 - tau0) / (0.1973269804 * dt)))


def run(w, precisions=(qtraj.FP32,), use_rmin: int = 1) -> dict:
    """Runs the workload in FP64 and in each form of `precisions`; returns the report (a dict)."""
    ref, ref_t = _run(w, qtraj.FP64, use_rmin)
    medium_steps = np.array([medium_step_count(m.T0, m.tau0, m.Tf, w.grid.dt) for m in w.media])
    n = w.n_traj
    sem = ref["surv"].std(axis=0, ddof=1) / np.sqrt(n) if n > 1 else np.zeros(ref["surv"].shape[1])
    report = {"workload": w.name, "trajectories": n, "steps_per_trajectory": int(ref["n_steps_exec"].max()),
              "reference": {"form": "fp64 fused", **ref_t,
                            "survival_mean": {b: float(v) for b, v in zip(BASIS, ref["surv"].mean(axis=0))},
                            "survival_sem": {b: float(v) for b, v in zip(BASIS, sem)},
                            "mean_jumps": float(ref["n_jumps"].mean())},
              "forms": {}}
    for prec in precisions:
        o, t = _run(w, prec, use_rmin)
        # steps behind each trajectory's final state: a trajectory that took the rMin shortcut on
        # either side (n_steps_exec = 0) carries its group's no-jump evolution over the whole medium
        shortcut = ((o["flags"] | ref["flags"]) & qtraj.F_NOJUMP_SHORTCUT) != 0
        model_steps = np.where(shortcut, medium_steps[w.medium_idx],
                               np.maximum(np.maximum(o["n_steps_exec"], ref["n_steps_exec"]), 1)).astype(np.float64)
        # identical jump sequences: every jump at the same step with the same outcome (jump digests)
        same = (o["jump_digest"] == ref["jump_digest"]) & (o["n_jumps"] == ref["n_jumps"]) & \
               (o["l"] == ref["l"]) & (o["color"] == ref["color"])
        d = np.abs(o["surv"] - ref["surv"])
        dmean = np.abs(o["surv"].mean(axis=0) - ref["surv"].mean(axis=0))
        shift = np.abs(o["first_jump_step"] - ref["first_jump_step"])[(o["n_jumps"] == ref["n_jumps"]) & ~same]
        report["forms"][FORM_NAMES.get(prec, str(prec))] = {
            **t,
            "ensemble_mean_abs_error": {b: float(v) for b, v in zip(BASIS, dmean)},
            "ensemble_error_over_sem": {b: (float(v / s) if s > 0 else None) for b, v, s in zip(BASIS, dmean, sem)},
            "max_traj_error": float(d.max()),
            "max_traj_error_same_jumps": float(d[same].max()) if same.any() else None,
            "median_traj_error_same_jumps": float(np.median(d[same].max(axis=1))) if same.any() else None,
            "fraction_jump_steps_differ": float(1.0 - same.mean()),
            "max_traj_error_same_jumps_over_model": (
                float((d[same].max(axis=1) / np.maximum(1.0, np.abs(ref["surv"][same]).max(axis=1)) /
                       (5.5e-8 * np.sqrt(w.grid.N * model_steps[same]))).max())
                if same.any() else None),
            "first_jump_shift_steps_when_count_equal": (np.bincount(np.minimum(shift, 10)).tolist()
                                                        if len(shift) else []),
        }
    return report
