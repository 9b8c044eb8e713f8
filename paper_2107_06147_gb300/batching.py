"""Uneven batches: trajectories of different grid sizes, angular momenta and lifetimes in one call.

Trajectories are grouped by grid size N (a kernel instantiation and its shared-memory footprint
depend on N); each group runs as one persistent fused launch on its own CUDA stream, and all groups
are launched before any of them is waited for, so they share the GPU.  Inside a launch the CTAs take
trajectories from the launch's work counter, so trajectories of different l and different lifetimes
(media) refill the CTAs as they finish; a group is ordered longest medium first (Bjorken media;
tabulated ones keep their place), so that the last trajectories to start are short ones and the
launch's tail is short.  Results come back in the caller's order.
"""
from __future__ import annotations

import numpy as np

from . import qtraj


def _lifetime(m) -> float:
    """Proper-time span of a Bjorken medium, tau0 ((T0/Tf)^3 - 1) (fm/c); 0 for a tabulated one."""
    if m.kind == 0 and m.Tf > 0 and m.T0 > m.Tf:
        return m.tau0 * ((m.T0 / m.Tf) ** 3 - 1.0)
    return 0.0


class UnevenBatch:
    """A fixed layout of trajectories (per-trajectory N, L, initial state, medium); seeds per call."""

    def __init__(self, Ns, inits, media, dt: float = 0.001, dr: float = 5.0 / 512, precision=qtraj.FP32,
                 use_rmin: int = 1, Ls=None):
        import torch
        Ns = np.asarray(Ns)
        self.n = len(Ns)
        self.groups = []
        for N in sorted(set(int(x) for x in Ns)):
            ids = np.nonzero(Ns == N)[0]
            ids = ids[np.argsort([-_lifetime(media[t]) for t in ids], kind="stable")]
            L = float(Ls[ids[0]]) if Ls is not None else N * dr
            spec_keys, spec_list, spec_idx = {}, [], []
            for t in ids:
                s = inits[t]
                key = (s.kind, s.width, s.n, s.l, s.color)
                if key not in spec_keys:
                    spec_keys[key] = len(spec_list)
                    spec_list.append(s)
                spec_idx.append(spec_keys[key])
            eng = qtraj.Engine(qtraj.Config(N=N, L=L, dt=dt, precision=precision, use_rmin=use_rmin))
            eng.init(spec_list, len(ids), spec_idx=np.array(spec_idx, np.int32))
            self.groups.append({"N": N, "ids": ids, "eng": eng, "media": [media[t] for t in ids],
                                "stream": torch.cuda.Stream()})

    def evolve(self, seeds):
        """Launches every group on its own stream; returns immediately."""
        seeds = np.asarray(seeds, dtype=np.uint64)
        for g in self.groups:
            g["eng"].evolve(g["media"], seeds[g["ids"]], np.arange(len(g["ids"]), dtype=np.int32),
                            stream=g["stream"])

    def observables(self):
        out = np.zeros(self.n, dtype=qtraj.OBS_DTYPE)
        for g in self.groups:
            out[g["ids"]] = g["eng"].observables(stream=g["stream"], check_finite=False)
        return out

    def run(self, seeds):
        self.evolve(seeds)
        return self.observables()

    def stats(self):
        return {g["N"]: g["eng"].stats() for g in self.groups}

    def close(self):
        for g in self.groups:
            g["eng"].close()
