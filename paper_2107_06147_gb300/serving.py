"""Continuous-batching request loop over libqtraj.

A request asks for `ntraj` trajectories of one initial state (1S Gaussian, Coulomb 2S or 1P Gaussian)
in one Bjorken medium (T0, kappa_hat, gamma_hat) on an N-point grid.  The server keeps, for every
grid size N it serves, a few engine slots (a libqtraj context with its own workspace and CUDA
stream).  Whenever a slot is free, the scheduler fills it with up to one full wave of trajectories
taken first-come-first-served from the pending requests of that N -- trajectories of several
requests share a launch, and a request that arrives while others run joins the next launch that
frees up.  Slots of different N (and several slots of one N) run concurrently on separate streams, so
their work overlaps on the device.  Admission is bounded by a budget of trajectories in flight.

Each trajectory's result depends only on its own inputs (initial state, medium, seed), never on the
batch it shares a launch with, so a request's results are the same alone and in the mix.

Arithmetic runs in libqtraj; this module only schedules (host bookkeeping, torch streams and events).
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import qtraj

INIT_SPECS = (qtraj.init_spec("gauss", 0.2, 1, 0, 0),     # 1S-like Gaussian S wave
              qtraj.init_spec("coulomb", 0.0, 2, 0, 0),   # Coulomb 2S
              qtraj.init_spec("gauss", 0.2, 2, 1, 0))     # 1P-like Gaussian P wave


@dataclass
class Request:
    rid: int
    N: int
    init: int            # index into INIT_SPECS
    T0: float
    kappa_hat: float
    gamma_hat: float
    ntraj: int
    seed0: int
    Tf: float = 0.25
    arrival: float = 0.0
    admitted: float = -1.0
    done_time: float = -1.0
    next_traj: int = 0   # trajectories handed to launches so far
    n_done: int = 0
    obs: np.ndarray = field(default=None, repr=False)

    def medium(self):
        return qtraj.medium(self.T0, 0.6, self.Tf, self.kappa_hat, self.gamma_hat)


class _Slot:
    def __init__(self, N, L, dt, precision, cap, device):
        import torch
        self.eng = qtraj.Engine(qtraj.Config(N=N, L=L, dt=dt, precision=precision, use_rmin=0))
        self.cap = cap
        self.eng.init(list(INIT_SPECS), cap, spec_idx=np.zeros(cap, np.int32))
        self.stream = torch.cuda.Stream(device=device)
        self.event = torch.cuda.Event()
        self.busy = False
        self.parts = []      # (request, first trajectory, count) in launch order


class Server:
    """Per-N engine slots; see the module docstring."""

    def __init__(self, Ns=(1024, 2048, 4096, 8192, 16384), slots_per_n: int = 2, precision=qtraj.FP32,
                 max_inflight_traj: int = 1 << 20, dr: float = 5.0 / 512, dt: float = 0.001, wave_mult: int = 1):
        import torch
        self.device = torch.cuda.current_device()
        self.slots = {}
        self.pending = {}
        self.max_inflight = max_inflight_traj
        self.inflight = 0
        for N in Ns:
            probe = qtraj.Engine(qtraj.Config(N=N, L=N * dr, dt=dt, precision=precision, use_rmin=0))
            ki = probe.kernel_info()
            probe.close()
            cap = ki.sm_count * ki.ctas_per_sm * wave_mult
            self.slots[N] = [_Slot(N, N * dr, dt, precision, cap, self.device) for _ in range(slots_per_n)]
            self.pending[N] = deque()
        self.waiting = deque()    # arrived, not yet admitted
        self.completed = []

    # ------------------------------------------------------------------------------------------
    def submit(self, req: Request, now: float | None = None):
        req.arrival = time.perf_counter() if now is None else now
        req.obs = np.zeros(req.ntraj, dtype=qtraj.OBS_DTYPE)
        self.waiting.append(req)

    def _admit(self, now):
        while self.waiting and self.inflight + self.waiting[0].ntraj <= self.max_inflight:
            r = self.waiting.popleft()
            r.admitted = now
            self.inflight += r.ntraj
            self.pending[r.N].append(r)

    def _launch(self, N, slot):
        q = self.pending[N]
        parts, n = [], 0
        while q and n < slot.cap:
            r = q[0]
            take = min(r.ntraj - r.next_traj, slot.cap - n)
            parts.append((r, r.next_traj, take))
            r.next_traj += take
            n += take
            if r.next_traj == r.ntraj:
                q.popleft()
        if n == 0:
            return False
        spec_idx = np.concatenate([np.full(c, r.init, np.int32) for r, _, c in parts])
        media_idx = np.concatenate([np.full(c, i, np.int32) for i, (r, _, c) in enumerate(parts)])
        seeds = np.concatenate([np.arange(f, f + c, dtype=np.uint64) + np.uint64(r.seed0) for r, f, c in parts])
        media = [r.medium() for r, _, _ in parts]
        slot.eng.set_spec_idx(spec_idx)
        slot.eng.evolve(media, seeds, media_idx, stream=slot.stream)
        slot.event.record(slot.stream)
        slot.parts = parts
        slot.busy = True
        return True

    def _collect(self, slot, now):
        obs = slot.eng.observables(stream=slot.stream, check_finite=False)
        o = 0
        for r, f, c in slot.parts:
            r.obs[f:f + c] = obs[o:o + c]
            o += c
            r.n_done += c
            if r.n_done == r.ntraj:
                r.done_time = now
                self.inflight -= r.ntraj
                self.completed.append(r)
        slot.busy = False
        slot.parts = []

    def poll(self) -> int:
        """One scheduling pass: retire finished launches, admit, launch into free slots.  Returns the
        number of launches in flight."""
        now = time.perf_counter()
        for N, slots in self.slots.items():
            for s in slots:
                if s.busy and s.event.query():
                    self._collect(s, now)
        self._admit(now)
        busy = 0
        for N, slots in self.slots.items():
            for s in slots:
                if not s.busy:
                    self._launch(N, s)
                busy += s.busy
        return busy

    def idle(self) -> bool:
        return not self.waiting and all(not q for q in self.pending.values()) and \
            all(not s.busy for sl in self.slots.values() for s in sl)

    def run_stream(self, requests, arrivals_s, poll_interval_s: float = 0.0005, timeout_s: float = 3600.0):
        """Replays a request stream: request i is submitted at arrivals_s[i] seconds after the start.
        Returns the wall time of the whole stream."""
        t0 = time.perf_counter()
        i = 0
        while True:
            now = time.perf_counter() - t0
            while i < len(requests) and arrivals_s[i] <= now:
                self.submit(requests[i], now=t0 + arrivals_s[i])
                i += 1
            self.poll()
            if i == len(requests) and self.idle():
                break
            if now > timeout_s:
                raise TimeoutError("request stream did not finish")
            time.sleep(poll_interval_s)
        return time.perf_counter() - t0

    def close(self):
        for sl in self.slots.values():
            for s in sl:
                s.eng.close()


def latency_stats(reqs):
    lat = np.array([r.done_time - r.arrival for r in reqs])
    return {"n": int(len(lat)), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}


def requests_from_stream(stream: dict, seed_stride: int = 1 << 20):
    """Builds Request objects from inputs.serving_stream()."""
    reqs = []
    for i in range(len(stream["arrival_s"])):
        reqs.append(Request(rid=i, N=int(stream["N"][i]), init=int(stream["init"][i]), T0=float(stream["T0"][i]),
                            kappa_hat=float(stream["kappa_hat"][i]), gamma_hat=float(stream["gamma_hat"][i]),
                            ntraj=int(stream["ntraj"][i]), seed0=i * seed_stride))
    return reqs
