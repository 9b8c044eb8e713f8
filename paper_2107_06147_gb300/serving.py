"""Continuous batching of trajectory requests: a thin binding of libqtraj's server.

The scheduler is native (include/qtraj.h, "Serving"; csrc/serve.cu): for every grid size N the
server keeps a few engine slots (a context with its share of the workspace, its own CUDA stream and
a pinned result buffer).  qtraj_poll never blocks: it retires finished launches, admits queued
requests first come first served within a budget of trajectories in flight, and fills every idle
slot with up to `wave_mult` waves of trajectories taken across the admitted requests of that N in
arrival order or least work first (`order`) -- trajectories of several requests share a launch, a request that arrives while others run joins
the next launch that frees up, and slots of different N run concurrently on the device.

Each trajectory's result depends only on its own inputs (initial state, medium, seed), never on the
launch it shares, so a request's results are the same alone and in the mix.

This module marshals requests into trajectory descriptors, holds the workspace (a torch tensor), and
replays timed request streams; it does no arithmetic of the method.
"""
from __future__ import annotations

import ctypes as C
import time
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
    init: int            # index into the server's initial-state catalogue (INIT_SPECS by default)
    T0: float
    kappa_hat: float
    gamma_hat: float
    ntraj: int
    seed0: int
    Tf: float = 0.25
    arrival: float = 0.0
    done_time: float = -1.0
    obs: np.ndarray = field(default=None, repr=False)

    def descriptors(self) -> np.ndarray:
        """The request's trajectories: seeds seed0 .. seed0 + ntraj - 1, all on grid N."""
        d = np.zeros(self.ntraj, dtype=qtraj.TRAJ_DESC_DTYPE)
        d["N"] = self.N
        d["spec"] = self.init
        d["T0"], d["tau0"], d["Tf"] = self.T0, 0.6, self.Tf
        d["kappa_hat"], d["gamma_hat"] = self.kappa_hat, self.gamma_hat
        d["seed"] = np.uint64(self.seed0) + np.arange(self.ntraj, dtype=np.uint64)
        return d


class Server:
    """A libqtraj server over the grid sizes Ns (L = N dr); see the module docstring."""

    def __init__(self, Ns=(1024, 2048, 4096, 8192, 16384), slots_per_n: int = 2, precision=qtraj.FP32,
                 max_inflight_traj: int = 1 << 20, dr: float = 5.0 / 512, dt: float = 0.001, wave_mult: int = 1,
                 specs=INIT_SPECS, cfg: qtraj.Config | None = None, order: int = qtraj.ORDER_ARRIVAL):
        import torch
        self.lib = qtraj.load()
        base = cfg or qtraj.Config(precision=precision)
        self._params = base.params()
        self._Ns = (C.c_int * len(Ns))(*Ns)
        self._specs = (qtraj.InitSpec * len(specs))(*specs)
        self._cfg = qtraj.ServerConfig(self._Ns, len(Ns), dr, dt, base.M, C.pointer(self._params), self._specs,
                                       len(specs), slots_per_n, wave_mult, max_inflight_traj, order)
        nb = C.c_size_t()
        qtraj._check(self.lib.qtraj_server_workspace_bytes(C.byref(self._cfg), C.byref(nb)))
        self.ws = torch.empty(nb.value + 256, dtype=torch.uint8, device="cuda")
        ptr = (self.ws.data_ptr() + 255) & ~255
        h = C.c_void_p()
        qtraj._check(self.lib.qtraj_server_create(C.byref(self._cfg), C.c_void_p(ptr), nb.value, C.byref(h)))
        self.h = h
        self.requests = {}
        self.completed = []
        self._ids = (C.c_uint64 * 256)()

    def submit(self, req: Request, now: float | None = None):
        req.arrival = time.perf_counter() if now is None else now
        d = req.descriptors()
        qtraj._check(self.lib.qtraj_submit(self.h, C.c_void_p(d.ctypes.data), len(d), req.rid))
        self.requests[req.rid] = req

    def poll(self) -> list:
        """One scheduling pass; returns the requests that finished in it (their .obs filled)."""
        n = C.c_int()
        qtraj._check(self.lib.qtraj_poll(self.h, self._ids, len(self._ids), C.byref(n)))
        now = time.perf_counter()
        out = []
        for i in range(n.value):
            r = self.requests.pop(int(self._ids[i]))
            r.obs = np.zeros(r.ntraj, dtype=qtraj.OBS_DTYPE)
            qtraj._check(self.lib.qtraj_request_result(self.h, r.rid, C.c_void_p(r.obs.ctypes.data), r.ntraj))
            r.done_time = now
            self.completed.append(r)
            out.append(r)
        return out

    def counts(self):
        """(requests waiting for admission, admitted and unfinished, launches in flight)."""
        w, a, l = C.c_int(), C.c_int(), C.c_int()
        qtraj._check(self.lib.qtraj_server_counts(self.h, C.byref(w), C.byref(a), C.byref(l)))
        return w.value, a.value, l.value

    def launch_log(self, clear: bool = False) -> np.ndarray:
        """The finished launches (grid size, trajectories, requests, device start/end in ms)."""
        out = np.zeros(4096, dtype=qtraj.LAUNCH_DTYPE)
        n = C.c_int()
        qtraj._check(self.lib.qtraj_server_launch_log(self.h, C.c_void_p(out.ctypes.data), len(out), C.byref(n),
                                                      1 if clear else 0))
        return out[: n.value].copy()

    def idle(self) -> bool:
        return not self.requests and self.counts() == (0, 0, 0)

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
        if self.h:
            self.lib.qtraj_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


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
