"""Thin ctypes binding of libqtraj (include/qtraj.h).

Argument marshalling only: every step of the trajectory path runs in the library's CUDA kernels.
PyTorch provides device memory (the workspace) and streams.  Importing this module never falls
back to anything: if the library is missing or fails to load, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from .build import LIB

NBASIS = 6
BASIS_NAMES = ("1S", "2S", "1P", "3S", "2P", "1D")
FP64, FP32 = 0, 1
FUSED, PLAIN = 0, 1
F_NOJUMP_SHORTCUT, F_BORDERLINE, F_RMAX, F_MAXJUMPS, F_LCAP, F_NONFINITE = 1, 2, 4, 8, 16, 32
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENONFINITE", 6: "EBUSY"}


class QtrajError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"qtraj {STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("alpha_s", C.c_double), ("Nc", C.c_double), ("deriv_type", C.c_int), ("max_jumps", C.c_int),
                ("r_max", C.c_double), ("l_cap", C.c_int), ("use_rmin", C.c_int), ("precision", C.c_int),
                ("form", C.c_int), ("save_states", C.c_int), ("variant", C.c_int), ("t_vacuum", C.c_double),
                ("basis", C.c_int), ("potential", C.c_int), ("ksu_mD_factor", C.c_double)]


class InitSpec(C.Structure):
    _fields_ = [("kind", C.c_int), ("width", C.c_double), ("n", C.c_int), ("l", C.c_int), ("color", C.c_int)]


class Medium(C.Structure):
    _fields_ = [("kind", C.c_int), ("T0", C.c_double), ("tau0", C.c_double), ("Tf", C.c_double),
                ("kappa_hat", C.c_double), ("gamma_hat", C.c_double), ("table_offset", C.c_int),
                ("table_len", C.c_int)]


class RunStats(C.Structure):
    _fields_ = [("steps_executed", C.c_int64), ("nojump_steps", C.c_int64), ("n_traj", C.c_int),
                ("n_shortcut", C.c_int), ("n_groups", C.c_int), ("launches", C.c_int), ("ms_nojump", C.c_float),
                ("ms_main", C.c_float)]


class KernelInfo(C.Structure):
    _fields_ = [("threads_per_traj", C.c_int), ("ctas_per_sm", C.c_int), ("smem_bytes", C.c_int),
                ("regs_per_thread", C.c_int), ("radix", C.c_int), ("sm_count", C.c_int)]


class TrajDesc(C.Structure):
    _fields_ = [("N", C.c_int), ("spec", C.c_int), ("medium", Medium), ("seed", C.c_uint64)]


class ServerConfig(C.Structure):
    _fields_ = [("Ns", C.POINTER(C.c_int)), ("n_N", C.c_int), ("dr", C.c_double), ("dt", C.c_double),
                ("M", C.c_double), ("params", C.POINTER(Params)), ("specs", C.POINTER(InitSpec)), ("n_specs", C.c_int),
                ("slots_per_n", C.c_int), ("waves_per_launch", C.c_int), ("max_inflight_traj", C.c_int64),
                ("order", C.c_int)]


ORDER_ARRIVAL, ORDER_SHORTEST = 0, 1

# qtraj_launch_rec: one finished launch of a server slot
LAUNCH_DTYPE = np.dtype([("N", "<i4"), ("n_traj", "<i4"), ("n_requests", "<i4"), ("pad", "<i4"),
                         ("start_ms", "<f8"), ("end_ms", "<f8")])


# qtraj_traj_desc as a numpy record, to build large requests without a Python loop
TRAJ_DESC_DTYPE = np.dtype([("N", "<i4"), ("spec", "<i4"), ("kind", "<i4"), ("_pad", "<i4"), ("T0", "<f8"),
                            ("tau0", "<f8"), ("Tf", "<f8"), ("kappa_hat", "<f8"), ("gamma_hat", "<f8"),
                            ("table_offset", "<i4"), ("table_len", "<i4"), ("seed", "<u8")])
assert TRAJ_DESC_DTYPE.itemsize == C.sizeof(TrajDesc) == 72

# qtraj_trace_rec: one row of a trajectory's per-step summary
TRACE_DTYPE = np.dtype([("step", "<i4"), ("color", "<i4"), ("l", "<i4"), ("flags", "<i4"), ("norm2", "<f8"),
                        ("ov2", "<f8", NBASIS), ("r_ratio", "<f8")])
assert TRACE_DTYPE.itemsize == 80

OBS_DTYPE = np.dtype([("surv", "<f8", NBASIS), ("ov_re", "<f8", NBASIS), ("ov_im", "<f8", NBASIS),
                      ("norm2", "<f8"), ("r0", "<f8"), ("l", "<i4"), ("color", "<i4"), ("n_jumps", "<i4"),
                      ("n_steps_exec", "<i4"), ("flags", "<i4"), ("first_jump_step", "<i4"),
                      ("last_jump_step", "<i4"), ("jump_digest", "<u4")])
assert OBS_DTYPE.itemsize == 192

# every entry point of include/qtraj.h with its argument and result types
_PROTOS = {
    "qtraj_create": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, C.POINTER(Params), C.POINTER(C.c_void_p)]),
    "qtraj_destroy": (None, [C.c_void_p]),
    "qtraj_last_error": (C.c_char_p, [C.c_void_p]),
    "qtraj_workspace_bytes": (C.c_size_t, [C.c_void_p, C.c_int]),
    "qtraj_init": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int, C.POINTER(InitSpec), C.c_int,
                             C.POINTER(C.c_int)]),
    "qtraj_set_spec_idx": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.c_int]),
    "qtraj_basis_get": (C.c_int, [C.c_void_p, C.c_void_p]),
    "qtraj_fma_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "qtraj_set_trace": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "qtraj_set_profiles": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int]),
    "qtraj_evolve": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Medium), C.c_int, C.POINTER(C.c_int),
                               C.POINTER(C.c_uint64), C.c_void_p]),
    "qtraj_observables": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "qtraj_states": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "qtraj_nojump_results": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "qtraj_last_run_stats": (C.c_int, [C.c_void_p, C.POINTER(RunStats)]),
    "qtraj_kernel_info_get": (C.c_int, [C.c_void_p, C.POINTER(KernelInfo)]),
    "qtraj_server_workspace_bytes": (C.c_int, [C.POINTER(ServerConfig), C.POINTER(C.c_size_t)]),
    "qtraj_server_create": (C.c_int, [C.POINTER(ServerConfig), C.c_void_p, C.c_size_t, C.POINTER(C.c_void_p)]),
    "qtraj_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_uint64]),
    "qtraj_poll": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.c_int, C.POINTER(C.c_int)]),
    "qtraj_request_result": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int]),
    "qtraj_server_counts": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "qtraj_server_destroy": (None, [C.c_void_p]),
    "qtraj_server_launch_log": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_int]),
    "qtraj_dft16_study": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "qtraj_philox4x32_10": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "qtraj_period_draws": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "qtraj_evolve_static": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(InitSpec), C.c_int, C.POINTER(C.c_int),
                                      C.POINTER(Medium), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_uint64),
                                      C.c_void_p, C.c_void_p]),
}

_lib = None


def load(path: str = LIB):
    """Loads libqtraj.so (built by build.build()) and declares its prototypes."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"{path} not found: run paper_2107_06147_gb300.build.build() first")
        L = C.CDLL(path)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int, ctx=None):
    if st != 0:
        raise QtrajError(st, load().qtraj_last_error(ctx).decode())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


@dataclass
class Config:
    N: int = 512
    L: float = 20.0
    dt: float = 0.001
    M: float = 4.65
    alpha_s: float = 0.3
    Nc: float = 3.0
    deriv_type: int = 0
    max_jumps: int = -1
    r_max: float = 1.0
    l_cap: int = -1
    use_rmin: int = 1
    precision: int = FP64
    form: int = FUSED
    save_states: int = 0
    variant: int = 0
    t_vacuum: float = 0.0
    basis: int = 0
    potential: int = 0           # 0: OQS+pNRQCD with jumps (App. E); 1: isotropic KSU, no jumps
    ksu_mD_factor: float = 1.0

    def params(self) -> Params:
        return Params(self.alpha_s, self.Nc, self.deriv_type, self.max_jumps, self.r_max, self.l_cap, self.use_rmin,
                      self.precision, self.form, self.save_states, self.variant, self.t_vacuum, self.basis,
                      self.potential, self.ksu_mD_factor)


def fma_peak(precision=FP32) -> float:
    """Measured FMA throughput of the current device, TFLOP/s."""
    v = C.c_double()
    _check(load().qtraj_fma_peak(precision, C.byref(v)))
    return v.value


def init_spec(kind="gauss", width=0.2, n=1, l=0, color=0) -> InitSpec:
    """kind 'gauss', 'coulomb' (analytic eigenstate) or 'numerical' (eigenstate of the grid's H)."""
    return InitSpec({"gauss": 0, "coulomb": 1, "numerical": 2}[kind], width, n, l, color)


def medium(T0=0.425, tau0=0.6, Tf=0.25, kappa_hat=5.0, gamma_hat=0.0) -> Medium:
    return Medium(0, T0, tau0, Tf, kappa_hat, gamma_hat, 0, 0)


def table_medium(table_offset: int, table_len: int, Tf=0.25, kappa_hat=5.0, gamma_hat=0.0) -> Medium:
    """A tabulated T(tau) medium: points [table_offset, table_offset + table_len) of the context's
    profile store (Engine.set_profiles)."""
    return Medium(1, 0.0, 0.0, Tf, kappa_hat, gamma_hat, table_offset, table_len)


class Engine:
    """One libqtraj context plus its workspace (a torch uint8 tensor on the current device)."""

    def __init__(self, cfg: Config):
        self.cfg = cfg
        self.lib = load()
        h = C.c_void_p()
        p = cfg.params()
        _check(self.lib.qtraj_create(cfg.N, cfg.L, cfg.dt, cfg.M, C.byref(p), C.byref(h)))
        self.ctx = h
        self.ws = None
        self.n_traj = 0
        self.batch = 0

    def close(self):
        if self.ctx:
            self.lib.qtraj_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self, n_traj: int) -> int:
        return int(self.lib.qtraj_workspace_bytes(self.ctx, n_traj))

    def init(self, specs, n_traj: int, spec_idx=None, workspace=None):
        """Binds a workspace for n_traj trajectories (allocated with torch unless given) and sets the
        initial states."""
        import torch
        nb = self.workspace_bytes(n_traj)
        if workspace is None:
            workspace = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        self.ws = workspace
        base = workspace.data_ptr()
        ptr = (base + 255) & ~255
        have = max(0, workspace.numel() * workspace.element_size() - (ptr - base))
        arr = (InitSpec * len(specs))(*specs)
        idx = None
        if spec_idx is not None:
            self._spec_idx = np.ascontiguousarray(spec_idx, dtype=np.int32)
            idx = self._spec_idx.ctypes.data_as(C.POINTER(C.c_int))
        _check(self.lib.qtraj_init(self.ctx, C.c_void_p(ptr), have, n_traj, arr, len(specs), idx), self.ctx)
        self.n_traj = n_traj

    def basis(self) -> np.ndarray:
        """The overlap basis, (NBASIS, N) in the order of the survival ratios."""
        out = np.zeros((NBASIS, self.cfg.N))
        _check(self.lib.qtraj_basis_get(self.ctx, C.c_void_p(out.ctypes.data)), self.ctx)
        return out

    def set_trace(self, every: int, n_traced: int = 1, max_records: int = 1024):
        """Per-step summary rows for the first n_traced trajectories of later evolves (every = 0: off).
        The row buffers are torch device tensors held by the engine."""
        import torch
        if every <= 0:
            _check(self.lib.qtraj_set_trace(self.ctx, 0, 0, 0, None, None), self.ctx)
            self._trace = None
            return
        rec = torch.zeros(n_traced * max_records * TRACE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        cnt = torch.zeros(n_traced, dtype=torch.int32, device="cuda")
        _check(self.lib.qtraj_set_trace(self.ctx, every, n_traced, max_records, C.c_void_p(rec.data_ptr()),
                                        C.c_void_p(cnt.data_ptr())), self.ctx)
        self._trace = (rec, cnt, n_traced, max_records)

    def trace(self) -> list:
        """The summary rows of each traced trajectory of the last evolve (synchronises the device)."""
        import torch
        rec, cnt, n, cap = self._trace
        torch.cuda.synchronize()
        r = np.frombuffer(rec.cpu().numpy().tobytes(), dtype=TRACE_DTYPE).reshape(n, cap)
        c = cnt.cpu().numpy()
        return [r[i, : c[i]].copy() for i in range(n)]

    def set_profiles(self, tau, T):
        """Sets the profile store of tabulated media: points (tau [fm/c], T [GeV]); synchronous."""
        t = np.ascontiguousarray(tau, dtype=np.float64)
        v = np.ascontiguousarray(T, dtype=np.float64)
        dp = C.POINTER(C.c_double)
        _check(self.lib.qtraj_set_profiles(self.ctx, t.ctypes.data_as(dp), v.ctypes.data_as(dp), len(t)), self.ctx)

    def set_spec_idx(self, spec_idx):
        """Re-binds the initial state of trajectories [0, len(spec_idx)) (host-side, no device sync)."""
        self._spec_idx2 = np.ascontiguousarray(spec_idx, dtype=np.int32)
        _check(self.lib.qtraj_set_spec_idx(self.ctx, self._spec_idx2.ctypes.data_as(C.POINTER(C.c_int)),
                                           len(self._spec_idx2)), self.ctx)

    def evolve(self, media, seeds, medium_idx=None, batch: int | None = None, stream=None):
        batch = len(seeds) if batch is None else batch
        arr = (Medium * len(media))(*media)
        self._seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        idx = None
        if medium_idx is not None:
            self._midx = np.ascontiguousarray(medium_idx, dtype=np.int32)
            idx = self._midx.ctypes.data_as(C.POINTER(C.c_int))
        _check(self.lib.qtraj_evolve(self.ctx, batch, arr, len(media), idx,
                                     self._seeds.ctypes.data_as(C.POINTER(C.c_uint64)),
                                     C.c_void_p(_stream_ptr(stream))), self.ctx)
        self.batch = batch

    def observables(self, stream=None, check_finite: bool = True) -> np.ndarray:
        out = np.zeros(self.batch, dtype=OBS_DTYPE)
        st = self.lib.qtraj_observables(self.ctx, C.c_void_p(out.ctypes.data), 0, C.c_void_p(_stream_ptr(stream)))
        if st != 5 or check_finite:
            _check(st, self.ctx)
        return out

    def observables_device(self, out_tensor, stream=None):
        _check(self.lib.qtraj_observables(self.ctx, C.c_void_p(out_tensor.data_ptr()), 1,
                                          C.c_void_p(_stream_ptr(stream))), self.ctx)

    def states(self, stream=None) -> np.ndarray:
        out = np.zeros((self.batch, self.cfg.N), dtype=np.complex128)
        _check(self.lib.qtraj_states(self.ctx, C.c_void_p(out.ctypes.data), 0, C.c_void_p(_stream_ptr(stream))),
               self.ctx)
        return out

    def nojump_results(self, n_pairs: int) -> np.ndarray:
        out = np.zeros(n_pairs, dtype=OBS_DTYPE)
        nw = C.c_int()
        _check(self.lib.qtraj_nojump_results(self.ctx, C.c_void_p(out.ctypes.data), n_pairs, C.byref(nw)), self.ctx)
        return out[: nw.value]

    def stats(self) -> RunStats:
        s = RunStats()
        _check(self.lib.qtraj_last_run_stats(self.ctx, C.byref(s)), self.ctx)
        return s

    def kernel_info(self) -> KernelInfo:
        k = KernelInfo()
        _check(self.lib.qtraj_kernel_info_get(self.ctx, C.byref(k)), self.ctx)
        return k


def philox4x32_10(ctr, key, stream=None):
    """Philox4x32-10 words of the device generator: ctr (n, 4) and key (n, 2) uint32 torch device
    tensors in, an (n, 4) uint32 device tensor out (int32 storage)."""
    import torch
    n = int(ctr.shape[0])
    out = torch.empty((n, 4), dtype=torch.int32, device=ctr.device)
    _check(load().qtraj_philox4x32_10(C.c_void_p(ctr.data_ptr()), C.c_void_p(key.data_ptr()), n,
                                      C.c_void_p(out.data_ptr()), C.c_void_p(_stream_ptr(stream))))
    return out


def period_draws(seeds, k, stream=None):
    """The (r, u_l, u_c) uniforms of waiting period k[i] of seed seeds[i] (int64 / int32 torch device
    tensors holding uint64 / uint32 values), as the trajectory kernels draw them: an (n, 3) float64
    device tensor."""
    import torch
    n = int(seeds.shape[0])
    out = torch.empty((n, 3), dtype=torch.float64, device=seeds.device)
    _check(load().qtraj_period_draws(C.c_void_p(seeds.data_ptr()), C.c_void_p(k.data_ptr()), n,
                                     C.c_void_p(out.data_ptr()), C.c_void_p(_stream_ptr(stream))))
    return out


def dft16_study(method: int, x: np.ndarray, passes: int):
    """Radix-16 DFT blocks y = (F/4) x on the CUDA cores (method 0) or the tensor cores (1 BF16X3,
    2 BF16X9, 3 FP16X3, 4 FP16X5), qtraj_dft16_study: x (n_batches, 256, 16) complex, converted to
    FP32; returns ((F/4)^passes applied to every 16-point column, ms of the timed launch)."""
    xi = np.ascontiguousarray(x, dtype=np.complex128)
    if xi.ndim != 3 or xi.shape[1:] != (256, 16):
        raise ValueError("x must have shape (n_batches, 256, 16)")
    y = np.zeros_like(xi)
    ms = C.c_double()
    _check(load().qtraj_dft16_study(method, xi.shape[0], passes, C.c_void_p(xi.ctypes.data), C.c_void_p(y.ctypes.data),
                                    C.byref(ms)))
    return y, ms.value
