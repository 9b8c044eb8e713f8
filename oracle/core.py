"""ctypes wrapper of ``qtraj_oracle.c`` (test infrastructure only).

Every function here marshals numpy arrays into the C oracle and back; the arithmetic of the method
lives in ``qtraj_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qtraj_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboqt.so")

NBASIS = 6
BASIS_NAMES = ("1S", "2S", "1P", "3S", "2P", "1D")
F_NOJUMP_SHORTCUT, F_BORDERLINE, F_RMAX, F_MAXJUMPS, F_LCAP, F_NONFINITE = 1, 2, 4, 8, 16, 32


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_lib/liboqt.so`` with gcc (plain C99, -O2)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("N", C.c_int), ("L", C.c_double), ("dt", C.c_double), ("M", C.c_double),
                ("alpha_s", C.c_double), ("Nc", C.c_double), ("deriv_type", C.c_int),
                ("max_jumps", C.c_int), ("r_max", C.c_double), ("l_cap", C.c_int),
                ("use_rmin", C.c_int), ("t_vac", C.c_double), ("basis", C.POINTER(C.c_double)),
                ("potential", C.c_int), ("ksu_fmd", C.c_double)]


class Init(C.Structure):
    _fields_ = [("kind", C.c_int), ("width", C.c_double), ("n", C.c_int), ("l", C.c_int),
                ("color", C.c_int), ("u0", C.POINTER(C.c_double))]


class Medium(C.Structure):
    _fields_ = [("T0", C.c_double), ("tau0", C.c_double), ("Tf", C.c_double),
                ("kappa_hat", C.c_double), ("gamma_hat", C.c_double), ("kind", C.c_int),
                ("tab_tau", C.POINTER(C.c_double)), ("tab_T", C.POINTER(C.c_double)), ("tab_n", C.c_int)]


class Obs(C.Structure):
    _fields_ = [("surv", C.c_double * NBASIS), ("ov_re", C.c_double * NBASIS),
                ("ov_im", C.c_double * NBASIS), ("norm2", C.c_double), ("r0", C.c_double),
                ("l", C.c_int), ("color", C.c_int), ("n_jumps", C.c_int), ("n_steps_exec", C.c_int),
                ("flags", C.c_int), ("first_jump_step", C.c_int), ("last_jump_step", C.c_int),
                ("jump_digest", C.c_uint32)]


TRACE_DTYPE = np.dtype([("step", "<i4"), ("color", "<i4"), ("l", "<i4"), ("flags", "<i4"), ("norm2", "<f8"),
                        ("ov2", "<f8", NBASIS), ("r_ratio", "<f8")])

OBS_DTYPE = np.dtype([("surv", "<f8", NBASIS), ("ov_re", "<f8", NBASIS), ("ov_im", "<f8", NBASIS),
                      ("norm2", "<f8"), ("r0", "<f8"), ("l", "<i4"), ("color", "<i4"),
                      ("n_jumps", "<i4"), ("n_steps_exec", "<i4"), ("flags", "<i4"),
                      ("first_jump_step", "<i4"), ("last_jump_step", "<i4"), ("jump_digest", "<u4")])
assert OBS_DTYPE.itemsize == C.sizeof(Obs)

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        cd = C.POINTER(C.c_double)
        L.oqt_fft.argtypes = [C.c_int, cd, C.c_int]
        L.oqt_fft.restype = C.c_int
        L.oqt_dft.argtypes = [C.c_int, cd, cd, C.c_int]
        L.oqt_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
        L.oqt_draws.argtypes = [C.c_uint64, C.c_uint32, cd, cd, cd]
        L.oqt_philox_many.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oqt_draws_many.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oqt_bohr_radius.argtypes = [C.POINTER(Params)]
        L.oqt_bohr_radius.restype = C.c_double
        L.oqt_n_steps.argtypes = [C.POINTER(Params), C.POINTER(Medium)]
        L.oqt_n_steps.restype = C.c_int
        L.oqt_T3.argtypes = [C.POINTER(Params), C.POINTER(Medium), C.c_int]
        L.oqt_T3.restype = C.c_double
        L.oqt_kinetic.argtypes = [C.POINTER(Params), C.c_int]
        L.oqt_kinetic.restype = C.c_double
        L.oqt_norm2.argtypes = [C.POINTER(Params), cd]
        L.oqt_norm2.restype = C.c_double
        L.oqt_eigenstate.argtypes = [C.POINTER(Params), C.c_int, C.c_int, cd]
        L.oqt_initial_state.argtypes = [C.POINTER(Params), C.POINTER(Init), cd]
        L.oqt_strang_step.argtypes = [C.POINTER(Params), cd, C.c_int, C.c_int, C.c_double, C.c_double,
                                      C.c_double]
        L.oqt_evolve_nojump.argtypes = [C.POINTER(Params), cd, C.c_int, C.c_int, C.POINTER(Medium), C.c_int,
                                        C.c_int, cd]
        L.oqt_nojump_run.argtypes = [C.POINTER(Params), C.POINTER(Init), C.POINTER(Medium), C.POINTER(Obs), cd]
        L.oqt_trajectory.argtypes = [C.POINTER(Params), C.POINTER(Init), C.POINTER(Medium), C.c_uint64,
                                     C.POINTER(Obs), C.POINTER(Obs), cd]
        L.oqt_run_batch.argtypes = [C.POINTER(Params), C.c_int, C.POINTER(Init), C.c_int, C.POINTER(C.c_int),
                                    C.POINTER(Medium), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_uint64),
                                    C.POINTER(Obs), cd, C.POINTER(Obs), C.c_int]
        L.oqt_run_batch.restype = C.c_int
        L.oqt_jump_l.argtypes = [C.c_int, C.c_double]
        L.oqt_jump_l.restype = C.c_int
        L.oqt_jump_color.argtypes = [C.POINTER(Params), C.c_int, C.c_double]
        L.oqt_jump_color.restype = C.c_int
        L.oqt_potential_parts.argtypes = [C.POINTER(Params), C.c_int, C.c_int, C.c_double, C.c_double,
                                          C.c_double, C.c_double, cd, cd]
        L.oqt_vacuum_steps.argtypes = [C.POINTER(Params)]
        L.oqt_vacuum_steps.restype = C.c_int
        L.oqt_start_state.argtypes = [C.POINTER(Params), C.POINTER(Init), cd]
        L.oqt_trajectory_traced.argtypes = [C.POINTER(Params), C.POINTER(Init), C.POINTER(Medium), C.c_uint64,
                                            C.POINTER(Obs), C.POINTER(Obs), cd, C.c_int, C.c_void_p, C.c_int,
                                            C.POINTER(C.c_int)]
        L.oqt_kappa_fit.argtypes = [C.c_int, C.c_double]
        L.oqt_kappa_fit.restype = C.c_double
        for f in ("oqt_expE1", "oqt_expmEi", "oqt_ksu_phi"):
            getattr(L, f).argtypes = [C.c_double]
            getattr(L, f).restype = C.c_double
        L.oqt_alpha_s_run.argtypes = [C.c_double, C.c_double]
        L.oqt_alpha_s_run.restype = C.c_double
        L.oqt_ksu_debye_mass.argtypes = [C.POINTER(Params), C.c_double]
        L.oqt_ksu_debye_mass.restype = C.c_double
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ------------------------------------------------------------------------------------------------
# parameter records
# ------------------------------------------------------------------------------------------------
@dataclass
class Grid:
    """Grid and physics constants of one run (paper Table 1: num, L, dt, m, alpha)."""
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
    t_vac: float = 0.0
    basis: object = None          # (NBASIS, N) overlap basis (numerical eigenstates); None: analytic
    potential: int = 0            # 0: App. E OQS+pNRQCD with jumps; 1: isotropic KSU (no jumps)
    ksu_fmd: float = 1.0          # F_mD of the KSU Debye mass

    def c(self) -> Params:
        b = None
        if self.basis is not None:
            self._basis_c = np.ascontiguousarray(self.basis, dtype=np.float64)
            b = _dp(self._basis_c)
        return Params(self.N, self.L, self.dt, self.M, self.alpha_s, self.Nc, self.deriv_type,
                      self.max_jumps, self.r_max, self.l_cap, self.use_rmin, self.t_vac, b, self.potential,
                      self.ksu_fmd)


def init_spec(kind: str = "gauss", width: float = 0.2, n: int = 1, l: int = 0, color: int = 0) -> Init:
    return Init(0 if kind == "gauss" else 1, width, n, l, color, None)


def given_state(u0, n: int, l: int, color: int = 0) -> Init:
    """Initial state kind 2: the given (numerical) eigenstate (n, l), discretely normalised; the
    record keeps its own copy of the values alive."""
    a = np.ascontiguousarray(np.real(u0), dtype=np.float64)
    s = Init(2, 0.0, n, l, color, _dp(a))
    s._keep = a
    return s


def medium(T0=0.425, tau0=0.6, Tf=0.25, kappa_hat=5.0, gamma_hat=0.0) -> Medium:
    return Medium(T0, tau0, Tf, kappa_hat, gamma_hat, 0, None, None, 0)


def table_medium(tau, T, Tf=0.25, kappa_hat=5.0, gamma_hat=0.0) -> Medium:
    """A tabulated T(tau) medium (tau ascending, fm/c; T in GeV).  The record points into its own
    copies of the arrays, kept alive on the record."""
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    m = Medium(float(T[0]), float(tau[0]), Tf, kappa_hat, gamma_hat, 1, _dp(tau), _dp(T), len(tau))
    m._keep = (tau, T)
    return m


# ------------------------------------------------------------------------------------------------
# thin wrappers
# ------------------------------------------------------------------------------------------------
def fft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    y = np.ascontiguousarray(x, dtype=np.complex128).copy()
    rc = lib().oqt_fft(len(y), _dp(y), sign)
    if rc != 0:
        raise ValueError("length must be a power of two")
    return y


def dft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    xx = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(xx)
    lib().oqt_dft(len(xx), _dp(xx), _dp(out), sign)
    return out


def philox4x32_10(ctr, key) -> tuple:
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().oqt_philox4x32_10(c, k, o)
    return tuple(o)


def philox_many(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x32-10 words of n (counter, key) pairs: ctr (n, 4), key (n, 2) uint32 -> (n, 4) uint32."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros((len(c), 4), dtype=np.uint32)
    lib().oqt_philox_many(len(c), c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def draws_many(seeds: np.ndarray, k: np.ndarray) -> np.ndarray:
    """The (r, u_l, u_c) uniforms of waiting period k[i] of seed seeds[i] -> (n, 3) float64."""
    s = np.ascontiguousarray(seeds, dtype=np.uint64)
    kk = np.ascontiguousarray(k, dtype=np.uint32)
    out = np.zeros((len(s), 3))
    lib().oqt_draws_many(len(s), s.ctypes.data, kk.ctypes.data, out.ctypes.data)
    return out


def draws(seed: int, k: int):
    r, ul, uc = C.c_double(), C.c_double(), C.c_double()
    lib().oqt_draws(C.c_uint64(seed), C.c_uint32(k), C.byref(r), C.byref(ul), C.byref(uc))
    return r.value, ul.value, uc.value


def bohr_radius(g: Grid) -> float:
    p = g.c()
    return lib().oqt_bohr_radius(C.byref(p))


def n_steps(g: Grid, m: Medium) -> int:
    p = g.c()
    return lib().oqt_n_steps(C.byref(p), C.byref(m))


def T3(g: Grid, m: Medium, n: int) -> float:
    p = g.c()
    return lib().oqt_T3(C.byref(p), C.byref(m), n)


def kinetic(g: Grid, k: int) -> float:
    p = g.c()
    return lib().oqt_kinetic(C.byref(p), k)


def norm2(g: Grid, u: np.ndarray) -> float:
    p = g.c()
    uu = np.ascontiguousarray(u, dtype=np.complex128)
    return lib().oqt_norm2(C.byref(p), _dp(uu))


def eigenstate(g: Grid, n: int, l: int) -> np.ndarray:
    p = g.c()
    phi = np.zeros(g.N)
    lib().oqt_eigenstate(C.byref(p), n, l, _dp(phi))
    return phi


def initial_state(g: Grid, spec: Init) -> np.ndarray:
    p = g.c()
    u = np.zeros(g.N, dtype=np.complex128)
    lib().oqt_initial_state(C.byref(p), C.byref(spec), _dp(u))
    return u


def vacuum_steps(g: Grid) -> int:
    p = g.c()
    return lib().oqt_vacuum_steps(C.byref(p))


def start_state(g: Grid, spec: Init) -> np.ndarray:
    """The initial state after the vacuum evolution of g.t_vac (the initial state itself if 0)."""
    p = g.c()
    u = np.zeros(g.N, dtype=np.complex128)
    lib().oqt_start_state(C.byref(p), C.byref(spec), _dp(u))
    return u


def strang_step(g: Grid, u: np.ndarray, color: int, l: int, T3v: float, kappa_hat: float,
                gamma_hat: float) -> np.ndarray:
    p = g.c()
    v = np.ascontiguousarray(u, dtype=np.complex128).copy()
    lib().oqt_strang_step(C.byref(p), _dp(v), color, l, T3v, kappa_hat, gamma_hat)
    return v


def evolve_nojump(g: Grid, u: np.ndarray, color: int, l: int, m: Medium, n0: int, nsteps: int):
    """H_eff evolution from step n0 for nsteps steps; returns (state, norm^2 after every step)."""
    p = g.c()
    v = np.ascontiguousarray(u, dtype=np.complex128).copy()
    hist = np.zeros(max(nsteps, 1))
    lib().oqt_evolve_nojump(C.byref(p), _dp(v), color, l, C.byref(m), n0, nsteps, _dp(hist))
    return v, hist[:nsteps]


def jump_l(l: int, ul: float) -> int:
    return lib().oqt_jump_l(l, ul)


def jump_color(g: Grid, color: int, uc: float) -> int:
    p = g.c()
    return lib().oqt_jump_color(C.byref(p), color, uc)


def trajectory_trace(g: Grid, spec: Init, m: Medium, seed: int, every: int, cap: int = 100000):
    """One trajectory without the rMin shortcut, with its per-step summary rows (TRACE_DTYPE)."""
    p = g.c()
    p.use_rmin = 0
    o = Obs()
    rec = np.zeros(cap, dtype=TRACE_DTYPE)
    n = C.c_int()
    lib().oqt_trajectory_traced(C.byref(p), C.byref(spec), C.byref(m), C.c_uint64(seed), None, C.byref(o), None,
                                every, C.c_void_p(rec.ctypes.data), cap, C.byref(n))
    return np.frombuffer(bytes(o), dtype=OBS_DTYPE).copy()[0], rec[: n.value].copy()


def expE1(x: float) -> float:
    """e^x E1(x) for x > 0 (the oracle's own evaluation)."""
    return lib().oqt_expE1(x)


def expmEi(x: float) -> float:
    """e^-x Ei(x) for x > 0 (the oracle's own evaluation)."""
    return lib().oqt_expmEi(x)


def ksu_phi(rhat: float) -> float:
    """phi(rhat) of the isotropic KSU potential's imaginary part (App. E)."""
    return lib().oqt_ksu_phi(rhat)


def alpha_s_run(mu: float, Nc: float = 3.0) -> float:
    """The one-loop running coupling from alpha_s(5 GeV) = 0.2034 (N_F = 3)."""
    return lib().oqt_alpha_s_run(mu, Nc)


def ksu_debye_mass(g: Grid, T: float) -> float:
    p = g.c()
    return lib().oqt_ksu_debye_mass(C.byref(p), T)


def ksu_potential(g: Grid, l: int, T: float, r: float) -> complex:
    """The KSU potential V_R + i V_I + l(l+1)/(M r^2) at temperature T (GeV) and r (GeV^-1)."""
    h = Grid(**{k: getattr(g, k) for k in g.__dataclass_fields__})
    h.potential = 1
    return potential(h, 0, l, T ** 3, 0.0, 0.0, r)


def kappa_fit(which: int, T: float) -> float:
    """kappa_hat(T) of lattice fit `which` (1 central, 2 lower, 3 upper; App. E)."""
    return lib().oqt_kappa_fit(which, T)


def potential(g: Grid, color: int, l: int, T3v: float, kappa_hat: float, gamma_hat: float, r: float) -> complex:
    p = g.c()
    re, im = C.c_double(), C.c_double()
    lib().oqt_potential_parts(C.byref(p), color, l, T3v, kappa_hat, gamma_hat, r, C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def obs_to_numpy(obs_arr) -> np.ndarray:
    return np.frombuffer(bytes(obs_arr), dtype=OBS_DTYPE).copy()


def nojump_run(g: Grid, spec: Init, m: Medium, want_state: bool = False):
    p = g.c()
    o = Obs()
    u = np.zeros(g.N, dtype=np.complex128)
    lib().oqt_nojump_run(C.byref(p), C.byref(spec), C.byref(m), C.byref(o), _dp(u) if want_state else None)
    rec = np.frombuffer(bytes(o), dtype=OBS_DTYPE).copy()[0]
    return (rec, u) if want_state else rec


def trajectory(g: Grid, spec: Init, m: Medium, seed: int, nojump=None, want_state: bool = False):
    p = g.c()
    o = Obs()
    nj = None
    if nojump is not None:
        nj = Obs.from_buffer_copy(np.asarray(nojump, dtype=OBS_DTYPE).tobytes())
    u = np.zeros(g.N, dtype=np.complex128)
    lib().oqt_trajectory(C.byref(p), C.byref(spec), C.byref(m), C.c_uint64(seed),
                         C.byref(nj) if nj is not None else None, C.byref(o), _dp(u) if want_state else None)
    rec = np.frombuffer(bytes(o), dtype=OBS_DTYPE).copy()[0]
    return (rec, u) if want_state else rec


def run_batch(g: Grid, inits, init_idx, media, medium_idx, seeds, n_threads: int | None = None,
              want_states: bool = False):
    """Runs len(seeds) trajectories; returns (obs records, no-jump records per (init, medium) pair,
    final states or None)."""
    p = g.c()
    n = len(seeds)
    ni, nm = len(inits), len(media)
    ci = (Init * ni)(*inits)
    cm = (Medium * nm)(*media)
    ii = np.ascontiguousarray(init_idx, dtype=np.int32)
    mi = np.ascontiguousarray(medium_idx, dtype=np.int32)
    sd = np.ascontiguousarray(seeds, dtype=np.uint64)
    out = (Obs * max(n, 1))()
    nj = (Obs * (ni * nm))()
    u = np.zeros((n, g.N), dtype=np.complex128) if want_states else None
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    lib().oqt_run_batch(C.byref(p), n, ci, ni, ii.ctypes.data_as(C.POINTER(C.c_int)), cm, nm,
                        mi.ctypes.data_as(C.POINTER(C.c_int)), sd.ctypes.data_as(C.POINTER(C.c_uint64)),
                        out, _dp(u) if want_states else None, nj, n_threads)
    return obs_to_numpy(out)[:n], obs_to_numpy(nj), u
