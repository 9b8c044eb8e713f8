"""Seeded synthetic workloads for the quantum-trajectory engine.

This module only draws and lists inputs (grids, initial-state specs, media, seeds, request
streams); it holds none of the method's arithmetic, so the tests can feed the same inputs to the
CUDA path and to the CPU oracle.  Every recipe follows the paper's own benchmark workload -- a
Gaussian S wave in a Bjorken-cooled medium, T0 = 425 MeV at tau0 = 0.6 fm/c down to Tf = 250 MeV
(Sec. 5) -- with the sizes of the engine's headline configurations.  Random parameters come from
numpy's PCG64 with a fixed seed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class InitSpec:
    """Initial state: kind 'gauss' is r^{l+1} exp(-r^2/(2 width^2)); kind 'coulomb' is the
    Coulomb eigenstate (n, l).  color 0 = singlet, 1 = octet."""
    kind: str = "gauss"
    width: float = 0.2
    n: int = 1
    l: int = 0
    color: int = 0


@dataclass
class MediumSpec:
    """Bjorken medium T(tau) = T0 (tau0/tau)^{1/3} from tau0 (fm/c) until T < Tf (GeV), with the
    transport coefficients kappa_hat, gamma_hat."""
    T0: float = 0.425
    tau0: float = 0.6
    Tf: float = 0.25
    kappa_hat: float = 5.0
    gamma_hat: float = 0.0


@dataclass
class GridSpec:
    N: int = 512
    L: float = 20.0
    dt: float = 0.001
    M: float = 4.65
    alpha_s: float = 0.3
    Nc: float = 3.0


@dataclass
class Workload:
    name: str
    grid: GridSpec
    inits: list
    media: list
    init_idx: np.ndarray
    medium_idx: np.ndarray
    seeds: np.ndarray
    notes: dict = field(default_factory=dict)

    @property
    def n_traj(self) -> int:
        return int(len(self.seeds))


GAUSS_1S = InitSpec("gauss", 0.2, 1, 0, 0)
COULOMB_2S = InitSpec("coulomb", 0.0, 2, 0, 0)
GAUSS_1P = InitSpec("gauss", 0.2, 2, 1, 0)


def tiny(n_traj: int = 8) -> Workload:
    """8 trajectories, singlet Gaussian S wave (width 0.2 GeV^-1), N=512, L=20, dt=0.001,
    kappa_hat=5, gamma_hat=0, Bjorken 0.425 GeV at 0.6 fm/c down to 0.25 GeV, seeds 0..7."""
    return Workload("tiny N=512 L=20 dt=0.001 kappa=5 gamma=0", GridSpec(512, 20.0, 0.001),
                    [GAUSS_1S], [MediumSpec()], np.zeros(n_traj, np.int32), np.zeros(n_traj, np.int32),
                    np.arange(n_traj, dtype=np.uint64))


def uniform(per_group: int = 10000, N: int = 4096, L: float = 40.0, dt: float = 0.001,
            kappas=(4.0, 5.0, 6.0), gammas=(-3.5, 0.0), shuffle_seed: int | None = 0) -> Workload:
    """Uniform batch: per_group trajectories of each initial state (Gaussian 1S-like l=0, Coulomb 2S,
    Gaussian 1P-like l=1) for every (kappa_hat, gamma_hat) pair, same Bjorken profile.  Seed =
    trajectory id.  The trajectory order is shuffled (PCG64) so that a prefix is a fair sample."""
    inits = [GAUSS_1S, COULOMB_2S, GAUSS_1P]
    media = [MediumSpec(0.425, 0.6, 0.25, k, g) for k in kappas for g in gammas]
    ii, mi = np.meshgrid(np.arange(len(inits)), np.arange(len(media)), indexing="ij")
    ii = np.repeat(ii.ravel(), per_group).astype(np.int32)
    mi = np.repeat(mi.ravel(), per_group).astype(np.int32)
    if shuffle_seed is not None:
        perm = np.random.Generator(np.random.PCG64(shuffle_seed)).permutation(len(ii))
        ii, mi = ii[perm], mi[perm]
    seeds = np.arange(len(ii), dtype=np.uint64)
    return Workload(f"uniform N={N} L={L:g} dt={dt:g} {per_group}/group x {len(inits)} inits x {len(media)} media",
                    GridSpec(N, L, dt), inits, media, ii, mi, seeds)


def uniform_interleaved(per_group: int = 10000, N: int = 4096, L: float = 40.0, dt: float = 0.001,
                        kappas=(4.0, 5.0, 6.0), gammas=(-3.5, 0.0)) -> Workload:
    """The uniform batch in a fixed interleaved order: trajectory t has initial state t % 3 and
    medium (t // 3) % 6, seed t.  Any slice that starts at a multiple of 18 has the same pattern of
    (initial state, medium) pairs, so consecutive slices differ only in their seeds."""
    inits = [GAUSS_1S, COULOMB_2S, GAUSS_1P]
    media = [MediumSpec(0.425, 0.6, 0.25, k, g) for k in kappas for g in gammas]
    n = per_group * len(inits) * len(media)
    t = np.arange(n)
    return Workload(f"uniform N={N} L={L:g} dt={dt:g} {per_group}/group x {len(inits)} inits x {len(media)} media",
                    GridSpec(N, L, dt), inits, media, (t % 3).astype(np.int32), ((t // 3) % 6).astype(np.int32),
                    t.astype(np.uint64))


def headline(n_traj: int = 16384, N: int = 4096) -> Workload:
    """One (kappa_hat, gamma_hat) = (5, 0) slice of the uniform N=4096 batch: 1S/2S/1P initial states
    in equal thirds, L=40, dt=0.001, Bjorken 0.425 -> 0.25 GeV."""
    inits = [GAUSS_1S, COULOMB_2S, GAUSS_1P]
    ii = (np.arange(n_traj) % 3).astype(np.int32)
    return Workload(f"uniform N={N} L=40 dt=0.001 kappa=5 gamma=0 1S/2S/1P thirds", GridSpec(N, 40.0 * N / 4096, 0.001),
                    inits, [MediumSpec(0.425, 0.6, 0.25, 5.0, 0.0)], ii, np.zeros(n_traj, np.int32),
                    np.arange(n_traj, dtype=np.uint64))


def precision(n_traj: int = 4096, N: int = 8192, L: float = 80.0, dt: float = 0.0005) -> Workload:
    """Precision study: N=8192, L=80, dt=0.0005, singlet Gaussian S wave, kappa_hat=5, gamma_hat=0,
    Bjorken 0.425 -> 0.25 GeV (23,797 steps); seeds = trajectory ids."""
    return Workload(f"precision N={N} L={L:g} dt={dt:g} 1S Gaussian kappa=5 gamma=0", GridSpec(N, L, dt), [GAUSS_1S],
                    [MediumSpec()], np.zeros(n_traj, np.int32), np.zeros(n_traj, np.int32),
                    np.arange(n_traj, dtype=np.uint64))


def small_parity(N: int = 64, n_traj: int = 16, seed: int = 7) -> Workload:
    """A small mixed case for element-wise parity: random initial states (Gaussian l in 0..2, Coulomb
    1S/2S/2P, singlet and octet), random media (T0 in [0.3, 0.6], kappa in [3, 7], gamma in [-3.5, 0],
    short profiles) on an N-point grid with dr = 5/256."""
    rng = np.random.Generator(np.random.PCG64(seed))
    inits = [InitSpec("gauss", 0.2, 1, 0, 0), InitSpec("gauss", 0.3, 2, 1, 0), InitSpec("gauss", 0.25, 3, 2, 1),
             InitSpec("coulomb", 0.0, 1, 0, 0), InitSpec("coulomb", 0.0, 2, 0, 0), InitSpec("coulomb", 0.0, 2, 1, 1)]
    media = []
    for _ in range(4):
        T0 = float(rng.uniform(0.3, 0.6))
        media.append(MediumSpec(T0, 0.6, T0 * float(rng.uniform(0.8, 0.95)), float(rng.uniform(3, 7)),
                                float(rng.uniform(-3.5, 0))))
    ii = rng.integers(0, len(inits), n_traj).astype(np.int32)
    mi = rng.integers(0, len(media), n_traj).astype(np.int32)
    seeds = rng.integers(0, 2**63, n_traj, dtype=np.uint64)
    return Workload(f"small parity N={N}", GridSpec(N, N * 5.0 / 256, 0.001), inits, media, ii, mi, seeds)


def uneven(n_traj: int = 1 << 16, seed: int = 0, Ns=(1024, 2048, 4096, 8192)) -> dict:
    """Uneven batch: N drawn from Ns (L = N*5/512, i.e. fixed dr), l0 in {0, 1, 2} (Gaussian
    r^{l+1}e^{-r^2/(2*0.2^2)} singlets), T0 ~ U[0.30, 0.60] GeV at tau0 = 0.6 fm/c cut at 0.25 GeV,
    kappa_hat ~ U[3, 7], gamma_hat ~ U[-3.5, 0]; seeds = trajectory ids.  Returned as per-trajectory
    arrays."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ns = rng.choice(np.array(Ns), n_traj)
    l0 = rng.integers(0, 3, n_traj)
    T0 = rng.uniform(0.30, 0.60, n_traj)
    kap = rng.uniform(3.0, 7.0, n_traj)
    gam = rng.uniform(-3.5, 0.0, n_traj)
    return {"N": Ns, "l0": l0, "T0": T0, "kappa_hat": kap, "gamma_hat": gam,
            "seeds": np.arange(n_traj, dtype=np.uint64)}


def serving_stream(n_requests: int = 256, rate_hz: float = 200.0, seed: int = 1,
                   N_choices=(1024, 2048, 4096, 8192, 16384), ntraj_range=(64, 4096)):
    """Poisson request stream: arrival times (s), initial state in {1S, 2S, 1P}, kappa_hat ~ U[3,7],
    gamma_hat ~ U[-3.5,0], T0 ~ U[0.3,0.6] GeV Bjorken, ntraj log-uniform in ntraj_range, N from
    N_choices (L = N*5/512, dt = 0.001)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, n_requests)
    arrival = np.cumsum(gaps) - gaps[0]
    init = rng.integers(0, 3, n_requests)
    kap = rng.uniform(3.0, 7.0, n_requests)
    gam = rng.uniform(-3.5, 0.0, n_requests)
    T0 = rng.uniform(0.3, 0.6, n_requests)
    lo, hi = np.log(ntraj_range[0]), np.log(ntraj_range[1])
    ntraj = np.exp(rng.uniform(lo, hi, n_requests)).astype(np.int64)
    N = rng.choice(np.array(N_choices), n_requests)
    return {"arrival_s": arrival, "init": init, "kappa_hat": kap, "gamma_hat": gam, "T0": T0,
            "ntraj": ntraj, "N": N}


def serving_prefix(n: int, rate_hz: float = 200.0, seed: int = 1) -> dict:
    """The first n requests of the 256-request serving stream.  (serving_stream draws each field for
    all requests in turn, so a stream generated with n_requests = n is a different set of requests,
    not a prefix.)"""
    st = serving_stream(n_requests=max(256, n), rate_hz=rate_hz, seed=seed)
    return {k: v[:n] for k, v in st.items()}
