"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test names the passage or the closed form it checks.  None retypes an oracle formula: the
expected values come from the paper's printed numbers (tests/golden), closed-form solutions,
brute force, invariants, or an independent integration of the density matrix.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from conftest import oracle_inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------------------------------------
# FFT and random numbers
# ------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64, 256])
def test_fft_matches_bruteforce_dft(oracle_lib, n):
    o = oracle_lib
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, 1):
        X = o.fft(x, sign)
        Xd = o.dft(x, sign)
        # the DFT definition, also checked against the textbook formula written with numpy
        jk = np.outer(np.arange(n), np.arange(n))
        Xm = np.exp(sign * 2j * np.pi * jk / n) @ x
        assert np.abs(Xd - Xm).max() <= 1e-12 * max(1.0, np.abs(Xm).max())
        assert np.abs(X - Xd).max() <= 1e-13 * max(1.0, np.abs(Xd).max()) * max(1, np.log2(n))


def test_fft_inverse_and_parseval(oracle_lib):
    o = oracle_lib
    rng = np.random.default_rng(3)
    n = 4096
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = o.fft(x, -1)
    assert abs(np.vdot(X, X).real / n - np.vdot(x, x).real) < 1e-12 * np.vdot(x, x).real
    y = o.fft(X, +1) / n
    assert np.abs(y - x).max() < 1e-13 * np.abs(x).max() * 12


def test_philox_known_answers(oracle_lib):
    for row in _read_golden("philox4x32_10_kat.txt"):
        v = [int(t, 16) for t in row]
        assert oracle_lib.philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def test_draws_uniform_in_open_interval(oracle_lib):
    from scipy import stats
    o = oracle_lib
    d = np.array([o.draws(12345, k) for k in range(20000)])
    assert (d > 0).all() and (d < 1).all()
    for col in range(3):
        assert stats.kstest(d[:, col], "uniform").pvalue > 1e-3
    # different seeds give different streams, a given (seed, k) is reproducible
    assert o.draws(1, 0) != o.draws(2, 0)
    assert o.draws(7, 5) == o.draws(7, 5)


# ------------------------------------------------------------------------------------------------
# paper's printed constants
# ------------------------------------------------------------------------------------------------
def test_jump_matrix_matches_paper(oracle_lib):
    """p(l -> l') of Eq. (pjump): the threshold of the oracle's rule on u_l in (0,1), found by
    bisection, is the printed probability of jumping down."""
    o = oracle_lib
    M = np.array([[float(Fraction(t)) for t in row] for row in _read_golden("jump_matrix.txt")])
    for l in range(4):
        lo, hi = 0.0, 1.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if o.jump_l(l, mid) == l - 1:
                lo = mid
            else:
                hi = mid
        p_down = lo
        if l - 1 >= 0:
            assert abs(p_down - M[l - 1, l]) < 1e-12
        else:
            assert p_down == 0.0
        if l + 1 < 4:
            assert abs((1 - p_down) - M[l + 1, l]) < 1e-12
        for lp in range(4):
            if abs(lp - l) != 1:
                assert M[lp, l] == 0.0
    # empirical frequencies with the oracle's own draws, 2e5 samples, within 4 sigma
    d = np.array([o.draws(99, k) for k in range(200000)])
    for l in (1, 2, 3):
        f = np.mean([o.jump_l(l, u) == l - 1 for u in d[:50000, 1]])
        p = l / (2 * l + 1)
        assert abs(f - p) < 4 * np.sqrt(p * (1 - p) / 50000)


def test_jump_rule_at_large_l(oracle_lib):
    """Eq. (pjump) beyond the printed matrix: for every l up to 300 the oracle jumps down with
    probability l/(2l+1) (threshold found by bisection on u_l), so that l(l+1) grows by exactly 2 per
    jump on average, (l+1)/(2l+1) (l+1)(l+2) + l/(2l+1) (l-1)l - l(l+1) = 2 -- the growth that takes
    trajectories with hundreds of jumps to l ~ 30..130."""
    o = oracle_lib
    for l in list(range(0, 40)) + [63, 64, 65, 127, 128, 255, 256, 257, 300]:
        lo, hi = 0.0, 1.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if o.jump_l(l, mid) == l - 1:
                lo = mid
            else:
                hi = mid
        p_down = lo
        assert abs(p_down - l / (2 * l + 1)) < 1e-12, l
        growth = (1 - p_down) * (l + 1) * (l + 2) + p_down * (l - 1) * l - l * (l + 1)
        assert abs(growth - 2.0) < 1e-6 * max(1, l * l), (l, growth)


def test_gaussian_initial_state_at_large_l(oracle_lib):
    """The Gaussian initial state r^{l+1} e^{-r^2/(2 w^2)}, discretely normalised: at small l equal to
    the formula evaluated directly (1e-13); at l = 300, w = 0.31, where r^{l+1} alone overflows, finite,
    normalised, and peaked at the maximum of (l+1) ln r - r^2/(2 w^2), r = w sqrt(l+1) (to one dr)."""
    o = oracle_lib
    g = o.Grid(N=1024, L=10.0)
    dr = g.L / g.N
    r = np.arange(g.N) * dr
    for l, w in ((0, 0.2), (2, 0.3), (20, 0.3)):
        u = o.initial_state(g, o.init_spec("gauss", w, 1, l, 0)).real
        v = r ** (l + 1) * np.exp(-r * r / (2 * w * w))
        v /= np.sqrt((v * v).sum() * dr)
        assert np.abs(u - v).max() < 1e-13 * np.abs(v).max(), l
    u = o.initial_state(g, o.init_spec("gauss", 0.31, 1, 300, 0)).real
    assert np.isfinite(u).all() and u[0] == 0.0
    assert abs((u * u).sum() * dr - 1.0) < 1e-12
    assert abs(r[np.argmax(u)] - 0.31 * np.sqrt(301)) <= dr


def test_colour_rule_and_potential_constants(oracle_lib):
    o = oracle_lib
    g = o.Grid()
    consts = {k: float(Fraction(v)) for k, v in _read_golden("colour_and_potential_constants.txt")}
    # colour thresholds by bisection on u_c
    assert all(o.jump_color(g, 0, u) == 1 for u in np.linspace(1e-9, 1 - 1e-9, 101))
    lo, hi = 0.0, 1.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if o.jump_color(g, 1, mid) == 0:
            lo = mid
        else:
            hi = mid
    assert abs(lo - consts["p_o_to_s"]) < 1e-12
    assert abs((1 - lo) - consts["p_o_to_o"]) < 1e-12
    # potential: singlet -alpha/r, octet +alpha/(8 r), r^2 coefficients 1/2 and 7/32 (App. E)
    alpha = consts["C_F"] * g.alpha_s
    r = 0.7
    vs = o.potential(g, 0, 0, 0.0, 0.0, 0.0, r)
    vo = o.potential(g, 1, 0, 0.0, 0.0, 0.0, r)
    assert abs(vs - (-alpha / r)) < 1e-15
    assert abs(vo - consts["octet_coulomb_over_alpha"] * alpha / r) < 1e-15
    T3, kap, gam = 0.07, 4.5, -1.3
    for c, f in ((0, consts["singlet_r2_factor"]), (1, consts["octet_r2_factor"])):
        dv = o.potential(g, c, 0, T3, kap, gam, r) - o.potential(g, c, 0, 0.0, 0.0, 0.0, r)
        assert abs(dv.real - f * gam * T3 * r * r) < 1e-15
        assert abs(dv.imag + f * kap * T3 * r * r) < 1e-15


# ------------------------------------------------------------------------------------------------
# split step: closed forms and invariants
# ------------------------------------------------------------------------------------------------
def _free_gaussian(r, D, t, M):
    # free s-wave Gaussian u = r R of a particle of reduced mass M/2 (hbar = 1):
    # R(r,t) = (D^2/a)^{3/2} exp(-r^2/(2a)),  a = D^2 + 2 i t / M
    a = D * D + 2j * t / M
    return D ** 3 * a ** -1.5 * r * np.exp(-r * r / (2 * a))


@pytest.mark.parametrize("dt,steps", [(0.001, 2000), (0.05, 40)])
def test_free_gaussian_spreading_closed_form(oracle_lib, dt, steps):
    o = oracle_lib
    g = o.Grid(N=512, L=20.0, dt=dt, alpha_s=0.0)
    D = 0.5
    r = np.arange(g.N) * (g.L / g.N)
    u0 = _free_gaussian(r, D, 0.0, g.M).astype(np.complex128)
    m = o.medium(kappa_hat=0.0, gamma_hat=0.0)
    u, _ = o.evolve_nojump(g, u0, 0, 0, m, 0, steps)
    ue = _free_gaussian(r, D, steps * dt, g.M)
    assert np.linalg.norm(u - ue) / np.linalg.norm(ue) < 1e-10


def test_vacuum_evolution_free_gaussian_and_coulomb_phase(oracle_lib):
    """Vacuum evolution before the medium (Sec. 3.5 item 3; Table 1 tmed - t0): t_vac / dt rounded
    steps with T = 0.  With alpha_s = 0 the start state of a Gaussian S wave is the spreading free
    Gaussian at t_vac (closed form); a Coulomb 1S only turns its phase by -E_1 t_vac with
    E_1 = -M (C_F alpha_s)^2 / 4, keeping its norm."""
    o = oracle_lib
    g = o.Grid(N=512, L=20.0, dt=0.001, alpha_s=0.0, t_vac=0.7504)
    assert o.vacuum_steps(g) == 750
    D = 0.5
    r = np.arange(g.N) * (g.L / g.N)
    spec = o.init_spec("gauss", D, 1, 0, 0)
    u0 = o.initial_state(g, spec)
    e0 = _free_gaussian(r, D, 0.0, g.M)
    c = u0[100] / e0[100]                       # the discrete normalisation, a real constant
    u = o.start_state(g, spec)
    ue = c * _free_gaussian(r, D, 750 * g.dt, g.M)
    assert np.linalg.norm(u - ue) / np.linalg.norm(ue) < 1e-10
    g = o.Grid(N=2048, L=20.0, dt=0.001, t_vac=2.0)
    phi = o.eigenstate(g, 1, 0)
    u = o.start_state(g, o.init_spec("coulomb", 0.0, 1, 0, 0))
    A = (g.L / g.N) * np.dot(phi, u)
    E = -np.angle(A) / (o.vacuum_steps(g) * g.dt)
    E1 = -g.M * (4.0 / 3.0 * 0.3) ** 2 / 4
    assert abs(E - E1) / abs(E1) < 1e-4 and abs(abs(A) - 1) < 1e-3
    assert abs(o.norm2(g, u) - 1) < 1e-12
    assert np.array_equal(o.start_state(o.Grid(N=64, L=2.0), spec), o.initial_state(o.Grid(N=64, L=2.0), spec))


def test_derivtype1_matches_three_point_laplacian(oracle_lib):
    """derivType 1 (Sec. 2.4): the kinetic operator is -(u_{j+1} - 2u_j + u_{j-1})/(M dr^2) with
    Dirichlet walls; with V = 0 one step equals exp(-i dt H3) applied with a dense eigen-solver."""
    o = oracle_lib
    N, L, dt = 64, 8.0, 0.01
    g = o.Grid(N=N, L=L, dt=dt, alpha_s=0.0, deriv_type=1)
    dr = L / N
    n = N - 1
    H = (np.diag(np.full(n, 2.0)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)) / (g.M * dr * dr)
    w, V = np.linalg.eigh(H)
    rng = np.random.default_rng(0)
    u0 = np.zeros(N, np.complex128)
    u0[1:] = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    m = o.medium(kappa_hat=0.0, gamma_hat=0.0)
    u, _ = o.evolve_nojump(g, u0, 0, 0, m, 0, 5)
    ue = V @ (np.exp(-1j * w * 5 * dt) * (V.T @ u0[1:]))
    assert np.abs(u[1:] - ue).max() < 1e-12 * np.abs(ue).max()
    assert u[0] == 0


def test_unitarity_for_real_potential(oracle_lib):
    """kappa_hat = 0: Strang splitting of a real potential is unitary (Sec. 3.3); the discrete norm
    stays 1 to rounding over the whole Bjorken profile (11,899 steps)."""
    o = oracle_lib
    g = o.Grid(N=512, L=20.0, dt=0.001)
    m = o.medium(kappa_hat=0.0, gamma_hat=-2.0)
    u0 = o.initial_state(g, o.init_spec())
    assert abs(o.norm2(g, u0) - 1) < 1e-14
    ns = o.n_steps(g, m)
    assert ns == 11899
    _, h = o.evolve_nojump(g, u0, 0, 0, m, 0, ns)
    assert np.abs(h - 1).max() < 1e-12
    _, h = o.evolve_nojump(g, u0, 1, 3, m, 0, 2000)   # octet, l = 3
    assert np.abs(h - 1).max() < 1e-12


def test_coulomb_energies_converge(oracle_lib):
    """T = 0 Coulomb problem of reduced mass M/2: E_n = -M (C_F alpha_s)^2 / (4 n^2).  The energy is
    read from the phase of <phi|psi(t)>.  The 1S error must fall under refinement of the grid at
    fixed L (the analytic 1S has a kink in its odd extension, so convergence is algebraic); at the
    finest grid the bounds below hold (1P pins the centrifugal term)."""
    o = oracle_lib
    M, alpha = 4.65, 4.0 / 3.0 * 0.3
    t_steps = 5000
    errs = {}
    for N in (512, 2048):
        g = o.Grid(N=N, L=20.0, dt=0.001)
        m = o.medium(kappa_hat=0.0, gamma_hat=0.0)
        dr = g.L / g.N
        for (n, l) in ((1, 0), (2, 0), (2, 1)):
            phi = o.eigenstate(g, n, l)
            u, _ = o.evolve_nojump(g, phi.astype(np.complex128), 0, l, m, 0, t_steps)
            A = dr * np.dot(phi, u)
            E = -np.angle(A) / (t_steps * g.dt)
            Eex = -M * alpha ** 2 / (4 * n * n)
            errs[(N, n, l)] = abs(E - Eex) / abs(Eex)
    assert errs[(2048, 1, 0)] < errs[(512, 1, 0)] / 4
    assert errs[(2048, 1, 0)] < 1e-4
    assert errs[(2048, 2, 0)] < 1e-3
    assert errs[(2048, 2, 1)] < 5e-4


def test_nonhermitian_decay_rate(oracle_lib):
    """With jumps off the norm is p_NoJump(t) and -d|psi|^2/dt = <psi|Gamma|psi> (Eq. wta), with
    Gamma_s = kappa_hat T^3 r^2 and Gamma_o = (7/16) kappa_hat T^3 r^2 (Sec. 3.4.2, Gamma).  The
    centred difference of the norm agrees to O(dt^2)."""
    o = oracle_lib
    T3 = 0.4 ** 3
    m = o.medium(T0=0.4, tau0=1e9, Tf=0.39, kappa_hat=5.0, gamma_hat=-1.0)   # T constant over the window
    for color, frac in ((0, 1.0), (1, 7.0 / 16.0)):
        errs = []
        for dt in (0.001, 0.0005):
            g = o.Grid(N=256, L=10.0, dt=dt)
            dr = g.L / g.N
            r = np.arange(g.N) * dr
            nst = int(round(0.2 / dt))
            u0 = o.initial_state(g, o.init_spec("gauss", 0.6, 1, 1, color))
            u, h = o.evolve_nojump(g, u0, color, 1, m, 0, nst)
            _, h1 = o.evolve_nojump(g, u, color, 1, m, nst, 1)
            rate = -(h1[0] - h[-2]) / (2 * dt)          # centred at u, the state after step nst-1
            gam = frac * 5.0 * T3 * dr * np.sum(r * r * np.abs(u) ** 2)
            errs.append(abs(rate - gam) / gam)
            assert np.all(np.diff(h) < 0)
        assert errs[0] < 2e-6
        assert 3.0 < errs[0] / errs[1] < 5.0            # second order in dt


def _fnv1a32(words):
    """FNV-1a, 32 bit (Fowler, Noll, Vo), over the little-endian bytes of 32-bit words."""
    h = 2166136261
    for w in words:
        for b in int(w & 0xFFFFFFFF).to_bytes(4, "little"):
            h = ((h ^ b) * 16777619) & 0xFFFFFFFF
    return h


def test_jump_digest_and_last_jump_step_follow_the_jumps(oracle_lib):
    """The record's jump digest is FNV-1a over (step, new l, new colour) of every jump in order, and
    last_jump_step the step of the last jump (0-based, as first_jump_step): both recomputed here from
    the per-step rows (rows count steps from 1; a jump after step n shows as a change of l between
    the rows n and n+1), for trajectories with 0 to ~30 jumps."""
    o = oracle_lib
    from paper_2107_06147_gb300 import inputs
    w = inputs.small_parity(N=128, n_traj=12, seed=17)
    w.grid.L = 8.0                       # a wide box: large r, many jumps
    for m in w.media:
        m.Tf = 0.8 * m.T0
    g, inits, media = oracle_inputs(w)
    g.use_rmin = 0
    seen = 0
    for t in range(12):
        ob, rows = o.trajectory_trace(g, inits[w.init_idx[t]], media[w.medium_idx[t]], int(w.seeds[t]), every=1)
        if ob["n_steps_exec"] < 2 or ob["flags"] & (o.F_MAXJUMPS | o.F_LCAP):
            continue
        ch = np.nonzero(rows["l"][1:] != rows["l"][:-1])[0]
        words = []
        for i in ch:
            words += [int(rows["step"][i]) - 1, int(rows["l"][i + 1]), int(rows["color"][i + 1])]
        last_row_jump = ob["n_jumps"] == len(ch) + 1      # a jump after the final step has no next row
        if last_row_jump:
            words += [int(rows["step"][-1]) - 1, int(ob["l"]), int(ob["color"])]
        assert ob["n_jumps"] == len(words) // 3
        assert ob["first_jump_step"] == (words[0] if words else -1)
        assert ob["jump_digest"] == _fnv1a32(words)
        assert ob["last_jump_step"] == (words[-3] if words else -1)
        seen += ob["n_jumps"] > 0
    assert seen >= 4
    assert _fnv1a32([]) == 2166136261 and _fnv1a32([0]) == 0x4B95F515   # FNV-1a of four zero bytes


def test_kappa_fit_coefficients_match_the_printed_fits(oracle_lib):
    """App. E prints the three lattice fits of kappa_hat(T) coefficient by coefficient
    (tests/golden/kappa_hat_lattice_fits.txt, transcribed from the paper).  Evaluated at x = T/T_c
    from 1 to 60 with those printed numbers, the oracle's fit must agree to rounding: a typo in any
    of the twelve coefficients, a swapped row (the kappa = -1/-2/-3 labels) or another T_c breaks it."""
    rows = _read_golden("kappa_hat_lattice_fits.txt")
    assert [r[1] for r in rows] == ["central", "lower", "upper"]
    x = np.array([1.0, 1.3, 2.0, 3.7, 6.0, 11.0, 25.0, 60.0])
    for r in rows:
        which = int(r[0])
        a, b, c, d = (float(t) for t in r[2:6])
        printed = 1.0 / (a * x ** 1.5 + b * x + c * np.sqrt(x) + d)
        got = np.array([oracle_lib.kappa_fit(which, 0.155 * xi) for xi in x])
        np.testing.assert_allclose(got, printed, rtol=1e-13, atol=0)
    # and each printed fit is distinct at every x, so the comparison above separates the rows
    f = np.array([[oracle_lib.kappa_fit(w, 0.155 * xi) for xi in x] for w in (1, 2, 3)])
    assert (np.abs(np.diff(f, axis=0)) > 1e-3 * np.abs(f[1:])).all()


def test_kappa_fits_positive_ordered_decreasing(oracle_lib):
    """The three lattice fits of kappa_hat(T) (App. E; parameter kappa = -1, -2, -3): positive and
    decreasing in T over T_c..100 T_c, and the lower-limit fit below the central below the upper-limit
    fit everywhere there (a swapped or mislabelled coefficient row breaks the order)."""
    o = oracle_lib
    T = 0.155 * np.geomspace(1.0, 100.0, 400)
    k = np.array([[o.kappa_fit(w, t) for t in T] for w in (1, 2, 3)])
    assert (k > 0).all()
    assert (np.diff(k, axis=1) < 0).all()
    assert (k[1] < k[0]).all() and (k[0] < k[2]).all()


@pytest.mark.parametrize("which", [1, 2, 3])
def test_kappa_fit_medium_decays_with_kappa_of_T(oracle_lib, which):
    """A medium with kappa = -which evolves with Gamma = kappa_hat(T_n) T_n^3 r^2 at step n: the
    centred decay rate of the norm matches <Gamma> with the fit evaluated at the temperature of that
    time, early and late in a Bjorken medium (where kappa_hat changes by ~30%), and does not match the
    other time's value."""
    o = oracle_lib
    g = o.Grid(N=256, L=10.0, dt=0.001)
    dr = g.L / g.N
    r = np.arange(g.N) * dr
    m = o.medium(T0=0.45, tau0=0.6, Tf=0.3, kappa_hat=float(-which), gamma_hat=-1.0)
    u = o.initial_state(g, o.init_spec("gauss", 0.6, 1, 0, 0))
    rates, gams, k = [], [], []
    n = 0
    for stop in (200, 6500):
        u, h = o.evolve_nojump(g, u, 0, 0, m, n, stop - n)
        _, h1 = o.evolve_nojump(g, u, 0, 0, m, stop, 1)
        rates.append(-(h1[0] - h[-2]) / (2 * g.dt))
        T3 = o.T3(g, m, stop)
        k.append(o.kappa_fit(which, T3 ** (1 / 3)))
        gams.append(k[-1] * T3 * dr * np.sum(r * r * np.abs(u) ** 2))
        n = stop
    for a, b in zip(rates, gams):
        assert abs(a - b) / b < 5e-3
    assert k[1] / k[0] > 1.2                                             # kappa_hat really changed ...
    assert abs(rates[1] / (gams[1] * k[0] / k[1]) - 1) > 0.15            # ... and the early value is wrong late


def test_summary_trace_coulomb_r_ratios(oracle_lib):
    """The per-step summary (App. C summary.tsv): R = <psi|r|psi>/<1S|r|1S> of a Coulomb state in a
    medium without kappa and gamma is the closed-form <r>_nl / <r>_1S = (3n^2 - l(l+1)) / 3, its own
    overlap |<nl|psi>|^2 stays 1; rows every `every` steps and after the last."""
    o = oracle_lib
    g = o.Grid(N=2048, L=60.0, dt=0.001)
    m = o.medium(0.4, 0.6, 0.39, 0.0, 0.0)
    for s, (n, l) in enumerate(((1, 0), (2, 0), (2, 1), (3, 0), (3, 1), (3, 2))):
        ob, rec = o.trajectory_trace(g, o.init_spec("coulomb", 0.0, n, l, 0), m, 5, every=100)
        assert list(rec["step"]) == [100, 200, ob["n_steps_exec"]]
        assert np.abs(rec["r_ratio"] - (3 * n * n - l * (l + 1)) / 3.0).max() < 1e-4 * n * n
        assert np.abs(rec["ov2"][:, s] - 1).max() < 1e-5
        assert np.abs(rec["norm2"] - 1).max() < 1e-12 and (rec["color"] == 0).all() and (rec["l"] == l).all()


def test_summary_trace_follows_the_trajectory(oracle_lib):
    """The summary rows of a trajectory with jumps: before the first jump the norm is the no-jump
    norm history at those steps (the same evolution), and the rows' (colour, l) change at the jumps."""
    o = oracle_lib
    g = o.Grid(N=64, L=2.5, dt=0.001)
    spec = o.init_spec("gauss", 0.3, 1, 0, 0)
    m = o.medium(T0=0.5, tau0=0.6, Tf=0.3, kappa_hat=6.0, gamma_hat=-1.0)
    for seed in range(40):
        ob, rec = o.trajectory_trace(g, spec, m, seed, every=10)
        if ob["n_jumps"] >= 2:
            break
    assert ob["n_jumps"] >= 2
    fj = ob["first_jump_step"]
    _, h = o.evolve_nojump(g, o.initial_state(g, spec), 0, 0, m, 0, fj + 1)
    pre = rec[rec["step"] <= fj + 1]
    assert len(pre) >= 3 and np.array_equal(pre["norm2"], h[pre["step"] - 1])
    post = rec[rec["step"] > fj + 1]
    assert (post["color"] == 1).any() and (pre["color"] == 0).all()


def test_numerical_eigenstates_energies_and_propagation(oracle_lib):
    """Numerical eigenstates of the discretised vacuum Hamiltonian (initType 100 / ProjType 1):
    their energies approach E_n = -M (C_F alpha_s)^2 / (4 n^2) under refinement, and they are
    eigenstates of the oracle's own propagator: after 1000 vacuum steps a numerical 1S has turned
    its phase by -E t and kept |<phi|psi>| = 1 to O(dt^2), far closer than the analytic 1S (which
    the grid's Hamiltonian does not hold exactly)."""
    from oracle import eigen
    o = oracle_lib
    M, alpha = 4.65, 4.0 / 3.0 * 0.3
    errs = {}
    for N in (512, 1024):
        g = o.Grid(N=N, L=40.0, dt=0.001)
        for l, m in ((0, 2), (1, 1)):
            lam, _ = eigen.vacuum_eigenstates(g, l, m)
            for k in range(m):
                n = l + 1 + k
                errs[(N, n, l)] = abs(lam[k] + M * alpha ** 2 / (4 * n * n)) / (M * alpha ** 2 / (4 * n * n))
    assert errs[(1024, 1, 0)] < errs[(512, 1, 0)] and errs[(1024, 1, 0)] < 2e-3
    assert errs[(1024, 2, 0)] < 2e-3 and errs[(1024, 2, 1)] < 2e-3
    m0 = o.medium(kappa_hat=0.0, gamma_hat=0.0)
    perr = []
    for dt in (0.001, 0.0005):
        g = o.Grid(N=512, L=20.0, dt=dt)
        lam, v = eigen.vacuum_eigenstates(g, 0, 1)
        dr = g.L / g.N
        nst = int(round(1.0 / dt))
        u, _ = o.evolve_nojump(g, v[0].astype(np.complex128), 0, 0, m0, 0, nst)
        A = dr * np.dot(v[0], u)
        assert abs(abs(A) - 1) < 1e-7
        perr.append(abs(-np.angle(A) / (nst * dt) - lam[0]) / abs(lam[0]))
    assert perr[0] < 3e-6 and 3.0 < perr[0] / perr[1] < 5.0        # the splitting's O(dt^2) only
    g = o.Grid(N=512, L=20.0, dt=0.001)
    lam, v = eigen.vacuum_eigenstates(g, 0, 1)
    dr = g.L / g.N
    u, _ = o.evolve_nojump(g, v[0].astype(np.complex128), 0, 0, m0, 0, 1000)
    A = dr * np.dot(v[0], u)
    phi = o.eigenstate(g, 1, 0)
    ua, _ = o.evolve_nojump(g, phi.astype(np.complex128), 0, 0, m0, 0, 1000)
    assert abs(abs(dr * np.dot(phi, ua)) - 1) > 100 * abs(abs(A) - 1)
    # a numerical 1S start, measured in the numerical basis, keeps S(1S) = 1 in vacuum
    g.basis = eigen.numerical_basis(g)
    rec = o.nojump_run(g, o.given_state(g.basis[0], 1, 0), o.medium(0.4, 0.6, 0.39, 0.0, 0.0))
    assert abs(rec["surv"][0] - 1) < 1e-7 and abs(rec["surv"][1]) < 1e-12


def test_table_profile_linear_pieces_and_end(oracle_lib):
    """Tabulated T(tau) (Table 1 temperatureEvolution 1/2; App. B formats): step n uses T linearly
    interpolated at tau_n = tau_1 + n dt hbar c; the evolution ends at the first crossing of Tf
    (ceil of the steps to it), at the table's last tau if T never falls below Tf, and at once if it
    starts below Tf."""
    o = oracle_lib
    g = o.Grid(N=64, L=2.0, dt=0.001)
    hc = 0.1973269804
    tau, T = np.array([0.6, 1.0, 2.0]), np.array([0.5, 0.4, 0.2])
    m = o.table_medium(tau, T, Tf=0.3)
    assert o.n_steps(g, m) == int(np.ceil((1.5 - 0.6) / (hc * g.dt)))      # crossing at tau = 1.5
    for n in (0, 700, 2027, 2028, 4000):
        t = 0.6 + n * g.dt * hc
        Tex = 0.5 - 0.25 * (t - 0.6) if t < 1.0 else 0.4 - 0.2 * (t - 1.0)
        assert abs(o.T3(g, m, n) - Tex ** 3) < 1e-14
    assert o.n_steps(g, o.table_medium(tau, T, Tf=0.1)) == int(np.ceil((2.0 - 0.6) / (hc * g.dt)))
    assert abs(o.T3(g, o.table_medium(tau, T, Tf=0.1), 10 ** 5) - 0.2 ** 3) < 1e-15   # held after the end
    assert o.n_steps(g, o.table_medium(tau, T, Tf=0.6)) == 0


def test_table_sampled_from_bjorken_converges(oracle_lib):
    """A table sampled from a Bjorken profile reproduces the Bjorken evolution: after 5000 steps the
    no-jump norm differs by O(dtau^2) of the sampling (the difference falls ~4x when dtau halves)."""
    o = oracle_lib
    g = o.Grid(N=128, L=5.0, dt=0.001)
    u0 = o.initial_state(g, o.init_spec("gauss", 0.3, 1, 0, 0))
    bj = o.medium(T0=0.45, tau0=0.6, Tf=0.3, kappa_hat=5.0, gamma_hat=-1.0)
    _, href = o.evolve_nojump(g, u0, 0, 0, bj, 0, 5000)
    errs = []
    for d in (0.04, 0.02):
        tau = np.arange(0.6, 2.6, d)
        T = 0.45 * (0.6 / tau) ** (1.0 / 3.0)
        tm = o.table_medium(tau, T, Tf=0.3, kappa_hat=5.0, gamma_hat=-1.0)
        _, h = o.evolve_nojump(g, u0, 0, 0, tm, 0, 5000)
        errs.append(abs(h[-1] - href[-1]) / href[-1])
        # the interpolated profile lies above the convex Bjorken one, so it crosses Tf a little later
        assert 0 <= o.n_steps(g, tm) - o.n_steps(g, bj) <= 4
    assert errs[0] < 3e-4 and 3.0 < errs[0] / errs[1] < 5.0


# ------------------------------------------------------------------------------------------------
# trajectories: waiting-time statistics, shortcut exactness, options
# ------------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_batch(oracle_lib):
    o = oracle_lib
    g = o.Grid(N=64, L=2.5, dt=0.002)
    spec = o.init_spec("gauss", 0.3, 1, 0, 0)
    m = o.medium(T0=0.5, tau0=0.6, Tf=0.42, kappa_hat=4.0, gamma_hat=-1.0)
    n = 4000
    obs, nj, _ = o.run_batch(g, [spec], np.zeros(n, int), [m], np.zeros(n, int), np.arange(n, dtype=np.uint64) + 1000)
    return g, spec, m, obs, nj[0]


def test_zero_jump_fraction_is_p_nojump(oracle_lib, small_batch):
    g, spec, m, obs, nj = small_batch
    p = nj["norm2"]
    n = len(obs)
    frac = np.mean(obs["n_jumps"] == 0)
    assert 0.05 < p < 0.95
    assert abs(frac - p) < 3.5 * np.sqrt(p * (1 - p) / n)
    # zero-jump trajectories are exactly the rMin shortcuts
    assert np.array_equal(obs["n_jumps"] == 0, (obs["flags"] & oracle_lib.F_NOJUMP_SHORTCUT) != 0)


def test_first_jump_time_distribution(oracle_lib, small_batch):
    """P(first jump after step <= n) = 1 - |psi_nojump(n)|^2 (Eq. wta with a uniform threshold)."""
    o = oracle_lib
    g, spec, m, obs, nj = small_batch
    u0 = o.initial_state(g, spec)
    _, h = o.evolve_nojump(g, u0, spec.color, spec.l, m, 0, o.n_steps(g, m))
    fj = obs["first_jump_step"]
    n = len(fj)
    steps = np.arange(len(h))
    emp = np.searchsorted(np.sort(fj[fj >= 0]), steps, side="right") / n
    D = np.abs(emp - (1 - h)).max()
    assert D < 1.63 / np.sqrt(n)      # Kolmogorov-Smirnov at the 1% level


def test_rmin_shortcut_is_exact(oracle_lib):
    """A trajectory with r0 < p_NoJump never jumps, so its full evolution equals the zeroth
    trajectory bit for bit (Sec. 3.5 item 4a)."""
    o = oracle_lib
    g = o.Grid(N=64, L=2.5, dt=0.002, use_rmin=0)
    spec = o.init_spec("gauss", 0.3, 1, 0, 0)
    m = o.medium(T0=0.5, tau0=0.6, Tf=0.42, kappa_hat=4.0, gamma_hat=-1.0)
    nj = o.nojump_run(g, spec, m)
    found = 0
    for seed in range(200):
        r0 = o.draws(seed, 0)[0]
        if r0 < nj["norm2"]:
            rec = o.trajectory(g, spec, m, seed)
            assert rec["n_jumps"] == 0
            for f in ("surv", "ov_re", "ov_im", "norm2"):
                assert np.array_equal(rec[f], nj[f])
            found += 1
            if found == 5:
                break
    assert found == 5


def test_options_rmax_maxjumps_lcap(oracle_lib):
    o = oracle_lib
    spec = o.init_spec("gauss", 0.3, 1, 0, 0)
    m = o.medium(T0=0.5, tau0=0.6, Tf=0.42, kappa_hat=4.0, gamma_hat=-1.0)
    seeds = np.arange(300, dtype=np.uint64)
    base = o.Grid(N=64, L=2.5, dt=0.002)
    obs, _, _ = o.run_batch(base, [spec], np.zeros(300, int), [m], np.zeros(300, int), seeds)
    g = o.Grid(N=64, L=2.5, dt=0.002, r_max=0.5)
    ob2, _, _ = o.run_batch(g, [spec], np.zeros(300, int), [m], np.zeros(300, int), seeds)
    cut = obs["r0"] > 0.5
    assert cut.any() and (~cut).any()
    assert np.all(ob2["surv"][cut] == 0) and np.all(ob2["flags"][cut] & o.F_RMAX)
    assert np.array_equal(ob2["surv"][~cut], obs["surv"][~cut])
    g = o.Grid(N=64, L=2.5, dt=0.002, max_jumps=1)
    ob3, _, _ = o.run_batch(g, [spec], np.zeros(300, int), [m], np.zeros(300, int), seeds)
    two = obs["n_jumps"] >= 2
    assert two.any()
    assert np.all(ob3["flags"][two] & o.F_MAXJUMPS) and np.all(ob3["surv"][two] == 0)
    assert np.array_equal(ob3["surv"][obs["n_jumps"] <= 1], obs["surv"][obs["n_jumps"] <= 1])
    g = o.Grid(N=64, L=2.5, dt=0.002, l_cap=1)
    ob4, _, _ = o.run_batch(g, [spec], np.zeros(300, int), [m], np.zeros(300, int), seeds)
    assert np.all(ob4["l"][(ob4["flags"] & o.F_LCAP) == 0] <= 1)


def test_determinism_and_thread_independence(oracle_lib):
    from paper_2107_06147_gb300 import inputs
    o = oracle_lib
    w = inputs.small_parity(N=32, n_traj=24)
    g, inits, media = oracle_inputs(w)
    a, _, ua = o.run_batch(g, inits, w.init_idx, media, w.medium_idx, w.seeds, n_threads=1, want_states=True)
    b, _, ub = o.run_batch(g, inits, w.init_idx, media, w.medium_idx, w.seeds, n_threads=8, want_states=True)
    assert a.tobytes() == b.tobytes()
    assert np.array_equal(ua, ub)


# ------------------------------------------------------------------------------------------------
# the whole unravelling against the density matrix
# ------------------------------------------------------------------------------------------------
def test_trajectory_average_matches_lindblad(oracle_lib):
    """N = 32, l <= 3: the mean survival probabilities and the colour/l populations of 20,000
    trajectories equal the RK4 solution of the Lindblad equation (Eq. Lindblad with the collapse
    operators of Eq. collapse) within 3.5 standard errors.  This pins the jump rules, the waiting
    time, and the normalised read-out of the overlaps."""
    from oracle import lindblad
    o = oracle_lib
    N, L, dt = 32, 8.0, 0.002
    g = o.Grid(N=N, L=L, dt=dt, l_cap=3)
    spec = o.init_spec("gauss", 0.5, 1, 0, 0)
    m = o.medium(T0=0.45, tau0=0.6, Tf=0.35, kappa_hat=3.0, gamma_hat=-1.0)
    u0 = o.initial_state(g, spec)
    rho, ns = lindblad.evolve(N, L, dt, g.M, g.alpha_s, g.Nc, u0, 0, 0, 3, m.T0, m.tau0, m.Tf,
                              m.kappa_hat, m.gamma_hat)
    assert ns == o.n_steps(g, m)
    dr = L / N
    nt = 20000
    obs, nj, _ = o.run_batch(g, [spec], np.zeros(nt, int), [m], np.zeros(nt, int), np.arange(nt, dtype=np.uint64))
    basis = [(1, 0), (2, 0), (2, 1), (3, 0), (3, 1), (3, 2)]
    for s, (n, l) in enumerate(basis):
        phi = o.eigenstate(g, n, l)
        expect = lindblad.expectation(rho[0, l], phi, dr)
        if l == 0:   # survival ratio -> probability
            o0 = dr * np.dot(phi[1:], u0[1:].real)
            v = obs["surv"][:, s] * o0 * o0
        else:
            v = obs["surv"][:, s]
        sem = v.std() / np.sqrt(nt)
        assert abs(v.mean() - expect) < 3.5 * sem + 1e-12, (s, v.mean(), expect, sem)
    pops = np.real(np.trace(rho, axis1=2, axis2=3))
    alive = (obs["flags"] & o.F_LCAP) == 0
    for c in range(2):
        for l in range(4):
            f = np.mean((obs["color"] == c) & (obs["l"] == l) & alive)
            p = pops[c, l]
            assert abs(f - p) < 3.5 * np.sqrt(max(p * (1 - p), 1e-6) / nt), (c, l, f, p)


# ------------------------------------------------------------------------------------------------
# the isotropic KSU potential (App. E, "Isotropic KSU potential")
# ------------------------------------------------------------------------------------------------
def test_ksu_special_functions_match_library(oracle_lib):
    """The oracle's own e^x E1(x) (series / continued fraction) and e^-x Ei(x) (series / asymptotic
    series) against scipy's exp1 and expi, across the switch points."""
    special = pytest.importorskip("scipy.special")
    o = oracle_lib
    for x in (1e-4, 0.01, 0.3, 0.999, 1.001, 2.0, 7.0, 20.0, 59.9, 60.1, 90.0, 300.0):
        assert abs(o.expE1(x) / (np.exp(x) * special.exp1(x)) - 1) < 1e-13, x
        assert abs(o.expmEi(x) / (np.exp(-x) * special.expi(x)) - 1) < 1e-13, x


def test_ksu_phi_is_the_printed_integral(oracle_lib):
    """phi(rhat) = 2 int_0^inf dz z/(z^2+1)^2 [1 - sin(z rhat)/(z rhat)] as printed: the oracle's
    closed form and small-argument series against the integral itself (2 int z/(z^2+1)^2 = 1, and the
    sine part by mpmath's oscillatory quadrature at 30 digits), and its limits phi(0) = 0,
    phi -> 1 - 2/rhat^2."""
    mp = pytest.importorskip("mpmath")
    o = oracle_lib
    mp.mp.dps = 30
    for a in (0.05, 0.3, 1.0, 1.9, 2.1, 3.0, 10.0, 30.0):   # both sides of the series/closed-form switch
        am = mp.mpf(a)
        sine = mp.quadosc(lambda z: mp.sin(am * z) / (1 + z * z) ** 2, [0, mp.inf], omega=am)
        assert abs(o.ksu_phi(a) - float(1 - 2 * sine / am)) < 1e-15, a
    assert o.ksu_phi(0.0) == 0.0
    xs = np.linspace(1e-3, 50, 400)
    ph = np.array([o.ksu_phi(x) for x in xs])
    assert (np.diff(ph) > 0).all() and 0 < ph[0] < 1e-5
    assert abs(o.ksu_phi(200.0) - (1 - 2 / 200.0 ** 2)) < 1e-7


def test_ksu_running_coupling(oracle_lib):
    """alpha_s(5 GeV) = 0.2034 as printed, and the one-loop renormalisation-group equation
    d alpha_s / d ln mu^2 = -b0 alpha_s^2, b0 = (11 Nc - 2 N_F)/(12 pi) with N_F = 3, by finite
    differences."""
    o = oracle_lib
    assert o.alpha_s_run(5.0) == pytest.approx(0.2034, abs=1e-15)
    b0 = (33.0 - 6.0) / (12 * np.pi)
    for mu in (1.5, 2.5, 4.0, 12.0):
        h = 1e-4                                                 # a step in ln mu^2
        d = (o.alpha_s_run(mu * np.exp(h / 4)) - o.alpha_s_run(mu * np.exp(-h / 4))) / h
        assert abs(d / (-b0 * o.alpha_s_run(mu) ** 2) - 1) < 1e-7, mu
    assert o.alpha_s_run(2.0) > o.alpha_s_run(3.0) > o.alpha_s_run(5.0)


def test_ksu_potential_limits(oracle_lib):
    """The KSU potential (App. E): as T -> 0 (m_D -> 0) the KMS form becomes the Cornell -a/r + sigma r;
    its real part never exceeds V_vac(r_SB) = -a/r_SB + sigma r_SB and equals it where the KMS form
    would; the imaginary part is -alpha_s(2 pi T) C_F T phi(m_D r): 0 at r -> 0, tending to
    -alpha_s C_F T; at T = 0 the potential is the vacuum Cornell with string breaking."""
    o = oracle_lib
    g = o.Grid(N=256, L=20.0)
    a, sig, rsb = 0.409, 0.21, 1.25 / 0.1973269804
    vcap = -a / rsb + sig * rsb
    g0 = o.Grid(N=256, L=20.0, ksu_fmd=1e-9)               # m_D -> 0 at a physical temperature
    for r in (0.05, 0.5, 2.0, 5.0):
        v = o.ksu_potential(g0, 0, 0.3, r)
        assert abs(v.real - (-a / r + sig * r)) < 1e-7 and abs(v.imag) < 1e-12, r
    for r in (0.05, 0.5, 2.0, 6.0, 8.0):
        v = o.ksu_potential(g, 0, 0.0, r)
        assert v.imag == 0 and abs(v.real - ((-a / r + sig * r) if r <= rsb else vcap)) < 1e-14
    T = 0.3
    mD = o.ksu_debye_mass(g, T)
    rs = np.linspace(0.02, 40.0, 2000)
    v = np.array([o.ksu_potential(g, 0, T, r) for r in rs])
    assert (v.real <= vcap + 1e-15).all() and abs(v.real[-1] - 2 * sig / mD) < 1e-10   # screened: 2 sigma/m_D
    gc = o.Grid(N=256, L=20.0, ksu_fmd=0.3)                  # weak screening: 2 sigma/m_D above the cap
    vc = np.array([o.ksu_potential(gc, 0, T, r) for r in rs])
    assert 2 * sig / o.ksu_debye_mass(gc, T) > vcap
    assert (vc.real <= vcap + 1e-15).all() and vc.real[-1] == vcap and (vc.real == vcap).sum() > 100
    assert (np.abs(np.diff(vc.real[rs > 1.0])) < 0.02).all()   # continuous across the cap (slope < 1 GeV^2)
    assert (v.imag <= 0).all() and abs(v.imag[0]) < 1e-3
    asym = -o.alpha_s_run(2 * np.pi * T) * (4.0 / 3.0) * T
    x = mD * rs[-1]
    assert abs(v.imag[-1] / asym - (1 - 2 / x ** 2 - 8 / x ** 4)) < 1e-6   # phi's asymptotic series
    assert o.ksu_potential(g, 2, T, 1.0).real - o.ksu_potential(g, 0, T, 1.0).real == pytest.approx(6.0 / 4.65, rel=1e-12)
    assert o.ksu_debye_mass(g, 0.0) == 0.0
    g2 = o.Grid(N=256, L=20.0, ksu_fmd=1.5)
    assert o.ksu_debye_mass(g2, T) == pytest.approx(1.5 * mD, rel=1e-14)


def test_ksu_vacuum_spectrum_independent_discretisation(oracle_lib):
    """The KSU vacuum basis: eigenstates of the grid Hamiltonian with the Cornell potential (string
    breaking at r_SB).  Its 1S and 1P energies agree with a second discretisation of the same radial
    problem (a three-point Laplacian on a 4x finer grid, scipy's tridiagonal eigensolver)."""
    linalg = pytest.importorskip("scipy.linalg")
    from oracle import eigen
    o = oracle_lib
    g = o.Grid(N=1024, L=16.0, potential=1)
    for l in (0, 1):
        w, _ = eigen.vacuum_eigenstates(g, l, 1)
        Nf = 8192
        dr = g.L / Nf
        r = np.arange(1, Nf) * dr
        V = eigen.vacuum_potential(g, r) + l * (l + 1) / (g.M * r * r)
        d = V + 2.0 / (g.M * dr * dr)                          # -u''/M with the reduced mass M/2
        e = np.full(len(r) - 1, -1.0 / (g.M * dr * dr))
        wf = linalg.eigh_tridiagonal(d, e, select="i", select_range=(0, 0))[0][0]
        assert abs(w[0] - wf) < 2e-4, (l, w[0], wf)


def test_ksu_evolution_has_no_jumps_and_decays_by_v_i(oracle_lib):
    """Evolution with the KSU potential (singlet, H_eff, no collapse operator): no jump and r0 = 0 in
    any record; the norm falls at the rate -d|psi|^2/dt = -2 <psi|V_I|psi> (to O(dt^2)); the survival
    ratio is the unnormalised |<1S|psi>|^2 / |<1S|psi_0>|^2; at a vanishing temperature the vacuum
    1S stays put (S = 1, norm 1)."""
    from oracle import eigen
    o = oracle_lib
    g = o.Grid(N=256, L=12.0, dt=0.001, potential=1)
    g.basis = eigen.numerical_basis(g)
    _, v1s = eigen.vacuum_eigenstates(g, 0, 1)
    inits = [o.given_state(v1s[0], 1, 0, 0), o.init_spec("gauss", 0.5, 1, 0, 0)]
    media = [o.medium(T0=0.45, tau0=0.6, Tf=0.35, kappa_hat=0.0)]
    idx = np.array([0, 1, 0, 1], np.int32)
    mi = np.zeros(4, np.int32)
    ref, _, u = o.run_batch(g, inits, idx, media, mi, np.arange(4, dtype=np.uint64), want_states=True)
    assert (ref["n_jumps"] == 0).all() and (ref["r0"] == 0).all() and (ref["n_steps_exec"] > 100).all()
    assert (ref["norm2"] < 0.99).all() and np.array_equal(ref["surv"][0], ref["surv"][2])   # deterministic
    ov2 = ref["ov_re"][:, 0] ** 2 + ref["ov_im"][:, 0] ** 2
    o0 = (g.L / g.N) * np.dot(g.basis[0], v1s[0])
    assert np.allclose(ref["surv"][0, 0], ov2[0] / o0 ** 2, rtol=1e-12)   # not divided by the norm
    # with m_D -> 0 the potential is the vacuum one: the vacuum 1S keeps S = 1 and its norm
    g0 = o.Grid(N=256, L=12.0, dt=0.001, potential=1, ksu_fmd=1e-12)
    g0.basis = g.basis
    r0_, _, _ = o.run_batch(g0, inits[:1], np.zeros(1, np.int32), media, np.zeros(1, np.int32), np.zeros(1, np.uint64))
    assert abs(r0_["norm2"][0] - 1) < 1e-10 and abs(r0_["surv"][0, 0] - 1) < 1e-8
    # decay rate at constant T
    m = o.medium(T0=0.4, tau0=1e9, Tf=0.39, kappa_hat=0.0)
    errs = []
    for dt in (0.001, 0.0005):
        h_ = o.Grid(N=256, L=12.0, dt=dt, potential=1)
        dr = h_.L / h_.N
        r = np.arange(h_.N) * dr
        u0 = o.initial_state(h_, o.init_spec("gauss", 0.8, 1, 0, 0))
        nst = int(round(0.1 / dt))
        uu, hh = o.evolve_nojump(h_, u0, 0, 0, m, 0, nst)
        _, h1 = o.evolve_nojump(h_, uu, 0, 0, m, nst, 1)
        rate = -(h1[0] - hh[-2]) / (2 * dt)
        VI = np.array([o.ksu_potential(h_, 0, 0.4, x).imag if x > 0 else 0.0 for x in r])
        gam = -2.0 * dr * np.sum(VI * np.abs(uu) ** 2)
        errs.append(abs(rate - gam) / gam)
    assert errs[0] < 1e-5 and 3.0 < errs[0] / errs[1] < 5.0


def test_dft16_oracle_pins():
    """The 16-point DFT of oracle/dft16.py: numpy's FFT (a library routine), F^2 = 16 x (m -> -m mod 16),
    and F^4 = 256 I."""
    from oracle import dft16 as odft
    rng = np.random.default_rng(4)
    x = rng.standard_normal((3, 7, 16)) + 1j * rng.standard_normal((3, 7, 16))
    assert np.allclose(odft.passes(x, 1), np.fft.fft(x, axis=-1), rtol=0, atol=1e-12)
    rev = x[..., (-np.arange(16)) % 16]
    assert np.allclose(odft.passes(x, 2), 16 * rev, rtol=0, atol=1e-11)
    assert np.allclose(odft.passes(x, 4), 256 * x, rtol=0, atol=1e-10)
    assert np.array_equal(odft.passes(x, 0), x)
