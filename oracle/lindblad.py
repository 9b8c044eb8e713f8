"""Brute-force density-matrix integration of the quarkonium Lindblad equation (test infrastructure).

This is the object the quantum trajectories unravel (Sec. 3.1, Eq. Lindblad; Sec. 3.4, Eqs.
hamiltonian, collapse, Pl+- and pjump), integrated directly with classical RK4 so that the
trajectory average of the oracle can be checked against it.  It is used only by the tests.

Discretisation (the same grid as the trajectories): interior points r_j = j*dr, j = 1..N-1, with
the sine basis of the box (0, L).  The kinetic operator is the dense matrix
    H_kin = (2/N) S diag(T_kin(p_k)) S,   S_kj = sin(pi j k / N),   p_k = pi k / L,
i.e. exactly the operator whose exponential the split step applies in momentum space.  The
density matrix is block diagonal in colour c and angular momentum l (Eq. rhoso); the block
rho_cl holds dr * u u^dagger for a pure state, so Tr rho_cl is the probability of (c, l).

    d rho_cl/dt = -i (H_cl rho_cl - rho_cl H_cl^dagger)
                  + kappa T^3 sum_{c', l'} w(c'->c) p(l'->l) R rho_c'l' R,      R = diag(r_j)

with H_cl = H_kin + diag(V_eff), Im V_eff = -Gamma/2, Gamma_s = kappa T^3 r^2,
Gamma_o = (Nc^2-2)/(2(Nc^2-1)) kappa T^3 r^2, and the colour weights of the collapse operators:
w(s->o) = 1, w(o->s) = 1/(Nc^2-1), w(o->o) = (Nc^2-4)/(2(Nc^2-1)) (Sec. 3.4.2, Gamma^0 and
Gamma^1).  p(l->l+1) = (l+1)/(2l+1), p(l->l-1) = l/(2l+1) (Eq. Pl+-).  Blocks with l > l_max are
dropped (their population is lost), which the trajectories mirror with their l_cap option.

Time: step n covers [n dt, (n+1) dt) with the temperature T(tau_n) held fixed, the same
piecewise-constant profile the split step sees; one RK4 step of size dt per step.
"""
from __future__ import annotations

import numpy as np

HBARC = 0.1973269804


def _potential_diag(r, color, l, T3, kap, gam, M, alpha_s, Nc):
    CF = (Nc * Nc - 1) / (2 * Nc)
    if color == 0:
        coul, f = -CF * alpha_s / r, 0.5
    else:
        coul, f = alpha_s / (2 * Nc * r), (Nc * Nc - 2) / (4 * (Nc * Nc - 1))
    return coul + l * (l + 1) / (M * r * r) + f * gam * T3 * r * r - 1j * f * kap * T3 * r * r


def evolve(N, L, dt, M, alpha_s, Nc, u0, c0, l0, l_max, T0, tau0, Tf, kappa_hat, gamma_hat,
           deriv_type=0):
    """Returns rho[c][l] (interior-point matrices) at the end of the Bjorken profile and the number
    of steps taken.  u0 is the normalised initial state on the full grid (index 0 ignored)."""
    n = N - 1
    dr = L / N
    j = np.arange(1, N)
    r = j * dr
    S = np.sin(np.pi * np.outer(j, j) / N)
    p = np.pi * j / L
    if deriv_type == 1:
        tk = 2 * (1 - np.cos(p * dr)) / (M * dr * dr)
    else:
        tk = p * p / M
    Hkin = (2.0 / N) * (S * tk[None, :]) @ S
    nl = l_max + 1
    Vstat = np.zeros((2, nl, n), dtype=np.complex128)
    Vr2 = np.zeros((2, n), dtype=np.complex128)   # coefficient of T^3 in V_eff
    for c in range(2):
        for l in range(nl):
            Vstat[c, l] = _potential_diag(r, c, l, 0.0, 0.0, 0.0, M, alpha_s, Nc)
        Vr2[c] = _potential_diag(r, c, 0, 1.0, kappa_hat, gamma_hat, M, 0.0, Nc)
    # colour weights of the gain term, indexed [from][to]
    w = np.zeros((2, 2))
    w[0, 1] = 1.0
    w[1, 0] = 1.0 / (Nc * Nc - 1)
    w[1, 1] = (Nc * Nc - 4) / (2 * (Nc * Nc - 1))

    rho = np.zeros((2, nl, n, n), dtype=np.complex128)
    u = np.asarray(u0)[1:]
    rho[c0, l0] = dr * np.outer(u, u.conj())

    tau_f = tau0 * (T0 / Tf) ** 3
    nsteps = int(np.ceil((tau_f - tau0) / (HBARC * dt)))

    def rhs(rh, H, T3):
        out = -1j * (H @ rh - rh @ np.conj(np.swapaxes(H, -1, -2)))
        rr = r[None, None, :, None] * rh * r[None, None, None, :]
        for c in range(2):
            for l in range(nl):
                gain = np.zeros((n, n), dtype=np.complex128)
                for cf in range(2):
                    if w[cf, c] == 0.0:
                        continue
                    if l - 1 >= 0:
                        lf = l - 1
                        gain += w[cf, c] * (lf + 1) / (2 * lf + 1) * rr[cf, lf]
                    if l + 1 < nl:
                        lf = l + 1
                        gain += w[cf, c] * lf / (2 * lf + 1) * rr[cf, lf]
                out[c, l] += kappa_hat * T3 * gain
        return out

    for step in range(nsteps):
        tau = tau0 + step * dt * HBARC
        T = T0 * (tau0 / tau) ** (1.0 / 3.0)
        T3 = T * T * T
        H = np.empty((2, nl, n, n), dtype=np.complex128)
        for c in range(2):
            for l in range(nl):
                H[c, l] = Hkin + np.diag(Vstat[c, l] + T3 * Vr2[c])
        k1 = rhs(rho, H, T3)
        k2 = rhs(rho + 0.5 * dt * k1, H, T3)
        k3 = rhs(rho + 0.5 * dt * k2, H, T3)
        k4 = rhs(rho + dt * k3, H, T3)
        rho = rho + (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return rho, nsteps


def expectation(rho_block, phi, dr):
    """<phi| rho |phi> for a real grid state phi (full grid, index 0 ignored) normalised with the
    discrete norm."""
    f = np.asarray(phi)[1:]
    return float(np.real(dr * f @ rho_block @ f))
