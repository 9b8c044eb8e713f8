// eigen.h -- numerical vacuum eigenstates of the discretised singlet Hamiltonian (host code).
#pragma once
#include <vector>

namespace qt {

struct EigenProblem {
    int N;           // grid points, r_j = j L / N
    double L, M;     // box (GeV^-1), heavy-quark mass (GeV)
    double coul;     // coefficient of 1/r (the singlet's -C_F alpha_s)
    int deriv_type;  // kinetic factor as in the propagator: 0 p^2/M, 1 2[1 - cos(p dr)]/(M dr^2)
    // vacuum potential of the isotropic KSU model instead of coul / r (potential 1): the Cornell
    // -a/r + sigma r, constant beyond r_sb; its states are signed positive at their first point
    // above 1e-3 of their largest value (the others: positive overlap with the start vector)
    int potential = 0;
    double a = 0, sigma = 0, r_sb = 0;
};

// The m lowest eigenvectors of H = V_l + K for angular momentum l, started from `start` (m vectors of
// length N, e.g. the analytic Coulomb states of n = l+1 .. l+m), discretely normalised, each signed
// to overlap positively with its start vector; lam their eigenvalues.  Returns the iterations used,
// or a negative value if the residual did not fall below 1e-13 |H|.
int vacuum_eigenstates(const EigenProblem &ep, int l, int m, const std::vector<std::vector<double>> &start,
                       std::vector<std::vector<double>> &out, std::vector<double> &lam);

} // namespace qt
