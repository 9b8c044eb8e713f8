// eigen.cu -- numerical vacuum eigenstates (host code): the lowest eigenvectors of the discretised
// singlet vacuum Hamiltonian of one angular momentum on the trajectory grid, H = V + K with
// V_j = -C_F alpha_s / r_j + l(l+1) / (M r_j^2) on r_j = j dr and K diagonal in the sine basis of the
// grid (the kinetic factor the propagator uses: p_k^2/M, or 2[1 - cos(p_k dr)]/(M dr^2) for
// derivType 1, p_k = pi k / L).  These are the computed eigenstates of Sec. 2.5 (the paper's
// ProjType 1 / initType 100), obtained here by LOBPCG (Knyazev's locally optimal block
// preconditioned conjugate gradient) with the kinetic preconditioner (K + s)^-1, H applied through
// sine transforms in O(N log N).
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "eigen.h"

namespace qt {
namespace {

using cplx = std::complex<double>;
using Vec = std::vector<double>;

// in-place radix-2 complex FFT (forward, e^{-2 pi i jk/n}); n a power of two
void fft(std::vector<cplx> &a)
{
    const size_t n = a.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(a[i], a[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = -2.0 * M_PI / (double)len;
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const cplx w(std::cos(ang * (double)k), std::sin(ang * (double)k));
                const cplx u = a[i + k], v = a[i + k + len / 2] * w;
                a[i + k] = u + v;
                a[i + k + len / 2] = u - v;
            }
    }
}

struct Problem {
    int N;
    Vec V, K;          // potential on the grid, kinetic factor per sine mode
    double shift;      // preconditioner shift
    double hnorm;      // bound of |H|
    mutable std::vector<cplx> z;

    // S_k = sum_j x_j sin(pi j k / N): the length-2N FFT of the odd extension, Im part / -2
    void dst(const Vec &x, Vec &out) const
    {
        z.assign(2 * (size_t)N, cplx(0.0, 0.0));
        for (int j = 1; j < N; ++j) {
            z[j] = x[j];
            z[2 * N - j] = -x[j];
        }
        fft(z);
        out.assign(N, 0.0);
        for (int k = 1; k < N; ++k) out[k] = -z[k].imag() / 2.0;
    }
    void apply_h(const Vec &x, Vec &y) const
    {
        Vec s, t;
        dst(x, s);
        for (int k = 0; k < N; ++k) s[k] *= K[k];
        dst(s, t);
        y.assign(N, 0.0);
        for (int j = 1; j < N; ++j) y[j] = V[j] * x[j] + t[j] * 2.0 / N;
    }
    void precondition(const Vec &r, Vec &w) const
    {
        Vec s, t;
        dst(r, s);
        for (int k = 0; k < N; ++k) s[k] /= (K[k] + shift);
        dst(s, t);
        w.assign(N, 0.0);
        for (int j = 1; j < N; ++j) w[j] = t[j] * 2.0 / N;
    }
};

double dot(const Vec &a, const Vec &b)
{
    double s = 0.0;
    for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
    return s;
}

// modified Gram-Schmidt, twice; vectors that become (numerically) dependent are dropped
void orthonormalise(std::vector<Vec> &v)
{
    std::vector<Vec> q;
    for (Vec &x : v) {
        const double n0 = std::sqrt(dot(x, x));
        if (!(n0 > 0)) continue;
        for (int pass = 0; pass < 2; ++pass)
            for (const Vec &e : q) {
                const double c = dot(e, x);
                for (size_t i = 0; i < x.size(); ++i) x[i] -= c * e[i];
            }
        const double n1 = std::sqrt(dot(x, x));
        if (n1 < 1e-10 * n0) continue;
        for (double &e : x) e /= n1;
        q.push_back(std::move(x));
    }
    v.swap(q);
}

// eigenpairs of a small symmetric matrix (cyclic Jacobi), ascending
void jacobi(std::vector<double> a, int n, std::vector<double> &w, std::vector<double> &vecs)
{
    vecs.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) vecs[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += a[(size_t)i * n + j] * a[(size_t)i * n + j];
        if (off < 1e-30) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = a[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double theta = (a[(size_t)q * n + q] - a[(size_t)p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {   // columns p, q
                    const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
                    a[(size_t)k * n + p] = c * akp - s * akq;
                    a[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {   // rows p, q
                    const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
                    a[(size_t)p * n + k] = c * apk - s * aqk;
                    a[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = vecs[(size_t)k * n + p], vkq = vecs[(size_t)k * n + q];
                    vecs[(size_t)k * n + p] = c * vkp - s * vkq;
                    vecs[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return a[(size_t)x * n + x] < a[(size_t)y * n + y]; });
    std::vector<double> v2((size_t)n * n);
    w.assign(n, 0.0);
    for (int c = 0; c < n; ++c) {
        w[c] = a[(size_t)idx[c] * n + idx[c]];
        for (int k = 0; k < n; ++k) v2[(size_t)k * n + c] = vecs[(size_t)k * n + idx[c]];
    }
    vecs.swap(v2);
}

} // namespace

int vacuum_eigenstates(const EigenProblem &ep, int l, int m, const std::vector<std::vector<double>> &start,
                       std::vector<std::vector<double>> &out, std::vector<double> &lam)
{
    const int N = ep.N;
    Problem P;
    P.N = N;
    P.V.assign(N, 0.0);
    P.K.assign(N, 0.0);
    const double dr = ep.L / N;
    double vmax = 0.0, kmax = 0.0;
    for (int j = 1; j < N; ++j) {
        const double r = j * dr;
        const double vac = ep.potential == 1 ? (r <= ep.r_sb ? -ep.a / r + ep.sigma * r : -ep.a / ep.r_sb + ep.sigma * ep.r_sb)
                                             : ep.coul / r;
        P.V[j] = vac + l * (l + 1.0) / (ep.M * r * r);
        vmax = std::max(vmax, std::fabs(P.V[j]));
    }
    for (int k = 0; k < N; ++k) {
        const double p = M_PI * k / ep.L;
        P.K[k] = ep.deriv_type == 1 ? 2.0 * (1.0 - std::cos(p * dr)) / (ep.M * dr * dr) : p * p / ep.M;
        kmax = std::max(kmax, P.K[k]);
    }
    P.shift = 1.0;
    P.hnorm = vmax + kmax;
    const double tol = 3e-15 * P.hnorm;

    std::vector<Vec> X = start, P_dir;
    for (Vec &x : X) x[0] = 0.0;
    orthonormalise(X);
    if ((int)X.size() != m) return -1;
    std::vector<Vec> HX(m);
    double res_max = 0.0;
    int it;
    for (it = 0; it < 6000; ++it) {
        lam.assign(m, 0.0);
        std::vector<Vec> W(m);
        res_max = 0.0;
        for (int i = 0; i < m; ++i) {
            P.apply_h(X[i], HX[i]);
            lam[i] = dot(X[i], HX[i]);
            Vec r(N);
            for (int j = 0; j < N; ++j) r[j] = HX[i][j] - lam[i] * X[i][j];
            res_max = std::max(res_max, std::sqrt(dot(r, r)));
            P.precondition(r, W[i]);
        }
        if (res_max < tol) break;
        std::vector<Vec> B = X;
        for (Vec &w : W) B.push_back(w);
        for (Vec &p : P_dir) B.push_back(p);
        orthonormalise(B);
        const int nb = (int)B.size();
        std::vector<Vec> HB(nb);
        for (int i = 0; i < nb; ++i) P.apply_h(B[i], HB[i]);
        std::vector<double> A((size_t)nb * nb), w, c;
        for (int i = 0; i < nb; ++i)
            for (int j = i; j < nb; ++j) A[(size_t)i * nb + j] = A[(size_t)j * nb + i] = dot(B[i], HB[j]);
        jacobi(A, nb, w, c);
        std::vector<Vec> Xn(m, Vec(N, 0.0));
        for (int i = 0; i < m; ++i)
            for (int b = 0; b < nb; ++b) {
                const double cb = c[(size_t)b * nb + i];
                for (int j = 0; j < N; ++j) Xn[i][j] += cb * B[b][j];
            }
        P_dir.assign(m, Vec(N, 0.0));
        for (int i = 0; i < m; ++i) {
            P_dir[i] = Xn[i];
            for (int k = 0; k < m; ++k) {
                const double ck = dot(X[k], Xn[i]);
                for (int j = 0; j < N; ++j) P_dir[i][j] -= ck * X[k][j];
            }
        }
        X.swap(Xn);
    }
    if (res_max >= 1e-13 * P.hnorm) return -2;
    // discrete normalisation (L/N) sum u^2 = 1, sign: positive overlap with the start vector (KSU:
    // positive at the first point above 1e-3 of the largest value)
    out.assign(m, Vec(N, 0.0));
    for (int i = 0; i < m; ++i) {
        double s = dot(X[i], start[i]) < 0 ? -1.0 : 1.0;
        if (ep.potential == 1) {
            double mx = 0.0;
            for (int j = 0; j < N; ++j) mx = std::max(mx, std::fabs(X[i][j]));
            for (int j = 0; j < N; ++j)
                if (std::fabs(X[i][j]) > 1e-3 * mx) {
                    s = X[i][j] < 0 ? -1.0 : 1.0;
                    break;
                }
        }
        for (int j = 0; j < N; ++j) out[i][j] = s * X[i][j] / std::sqrt(dr);
    }
    return it;
}

} // namespace qt
