/*
 * qtraj_oracle.c -- plain, slow FP64 CPU oracle of the QTraj 1.0 quantum-trajectory method
 * (Brambilla, Escobedo, Strickland, Vairo, Vander Griend, Weber, arXiv:2107.06147).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file's library.  It shares no code, header, table or constant generator
 * with the CUDA path; it has its own radix-2 FFT and its own Philox4x32-10.
 *
 * What it computes, step by step, in the paper's order:
 *   - grid and norm (Sec. 3.3, Eq. normcond): u_j = u(r_j), r_j = j*dr, dr = L/N, j = 0..N-1,
 *     u_0 = 0 and u(L) = 0; norm^2 = (L/N) sum_j |u_j|^2;
 *   - the Strang split step (Sec. 3.3, steps 1-5): exp(-i V dt/2), sine transform, exp(-i T dt),
 *     inverse sine transform, exp(-i V dt/2).  The sine transform is realised literally as a
 *     complex DFT of length 2N of the odd extension of u (zero at 0 and N) -- the plain definition;
 *   - T_kin = p^2/m with m the heavy-quark mass (Sec. 2.4), or 2[1-cos(p dr)]/(m dr^2);
 *   - the OQS+pNRQCD ("Munich") potential (App. E, Eqs. E.1-E.5 and the V_I lines after them),
 *     written for general N_c, with the centrifugal term l(l+1)/(m r^2);
 *   - Bjorken cooling T(tau) = T0 (tau0/tau)^{1/3} (Sec. 3.4, Table 1); step n uses T(tau_n)
 *     for both half-steps, as the evolution loop loads the space kernel with T[n] before each step;
 *   - the waiting-time Monte-Carlo wave-function algorithm (Sec. 3.2.1, Eq. wta; Sec. 3.5 items
 *     3-4): draw r, evolve until norm^2 <= r, jump (l -> l +- 1 with p_{l,-} = l/(2l+1), Eq. Pl+-;
 *     colour s -> o, o -> s with 2/(N_c^2-2), Sec. 3.4.2), multiply by r and renormalise, redraw;
 *   - the rMin shortcut, rMax and maxJumps options (Sec. 3.5 item 4);
 *   - survival ratios of the 1S, 2S, 1P, 3S, 2P, 1D Coulomb states (Sec. 5 and the ratios.tsv
 *     format of App. C with its footnote on zero initial overlaps).
 *
 * Readings where the paper is silent or garbled:
 *   hbar*c = 0.1973269804 GeV fm converts dt (GeV^-1) to fm/c; n_steps = ceil((tau_f-tau0)/(hbar c dt))
 *   with tau_f = tau0 (T0/Tf)^3; the generator is Philox4x32-10 keyed by the 64-bit trajectory seed with
 *   counter (k,0,0,0) for waiting period k; jumps may trigger after the final step; overlaps are taken
 *   with the normalised state; Coulomb eigenstates are normalised on the grid.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OQT_HBARC 0.1973269804      /* GeV fm */
#define OQT_PI 3.14159265358979323846

/* observable flags */
#define OQT_F_NOJUMP_SHORTCUT 1
#define OQT_F_BORDERLINE 2
#define OQT_F_RMAX 4
#define OQT_F_MAXJUMPS 8
#define OQT_F_LCAP 16
#define OQT_F_NONFINITE 32

#define OQT_NBASIS 6
#define OQT_BORDERLINE_EPS 1e-12

typedef struct {
    int N;            /* grid points (power of two) */
    double L, dt, M;  /* box (GeV^-1), time step (GeV^-1), heavy-quark mass (GeV) */
    double alpha_s, Nc;
    int deriv_type;   /* 0: p^2/M ; 1: 2[1-cos(p dr)]/(M dr^2) */
    int max_jumps;    /* < 0: unlimited */
    double r_max;     /* 1.0: off */
    int l_cap;        /* < 0: none; a jump to l > l_cap ends the trajectory with zero overlaps */
    int use_rmin;     /* 1: rMin shortcut */
    double t_vac;     /* vacuum evolution before the medium, GeV^-1 (Table 1: tmed - t0); 0: none */
    const double *basis; /* OQT_NBASIS x N overlap basis (numerical eigenstates), NULL: analytic Coulomb */
    int potential;    /* 0: the OQS+pNRQCD potential of App. E with jumps; 1: the isotropic KSU
                         potential of App. E (singlet, H_eff only, no jumps) */
    double ksu_fmd;   /* F_mD, the KSU Debye-mass factor */
} oqt_params;

/* kind 0 Gaussian, 1 analytic Coulomb eigenstate, 2 a given (numerical) eigenstate in u0 (N values,
 * discretely normalised) */
typedef struct { int kind; double width; int n, l, color; const double *u0; } oqt_init;
/* kind 0: Bjorken T0 (tau0/tau)^{1/3} from tau0; kind 1: T(tau) interpolated linearly in the table
 * (tab_tau[i], tab_T[i]), i < tab_n, tau ascending (fm/c), from tab_tau[0] (Table 1
 * temperatureEvolution 1/2; the file formats of App. B).  Both end once T < Tf. */
typedef struct {
    double T0, tau0, Tf, kappa_hat, gamma_hat;
    int kind;
    const double *tab_tau, *tab_T;
    int tab_n;
} oqt_medium;

typedef struct {
    double surv[OQT_NBASIS];
    double ov_re[OQT_NBASIS], ov_im[OQT_NBASIS];
    double norm2, r0;
    int l, color, n_jumps, n_steps_exec, flags, first_jump_step;
    int last_jump_step;      /* -1 if none */
    uint32_t jump_digest;    /* FNV-1a (32 bit) of the jump sequence, see oqt_digest_jump */
} oqt_obs;

/* FNV-1a, 32 bit (Fowler, Noll, Vo): h = (h XOR byte) * 16777619 per byte from the offset basis
 * 2166136261.  A trajectory's jump digest runs over the little-endian bytes of the three words
 * (step, new l, new colour) of each of its jumps in order; two runs share it when their jump
 * sequences are identical step for step. */
#define OQT_FNV_BASIS 2166136261u
static uint32_t oqt_fnv_bytes(uint32_t h, uint32_t word)
{
    unsigned char b[4] = {(unsigned char)(word & 255u), (unsigned char)((word >> 8) & 255u),
                          (unsigned char)((word >> 16) & 255u), (unsigned char)(word >> 24)};
    for (int i = 0; i < 4; i++) {
        h ^= b[i];
        h *= 16777619u;
    }
    return h;
}
static uint32_t oqt_digest_jump(uint32_t h, int step, int l, int color)
{
    h = oqt_fnv_bytes(h, (uint32_t)step);
    h = oqt_fnv_bytes(h, (uint32_t)l);
    return oqt_fnv_bytes(h, (uint32_t)color);
}

/* one row of the per-step summary (App. C, summary.tsv): after step `step` (1-based), before a jump
 * at that step -- the norm, colour, l, the overlaps |<nl|psi>|^2 of the normalised state (zero unless
 * a singlet of the basis state's l), and <psi|r|psi> / <psi|psi> / <1S|r|1S> */
typedef struct {
    int step, color, l, flags;
    double norm2;
    double ov2[OQT_NBASIS];
    double r_ratio;
} oqt_trace_rec;

/* basis order: 1S, 2S, 1P, 3S, 2P, 1D as (n, l) of the Coulomb problem */
static const int OQT_BASIS_N[OQT_NBASIS] = {1, 2, 2, 3, 3, 3};
static const int OQT_BASIS_L[OQT_NBASIS] = {0, 0, 1, 0, 1, 2};

/* ------------------------------------------------------------------------------------------ */
/* FFT: iterative radix-2 Cooley-Tukey with bit reversal.  X_k = sum_j x_j exp(sign*2 pi i jk/n). */
/* Twiddles are evaluated directly with cos/sin for every (stage, k) pair -- no recurrences.      */
/* ------------------------------------------------------------------------------------------ */
int oqt_fft(int n, double complex *x, int sign)
{
    if (n < 1 || (n & (n - 1))) return -1;
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { double complex t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1;
        for (int k = 0; k < half; k++) {
            double ang = sign * 2.0 * OQT_PI * (double)k / (double)len;
            double complex w = cos(ang) + I * sin(ang);
            for (int s = 0; s < n; s += len) {
                double complex a = x[s + k], b = w * x[s + k + half];
                x[s + k] = a + b;
                x[s + k + half] = a - b;
            }
        }
    }
    return 0;
}

/* brute-force O(n^2) DFT, the definition, used to pin oqt_fft */
void oqt_dft(int n, const double complex *x, double complex *X, int sign)
{
    for (int k = 0; k < n; k++) {
        double complex s = 0;
        for (int j = 0; j < n; j++) {
            long long jk = ((long long)j * k) % n;
            double ang = sign * 2.0 * OQT_PI * (double)jk / (double)n;
            s += x[j] * (cos(ang) + I * sin(ang));
        }
        X[k] = s;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",     */
/* SC'11): ten rounds of two 32x32->64 multiplies with a Weyl key schedule.                      */
/* ------------------------------------------------------------------------------------------ */
void oqt_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The three uniforms of waiting period k of a trajectory: threshold r (53 bits, in (0,1)),
 * the angular-momentum draw u_l and the colour draw u_c (32 bits each, in (0,1)). */
void oqt_draws(uint64_t seed, uint32_t k, double *r, double *ul, double *uc)
{
    uint32_t ctr[4] = {k, 0u, 0u, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    oqt_philox4x32_10(ctr, key, x);
    uint64_t w = ((uint64_t)x[1] << 32) | x[0];
    *r = ((double)(w >> 11) + 0.5) * 0x1.0p-53;
    *ul = ((double)x[2] + 0.5) * 0x1.0p-32;
    *uc = ((double)x[3] + 0.5) * 0x1.0p-32;
}

/* the same over arrays: the words of n (counter, key) pairs, and the uniforms of n (seed, k) pairs
 * (for comparing long streams with another implementation without a call per value) */
void oqt_philox_many(int n, const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    for (int i = 0; i < n; i++) oqt_philox4x32_10(ctr + 4 * (size_t)i, key + 2 * (size_t)i, out + 4 * (size_t)i);
}

void oqt_draws_many(int n, const uint64_t *seed, const uint32_t *k, double *out)
{
    for (int i = 0; i < n; i++)
        oqt_draws(seed[i], k[i], out + 3 * (size_t)i, out + 3 * (size_t)i + 1, out + 3 * (size_t)i + 2);
}

/* ------------------------------------------------------------------------------------------ */
/* physics helpers                                                                             */
/* ------------------------------------------------------------------------------------------ */
static double oqt_CF(double Nc) { return (Nc * Nc - 1.0) / (2.0 * Nc); }

/* Bohr radius a0 = 1/(mu alpha), mu = M/2 the reduced mass, alpha = C_F alpha_s */
double oqt_bohr_radius(const oqt_params *p) { return 2.0 / (p->M * oqt_CF(p->Nc) * p->alpha_s); }

/* a tabulated temperature at tau: linear between the two neighbouring points; before the first
 * point the first temperature, after the last the last */
static double oqt_table_T(const oqt_medium *m, double tau)
{
    if (tau <= m->tab_tau[0]) return m->tab_T[0];
    for (int i = 0; i + 1 < m->tab_n; i++)
        if (tau < m->tab_tau[i + 1])
            return m->tab_T[i] + (m->tab_T[i + 1] - m->tab_T[i]) * (tau - m->tab_tau[i]) /
                                     (m->tab_tau[i + 1] - m->tab_tau[i]);
    return m->tab_T[m->tab_n - 1];
}

/* the proper time the medium starts at */
static double oqt_tau_start(const oqt_medium *m) { return m->kind == 1 ? m->tab_tau[0] : m->tau0; }

/* number of steps until T(tau) falls below Tf: ceil((tau_f - tau_start) / (hbar c dt)), with tau_f
 * from T0 (tau0/tau_f)^{1/3} = Tf (Bjorken) or the first crossing of Tf by the table (its last tau if
 * it never falls below Tf) */
int oqt_n_steps(const oqt_params *p, const oqt_medium *m)
{
    double tau_f;
    if (m->kind == 1) {
        tau_f = m->tab_tau[m->tab_n - 1];
        if (m->tab_T[0] < m->Tf) tau_f = m->tab_tau[0];
        else
            for (int i = 0; i + 1 < m->tab_n; i++)
                if (m->tab_T[i + 1] < m->Tf) {
                    tau_f = m->tab_tau[i] + (m->tab_tau[i + 1] - m->tab_tau[i]) * (m->tab_T[i] - m->Tf) /
                                                (m->tab_T[i] - m->tab_T[i + 1]);
                    break;
                }
    } else {
        tau_f = m->tau0 * pow(m->T0 / m->Tf, 3.0);
    }
    double steps = ceil((tau_f - oqt_tau_start(m)) / (OQT_HBARC * p->dt));
    if (steps < 0) steps = 0;
    return (int)steps;
}

/* T(tau_n)^3 for step n, tau_n = tau_start + n dt hbar c: T0^3 tau0 / tau_n (Bjorken) or the
 * table's temperature cubed */
double oqt_T3(const oqt_params *p, const oqt_medium *m, int n)
{
    double tau = oqt_tau_start(m) + (double)n * p->dt * OQT_HBARC;
    double T = m->kind == 1 ? oqt_table_T(m, tau) : m->T0 * pow(m->tau0 / tau, 1.0 / 3.0);
    return T * T * T;
}

/* kappa_hat(T) from the lattice fits of App. E (the potential's parameter kappa = -1, -2, -3 selects the
 * central, lower and upper fit): kappa_hat = 1 / (a x^{3/2} + b x + c x^{1/2} + d), x = T / T_c with
 * T_c = 0.155 GeV.  which = 1, 2, 3. */
double oqt_kappa_fit(int which, double T)
{
    static const double coef[3][4] = {{0.00397, -0.08341, 0.98031, -0.51889},
                                      {0.00712, -0.14262, 1.55601, -0.80712},
                                      {0.00272, -0.05854, 0.71513, -0.38197}};
    const double *k = coef[which - 1];
    double x = T / 0.155;
    return 1.0 / (k[0] * pow(x, 1.5) + k[1] * x + k[2] * sqrt(x) + k[3]);
}

/* the kappa_hat a medium uses at temperature cubed T3: its constant, or a lattice fit of T */
double oqt_kappa_at(const oqt_medium *m, double T3)
{
    if (m->kappa_hat >= 0) return m->kappa_hat;
    return oqt_kappa_fit((int)(-m->kappa_hat), cbrt(T3));
}

/* ------------------------------------------------------------------------------------------ */
/* The isotropic KSU potential (App. E, "Isotropic KSU potential"): a Karsch-Mehr-Satz real part  */
/* capped at the vacuum Cornell potential's string-breaking value, and the leading-order          */
/* imaginary part of the chromoelectric screening regime.  Constants as printed: a = 0.409,       */
/* sigma = 0.21 GeV^2, r_SB = 1.25 fm, alpha_s(5 GeV) = 0.2034.  Readings (the paper leaves them    */
/* open): alpha_s(mu) runs at one loop from alpha_s(5 GeV) with N_F = 3 flavours, which also enter */
/* m_D; the alpha_s of V_I is the same alpha_s(2 pi T); C_F = (Nc^2-1)/(2 Nc) (4/3 at Nc = 3).      */
/* ------------------------------------------------------------------------------------------ */
#define OQT_KSU_A 0.409
#define OQT_KSU_SIGMA 0.21
#define OQT_KSU_RSB_FM 1.25
#define OQT_KSU_ALPHAS_MZ 0.2034   /* at mu0 = 5 GeV */
#define OQT_KSU_MU0 5.0
#define OQT_KSU_NF 3
#define OQT_EULER_GAMMA 0.57721566490153286061

/* one-loop running coupling: alpha_s(mu) = alpha_0 / (1 + alpha_0 b0 ln(mu^2/mu0^2)),
 * b0 = (11 Nc - 2 N_F) / (12 pi) */
double oqt_alpha_s_run(double mu, double Nc)
{
    double b0 = (11.0 * Nc - 2.0 * OQT_KSU_NF) / (12.0 * OQT_PI);
    return OQT_KSU_ALPHAS_MZ / (1.0 + OQT_KSU_ALPHAS_MZ * b0 * log(mu * mu / (OQT_KSU_MU0 * OQT_KSU_MU0)));
}

/* the isotropic Debye mass m_D = F_mD T sqrt(Nc (1 + N_F/6) pi alpha), alpha = C_F alpha_s(2 pi T) */
double oqt_ksu_debye_mass(const oqt_params *p, double T)
{
    if (T <= 0) return 0.0;
    double alpha = oqt_CF(p->Nc) * oqt_alpha_s_run(2.0 * OQT_PI * T, p->Nc);
    return p->ksu_fmd * T * sqrt(p->Nc * (1.0 + OQT_KSU_NF / 6.0) * OQT_PI * alpha);
}

/* E1(x) = int_x^inf e^-t / t dt for x > 0, times e^x: the power series of E1 (x <= 1) or the
 * continued fraction e^x E1(x) = 1/(x+1- 1/(x+3- 4/(x+5- 9/(x+7- ...)))) (x > 1), evaluated by
 * the modified Lentz method */
double oqt_expE1(double x)
{
    if (x <= 1.0) {
        double sum = 0.0, term = 1.0;
        for (int k = 1; k < 60; k++) {
            term *= -x / k;
            sum += term / k;
        }
        return exp(x) * (-OQT_EULER_GAMMA - log(x) - sum);
    }
    double b = x + 1.0, c = 1e300, d = 1.0 / b, h = d;
    for (int i = 1; i < 1000; i++) {
        double an = -(double)i * i;
        b += 2.0;
        d = 1.0 / (an * d + b);
        c = b + an / c;
        double del = c * d;
        h *= del;
        if (fabs(del - 1.0) < 1e-17) break;
    }
    return h;
}

/* Ei(x) = PV int_-inf^x e^t / t dt for x > 0, times e^-x: the power series
 * Ei(x) = gamma + ln x + sum_k x^k / (k k!) (all terms positive) for x <= 60, the asymptotic series
 * e^-x Ei(x) ~ sum_k k!/x^(k+1), cut before its terms grow, above (its error ~ e^-x) */
double oqt_expmEi(double x)
{
    if (x <= 60.0) {
        double sum = 0.0, term = 1.0;
        for (int k = 1; k < 400; k++) {
            term *= x / k;
            double t = term / k;
            sum += t;
            if (t < 1e-18 * sum) break;
        }
        return exp(-x) * (OQT_EULER_GAMMA + log(x) + sum);
    }
    double sum = 0.0, term = 1.0 / x, prev = 1e300;
    for (int k = 0; k < 200; k++) {
        if (term > prev) break;
        sum += term;
        prev = term;
        term *= (k + 1.0) / x;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

/* phi(rhat) = 2 int_0^inf dz z/(z^2+1)^2 [1 - sin(z rhat)/(z rhat)] (the V_I of the isotropic KSU
 * potential): with int_0^inf sin(a z)/(1+z^2)^2 dz = [(1+a) e^-a Ei(a) + (1-a) e^a E1(a)]/4 (the
 * derivative in b at b = 1 of int sin(a z)/(b^2+z^2) dz = [e^-ab Ei(ab) - e^ab Ei(-ab)]/(2b), and
 * 2 int z/(z^2+1)^2 dz = 1), phi(a) = 1 - [(1+a) e^-a Ei(a) + (1-a) e^a E1(a)] / (2a); phi(0) = 0. */
double oqt_ksu_phi(double a)
{
    if (a <= 0) return 0.0;
    if (a >= 2.0) return 1.0 - ((1.0 + a) * oqt_expmEi(a) + (1.0 - a) * oqt_expE1(a)) / (2.0 * a);
    /* below 2 the closed form loses digits to cancellation (phi ~ a^2 ln a while each term is O(1));
     * the same expression expanded instead: with f(a) = (1+a) e^-a = sum_n (-1)^n (1-n) a^n / n! and
     * P(a) = sum_{n>=1} a^n / (n n!) (so that Ei = gamma + ln a + P(a), E1 = -gamma - ln a - P(-a)),
     * phi(a) = -sum_{odd m>=3} [(gamma + ln a)(m-1)/m! + c_m] a^(m-1), c_m the a^m coefficient of f P
     * (the odd orders of f P above the first give the terms; its a^1 term cancels the 1) */
    enum { NT = 40 };
    double fc[NT], pc[NT], fact = 1.0;
    for (int n = 0; n < NT; n++) {
        if (n > 0) fact *= n;
        fc[n] = ((n & 1) ? -1.0 : 1.0) * (1.0 - n) / fact;
        pc[n] = n == 0 ? 0.0 : 1.0 / (n * fact);
    }
    double L = OQT_EULER_GAMMA + log(a), sum = 0.0, mfact = 1.0, apow = a * a;
    for (int m = 1; m < NT; m++) {
        mfact *= m;
        if (m < 3 || !(m & 1)) continue;
        double cm = 0.0;
        for (int n = 0; n <= m; n++) cm += fc[n] * pc[m - n];
        sum += (L * (m - 1) / mfact + cm) * apow;   /* apow = a^(m-1) */
        apow *= a * a;
    }
    return -sum;
}

/* the KSU potential at r (singlet, angular momentum l) and temperature T: V_R + i V_I + l(l+1)/(M r^2) */
double complex oqt_ksu_potential(const oqt_params *p, int l, double T, double r)
{
    const double a = OQT_KSU_A, sig = OQT_KSU_SIGMA, rsb = OQT_KSU_RSB_FM / OQT_HBARC;
    double vcap = -a / rsb + sig * rsb;           /* V_vac(r_SB) */
    double re, im = 0.0;
    double mD = oqt_ksu_debye_mass(p, T);
    if (mD <= 0) {                                 /* vacuum: the Cornell potential with string breaking */
        re = r <= rsb ? -a / r + sig * r : vcap;
    } else {
        double e = exp(-mD * r);
        double kms = -a / r * (1.0 + mD * r) * e + 2.0 * sig / mD * (1.0 - e) - sig * r * e;
        re = kms <= vcap ? kms : vcap;
        im = -oqt_alpha_s_run(2.0 * OQT_PI * T, p->Nc) * oqt_CF(p->Nc) * T * oqt_ksu_phi(mD * r);
    }
    re += (double)l * (l + 1) / (p->M * r * r);
    return re + I * im;
}

/* V_eff(r) for colour c (0 singlet, 1 octet), angular momentum l, temperature cubed T3.
 * singlet: -C_F a_s/r + gam T^3 r^2/2 - i kap T^3 r^2/2
 * octet  : +a_s/(2 Nc r) + f gam T^3 r^2 - i f kap T^3 r^2,  f = (Nc^2-2)/(4(Nc^2-1)) = 7/32
 * plus the centrifugal l(l+1)/(M r^2). */
double complex oqt_potential(const oqt_params *p, int color, int l, double T3, double kappa_hat,
                             double gamma_hat, double r)
{
    if (p->potential == 1) return oqt_ksu_potential(p, l, cbrt(T3), r);
    double Nc = p->Nc, coul, f;
    if (color == 0) { coul = -oqt_CF(Nc) * p->alpha_s / r; f = 0.5; }
    else { coul = p->alpha_s / (2.0 * Nc * r); f = (Nc * Nc - 2.0) / (4.0 * (Nc * Nc - 1.0)); }
    double cent = (double)l * (l + 1) / (p->M * r * r);
    double re = coul + cent + f * gamma_hat * T3 * r * r;
    double im = -f * kappa_hat * T3 * r * r;
    return re + I * im;
}

/* the same value through plain pointers, for callers that cannot take a C99 complex return */
void oqt_potential_parts(const oqt_params *p, int color, int l, double T3, double kappa_hat, double gamma_hat,
                         double r, double *re, double *im)
{
    double complex v = oqt_potential(p, color, l, T3, kappa_hat, gamma_hat, r);
    *re = creal(v);
    *im = cimag(v);
}

/* kinetic energy at momentum index k of the length-2N odd extension */
double oqt_kinetic(const oqt_params *p, int k)
{
    int N = p->N;
    int kk = k <= N ? k : 2 * N - k;
    double pk = OQT_PI * (double)kk / p->L;
    if (p->deriv_type == 1) {
        double dr = p->L / N;
        return 2.0 * (1.0 - cos(pk * dr)) / (p->M * dr * dr);
    }
    return pk * pk / p->M;
}

double oqt_norm2(const oqt_params *p, const double complex *u)
{
    double s = 0;
    for (int j = 1; j < p->N; j++) s += creal(u[j]) * creal(u[j]) + cimag(u[j]) * cimag(u[j]);
    return s * p->L / p->N;
}

/* generalised Laguerre L_k^{a}(x) by the three-term recurrence */
static double oqt_laguerre(int k, int a, double x)
{
    if (k == 0) return 1.0;
    double lm1 = 1.0, l0 = 1.0 + a - x;
    for (int i = 1; i < k; i++) {
        double lp1 = ((2.0 * i + 1 + a - x) * l0 - (i + a) * lm1) / (i + 1);
        lm1 = l0; l0 = lp1;
    }
    return l0;
}

/* Coulomb u_nl(r) = r R_nl(r) up to a constant: r^{l+1} e^{-r/(n a0)} L_{n-l-1}^{2l+1}(2r/(n a0)),
 * sampled on the grid and normalised with the discrete norm. */
void oqt_eigenstate(const oqt_params *p, int n, int l, double *phi)
{
    double a0 = oqt_bohr_radius(p), dr = p->L / p->N, s = 0;
    phi[0] = 0;
    for (int j = 1; j < p->N; j++) {
        double r = j * dr, x = 2.0 * r / (n * a0);
        phi[j] = pow(r, l + 1) * exp(-r / (n * a0)) * oqt_laguerre(n - l - 1, 2 * l + 1, x);
        s += phi[j] * phi[j];
    }
    double c = 1.0 / sqrt(s * dr);
    for (int j = 1; j < p->N; j++) phi[j] *= c;
}

/* initial state: Gaussian r^{l+1} exp(-r^2/(2 w^2)) (kind 0) or Coulomb u_nl (kind 1), normalised */
void oqt_initial_state(const oqt_params *p, const oqt_init *in, double complex *u)
{
    double dr = p->L / p->N;
    if (in->kind == 2) {
        u[0] = 0;
        for (int j = 1; j < p->N; j++) u[j] = in->u0[j];
        return;
    }
    if (in->kind == 1) {
        double *phi = malloc(sizeof(double) * p->N);
        oqt_eigenstate(p, in->n, in->l, phi);
        for (int j = 0; j < p->N; j++) u[j] = phi[j];
        free(phi);
        return;
    }
    /* the Gaussian through its logarithm, less the largest logarithm (the same normalised state;
       r^{l+1} alone would overflow at large l) */
    double *e = malloc(sizeof(double) * p->N);
    double emax = -HUGE_VAL, s = 0;
    for (int j = 1; j < p->N; j++) {
        double r = j * dr;
        e[j] = (in->l + 1) * log(r) - r * r / (2.0 * in->width * in->width);
        if (e[j] > emax) emax = e[j];
    }
    u[0] = 0;
    for (int j = 1; j < p->N; j++) {
        double v = exp(e[j] - emax);
        u[j] = v;
        s += v * v;
    }
    free(e);
    double c = 1.0 / sqrt(s * dr);
    for (int j = 1; j < p->N; j++) u[j] *= c;
}

/* ------------------------------------------------------------------------------------------ */
/* one Strang step (Sec. 3.3, steps 1-5)                                                        */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    const oqt_params *p;
    double complex *z;     /* 2N scratch */
    double complex *kin;   /* 2N momentum kernel exp(-i T_kin dt) */
    double complex *kv;    /* N space kernel */
} oqt_work;

static void oqt_work_init(oqt_work *w, const oqt_params *p)
{
    int N = p->N;
    w->p = p;
    w->z = malloc(sizeof(double complex) * 2 * N);
    w->kin = malloc(sizeof(double complex) * 2 * N);
    w->kv = malloc(sizeof(double complex) * N);
    for (int k = 0; k < 2 * N; k++) w->kin[k] = cexp(-I * oqt_kinetic(p, k) * p->dt);
}

static void oqt_work_free(oqt_work *w) { free(w->z); free(w->kin); free(w->kv); }

/* loads exp(-i V_eff dt/2) for the given (colour, l, T^3), like loadSpaceKernel(T[n]) */
static void oqt_load_space_kernel(oqt_work *w, int color, int l, double T3, double kap, double gam)
{
    const oqt_params *p = w->p;
    double dr = p->L / p->N;
    w->kv[0] = 0;
    for (int j = 1; j < p->N; j++) {
        double complex V = oqt_potential(p, color, l, T3, kap, gam, j * dr);
        w->kv[j] = cexp(-I * V * (p->dt / 2.0));
    }
}

static void oqt_make_step(oqt_work *w, double complex *u)
{
    const oqt_params *p = w->p;
    int N = p->N;
    double complex *z = w->z;
    for (int j = 1; j < N; j++) u[j] *= w->kv[j];                 /* step 1 */
    z[0] = 0; z[N] = 0;                                             /* step 2: odd extension */
    for (int j = 1; j < N; j++) { z[j] = u[j]; z[2 * N - j] = -u[j]; }
    oqt_fft(2 * N, z, -1);
    for (int k = 0; k < 2 * N; k++) z[k] *= w->kin[k];             /* step 3 */
    oqt_fft(2 * N, z, +1);                                          /* step 4 */
    u[0] = 0;
    for (int j = 1; j < N; j++) u[j] = z[j] / (2.0 * N);
    for (int j = 1; j < N; j++) u[j] *= w->kv[j];                 /* step 5 */
}

/* one step with explicit (colour, l, T^3); exported for the tests */
void oqt_strang_step(const oqt_params *p, double complex *u, int color, int l, double T3,
                     double kappa_hat, double gamma_hat)
{
    oqt_work w;
    oqt_work_init(&w, p);
    oqt_load_space_kernel(&w, color, l, T3, kappa_hat, gamma_hat);
    oqt_make_step(&w, u);
    oqt_work_free(&w);
}

/* steps of the vacuum evolution: t_vac / dt rounded to the nearest integer */
int oqt_vacuum_steps(const oqt_params *p)
{
    if (!(p->t_vac > 0)) return 0;
    return (int)llround(p->t_vac / p->dt);
}

/* the state a trajectory starts the medium with (Sec. 3.5 item 3): the initial state, evolved in
 * vacuum (T = 0: the Coulomb and centrifugal potential of its colour, no imaginary part, no jumps)
 * for oqt_vacuum_steps(p) Strang steps */
void oqt_start_state(const oqt_params *p, const oqt_init *in, double complex *u)
{
    oqt_initial_state(p, in, u);
    int nv = oqt_vacuum_steps(p);
    if (nv == 0) return;
    oqt_work w;
    oqt_work_init(&w, p);
    oqt_load_space_kernel(&w, in->color, in->l, 0.0, 0.0, 0.0);
    for (int n = 0; n < nv; n++) oqt_make_step(&w, u);
    oqt_work_free(&w);
}

/* H_eff evolution without jumps from step n0 for nsteps steps; norm2_hist[i] (optional) is the
 * norm after step n0+i. */
void oqt_evolve_nojump(const oqt_params *p, double complex *u, int color, int l, const oqt_medium *m,
                       int n0, int nsteps, double *norm2_hist)
{
    oqt_work w;
    oqt_work_init(&w, p);
    for (int n = n0; n < n0 + nsteps; n++) {
        double T3 = oqt_T3(p, m, n);
        oqt_load_space_kernel(&w, color, l, T3, oqt_kappa_at(m, T3), m->gamma_hat);
        oqt_make_step(&w, u);
        if (norm2_hist) norm2_hist[n - n0] = oqt_norm2(p, u);
    }
    oqt_work_free(&w);
}

/* ------------------------------------------------------------------------------------------ */
/* jump rules                                                                                  */
/* ------------------------------------------------------------------------------------------ */
/* new angular momentum from the draw u_l: down with p_{l,-} = l/(2l+1), else up (Eq. Pl+-) */
int oqt_jump_l(int l, double ul) { return (ul < (double)l / (2.0 * l + 1.0)) ? l - 1 : l + 1; }

/* new colour from the draw u_c: a singlet always becomes an octet; an octet becomes a singlet
 * with p_{o->s} = 2/(Nc^2-2) and stays an octet otherwise (Sec. 3.4.2) */
int oqt_jump_color(const oqt_params *p, int color, double uc)
{
    double p_os = 2.0 / (p->Nc * p->Nc - 2.0);
    return (color == 1 && uc < p_os) ? 0 : 1;
}

/* ------------------------------------------------------------------------------------------ */
/* observables                                                                                 */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    double *phi;                  /* OQT_NBASIS x N eigenstates */
    double complex ov0[OQT_NBASIS];
    int ov0_zero[OQT_NBASIS];     /* structural zero of the initial overlap */
} oqt_basis;

static void oqt_basis_init(oqt_basis *b, const oqt_params *p, const oqt_init *in)
{
    int N = p->N;
    double dr = p->L / N;
    b->phi = malloc(sizeof(double) * OQT_NBASIS * N);
    double complex *u0 = malloc(sizeof(double complex) * N);
    oqt_start_state(p, in, u0);          /* the survival ratios refer to the state entering the medium */
    for (int s = 0; s < OQT_NBASIS; s++) {
        if (p->basis) memcpy(b->phi + (size_t)s * N, p->basis + (size_t)s * N, sizeof(double) * N);
        else oqt_eigenstate(p, OQT_BASIS_N[s], OQT_BASIS_L[s], b->phi + (size_t)s * N);
        /* zero unless the initial state is a singlet of the same l; an eigenstate of the basis' own
         * kind (analytic Coulomb, or numerical with a numerical basis) is orthogonal to the basis
         * states of other n of its l */
        int same_family = (in->kind == 1 && !p->basis) || (in->kind == 2 && p->basis);
        int zero = in->color != 0 || in->l != OQT_BASIS_L[s] || (same_family && in->n != OQT_BASIS_N[s]);
        b->ov0_zero[s] = zero;
        double complex o = 0;
        if (!zero)
            for (int j = 1; j < N; j++) o += b->phi[(size_t)s * N + j] * u0[j];
        b->ov0[s] = o * dr;
    }
    free(u0);
}

static void oqt_basis_free(oqt_basis *b) { free(b->phi); }

static void oqt_zero_observables(oqt_obs *o)
{
    for (int s = 0; s < OQT_NBASIS; s++) { o->surv[s] = 0; o->ov_re[s] = 0; o->ov_im[s] = 0; }
}

/* survival ratio |<nl|psi>|^2 / n^2 / |<nl|psi_0>|^2, raw |<nl|psi>|^2/n^2 when the initial
 * overlap is zero, and 0 unless the state is a singlet of the basis state's l */
static void oqt_finalize(const oqt_params *p, const oqt_basis *b, const double complex *u, int color,
                         int l, oqt_obs *o)
{
    int N = p->N;
    double dr = p->L / N;
    double n2 = oqt_norm2(p, u);
    o->norm2 = n2;
    for (int s = 0; s < OQT_NBASIS; s++) {
        if (color != 0 || l != OQT_BASIS_L[s]) { o->surv[s] = 0; o->ov_re[s] = 0; o->ov_im[s] = 0; continue; }
        double complex ov = 0;
        for (int j = 1; j < N; j++) ov += b->phi[(size_t)s * N + j] * u[j];
        ov *= dr;
        o->ov_re[s] = creal(ov); o->ov_im[s] = cimag(ov);
        /* with jumps the ensemble estimator takes the normalised state; the KSU evolution has no
         * jumps, so the norm it loses is the dissociation and the overlap is taken unnormalised */
        double prob = (creal(ov) * creal(ov) + cimag(ov) * cimag(ov)) / (p->potential == 1 ? 1.0 : n2);
        if (b->ov0_zero[s]) o->surv[s] = prob;
        else {
            double d = creal(b->ov0[s]) * creal(b->ov0[s]) + cimag(b->ov0[s]) * cimag(b->ov0[s]);
            o->surv[s] = prob / d;
        }
    }
}

/* the zeroth trajectory: H_eff evolution over the whole profile, no jumps (Sec. 3.5 item 3) */
void oqt_nojump_run(const oqt_params *p, const oqt_init *in, const oqt_medium *m, oqt_obs *o,
                    double complex *u_final)
{
    int N = p->N;
    oqt_basis b;
    oqt_basis_init(&b, p, in);
    double complex *u = malloc(sizeof(double complex) * N);
    oqt_start_state(p, in, u);
    int ns = oqt_n_steps(p, m);
    oqt_evolve_nojump(p, u, in->color, in->l, m, 0, ns, NULL);
    memset(o, 0, sizeof(*o));
    oqt_finalize(p, &b, u, in->color, in->l, o);
    o->l = in->l; o->color = in->color; o->n_jumps = 0; o->n_steps_exec = ns;
    o->first_jump_step = -1; o->r0 = 0;
    o->last_jump_step = -1; o->jump_digest = OQT_FNV_BASIS;
    if (!isfinite(o->norm2)) o->flags |= OQT_F_NONFINITE;
    if (u_final) memcpy(u_final, u, sizeof(double complex) * N);
    free(u);
    oqt_basis_free(&b);
}

/* one quantum trajectory with jumps (Sec. 3.5 item 4).  nojump (may be NULL) is the zeroth
 * trajectory of the same initial state and medium; its norm is p_NoJump = rMin. */
/* the summary row of the state u (end of step `step`) in colour c, angular momentum l */
static void oqt_trace_row(const oqt_params *p, const oqt_basis *b, const double complex *u, int c, int l,
                          int step, double n2, oqt_trace_rec *rec)
{
    int N = p->N;
    double dr = p->L / N;
    memset(rec, 0, sizeof(*rec));
    rec->step = step; rec->color = c; rec->l = l; rec->norm2 = n2;
    double rr = 0, r1s = 0;
    for (int j = 1; j < N; j++) {
        double rj = j * dr;
        rr += rj * (creal(u[j]) * creal(u[j]) + cimag(u[j]) * cimag(u[j]));
        r1s += rj * b->phi[j] * b->phi[j];                       /* basis state 0 is 1S */
    }
    rec->r_ratio = (rr * dr / n2) / (r1s * dr);
    for (int s = 0; s < OQT_NBASIS; s++) {
        if (c != 0 || l != OQT_BASIS_L[s]) continue;
        double complex ov = 0;
        for (int j = 1; j < N; j++) ov += b->phi[(size_t)s * N + j] * u[j];
        ov *= dr;
        rec->ov2[s] = (creal(ov) * creal(ov) + cimag(ov) * cimag(ov)) / n2;
    }
}

/* oqt_trajectory with the per-step summary: every `every` steps and after the last step (before a
 * jump at that step), up to cap rows in rec; *n_rec rows written.  A trajectory resolved by the rMin
 * shortcut or by r_max evolves nothing and writes no row. */
void oqt_trajectory_traced(const oqt_params *p, const oqt_init *in, const oqt_medium *m, uint64_t seed,
                           const oqt_obs *nojump, oqt_obs *o, double complex *u_final, int every,
                           oqt_trace_rec *rec, int cap, int *n_rec);

void oqt_trajectory(const oqt_params *p, const oqt_init *in, const oqt_medium *m, uint64_t seed,
                    const oqt_obs *nojump, oqt_obs *o, double complex *u_final)
{
    oqt_trajectory_traced(p, in, m, seed, nojump, o, u_final, 0, NULL, 0, NULL);
}

void oqt_trajectory_traced(const oqt_params *p, const oqt_init *in, const oqt_medium *m, uint64_t seed,
                           const oqt_obs *nojump, oqt_obs *o, double complex *u_final, int every,
                           oqt_trace_rec *rec, int cap, int *n_rec)
{
    if (n_rec) *n_rec = 0;
    int N = p->N;
    double dr = p->L / N;
    memset(o, 0, sizeof(*o));
    o->first_jump_step = -1;
    o->last_jump_step = -1;
    o->jump_digest = OQT_FNV_BASIS;
    uint32_t k = 0;
    double r, ul, uc;
    oqt_draws(seed, k, &r, &ul, &uc);
    o->r0 = r;
    const int no_jumps = p->potential == 1;   /* the KSU potentials have no jump operators */
    if (no_jumps) { r = -1.0; o->r0 = 0.0; }
    o->l = in->l; o->color = in->color;
    double complex *u = malloc(sizeof(double complex) * N);
    oqt_start_state(p, in, u);

    if (p->use_rmin && nojump && !no_jumps) {
        if (fabs(r - nojump->norm2) < OQT_BORDERLINE_EPS) o->flags |= OQT_F_BORDERLINE;
        if (r < nojump->norm2) {   /* no jump can happen: the norm never increases */
            double r0 = o->r0;
            int flags = o->flags;
            *o = *nojump;
            o->r0 = r0;
            o->n_steps_exec = 0;
            o->flags = flags | OQT_F_NOJUMP_SHORTCUT;
            if (u_final) memset(u_final, 0, sizeof(double complex) * N);
            free(u);
            return;
        }
    }
    if (!no_jumps && r > p->r_max) {
        oqt_zero_observables(o);
        o->flags |= OQT_F_RMAX;
        o->norm2 = 1.0;
        if (u_final) memcpy(u_final, u, sizeof(double complex) * N);
        free(u);
        return;
    }

    oqt_basis b;
    oqt_basis_init(&b, p, in);
    oqt_work w;
    oqt_work_init(&w, p);
    int l = in->l, c = in->color, nj = 0, ns = oqt_n_steps(p, m);
    int ended = 0;
    for (int n = 0; n < ns; n++) {
        double T3 = oqt_T3(p, m, n);
        oqt_load_space_kernel(&w, c, l, T3, oqt_kappa_at(m, T3), m->gamma_hat);
        oqt_make_step(&w, u);
        o->n_steps_exec = n + 1;
        double n2 = oqt_norm2(p, u);
        if (every > 0 && ((n + 1) % every == 0 || n + 1 == ns) && *n_rec < cap)
            oqt_trace_row(p, &b, u, c, l, n + 1, n2, &rec[(*n_rec)++]);
        if (!isfinite(n2)) { o->flags |= OQT_F_NONFINITE; oqt_zero_observables(o); ended = 1; break; }
        if (fabs(n2 - r) < OQT_BORDERLINE_EPS) o->flags |= OQT_F_BORDERLINE;
        if (n2 <= r) {                                        /* a jump is triggered */
            if (p->max_jumps >= 0 && nj >= p->max_jumps) {
                o->flags |= OQT_F_MAXJUMPS; oqt_zero_observables(o); ended = 1; break;
            }
            int l_new = oqt_jump_l(l, ul);
            int c_new = oqt_jump_color(p, c, uc);
            if (p->l_cap >= 0 && l_new > p->l_cap) {
                o->flags |= OQT_F_LCAP; oqt_zero_observables(o);
                l = l_new; c = c_new; nj++;
                if (o->first_jump_step < 0) o->first_jump_step = n;
                o->last_jump_step = n;
                o->jump_digest = oqt_digest_jump(o->jump_digest, n, l, c);
                ended = 1; break;
            }
            /* u <- r u / ||r u|| */
            double s = 0;
            for (int j = 1; j < N; j++) {
                double rj = j * dr;
                u[j] *= rj;
                s += creal(u[j]) * creal(u[j]) + cimag(u[j]) * cimag(u[j]);
            }
            double inv = 1.0 / sqrt(s * dr);
            for (int j = 1; j < N; j++) u[j] *= inv;
            l = l_new; c = c_new; nj++;
            if (o->first_jump_step < 0) o->first_jump_step = n;
            o->last_jump_step = n;
            o->jump_digest = oqt_digest_jump(o->jump_digest, n, l, c);
            k++;
            oqt_draws(seed, k, &r, &ul, &uc);
        }
    }
    o->l = l; o->color = c; o->n_jumps = nj;
    if (!ended) oqt_finalize(p, &b, u, c, l, o);
    else o->norm2 = oqt_norm2(p, u);
    if (u_final) memcpy(u_final, u, sizeof(double complex) * N);
    free(u);
    oqt_work_free(&w);
    oqt_basis_free(&b);
}

/* ------------------------------------------------------------------------------------------ */
/* batch runner: zeroth trajectory per (initial state, medium) group, then every trajectory,    */
/* one trajectory per host thread.                                                              */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    const oqt_params *p;
    int n_traj;
    const oqt_init *inits; const int *init_idx;
    const oqt_medium *media; const int *medium_idx;
    const uint64_t *seeds;
    const oqt_obs *nojump; const int *group_of;   /* per trajectory group id, or NULL */
    oqt_obs *out;
    double complex *u_final;                      /* n_traj x N or NULL */
    int next;
} oqt_batch;

static void *oqt_batch_worker(void *arg)
{
    oqt_batch *bt = (oqt_batch *)arg;
    for (;;) {
        int t = __atomic_fetch_add(&bt->next, 1, __ATOMIC_RELAXED);
        if (t >= bt->n_traj) break;
        const oqt_obs *nj = bt->group_of ? &bt->nojump[bt->group_of[t]] : NULL;
        oqt_trajectory(bt->p, &bt->inits[bt->init_idx[t]], &bt->media[bt->medium_idx[t]], bt->seeds[t], nj,
                       &bt->out[t], bt->u_final ? bt->u_final + (size_t)t * bt->p->N : NULL);
    }
    return NULL;
}

typedef struct {
    const oqt_params *p;
    int n_groups;
    const oqt_init *inits; const oqt_medium *media;
    const int *g_init, *g_medium;
    oqt_obs *out;
    int next;
} oqt_group_batch;

static void *oqt_group_worker(void *arg)
{
    oqt_group_batch *gb = (oqt_group_batch *)arg;
    for (;;) {
        int g = __atomic_fetch_add(&gb->next, 1, __ATOMIC_RELAXED);
        if (g >= gb->n_groups) break;
        oqt_nojump_run(gb->p, &gb->inits[gb->g_init[g]], &gb->media[gb->g_medium[g]], &gb->out[g], NULL);
    }
    return NULL;
}

static void oqt_run_threads(void *(*fn)(void *), void *arg, int n_threads)
{
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = malloc(sizeof(pthread_t) * n_threads);
    for (int i = 0; i < n_threads; i++) pthread_create(&th[i], NULL, fn, arg);
    for (int i = 0; i < n_threads; i++) pthread_join(th[i], NULL);
    free(th);
}

/* Runs n_traj trajectories.  Trajectory t uses inits[init_idx[t]], media[medium_idx[t]] and
 * seeds[t].  When p->use_rmin is set, the zeroth trajectory of every (init, medium) pair that
 * occurs is run first and its results are written to nojump_out[init*n_media + medium] (if not
 * NULL).  Returns 0. */
int oqt_run_batch(const oqt_params *p, int n_traj, const oqt_init *inits, int n_inits, const int *init_idx,
                  const oqt_medium *media, int n_media, const int *medium_idx, const uint64_t *seeds,
                  oqt_obs *out, double complex *u_final, oqt_obs *nojump_out, int n_threads)
{
    int n_pairs = n_inits * n_media;
    oqt_obs *nojump = NULL;
    int *group_of = NULL;
    if (p->use_rmin) {
        int *used = calloc(n_pairs, sizeof(int));
        for (int t = 0; t < n_traj; t++) used[init_idx[t] * n_media + medium_idx[t]] = 1;
        int *g_init = malloc(sizeof(int) * n_pairs), *g_medium = malloc(sizeof(int) * n_pairs);
        int *pair_group = malloc(sizeof(int) * n_pairs);
        int ng = 0;
        for (int q = 0; q < n_pairs; q++) {
            pair_group[q] = -1;
            if (used[q]) { g_init[ng] = q / n_media; g_medium[ng] = q % n_media; pair_group[q] = ng; ng++; }
        }
        nojump = calloc(ng > 0 ? ng : 1, sizeof(oqt_obs));
        oqt_group_batch gb = {p, ng, inits, media, g_init, g_medium, nojump, 0};
        oqt_run_threads(oqt_group_worker, &gb, n_threads < ng ? n_threads : (ng > 0 ? ng : 1));
        group_of = malloc(sizeof(int) * (n_traj > 0 ? n_traj : 1));
        for (int t = 0; t < n_traj; t++) group_of[t] = pair_group[init_idx[t] * n_media + medium_idx[t]];
        if (nojump_out) {
            memset(nojump_out, 0, sizeof(oqt_obs) * n_pairs);
            for (int q = 0; q < n_pairs; q++) if (pair_group[q] >= 0) nojump_out[q] = nojump[pair_group[q]];
        }
        free(used); free(g_init); free(g_medium); free(pair_group);
    }
    oqt_batch bt = {p, n_traj, inits, init_idx, media, medium_idx, seeds, nojump, group_of, out, u_final, 0};
    oqt_run_threads(oqt_batch_worker, &bt, n_threads);
    free(nojump);
    free(group_of);
    return 0;
}
