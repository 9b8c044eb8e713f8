// api.cu -- the C ABI of libqtraj (include/qtraj.h): context, read-only tables, workspace layout,
// and the orchestration of an evolve (no-jump runs of every (initial state, medium) group first,
// then all trajectories).  All host-side tables are built in FP64.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "api_internal.h"
#include "eigen.h"
#include "fused_launch.cuh"
#include "plain.cuh"
#include "qtraj.h"

using namespace qt;

namespace {

constexpr double HBARC = 0.1973269804; // GeV fm
constexpr double PI = 3.14159265358979323846;
const int BASIS_N[NBASIS] = {1, 2, 2, 3, 3, 3};
const int BASIS_L[NBASIS] = {0, 0, 1, 0, 1, 2};

thread_local std::string g_err;

qtraj_status fail(qtraj_status st, const char *fmt, ...)
{
    char b[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof b, fmt, ap);
    va_end(ap);
    g_err = b;
    return st;
}

#define CK(call)                                                                                                   \
    do {                                                                                                           \
        cudaError_t e_ = (call);                                                                                   \
        if (e_ != cudaSuccess) return fail(QTRAJ_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                                           __LINE__);                                                              \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// generalised Laguerre polynomial L_k^{(a)}(x), three-term recurrence
double laguerre(int k, int a, double x)
{
    if (k == 0) return 1.0;
    double p0 = 1.0, p1 = 1.0 + a - x;
    for (int i = 1; i < k; ++i) {
        const double p2 = ((2.0 * i + 1.0 + a - x) * p1 - (i + a) * p0) / (i + 1.0);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

void st_coulomb(int N, double dr, double a0, int n, int l, double *u);

// discretely normalised Coulomb u_nl = r R_nl on r_j = j dr (j = 0..N-1; u_0 = 0)
void coulomb_u(int N, double dr, double a0, int n, int l, std::vector<double> &u)
{
    u.assign(N, 0.0);
    st_coulomb(N, dr, a0, n, l, u.data());
}

void st_gauss(int N, double dr, double w, int l, double *u);

// nullptr if the N values of an initial state are finite with a positive discrete norm, else why
// not (a Gaussian whose 2 w^2 underflows, for instance, evaluates to NaN)
const char *state_problem(int N, double dr, const double *u)
{
    double s = 0.0;
    for (int j = 0; j < N; ++j) {
        if (!std::isfinite(u[j])) return "is not finite";
        s += u[j] * u[j];
    }
    if (!(s * dr > 0.0) || !std::isfinite(s * dr)) return "has no finite positive norm";
    return nullptr;
}

void gauss_u(int N, double dr, double w, int l, std::vector<double> &u)
{
    u.assign(N, 0.0);
    st_gauss(N, dr, w, l, u.data());
}

} // namespace

struct qtraj_ctx {
    int N = 0;
    double L = 0, dt = 0, M = 0, dr = 0, a0 = 0;
    qtraj_params p{};
    int device = 0, sm_count = 0;
    // read-only tables
    void *W = nullptr, *WL = nullptr, *KT = nullptr, *sinpre = nullptr, *statV = nullptr, *statV2 = nullptr;
    double *eig = nullptr;
    double *ic = nullptr, *ov0 = nullptr;
    int *ov0_zero = nullptr, *spec_l = nullptr, *spec_color = nullptr;
    bool ic_cplx = false;   // ic holds complex states (after a vacuum evolution)
    double *prof = nullptr; // profile store of tabulated media: (tau, T) pairs
    std::vector<double> prof_host;
    double r1s = 1.0;       // <1S|r|1S> on the grid
    void *phi_tab = nullptr; // KSU: (phi, h phi') at the nodes of [KSU_PHI_A0, KSU_PHI_A1]
    std::vector<double> basis_host;   // [NBASIS][N] the overlap basis (analytic or numerical)
    qtraj_trace_rec *trace = nullptr;   // per-step summary (caller buffers), off when trace_every == 0
    int *trace_cnt = nullptr;
    int trace_every = 0, trace_n = 0, trace_cap = 0;
    int n_spec = 0;
    std::vector<qtraj_init_spec> specs;
    std::vector<int> spec_idx;
    MediumDev *media = nullptr;
    int media_cap = 0;
    // workspace
    char *ws = nullptr;
    size_t ws_bytes = 0;
    int n_traj = 0;
    size_t off_trajs = 0, off_obs = 0, off_gtrajs = 0, off_gobs = 0, off_gready = 0, off_ctr = 0, off_states = 0,
           off_plain = 0;
    // host staging and timing
    void *h_stage = nullptr;
    size_t h_stage_bytes = 0;
    cudaEvent_t ev_stage = nullptr, ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
    bool evolved = false;
    int last_batch = 0, last_groups = 0, last_n_media = 0, launches = 0;
    std::vector<int> group_pair;
    std::vector<int> host_steps;
};

namespace {

// ------------------------------------------------------------------------------------------------
// The isotropic KSU potential (App. E): constants as printed, and phi(rhat) tabulated for the kernels
// ------------------------------------------------------------------------------------------------
constexpr double KSU_A = 0.409, KSU_SIGMA = 0.21, KSU_RSB = 1.25 / HBARC;   // GeV^-1
constexpr double KSU_ALPHA0 = 0.2034, KSU_MU0 = 5.0;                        // alpha_s(5 GeV)
constexpr int KSU_NF = 3;
constexpr double KSU_TF_MIN = 0.1;   // GeV: the one-loop alpha_s(2 pi T) stays below ~0.5 above it
constexpr double EULER_G = 0.57721566490153286061;

// e^-x Ei(x) and e^x E1(x) for x >= 2 (power series of Ei -- positive terms -- up to 60 and its
// asymptotic series above; continued fraction of E1)
double ksu_eEi(double x)
{
    if (x <= 60.0) {
        double term = 1.0, sum = 0.0;
        for (int k = 1; k < 400; ++k) {
            term *= x / k;
            sum += term / k;
            if (term / k < 1e-18 * sum) break;
        }
        return std::exp(-x) * (EULER_G + std::log(x) + sum);
    }
    double t = 1.0 / x, sum = 0.0;
    for (int k = 0; k < 200 && t > 1e-18 * sum; ++k) {
        sum += t;
        t *= (k + 1.0) / x;
    }
    return sum;
}
double ksu_eE1(double x)
{
    // e^x E1(x) = 1/(x+1 - 1^2/(x+3 - 2^2/(x+5 - ...))), evaluated from the tail
    double f = x + 201.0;
    for (int i = 100; i >= 1; --i) f = x + 2.0 * i - 1.0 - (double)i * i / f;
    return 1.0 / f;
}

// phi(a) = 1 - [(1+a) e^-a Ei(a) + (1-a) e^a E1(a)] / (2a) and its derivative (a >= 2), for the
// table the kernels interpolate: d/da e^-a Ei(a) = 1/a - e^-a Ei(a), d/da e^a E1(a) = e^a E1(a) - 1/a
void ksu_phi_d(double a, double *phi, double *dphi)
{
    const double F = ksu_eEi(a), G = ksu_eE1(a);
    const double B = (1.0 + a) * F + (1.0 - a) * G;
    const double dB = 2.0 - a * (F + G);
    *phi = 1.0 - B / (2.0 * a);
    *dphi = -dB / (2.0 * a) + B / (2.0 * a * a);
}

struct Layout {
    size_t trajs, obs, gtrajs, gobs, gready, ctr, states, plain, total;
};

Layout layout(const qtraj_ctx *c, int n)
{
    Layout L{};
    size_t o = 0;
    L.trajs = o;
    o = align256(o + sizeof(TrajDev) * (size_t)n);
    L.obs = o;
    o = align256(o + sizeof(qtraj_obs) * (size_t)n);
    L.gtrajs = o;
    o = align256(o + sizeof(TrajDev) * (size_t)n);
    L.gobs = o;
    o = align256(o + sizeof(qtraj_obs) * (size_t)n);
    L.gready = o;
    o = align256(o + sizeof(int) * (size_t)n);
    L.ctr = o;
    o = align256(o + 256);
    L.states = o;
    if (c->p.save_states) o = align256(o + sizeof(double) * 2 * (size_t)c->N * n);
    L.plain = o;
    if (c->p.form == QTRAJ_PLAIN) {
        o = align256(o + 4 * sizeof(cpx<double>) * (size_t)c->N * n);   // psi, y, z, s
        o = align256(o + sizeof(double) * (size_t)n);                  // n2
        o = align256(o + sizeof(PlainState) * (size_t)n);
    }
    L.total = o;
    return L;
}

// the static part of the space kernel for every (colour, l < LTAB, j), rows [colour][l][j]:
// exp(-i V dt/2) (s1) and exp(-i V dt) (s2), V = coul_c / r + l(l+1) / (M r^2) at r = j dr, in FP64
// (entry j = 0 is zero: u(0) = 0).  Built on the device: 2 x 2 x LTAB x N phases.
template <typename T>
__global__ void stat_rows(typename Prec<T>::S *s1, typename Prec<T>::S *s2, int N, double dr, double M, double dt,
                          double coul0, double coul1)
{
    const size_t n = (size_t)2 * LTAB * N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % (size_t)N), row = (int)(i / (size_t)N);
        const int col = row / LTAB, l = row % LTAB;
        double c1 = 0.0, sn1 = 0.0, c2 = 0.0, sn2 = 0.0;
        if (j > 0) {
            const double r = j * dr;
            const double V = (col ? coul1 : coul0) / r + (double)l * (l + 1) / (M * r * r);
            const double ph = -V * dt * 0.5;
            sincos(ph, &sn1, &c1);
            sincos(2.0 * ph, &sn2, &c2);
        }
        s1[i] = Prec<T>::make_s(c1, sn1);
        s2[i] = Prec<T>::make_s(c2, sn2);
    }
}

template <typename T> qtraj_status build_tables(qtraj_ctx *c)
{
    using PC = typename Prec<T>::C;
    using PR = typename Prec<T>::Rl;
    const int N = c->N;
    std::vector<PC> W(N), KT(N);
    std::vector<PR> sp(N);
    for (int t = 0; t < N; ++t) {
        const double a = -2.0 * PI * (double)t / N;
        W[t] = Prec<T>::make(std::cos(a), std::sin(a));
        sp[t] = Prec<T>::make_r(std::sin(PI * (double)t / N));
    }
    for (int k = 0; k < N; ++k) {
        const double pk = PI * k / c->L;
        double Tk = pk * pk / c->M;
        if (c->p.deriv_type == 1) Tk = 2.0 * (1.0 - std::cos(pk * c->dr)) / (c->M * c->dr * c->dr);
        const double ph = -Tk * c->dt;
        KT[k] = Prec<T>::make(std::cos(ph) * 2.0 / N, std::sin(ph) * 2.0 / N);
    }
    const double Nc = c->p.Nc, CF = (Nc * Nc - 1.0) / (2.0 * Nc);
    double coul[2] = {-CF * c->p.alpha_s, c->p.alpha_s / (2.0 * Nc)};
    if (c->p.potential == 1) {
        // KSU: the static factor holds the Cornell -a/r (and the centrifugal term); the kernels apply
        // the rest of the potential, V_R + a/r and V_I, each step.  Phi is tabulated on
        // [KSU_PHI_A0, KSU_PHI_A1] as (phi, h phi') for cubic Hermite interpolation (error below
        // h^4/384 max|phi''''| ~ 3e-12), followed by the coefficients of its small-argument series
        // phi(a) = -sum_k [ln a (gamma_k) + c_k] a^(2k), from the expansion of the closed form in
        // Ei and E1: gamma_k = (m-1)/m!, c_k the a^m coefficient of (1+a)e^-a sum_{n>=1} a^n/(n n!),
        // m = 2k+1, plus gamma (m-1)/m! folded into c_k.
        coul[0] = coul[1] = -KSU_A;
        std::vector<T> tab(2 * (size_t)KSU_PHI_NODES + 2 * (size_t)KSU_PHI_SER);
        const double h = 1.0 / KSU_PHI_PER;
        for (int i = 0; i < KSU_PHI_NODES; ++i) {
            double ph, dph;
            const double a = KSU_PHI_A0 + i * h;
            if (a >= 2.0) {
                ksu_phi_d(a, &ph, &dph);
            } else {   // below 2 the series, and its derivative, in long double
                long double f[48], pc[48], fact = 1, sum = 0, dsum = 0;
                for (int n = 0; n < 48; ++n) {
                    if (n) fact *= n;
                    f[n] = ((n & 1) ? -1.0L : 1.0L) * (1.0L - n) / fact;
                    pc[n] = n ? 1.0L / (n * fact) : 0.0L;
                }
                const long double La = (long double)EULER_G + std::log((long double)a);
                long double mf = 1;
                for (int m = 1; m < 48; ++m) {
                    mf *= m;
                    if (m < 3 || !(m & 1)) continue;
                    long double cm = 0;
                    for (int n = 0; n <= m; ++n) cm += f[n] * pc[m - n];
                    const long double q = (long double)(m - 1) / mf;
                    const long double am = std::pow((long double)a, (long double)(m - 1));
                    sum += (La * q + cm) * am;
                    dsum += ((m - 1) * (La * q + cm) + q) * am / a;
                }
                ph = (double)-sum;
                dph = (double)-dsum;
            }
            tab[2 * (size_t)i] = (T)ph;
            tab[2 * (size_t)i + 1] = (T)(h * dph);
        }
        {
            double fact = 1.0, mf = 1.0;
            std::vector<double> f(40), pc(40);
            for (int n = 0; n < 40; ++n) {
                if (n) fact *= n;
                f[n] = ((n & 1) ? -1.0 : 1.0) * (1.0 - n) / fact;
                pc[n] = n ? 1.0 / (n * fact) : 0.0;
            }
            for (int m = 1, k = 0; m < 40 && k < KSU_PHI_SER; ++m) {
                mf *= m;
                if (m < 3 || !(m & 1)) continue;
                double cm = 0.0;
                for (int n = 0; n <= m; ++n) cm += f[n] * pc[m - n];
                const double q = (m - 1) / mf;
                tab[2 * (size_t)KSU_PHI_NODES + 2 * k] = (T)q;                    // times ln a
                tab[2 * (size_t)KSU_PHI_NODES + 2 * k + 1] = (T)(cm + EULER_G * q);
                ++k;
            }
        }
        CK(cudaMalloc(&c->phi_tab, sizeof(T) * tab.size()));
        CK(cudaMemcpy(c->phi_tab, tab.data(), sizeof(T) * tab.size(), cudaMemcpyHostToDevice));
    }
    // last-pass twiddles of the fused kernel, W^(m g) for m < R, g < G = N/(2R), one compact section
    // [R][G] (N/2 entries) per radix R = 16, 8, 4 at offsets 0, N/2, N: a kernel reads the section of
    // its own radix, and the threads of a warp read consecutive entries
    std::vector<PC> WL((size_t)3 * (N / 2));
    for (int sec = 0; sec < 3; ++sec) {
        const int R = 16 >> sec, G = N / (2 * R);
        for (int m = 0; m < R; ++m)
            for (int g = 0; g < G; ++g) WL[(size_t)sec * (N / 2) + (size_t)m * G + g] = W[(size_t)m * g];
    }
    CK(cudaMalloc(&c->WL, sizeof(PC) * WL.size()));
    CK(cudaMemcpy(c->WL, WL.data(), sizeof(PC) * WL.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&c->W, sizeof(PC) * N));
    CK(cudaMalloc(&c->KT, sizeof(PC) * N));
    CK(cudaMalloc(&c->sinpre, sizeof(PR) * N));
    using PS = typename Prec<T>::S;
    const size_t nstat = (size_t)2 * LTAB * N;
    if (cudaMalloc(&c->statV, sizeof(PS) * nstat) != cudaSuccess ||
        cudaMalloc(&c->statV2, sizeof(PS) * nstat) != cudaSuccess) {
        cudaGetLastError();
        return fail(QTRAJ_ENOMEM, "cudaMalloc of the static space-kernel tables (%zu bytes)", 2 * sizeof(PS) * nstat);
    }
    CK(cudaMemcpy(c->W, W.data(), sizeof(PC) * N, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->KT, KT.data(), sizeof(PC) * N, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->sinpre, sp.data(), sizeof(PR) * N, cudaMemcpyHostToDevice));
    // a private non-blocking stream: building a context waits for nothing else on the device
    cudaStream_t s = nullptr;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    const int blocks = (int)std::min<size_t>((nstat + 255) / 256, 4096);
    stat_rows<T><<<blocks, 256, 0, s>>>((PS *)c->statV, (PS *)c->statV2, N, c->dr, c->M, c->dt, coul[0], coul[1]);
    cudaError_t e = cudaGetLastError();
    const cudaError_t e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    cudaStreamDestroy(s);
    CK(e);
    return QTRAJ_OK;
}

template <typename T> Tables<T> tables(const qtraj_ctx *c)
{
    Tables<T> t;
    using PC = typename Prec<T>::C;
    t.W = (const PC *)c->W;
    t.WL = (const PC *)c->WL;
    t.KT = (const PC *)c->KT;
    t.sinpre = (const typename Prec<T>::Rl *)c->sinpre;
    t.statV = (const typename Prec<T>::S *)c->statV;
    t.statV2 = (const typename Prec<T>::S *)c->statV2;
    t.eig = c->eig;
    t.ic = c->ic;
    t.ov0 = c->ov0;
    t.ov0_zero = c->ov0_zero;
    t.spec_l = c->spec_l;
    t.spec_color = c->spec_color;
    t.media = c->media;
    t.dr = c->dr;
    t.dt = c->dt;
    t.M = c->M;
    const double Nc = c->p.Nc;
    t.p_os = 2.0 / (Nc * Nc - 2.0);
    t.coul[0] = -(Nc * Nc - 1.0) / (2.0 * Nc) * c->p.alpha_s;
    t.coul[1] = c->p.alpha_s / (2.0 * Nc);
    if (c->p.potential == 1) t.coul[0] = t.coul[1] = -KSU_A;   // the Cornell -a/r (static factor)
    t.max_jumps = c->p.max_jumps;
    t.l_cap = c->p.l_cap;
    t.use_rmin = c->p.use_rmin;
    t.r_max = c->p.r_max;
    t.ic_cplx = c->ic_cplx ? 1 : 0;
    t.prof = c->prof;
    t.r1s = c->r1s;
    t.potential = c->p.potential;
    t.phi_tab = (const T *)c->phi_tab;
    t.phi_ser = (const T *)c->phi_tab + 2 * (size_t)KSU_PHI_NODES;
    t.ksu_a_dr = (T)(KSU_A / c->dr);
    t.ksu_sig_dr = (T)(KSU_SIGMA * c->dr);
    t.ksu_two_sigma = (T)(2.0 * KSU_SIGMA);
    t.ksu_cap = (T)(-KSU_A / KSU_RSB + KSU_SIGMA * KSU_RSB);
    t.ksu_alpha0 = (T)KSU_ALPHA0;
    t.ksu_b0 = (T)((11.0 * c->p.Nc - 2.0 * KSU_NF) / (12.0 * PI));
    t.ksu_mu0sq = (T)(KSU_MU0 * KSU_MU0);
    {
        const double CF = (c->p.Nc * c->p.Nc - 1.0) / (2.0 * c->p.Nc);
        t.ksu_md2 = (T)(c->p.ksu_mD_factor * c->p.ksu_mD_factor * c->p.Nc * (1.0 + KSU_NF / 6.0) * PI * CF);
        t.ksu_cf = (T)CF;
    }
    t.ksu_dt = (T)c->dt;
    return t;
}

void free_ptr(void *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}
template <typename P> void free_typed(P *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

// steps until T falls below Tf: ceil((tau_f - tau_start) / (hbar c dt)) with tau_f where the Bjorken
// T0 (tau0/tau)^{1/3}, or the table's interpolated T, first crosses Tf (a table that stays >= Tf ends
// at its last tau, one that starts below Tf at once)
int medium_steps(double dt, const qtraj_medium &m, const double *prof)
{
    double tau_s = m.tau0, tau_f;
    if (m.kind == 1) {
        const double *p = prof + 2 * (size_t)m.table_offset;
        const int n = m.table_len;
        tau_s = p[0];
        tau_f = p[2 * (n - 1)];
        if (p[1] < m.Tf) {
            tau_f = tau_s;
        } else {
            for (int i = 0; i + 1 < n; ++i)
                if (p[2 * i + 3] < m.Tf) {
                    tau_f = p[2 * i] + (p[2 * i + 2] - p[2 * i]) * (p[2 * i + 1] - m.Tf) / (p[2 * i + 1] - p[2 * i + 3]);
                    break;
                }
        }
    } else {
        tau_f = m.tau0 * std::pow(m.T0 / m.Tf, 3.0);
    }
    double s = std::ceil((tau_f - tau_s) / (HBARC * dt));
    if (s < 0) s = 0;
    return (int)s;
}

// kappa_hat of a medium: >= 0 a constant; -1, -2, -3 the central, lower, upper lattice fit of
// kappa_hat(T) (App. E; the fits stay positive from T_c = 0.155 GeV up, so Tf >= T_c is required)
int kappa_fit_index(double k)
{
    return k == -1.0 ? 1 : k == -2.0 ? 2 : k == -3.0 ? 3 : 0;
}

// prof: the (tau, T) pairs of the context's profile store (n_prof points), or nullptr where
// tabulated media are not available
const char *medium_check(const qtraj_medium &q, const double *prof = nullptr, int n_prof = 0)
{
    if (q.kind == 1) {
        if (!prof) return "tabulated media (kind 1) need a context with a profile store (qtraj_set_profiles)";
        if (q.table_offset < 0 || q.table_len < 2 || q.table_offset > n_prof - q.table_len)
            return "table_offset/table_len outside the profile store (at least 2 points)";
        const double *p = prof + 2 * (size_t)q.table_offset;
        for (int i = 0; i + 1 < q.table_len; ++i)
            if (!(p[2 * i + 2] > p[2 * i])) return "the table's tau must be strictly ascending";
        if (!(p[0] > 0)) return "the table's tau must be positive";
        if (!(q.Tf > 0)) return "Tf must be positive";
    } else if (q.kind != 0) {
        return "kind must be 0 (Bjorken) or 1 (tabulated)";
    } else if (!(q.T0 > 0) || !(q.tau0 > 0) || !(q.Tf > 0)) {
        return "T0, tau0, Tf must be positive";
    }
    if (!std::isfinite(q.kappa_hat) || !std::isfinite(q.gamma_hat) || !std::isfinite(q.Tf) ||
        (q.kind == 0 && (!std::isfinite(q.T0) || !std::isfinite(q.tau0))))
        return "the medium's parameters must be finite";
    if (!(q.gamma_hat <= 0)) return "gamma_hat <= 0 required";
    if (kappa_fit_index(q.kappa_hat) != 0) {
        if (!(q.Tf >= 0.155)) return "a kappa_hat lattice fit needs Tf >= T_c = 0.155 GeV";
    } else if (!(q.kappa_hat >= 0)) {
        return "kappa_hat >= 0, or -1/-2/-3 for a lattice fit, required";
    }
    return nullptr;
}

// the device record of a medium on a context's grid
MediumDev encode_medium(const qtraj_ctx *c, const qtraj_medium &q)
{
    MediumDev d{};
    const double Nc = c->p.Nc;
    d.kind = q.kind;
    if (q.kind == 1) {
        d.tab_off = q.table_offset;
        d.tab_len = q.table_len;
        d.tau0 = c->prof_host[2 * (size_t)q.table_offset];
    } else {
        d.A = q.T0 * q.T0 * q.T0 * q.tau0;
        d.tau0 = q.tau0;
    }
    d.dtau = c->dt * HBARC;
    d.kfit = kappa_fit_index(q.kappa_hat);
    const double kap = d.kfit ? 1.0 : q.kappa_hat;
    for (int col = 0; col < 2; ++col) {
        const double f = col == 0 ? 0.5 : (Nc * Nc - 2.0) / (4.0 * (Nc * Nc - 1.0));
        d.er[col] = -f * kap * c->dt * 0.5;
        d.ei[col] = -f * q.gamma_hat * c->dt * 0.5;
        d.erj[col] = d.er[col] * c->dr * c->dr;
        d.eij[col] = d.ei[col] * c->dr * c->dr / PI;
    }
    return d;
}

} // namespace

namespace {
// The m lowest numerical eigenstates of the discretised singlet vacuum Hamiltonian of angular
// momentum l (n = l+1 .. l+m), started from the analytic Coulomb states of the same n.
qtraj_status numerical_states(const qtraj_ctx *c, int l, int m, std::vector<std::vector<double>> &out)
{
    const double Nc = c->p.Nc;
    EigenProblem ep{c->N, c->L, c->M, -(Nc * Nc - 1.0) / (2.0 * Nc) * c->p.alpha_s, c->p.deriv_type};
    if (c->p.potential == 1) {
        ep.potential = 1;
        ep.a = KSU_A;
        ep.sigma = KSU_SIGMA;
        ep.r_sb = KSU_RSB;
    }
    std::vector<std::vector<double>> start(m);
    for (int k = 0; k < m; ++k) coulomb_u(c->N, c->dr, c->a0, l + 1 + k, l, start[k]);
    std::vector<double> lam;
    const int it = vacuum_eigenstates(ep, l, m, start, out, lam);
    if (it < 0) return fail(QTRAJ_EINVAL, "numerical eigenstates of l = %d did not converge", l);
    return QTRAJ_OK;
}
} // namespace

namespace {
// Evolves every initial state of the context in vacuum for n_vac steps (T = 0: the Coulomb and
// centrifugal potential of its colour, no imaginary part, no jump test) with the fused kernel of the
// context's precision, then makes the results the context's (complex) initial states and their
// overlaps with the Coulomb basis the reference of the survival ratios (Sec. 3.5 item 3).
qtraj_status vacuum_evolution(qtraj_ctx *c, int n_specs, int n_vac)
{
    const int N = c->N;
    TrajDev *d_tr = nullptr;
    qtraj_obs *d_obs = nullptr;
    int *d_ctr = nullptr;
    double *d_st = nullptr;
    qtraj_status st = qt::reserve_media(c, 1);
    if (st != QTRAJ_OK) return st;
    auto cleanup = [&]() {
        free_typed(d_tr);
        free_typed(d_obs);
        free_typed(d_ctr);
        free_typed(d_st);
    };
    std::vector<TrajDev> tr(n_specs);
    for (int s = 0; s < n_specs; ++s) tr[s] = TrajDev{0ull, s, 0, n_vac, 0};
    MediumDev vac{};
    vac.tau0 = 1.0;   // A = 0: T^3 = 0 at every step; all exponent coefficients 0
    std::vector<double> states((size_t)n_specs * N * 2);
    int status = 0;
    cudaError_t e = cudaMalloc(&d_tr, sizeof(TrajDev) * n_specs);
    if (e == cudaSuccess) e = cudaMalloc(&d_obs, sizeof(qtraj_obs) * n_specs);
    if (e == cudaSuccess) e = cudaMalloc(&d_ctr, 256);
    if (e == cudaSuccess) e = cudaMalloc(&d_st, sizeof(double) * states.size());
    if (e == cudaSuccess) e = cudaMemcpy(d_tr, tr.data(), sizeof(TrajDev) * n_specs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->media, &vac, sizeof(MediumDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_ctr, 0, 256);
    if (e == cudaSuccess) {
        LaunchArgs va{d_tr, n_specs, d_obs, nullptr, d_ctr, d_ctr + 1, d_st, 1};
        FusedInfo fi;
        e = c->p.precision == QTRAJ_FP32
                ? fused_launch_f32(N, tables<float>(c), va, c->sm_count, 0, nullptr, &fi, false, c->p.variant)
                : fused_launch_f64(N, tables<double>(c), va, c->sm_count, 0, nullptr, &fi, false, c->p.variant);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(states.data(), d_st, sizeof(double) * states.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&status, d_ctr + 1, sizeof(int), cudaMemcpyDeviceToHost);
    cleanup();
    if (e != cudaSuccess) return fail(QTRAJ_ECUDA, "vacuum evolution: %s", cudaGetErrorString(e));
    if (status & 1) return fail(QTRAJ_ENONFINITE, "vacuum evolution: a norm became non-finite");
    // the overlaps of the evolved states with the Coulomb basis
    std::vector<double> ov0((size_t)n_specs * NBASIS * 2, 0.0), phi;
    std::vector<int> zero((size_t)n_specs * NBASIS);
    CK(cudaMemcpy(zero.data(), c->ov0_zero, sizeof(int) * zero.size(), cudaMemcpyDeviceToHost));
    for (int b = 0; b < NBASIS; ++b) {
        phi.assign(c->basis_host.begin() + (size_t)b * N, c->basis_host.begin() + (size_t)(b + 1) * N);
        for (int s = 0; s < n_specs; ++s) {
            if (zero[(size_t)s * NBASIS + b]) continue;
            const double *u = states.data() + (size_t)s * N * 2;
            double re = 0.0, im = 0.0;
            for (int j = 1; j < N; ++j) {
                re += phi[j] * u[2 * j];
                im += phi[j] * u[2 * j + 1];
            }
            ov0[((size_t)s * NBASIS + b) * 2] = re * c->dr;
            ov0[((size_t)s * NBASIS + b) * 2 + 1] = im * c->dr;
        }
    }
    free_typed(c->ic);
    CK(cudaMalloc(&c->ic, sizeof(double) * states.size()));
    CK(cudaMemcpy(c->ic, states.data(), sizeof(double) * states.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->ov0, ov0.data(), sizeof(double) * ov0.size(), cudaMemcpyHostToDevice));
    c->ic_cplx = true;
    return QTRAJ_OK;
}
} // namespace

extern "C" {

const char *qtraj_last_error(const qtraj_ctx *) { return g_err.c_str(); }

qtraj_status qtraj_create(int N, double L, double dt, double M, const qtraj_params *params, qtraj_ctx **out)
{
    g_err.clear();
    if (!out || !params) return fail(QTRAJ_EINVAL, "null argument");
    *out = nullptr;
    const qtraj_params &p = *params;
    if (!is_pow2(N) || N < 16 || N > 16384) return fail(QTRAJ_EINVAL, "N=%d must be a power of two in [16, 16384]", N);
    if (!(L > 0) || !(dt > 0) || !(M > 0)) return fail(QTRAJ_EINVAL, "L, dt and M must be positive");
    if (!(p.alpha_s >= 0) || !(p.Nc >= 2)) return fail(QTRAJ_EINVAL, "alpha_s >= 0 and Nc >= 2 required");
    if (p.deriv_type != 0 && p.deriv_type != 1) return fail(QTRAJ_EINVAL, "deriv_type must be 0 or 1");
    if (!(p.r_max > 0 && p.r_max <= 1)) return fail(QTRAJ_EINVAL, "r_max must be in (0, 1]");
    if (p.precision != QTRAJ_FP64 && p.precision != QTRAJ_FP32) return fail(QTRAJ_EINVAL, "unknown precision");
    if (p.form != QTRAJ_FUSED && p.form != QTRAJ_PLAIN) return fail(QTRAJ_EINVAL, "unknown form");
    if (p.form == QTRAJ_PLAIN && p.precision != QTRAJ_FP64) return fail(QTRAJ_EINVAL, "the plain form is FP64 only");
    if (p.variant < 0 || p.variant > 3) return fail(QTRAJ_EINVAL, "variant must be in 0..3");
    if (p.form == QTRAJ_FUSED && p.precision == QTRAJ_FP64 && N > 8192)
        return fail(QTRAJ_EINVAL, "the fused FP64 form supports N <= 8192");
    if (!(p.t_vacuum >= 0) || !std::isfinite(p.t_vacuum)) return fail(QTRAJ_EINVAL, "t_vacuum must be finite and >= 0");
    if (p.t_vacuum > 0 && p.precision == QTRAJ_FP64 && N > 8192)
        return fail(QTRAJ_EINVAL, "the vacuum evolution runs in the fused form: FP64 needs N <= 8192");
    if (p.basis != 0 && p.basis != 1) return fail(QTRAJ_EINVAL, "basis must be 0 (analytic) or 1 (numerical)");
    if (p.potential != 0 && p.potential != 1) return fail(QTRAJ_EINVAL, "potential must be 0 (OQS+pNRQCD) or 1 (KSU)");
    if (p.potential == 1) {
        if (!(p.ksu_mD_factor > 0) || !std::isfinite(p.ksu_mD_factor)) return fail(QTRAJ_EINVAL, "ksu_mD_factor must be > 0");
        if (p.form != QTRAJ_FUSED) return fail(QTRAJ_EINVAL, "the KSU potential runs in the fused form only");
        if (p.t_vacuum > 0) return fail(QTRAJ_EINVAL, "the KSU potential has no vacuum evolution (t_vacuum = 0)");
    } else if (p.basis == 1 && !(p.alpha_s > 0)) {
        return fail(QTRAJ_EINVAL, "the numerical basis needs alpha_s > 0");
    }

    qtraj_ctx *c = new qtraj_ctx();
    c->N = N;
    c->L = L;
    c->dt = dt;
    c->M = M;
    c->dr = L / N;
    c->p = p;
    c->a0 = 2.0 / (M * (p.Nc * p.Nc - 1.0) / (2.0 * p.Nc) * p.alpha_s);
    if (p.potential == 1) {
        c->p.basis = 1;                   // the Cornell vacuum eigenstates
        c->a0 = 2.0 / (M * KSU_A);       // Coulomb-like start vectors of the eigensolver
    }
    qtraj_status st = QTRAJ_OK;
    auto bail = [&](qtraj_status s) {
        qtraj_destroy(c);
        return s;
    };
    // the overlap basis: analytic Coulomb states, or the numerical eigenstates of the grid's H
    c->basis_host.assign((size_t)NBASIS * N, 0.0);
    if (c->p.basis == 1) {
        const int lm[3][2] = {{0, 3}, {1, 2}, {2, 1}};
        for (const auto &q : lm) {
            std::vector<std::vector<double>> v;
            if ((st = numerical_states(c, q[0], q[1], v)) != QTRAJ_OK) return bail(st);
            for (int k = 0; k < q[1]; ++k)
                for (int b = 0; b < NBASIS; ++b)
                    if (BASIS_L[b] == q[0] && BASIS_N[b] == q[0] + 1 + k)
                        std::memcpy(c->basis_host.data() + (size_t)b * N, v[k].data(), sizeof(double) * N);
        }
    } else {
        std::vector<double> u;
        for (int b = 0; b < NBASIS; ++b) {
            coulomb_u(N, c->dr, c->a0, BASIS_N[b], BASIS_L[b], u);
            std::memcpy(c->basis_host.data() + (size_t)b * N, u.data(), sizeof(double) * N);
        }
    }
    {
        double r1 = 0.0;
        for (int j = 1; j < N; ++j) r1 += j * c->dr * c->basis_host[j] * c->basis_host[j];
        c->r1s = std::isfinite(r1) && r1 > 0 ? r1 * c->dr : 1.0;
    }
    if (cudaGetDevice(&c->device) != cudaSuccess) return bail(fail(QTRAJ_ECUDA, "no CUDA device"));
    if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        return bail(fail(QTRAJ_ECUDA, "cannot query the SM count"));
    st = p.precision == QTRAJ_FP32 ? build_tables<float>(c) : build_tables<double>(c);
    if (st != QTRAJ_OK) return bail(st);
    const std::vector<double> &eig = c->basis_host;
    if (cudaMalloc(&c->eig, sizeof(double) * eig.size()) != cudaSuccess) return bail(fail(QTRAJ_ENOMEM, "cudaMalloc"));
    if (cudaMemcpy(c->eig, eig.data(), sizeof(double) * eig.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(QTRAJ_ECUDA, "upload of the Coulomb basis failed"));
    if (cudaEventCreateWithFlags(&c->ev_stage, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
        cudaEventCreate(&c->ev2) != cudaSuccess)
        return bail(fail(QTRAJ_ECUDA, "cudaEventCreate failed"));
    *out = c;
    return QTRAJ_OK;
}

void qtraj_destroy(qtraj_ctx *c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    free_ptr(c->W);
    free_ptr(c->WL);
    free_ptr(c->KT);
    free_ptr(c->sinpre);
    free_ptr(c->statV);
    free_ptr(c->statV2);
    free_ptr(c->phi_tab);
    free_typed(c->eig);
    free_typed(c->ic);
    free_typed(c->ov0);
    free_typed(c->ov0_zero);
    free_typed(c->spec_l);
    free_typed(c->spec_color);
    free_typed(c->prof);
    free_typed(c->media);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->ev_stage) cudaEventDestroy(c->ev_stage);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->ev2) cudaEventDestroy(c->ev2);
    delete c;
}

size_t qtraj_workspace_bytes(const qtraj_ctx *c, int n_traj)
{
    if (!c || n_traj < 0) return 0;
    return layout(c, n_traj).total;
}

qtraj_status qtraj_init(qtraj_ctx *c, void *d_ws, size_t bytes, int n_traj, const qtraj_init_spec *specs,
                        int n_specs, const int *spec_idx)
{
    g_err.clear();
    if (!c || !d_ws || !specs) return fail(QTRAJ_EINVAL, "null argument");
    if (n_traj <= 0 || n_specs <= 0) return fail(QTRAJ_EINVAL, "n_traj and n_specs must be positive");
    if (((uintptr_t)d_ws & 255) != 0) return fail(QTRAJ_EINVAL, "workspace must be 256-byte aligned");
    const Layout Lw = layout(c, n_traj);
    if (bytes < Lw.total) return fail(QTRAJ_ENOMEM, "workspace of %zu bytes < %zu required", bytes, Lw.total);
    if (!spec_idx && n_specs != 1 && n_specs != n_traj)
        return fail(QTRAJ_EINVAL, "spec_idx is required unless n_specs is 1 or n_traj");
    const int N = c->N;
    for (int s = 0; s < n_specs; ++s) {
        const qtraj_init_spec &q = specs[s];
        if (q.kind < 0 || q.kind > 2) return fail(QTRAJ_EINVAL, "spec %d: kind must be 0, 1 or 2", s);
        if (q.kind == 2 && !(c->p.alpha_s > 0)) return fail(QTRAJ_EINVAL, "spec %d: numerical eigenstates need alpha_s > 0", s);
        if (q.l < 0 || (q.color != 0 && q.color != 1)) return fail(QTRAJ_EINVAL, "spec %d: l >= 0, color 0/1", s);
        if (q.kind == 0 && !(q.width > 0)) return fail(QTRAJ_EINVAL, "spec %d: width must be positive", s);
        if (q.kind >= 1 && (q.n < 1 || q.l >= q.n)) return fail(QTRAJ_EINVAL, "spec %d: need 0 <= l < n", s);
        if (c->p.potential == 1 && q.color != 0) return fail(QTRAJ_EINVAL, "spec %d: the KSU potential is singlet only", s);
    }
    std::vector<int> idx(n_traj);
    for (int t = 0; t < n_traj; ++t) {
        idx[t] = spec_idx ? spec_idx[t] : (n_specs == 1 ? 0 : t);
        if (idx[t] < 0 || idx[t] >= n_specs) return fail(QTRAJ_EINVAL, "spec_idx[%d] out of range", t);
    }
    std::vector<double> ic((size_t)n_specs * N), ov0((size_t)n_specs * NBASIS * 2), u, phi;
    std::vector<int> zero((size_t)n_specs * NBASIS), sl(n_specs), sc(n_specs);
    for (int s = 0; s < n_specs; ++s) {
        const qtraj_init_spec &q = specs[s];
        if (q.kind == 1) {
            coulomb_u(N, c->dr, c->a0, q.n, q.l, u);
        } else if (q.kind == 2) {
            std::vector<std::vector<double>> v;
            const qtraj_status st = numerical_states(c, q.l, q.n - q.l, v);
            if (st != QTRAJ_OK) return st;
            u = v.back();
        } else {
            gauss_u(N, c->dr, q.width, q.l, u);
        }
        if (const char *why = state_problem(N, c->dr, u.data()))
            return fail(QTRAJ_EINVAL, "spec %d: the initial state %s", s, why);
        std::memcpy(ic.data() + (size_t)s * N, u.data(), sizeof(double) * N);
        sl[s] = q.l;
        sc[s] = q.color;
        // an eigenstate of the basis' own kind (analytic Coulomb with the analytic basis, numerical
        // with the numerical one) is orthogonal to the basis states of other n
        const bool same_family = (q.kind == 1 && c->p.basis == 0) || (q.kind == 2 && c->p.basis == 1);
        for (int b = 0; b < NBASIS; ++b) {
            const int z = q.color != 0 || q.l != BASIS_L[b] || (same_family && q.n != BASIS_N[b]);
            zero[(size_t)s * NBASIS + b] = z;
            double o = 0.0;
            if (!z) {
                const double *ph = c->basis_host.data() + (size_t)b * N;
                for (int j = 1; j < N; ++j) o += ph[j] * u[j];
                o *= c->dr;
            }
            ov0[((size_t)s * NBASIS + b) * 2] = o;
            ov0[((size_t)s * NBASIS + b) * 2 + 1] = 0.0;
        }
    }
    CK(cudaDeviceSynchronize());
    free_typed(c->ic);
    free_typed(c->ov0);
    free_typed(c->ov0_zero);
    free_typed(c->spec_l);
    free_typed(c->spec_color);
    CK(cudaMalloc(&c->ic, sizeof(double) * ic.size()));
    CK(cudaMalloc(&c->ov0, sizeof(double) * ov0.size()));
    CK(cudaMalloc(&c->ov0_zero, sizeof(int) * zero.size()));
    CK(cudaMalloc(&c->spec_l, sizeof(int) * n_specs));
    CK(cudaMalloc(&c->spec_color, sizeof(int) * n_specs));
    CK(cudaMemcpy(c->ic, ic.data(), sizeof(double) * ic.size(), cudaMemcpyHostToDevice));
    c->ic_cplx = false;
    CK(cudaMemcpy(c->ov0, ov0.data(), sizeof(double) * ov0.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->ov0_zero, zero.data(), sizeof(int) * zero.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->spec_l, sl.data(), sizeof(int) * n_specs, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->spec_color, sc.data(), sizeof(int) * n_specs, cudaMemcpyHostToDevice));
    c->specs.assign(specs, specs + n_specs);
    c->spec_idx = idx;
    c->n_spec = n_specs;
    c->ws = (char *)d_ws;
    c->ws_bytes = bytes;
    c->n_traj = n_traj;
    c->off_trajs = Lw.trajs;
    c->off_obs = Lw.obs;
    c->off_gtrajs = Lw.gtrajs;
    c->off_gobs = Lw.gobs;
    c->off_gready = Lw.gready;
    c->off_ctr = Lw.ctr;
    c->off_states = Lw.states;
    c->off_plain = Lw.plain;
    c->evolved = false;
    const int n_vac = c->p.t_vacuum > 0 ? (int)std::llround(c->p.t_vacuum / c->dt) : 0;
    if (n_vac > 0) return vacuum_evolution(c, n_specs, n_vac);
    return QTRAJ_OK;
}

qtraj_status qtraj_set_profiles(qtraj_ctx *c, const double *tau, const double *T, int n_points)
{
    g_err.clear();
    if (!c || !tau || !T) return fail(QTRAJ_EINVAL, "null argument");
    if (n_points < 2) return fail(QTRAJ_EINVAL, "n_points must be at least 2");
    std::vector<double> h(2 * (size_t)n_points);
    for (int i = 0; i < n_points; ++i) {
        if (!std::isfinite(tau[i]) || !std::isfinite(T[i]) || tau[i] < 0 || T[i] < 0)
            return fail(QTRAJ_EINVAL, "point %d: tau and T must be finite and >= 0", i);
        h[2 * (size_t)i] = tau[i];
        h[2 * (size_t)i + 1] = T[i];
    }
    CK(cudaDeviceSynchronize());
    free_typed(c->prof);
    CK(cudaMalloc(&c->prof, sizeof(double) * h.size()));
    CK(cudaMemcpy(c->prof, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice));
    c->prof_host = std::move(h);
    return QTRAJ_OK;
}

qtraj_status qtraj_set_trace(qtraj_ctx *c, int every, int n_traced, int max_records, qtraj_trace_rec *d_records,
                             int *d_counts)
{
    g_err.clear();
    if (!c) return fail(QTRAJ_EINVAL, "null argument");
    if (every < 0) return fail(QTRAJ_EINVAL, "every must be >= 0");
    if (every > 0) {
        if (c->p.form != QTRAJ_FUSED) return fail(QTRAJ_EINVAL, "the per-step summary needs the fused form");
        if (c->p.potential != 0) return fail(QTRAJ_EINVAL, "the per-step summary is for the OQS+pNRQCD potential");
        if (n_traced <= 0 || max_records <= 0 || !d_records || !d_counts)
            return fail(QTRAJ_EINVAL, "n_traced, max_records and the buffers are required");
    }
    c->trace_every = every;
    c->trace_n = every > 0 ? n_traced : 0;
    c->trace_cap = every > 0 ? max_records : 0;
    c->trace = every > 0 ? d_records : nullptr;
    c->trace_cnt = every > 0 ? d_counts : nullptr;
    return QTRAJ_OK;
}

qtraj_status qtraj_basis_get(const qtraj_ctx *c, double *out)
{
    g_err.clear();
    if (!c || !out) return fail(QTRAJ_EINVAL, "null argument");
    std::memcpy(out, c->basis_host.data(), sizeof(double) * c->basis_host.size());
    return QTRAJ_OK;
}

qtraj_status qtraj_set_spec_idx(qtraj_ctx *c, const int *spec_idx, int n)
{
    g_err.clear();
    if (!c || !spec_idx) return fail(QTRAJ_EINVAL, "null argument");
    if (!c->ws) return fail(QTRAJ_EINVAL, "qtraj_init has not bound a workspace");
    if (n <= 0 || n > c->n_traj) return fail(QTRAJ_EINVAL, "n %d outside [1, %d]", n, c->n_traj);
    for (int t = 0; t < n; ++t)
        if (spec_idx[t] < 0 || spec_idx[t] >= c->n_spec) return fail(QTRAJ_EINVAL, "spec_idx[%d] out of range", t);
    for (int t = 0; t < n; ++t) c->spec_idx[t] = spec_idx[t];
    return QTRAJ_OK;
}

qtraj_status qtraj_evolve(qtraj_ctx *c, int batch, const qtraj_medium *media, int n_media, const int *medium_idx,
                          const uint64_t *seeds, void *stream)
{
    g_err.clear();
    if (!c || !media || !seeds) return fail(QTRAJ_EINVAL, "null argument");
    if (!c->ws) return fail(QTRAJ_EINVAL, "qtraj_init has not bound a workspace");
    if (batch < 0 || batch > c->n_traj) return fail(QTRAJ_EINVAL, "batch %d outside [0, %d]", batch, c->n_traj);
    if (n_media <= 0) return fail(QTRAJ_EINVAL, "n_media must be positive");
    if (!medium_idx && n_media != 1 && n_media != batch)
        return fail(QTRAJ_EINVAL, "medium_idx is required unless n_media is 1 or batch");
    cudaStream_t s = (cudaStream_t)stream;
    const int N = c->N;

    std::vector<MediumDev> md(n_media);
    std::vector<int> steps(n_media);
    for (int m = 0; m < n_media; ++m) {
        const qtraj_medium &q = media[m];
        if (const char *why = medium_check(q, c->prof_host.empty() ? nullptr : c->prof_host.data(),
                                           (int)(c->prof_host.size() / 2)))
            return fail(QTRAJ_EINVAL, "medium %d: %s", m, why);
        if (c->p.potential == 1 && !(q.Tf >= KSU_TF_MIN))
            return fail(QTRAJ_EINVAL, "medium %d: the KSU potential needs Tf >= %g GeV", m, KSU_TF_MIN);
        steps[m] = medium_steps(c->dt, q, c->prof_host.data());
        md[m] = encode_medium(c, q);
    }
    std::vector<TrajDev> tr(batch);
    std::map<std::pair<int, int>, int> gmap;
    std::vector<TrajDev> gt;
    std::vector<int> gpair;
    int max_steps = 0;
    for (int t = 0; t < batch; ++t) {
        const int mi = medium_idx ? medium_idx[t] : (n_media == 1 ? 0 : t);
        if (mi < 0 || mi >= n_media) return fail(QTRAJ_EINVAL, "medium_idx[%d] out of range", t);
        const int sp = c->spec_idx[t];
        auto key = std::make_pair(sp, mi);
        auto it = gmap.find(key);
        int g;
        if (it == gmap.end()) {
            g = (int)gt.size();
            gmap[key] = g;
            gt.push_back(TrajDev{0ull, sp, mi, steps[mi], g});
            gpair.push_back(sp * n_media + mi);
        } else {
            g = it->second;
        }
        tr[t] = TrajDev{(unsigned long long)seeds[t], sp, mi, steps[mi], g};
        if (steps[mi] > max_steps) max_steps = steps[mi];
    }
    // the rMin shortcut belongs to the jump algorithm; the KSU evolution has no jumps
    const int n_groups = c->p.use_rmin && c->p.potential == 0 ? (int)gt.size() : 0;

    // staging: media | trajs | group trajs
    const size_t b_md = sizeof(MediumDev) * n_media, b_tr = sizeof(TrajDev) * batch, b_gt = sizeof(TrajDev) * gt.size();
    const size_t need = align256(b_md) + align256(b_tr) + align256(b_gt) + 256;
    CK(cudaEventSynchronize(c->ev_stage));   // the previous upload has left the staging buffer
    if (need > c->h_stage_bytes) {
        if (c->h_stage) cudaFreeHost(c->h_stage);
        c->h_stage = nullptr;
        c->h_stage_bytes = 0;
        CK(cudaMallocHost(&c->h_stage, need));
        c->h_stage_bytes = need;
    }
    if (n_media > c->media_cap) {
        CK(cudaStreamSynchronize(s));
        free_typed(c->media);
        CK(cudaMalloc(&c->media, sizeof(MediumDev) * n_media));
        c->media_cap = n_media;
    }
    char *h = (char *)c->h_stage;
    std::memcpy(h, md.data(), b_md);
    std::memcpy(h + align256(b_md), tr.data(), b_tr);
    std::memcpy(h + align256(b_md) + align256(b_tr), gt.data(), b_gt);
    TrajDev *d_tr = (TrajDev *)(c->ws + c->off_trajs);
    TrajDev *d_gt = (TrajDev *)(c->ws + c->off_gtrajs);
    qtraj_obs *d_obs = (qtraj_obs *)(c->ws + c->off_obs);
    qtraj_obs *d_gobs = (qtraj_obs *)(c->ws + c->off_gobs);
    int *d_ctr = (int *)(c->ws + c->off_ctr);
    int *d_status = d_ctr + 1;
    double *d_states = c->p.save_states ? (double *)(c->ws + c->off_states) : nullptr;
    CK(cudaMemcpyAsync(c->media, h, b_md, cudaMemcpyHostToDevice, s));
    if (b_tr) CK(cudaMemcpyAsync(d_tr, h + align256(b_md), b_tr, cudaMemcpyHostToDevice, s));
    if (b_gt) CK(cudaMemcpyAsync(d_gt, h + align256(b_md) + align256(b_tr), b_gt, cudaMemcpyHostToDevice, s));
    CK(cudaEventRecord(c->ev_stage, s));
    CK(cudaMemsetAsync(d_ctr, 0, 256, s));

    c->launches = 0;
    c->last_batch = batch;
    c->last_groups = n_groups;
    c->last_n_media = n_media;
    c->group_pair = gpair;
    c->host_steps = steps;

    LaunchArgs ga{d_gt, n_groups, d_gobs, nullptr, d_ctr, d_status, nullptr, 1};
    LaunchArgs ma{d_tr, batch, d_obs, d_gobs, d_ctr, d_status, d_states, 0};
    if (c->trace_every > 0 && c->p.form == QTRAJ_FUSED) {
        ma.trace = c->trace;
        ma.trace_cnt = c->trace_cnt;
        ma.trace_every = c->trace_every;
        ma.trace_n = c->trace_n;
        ma.trace_cap = c->trace_cap;
        CK(cudaMemsetAsync(c->trace_cnt, 0, sizeof(int) * (size_t)c->trace_n, s));
    }
    CK(cudaEventRecord(c->ev0, s));
    if (c->p.form == QTRAJ_PLAIN) {
        const size_t nN = (size_t)c->n_traj * N;
        cpx<double> *base = (cpx<double> *)(c->ws + c->off_plain);
        PlainBuffers pb;
        pb.psi = base;
        pb.y = base + nN;
        pb.z = base + 2 * nN;
        pb.s = base + 3 * nN;
        pb.n2 = (double *)(c->ws + align256(c->off_plain + 4 * sizeof(cpx<double>) * nN));
        pb.st = (PlainState *)((char *)pb.n2 + align256(sizeof(double) * c->n_traj));
        const Tables<double> tb = tables<double>(c);
        if (n_groups > 0) {
            int gmax = 0;
            for (auto &g : gt) gmax = g.n_steps > gmax ? g.n_steps : gmax;
            CK(plain_run(tb, ga, N, gmax, pb, s, &c->launches));
        }
        CK(cudaEventRecord(c->ev1, s));
        CK(plain_run(tb, ma, N, max_steps, pb, s, &c->launches));
    } else {
        // one launch: the groups' no-jump runs are its first work items, and a trajectory takes the
        // shortcut once its group's record is published (ms_nojump is then 0)
        FusedInfo fi;
        LaunchArgs fa = ma;
        fa.group = nullptr;
        fa.gtrajs = d_gt;
        fa.n_groups = n_groups;
        fa.gobs = d_gobs;
        fa.gready = n_groups > 0 ? (int *)(c->ws + c->off_gready) : nullptr;
        if (n_groups > 0) CK(cudaMemsetAsync(fa.gready, 0, sizeof(int) * (size_t)n_groups, s));
        CK(cudaEventRecord(c->ev1, s));
        if (c->p.precision == QTRAJ_FP32) CK(fused_launch_f32(N, tables<float>(c), fa, c->sm_count, 0, s, &fi, false, c->p.variant));
        else CK(fused_launch_f64(N, tables<double>(c), fa, c->sm_count, 0, s, &fi, false, c->p.variant));
        ++c->launches;
    }
    CK(cudaEventRecord(c->ev2, s));
    c->evolved = true;
    return QTRAJ_OK;
}

qtraj_status qtraj_observables(qtraj_ctx *c, void *out, int out_is_device, void *stream)
{
    g_err.clear();
    if (!c || !out) return fail(QTRAJ_EINVAL, "null argument");
    if (!c->evolved) return fail(QTRAJ_EINVAL, "no evolve has been enqueued");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(qtraj_obs) * c->last_batch;
    if (bytes) CK(cudaMemcpyAsync(out, c->ws + c->off_obs, bytes, out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!out_is_device) {
        int status = 0;
        CK(cudaMemcpyAsync(&status, (int *)(c->ws + c->off_ctr) + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (status & 1) return fail(QTRAJ_ENONFINITE, "a trajectory norm became non-finite");
    }
    return QTRAJ_OK;
}

} // extern "C"

namespace qt {
qtraj_status api_fail(qtraj_status st, const char *msg)
{
    g_err = msg;
    return st;
}

void api_clear_error() { g_err.clear(); }

qtraj_status obs_to_host_async(qtraj_ctx *c, void *host, cudaStream_t s)
{
    if (!c || !host) return fail(QTRAJ_EINVAL, "null argument");
    if (!c->evolved) return fail(QTRAJ_EINVAL, "no evolve has been enqueued");
    const size_t bytes = sizeof(qtraj_obs) * c->last_batch;
    if (bytes) CK(cudaMemcpyAsync(host, c->ws + c->off_obs, bytes, cudaMemcpyDeviceToHost, s));
    return QTRAJ_OK;
}

qtraj_status reserve_media(qtraj_ctx *c, int n)
{
    if (!c || n <= 0) return fail(QTRAJ_EINVAL, "bad argument");
    if (n > c->media_cap) {
        CK(cudaDeviceSynchronize());
        free_typed(c->media);
        CK(cudaMalloc(&c->media, sizeof(MediumDev) * n));
        c->media_cap = n;
    }
    // the pinned staging of an evolve of n trajectories with up to n media and n groups
    const size_t need = align256(sizeof(MediumDev) * n) + 2 * align256(sizeof(TrajDev) * n) + 256;
    if (need > c->h_stage_bytes) {
        CK(cudaDeviceSynchronize());
        if (c->h_stage) CK(cudaFreeHost(c->h_stage));
        c->h_stage = nullptr;
        c->h_stage_bytes = 0;
        CK(cudaMallocHost(&c->h_stage, need));
        c->h_stage_bytes = need;
    }
    return QTRAJ_OK;
}

const char *medium_problem(const qtraj_medium &q) { return medium_check(q); }
} // namespace qt

extern "C" {

qtraj_status qtraj_states(qtraj_ctx *c, void *out, int out_is_device, void *stream)
{
    g_err.clear();
    if (!c || !out) return fail(QTRAJ_EINVAL, "null argument");
    if (!c->p.save_states) return fail(QTRAJ_EINVAL, "the context was created without save_states");
    if (!c->evolved) return fail(QTRAJ_EINVAL, "no evolve has been enqueued");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * 2 * (size_t)c->N * c->last_batch;
    if (bytes) CK(cudaMemcpyAsync(out, c->ws + c->off_states, bytes, out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!out_is_device) CK(cudaStreamSynchronize(s));
    return QTRAJ_OK;
}

qtraj_status qtraj_nojump_results(qtraj_ctx *c, qtraj_obs *out, int capacity, int *n_written)
{
    g_err.clear();
    if (!c || !out || !n_written) return fail(QTRAJ_EINVAL, "null argument");
    if (!c->evolved) return fail(QTRAJ_EINVAL, "no evolve has been enqueued");
    const int n_pairs = c->n_spec * c->last_n_media;
    if (capacity < n_pairs) return fail(QTRAJ_EINVAL, "capacity %d < %d pairs", capacity, n_pairs);
    CK(cudaEventSynchronize(c->ev2));
    std::vector<qtraj_obs> g(c->last_groups);
    if (c->last_groups) CK(cudaMemcpy(g.data(), c->ws + c->off_gobs, sizeof(qtraj_obs) * c->last_groups, cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(qtraj_obs) * n_pairs);
    for (int i = 0; i < c->last_groups; ++i) out[c->group_pair[i]] = g[i];
    *n_written = n_pairs;
    return QTRAJ_OK;
}

qtraj_status qtraj_last_run_stats(qtraj_ctx *c, qtraj_run_stats *out)
{
    g_err.clear();
    if (!c || !out) return fail(QTRAJ_EINVAL, "null argument");
    if (!c->evolved) return fail(QTRAJ_EINVAL, "no evolve has been enqueued");
    CK(cudaEventSynchronize(c->ev2));
    std::vector<qtraj_obs> o(c->last_batch);
    if (c->last_batch) CK(cudaMemcpy(o.data(), c->ws + c->off_obs, sizeof(qtraj_obs) * c->last_batch, cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(*out));
    for (const qtraj_obs &r : o) {
        out->steps_executed += r.n_steps_exec;
        if (r.flags & QTRAJ_F_NOJUMP_SHORTCUT) ++out->n_shortcut;
    }
    std::vector<qtraj_obs> g(c->last_groups);
    if (c->last_groups) CK(cudaMemcpy(g.data(), c->ws + c->off_gobs, sizeof(qtraj_obs) * c->last_groups, cudaMemcpyDeviceToHost));
    for (const qtraj_obs &r : g) out->nojump_steps += r.n_steps_exec;
    out->steps_executed += out->nojump_steps;
    out->n_traj = c->last_batch;
    out->n_groups = c->last_groups;
    out->launches = c->launches;
    CK(cudaEventElapsedTime(&out->ms_nojump, c->ev0, c->ev1));
    CK(cudaEventElapsedTime(&out->ms_main, c->ev1, c->ev2));
    return QTRAJ_OK;
}

qtraj_status qtraj_kernel_info_get(const qtraj_ctx *c, qtraj_kernel_info *out)
{
    g_err.clear();
    if (!c || !out) return fail(QTRAJ_EINVAL, "null argument");
    std::memset(out, 0, sizeof(*out));
    out->sm_count = c->sm_count;
    if (c->p.form == QTRAJ_PLAIN) return QTRAJ_OK;
    FusedInfo fi{};
    LaunchArgs none{};
    if (c->p.precision == QTRAJ_FP32) CK(fused_launch_f32(c->N, tables<float>(c), none, c->sm_count, 0, nullptr, &fi, true, c->p.variant));
    else CK(fused_launch_f64(c->N, tables<double>(c), none, c->sm_count, 0, nullptr, &fi, true, c->p.variant));
    out->threads_per_traj = fi.G;
    out->ctas_per_sm = fi.ctas_per_sm;
    out->smem_bytes = fi.smem;
    out->regs_per_thread = fi.regs;
    out->radix = fi.R;
    return QTRAJ_OK;
}

} // extern "C"

// ------------------------------------------------------------------------------------------------
// qtraj_evolve_static: the fused evolve without any allocation.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where they evolve
// trajectories: a service that reserves all device memory for a pool at start-up and must not touch
// the CUDA allocator afterwards, or a latency-bound loop in which an allocation could synchronise the
// device or fail under fragmentation.  This entry point needs no workspace: everything the fused
// kernel uses besides its inputs and outputs (trajectory and group descriptors, the no-jump records,
// the media, the initial states, the work counter and the status word) lives in one file-scope
// device array of fixed size, and the host-side staging uses file-scope host arrays.  The caller
// passes host inputs and a device output buffer.
// ------------------------------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr int ST_MAX_TRAJ = QTRAJ_STATIC_MAX_TRAJ;
constexpr int ST_MAX_SPECS = QTRAJ_STATIC_MAX_SPECS;
constexpr int ST_MAX_MEDIA = QTRAJ_STATIC_MAX_MEDIA;
constexpr int ST_MAX_N = 16384;

struct StaticScratch {
    TrajDev trajs[ST_MAX_TRAJ];
    TrajDev gtrajs[ST_MAX_TRAJ];
    qtraj_obs gobs[ST_MAX_TRAJ];
    MediumDev media[ST_MAX_MEDIA];
    double ic[ST_MAX_SPECS * ST_MAX_N];
    double ov0[ST_MAX_SPECS * NBASIS * 2];
    int ov0_zero[ST_MAX_SPECS * NBASIS];
    int spec_l[ST_MAX_SPECS];
    int spec_color[ST_MAX_SPECS];
    int gready[ST_MAX_TRAJ];  // published flags of the groups' no-jump records; cleared by every call
    int counter_status[64];   // [0] work counter, [1] status word; cleared by every call
};

// The device scratch of every call on a device.  Host code must not use this name as an address:
// on the host it is only a stand-in for the symbol; its device address comes from
// cudaGetSymbolAddress (st_setup).
static __device__ __align__(256) unsigned char g_static_scratch[sizeof(StaticScratch)];

// host-side staging, also fixed in size
StaticScratch g_static_host;
int g_static_pair_group[ST_MAX_SPECS * ST_MAX_MEDIA];
std::mutex g_static_mutex;
constexpr int ST_MAX_DEVICES = 64;
StaticScratch *g_static_dev[ST_MAX_DEVICES] = {nullptr};

// once per device, with that device current: the device address of the scratch array
qtraj_status st_setup(int dev, StaticScratch **out)
{
    if (dev < 0 || dev >= ST_MAX_DEVICES) return fail(QTRAJ_EINVAL, "device %d beyond the static table", dev);
    if (!g_static_dev[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(QTRAJ_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        g_static_dev[dev] = (StaticScratch *)p;
    }
    *out = g_static_dev[dev];
    return QTRAJ_OK;
}

// discretely normalised initial states into a caller-provided array (no allocation)
void st_coulomb(int N, double dr, double a0, int n, int l, double *u)
{
    double s = 0.0;
    u[0] = 0.0;
    for (int j = 1; j < N; ++j) {
        const double r = j * dr;
        const double v = std::pow(r, l + 1) * std::exp(-r / (n * a0)) * laguerre(n - l - 1, 2 * l + 1, 2.0 * r / (n * a0));
        u[j] = v;
        s += v * v;
    }
    const double c = 1.0 / std::sqrt(s * dr);
    for (int j = 1; j < N; ++j) u[j] *= c;
}
// r^{l+1} exp(-r^2/(2 w^2)), discretely normalised: evaluated through its logarithm shifted by the
// largest value, so that no power of r overflows at large l (the normalisation removes the shift)
void st_gauss(int N, double dr, double w, int l, double *u)
{
    double mx = -HUGE_VAL;
    u[0] = 0.0;
    for (int j = 1; j < N; ++j) {
        const double r = j * dr;
        u[j] = (l + 1) * std::log(r) - r * r / (2.0 * w * w);
        mx = std::max(mx, u[j]);
    }
    double s = 0.0;
    for (int j = 1; j < N; ++j) {
        u[j] = std::exp(u[j] - mx);
        s += u[j] * u[j];
    }
    const double c = 1.0 / std::sqrt(s * dr);
    for (int j = 1; j < N; ++j) u[j] *= c;
}
} // namespace

extern "C" qtraj_status qtraj_evolve_static(qtraj_ctx *c, int batch, const qtraj_init_spec *specs, int n_specs,
                                            const int *spec_idx, const qtraj_medium *media, int n_media,
                                            const int *medium_idx, const uint64_t *seeds, qtraj_obs *d_out,
                                            void *stream)
{
    g_err.clear();
    if (!c || !specs || !media || !seeds || !d_out) return fail(QTRAJ_EINVAL, "null argument");
    if (c->p.form != QTRAJ_FUSED) return fail(QTRAJ_EINVAL, "qtraj_evolve_static runs the fused form only");
    if (c->p.t_vacuum > 0) return fail(QTRAJ_EINVAL, "qtraj_evolve_static does not run a vacuum evolution (t_vacuum > 0)");
    if (batch < 0 || batch > ST_MAX_TRAJ)
        return fail(QTRAJ_EINVAL, "batch %d outside [0, %d] (QTRAJ_STATIC_MAX_TRAJ)", batch, ST_MAX_TRAJ);
    if (n_specs <= 0 || n_specs > ST_MAX_SPECS)
        return fail(QTRAJ_EINVAL, "n_specs %d outside [1, %d] (QTRAJ_STATIC_MAX_SPECS)", n_specs, ST_MAX_SPECS);
    if (n_media <= 0 || n_media > ST_MAX_MEDIA)
        return fail(QTRAJ_EINVAL, "n_media %d outside [1, %d] (QTRAJ_STATIC_MAX_MEDIA)", n_media, ST_MAX_MEDIA);
    if (c->N > ST_MAX_N) return fail(QTRAJ_EINVAL, "N %d above %d", c->N, ST_MAX_N);
    if (!spec_idx && n_specs != 1 && n_specs != batch)
        return fail(QTRAJ_EINVAL, "spec_idx is required unless n_specs is 1 or batch");
    if (!medium_idx && n_media != 1 && n_media != batch)
        return fail(QTRAJ_EINVAL, "medium_idx is required unless n_media is 1 or batch");
    if (((uintptr_t)d_out & 7) != 0) return fail(QTRAJ_EINVAL, "d_out must be 8-byte aligned");

    std::lock_guard<std::mutex> lock(g_static_mutex);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(QTRAJ_ECUDA, "cudaGetDevice failed");
    // the context's tables live on c->device; the scratch address is looked up on the current one
    if (dev != c->device)
        return fail(QTRAJ_EINVAL, "the current device %d is not the context's device %d", dev, c->device);
    StaticScratch *ds = nullptr;
    const qtraj_status sst = st_setup(dev, &ds);
    if (sst != QTRAJ_OK) return sst;

    const int N = c->N;
    StaticScratch &h = g_static_host;
    for (int s = 0; s < n_specs; ++s) {
        const qtraj_init_spec &q = specs[s];
        if (q.kind != 0 && q.kind != 1) return fail(QTRAJ_EINVAL, "spec %d: kind must be 0 or 1", s);
        if (q.l < 0 || (q.color != 0 && q.color != 1)) return fail(QTRAJ_EINVAL, "spec %d: l >= 0, color 0/1", s);
        if (q.kind == 0 && !(q.width > 0)) return fail(QTRAJ_EINVAL, "spec %d: width must be positive", s);
        if (q.kind == 1 && (q.n < 1 || q.l >= q.n)) return fail(QTRAJ_EINVAL, "spec %d: need 0 <= l < n", s);
        double *u = h.ic + (size_t)s * N;
        if (q.kind == 1) st_coulomb(N, c->dr, c->a0, q.n, q.l, u);
        else st_gauss(N, c->dr, q.width, q.l, u);
        if (const char *why = state_problem(N, c->dr, u))
            return fail(QTRAJ_EINVAL, "spec %d: the initial state %s", s, why);
        h.spec_l[s] = q.l;
        h.spec_color[s] = q.color;
        // the overlaps and their structural zeros follow the context's basis, as in qtraj_init: an
        // analytic Coulomb state is orthogonal to the other n only in the analytic basis
        const bool same_family = q.kind == 1 && c->p.basis == 0;
        for (int b = 0; b < NBASIS; ++b) {
            const int z = q.color != 0 || q.l != BASIS_L[b] || (same_family && q.n != BASIS_N[b]);
            h.ov0_zero[s * NBASIS + b] = z;
            double o = 0.0;
            if (!z) {
                const double *ph = c->basis_host.data() + (size_t)b * N;
                for (int j = 1; j < N; ++j) o += ph[j] * u[j];
                o *= c->dr;
            }
            h.ov0[(s * NBASIS + b) * 2] = o;
            h.ov0[(s * NBASIS + b) * 2 + 1] = 0.0;
        }
    }
    int steps[ST_MAX_MEDIA];
    for (int m = 0; m < n_media; ++m) {
        const qtraj_medium &q = media[m];
        if (const char *why = medium_check(q)) return fail(QTRAJ_EINVAL, "medium %d: %s", m, why);
        if (c->p.potential == 1 && !(q.Tf >= KSU_TF_MIN))
            return fail(QTRAJ_EINVAL, "medium %d: the KSU potential needs Tf >= %g GeV", m, KSU_TF_MIN);
        steps[m] = medium_steps(c->dt, q, nullptr);
        h.media[m] = encode_medium(c, q);
    }
    for (int i = 0; i < n_specs * n_media; ++i) g_static_pair_group[i] = -1;
    int n_groups = 0;
    for (int t = 0; t < batch; ++t) {
        const int sp = spec_idx ? spec_idx[t] : (n_specs == 1 ? 0 : t);
        const int mi = medium_idx ? medium_idx[t] : (n_media == 1 ? 0 : t);
        if (sp < 0 || sp >= n_specs) return fail(QTRAJ_EINVAL, "spec_idx[%d] out of range", t);
        if (mi < 0 || mi >= n_media) return fail(QTRAJ_EINVAL, "medium_idx[%d] out of range", t);
        int &gidx = g_static_pair_group[sp * n_media + mi];
        if (gidx < 0) {
            gidx = n_groups;
            h.gtrajs[n_groups] = TrajDev{0ull, sp, mi, steps[mi], n_groups};
            ++n_groups;
        }
        h.trajs[t] = TrajDev{(unsigned long long)seeds[t], sp, mi, steps[mi], gidx};
    }
    if (!c->p.use_rmin || c->p.potential != 0) n_groups = 0;

    cudaStream_t s = (cudaStream_t)stream;
    auto up = [&](void *dst, const void *src, size_t n) -> cudaError_t {
        return n ? cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    CK(up(ds->ic, h.ic, sizeof(double) * (size_t)n_specs * N));
    CK(up(ds->ov0, h.ov0, sizeof(double) * n_specs * NBASIS * 2));
    CK(up(ds->ov0_zero, h.ov0_zero, sizeof(int) * n_specs * NBASIS));
    CK(up(ds->spec_l, h.spec_l, sizeof(int) * n_specs));
    CK(up(ds->spec_color, h.spec_color, sizeof(int) * n_specs));
    CK(up(ds->media, h.media, sizeof(MediumDev) * n_media));
    CK(up(ds->trajs, h.trajs, sizeof(TrajDev) * batch));
    CK(up(ds->gtrajs, h.gtrajs, sizeof(TrajDev) * (n_groups > 0 ? n_groups : 0)));
    // the work counter and the status word must start at zero in every call
    CK(cudaMemsetAsync(ds->counter_status, 0, sizeof(ds->counter_status), s));

    if (n_groups > 0) CK(cudaMemsetAsync(ds->gready, 0, sizeof(int) * (size_t)n_groups, s));

    int *d_ctr = ds->counter_status, *d_status = ds->counter_status + 1;
    LaunchArgs ma{ds->trajs, batch, d_out, nullptr, d_ctr, d_status, nullptr, 0};
    ma.gtrajs = ds->gtrajs;
    ma.n_groups = n_groups;
    ma.gobs = ds->gobs;
    ma.gready = ds->gready;
    FusedInfo fi;
    auto point = [&](auto tb) {
        tb.ic = ds->ic;
        tb.ic_cplx = 0;
        tb.ov0 = ds->ov0;
        tb.ov0_zero = ds->ov0_zero;
        tb.spec_l = ds->spec_l;
        tb.spec_color = ds->spec_color;
        tb.media = ds->media;
        return tb;
    };
    if (c->p.precision == QTRAJ_FP32) CK(fused_launch_f32(N, point(tables<float>(c)), ma, c->sm_count, 0, s, &fi, false, c->p.variant));
    else CK(fused_launch_f64(N, point(tables<double>(c)), ma, c->sm_count, 0, s, &fi, false, c->p.variant));
    return QTRAJ_OK;
}
