// qtraj_device.cuh -- device-side building blocks shared by the fused and the plain forms:
// complex arithmetic, Philox4x32-10, small in-register DFTs, and the device records.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "qtraj.h"

namespace qt {

constexpr int NBASIS = QTRAJ_NBASIS;
constexpr int LTAB = 256;            // l rows per colour of the static space-kernel tables
constexpr double BORDER_EPS = 1e-12; // |norm^2 - r| below this flags a borderline comparison (FP64)
// The FP32 forms flag at the error of their norm instead: the state is carried in FP32, and its
// norm after thousands of steps is good to ~1e-6 (the paired FP32/FP64 study: 3e-4 of the jumps
// moved by a step, at ~3e-3 mean norm change per step between jumps), so a threshold closer to the
// norm than that may be crossed a step earlier or later than in exact arithmetic.
constexpr double BORDER_EPS_F32 = 1e-6;
template <typename T> __host__ __device__ constexpr double border_eps()
{
    return sizeof(T) == 4 ? BORDER_EPS_F32 : BORDER_EPS;
}

// ------------------------------------------------------------------------------------------------
// complex numbers
// ------------------------------------------------------------------------------------------------
template <typename T> struct alignas(2 * sizeof(T)) cpx { T x, y; };

template <typename T> __host__ __device__ __forceinline__ cpx<T> mk(T a, T b) { return {a, b}; }
template <typename T> __device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T> __device__ __forceinline__ cpx<T> operator*(cpx<T> a, cpx<T> b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ cpx<T> scale(cpx<T> a, T s) { return {a.x * s, a.y * s}; }
template <typename T> __device__ __forceinline__ cpx<T> mul_i(cpx<T> a) { return {-a.y, a.x}; }   // i*a
template <typename T> __device__ __forceinline__ cpx<T> mul_mi(cpx<T> a) { return {a.y, -a.x}; }  // -i*a
// FP32: complex add, subtract and real scale as packed FP32x2 instructions (sm_100 and later): both
// components in one instruction, each with the same IEEE rounding as the scalar form (a - b is
// fma(-1, b, a), exact in the product), so results are bit-identical and the issue slots halve
template <> __device__ __forceinline__ cpx<float> operator+(cpx<float> a, cpx<float> b)
{
    const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
    return {r.x, r.y};
}
template <> __device__ __forceinline__ cpx<float> operator-(cpx<float> a, cpx<float> b)
{
    const float2 r = __ffma2_rn(make_float2(-1.f, -1.f), make_float2(b.x, b.y), make_float2(a.x, a.y));
    return {r.x, r.y};
}
template <> __device__ __forceinline__ cpx<float> scale(cpx<float> a, float s)
{
    const float2 r = __fmul2_rn(make_float2(a.x, a.y), make_float2(s, s));
    return {r.x, r.y};
}
// read-only-cache loads of complex values
__device__ __forceinline__ cpx<float> ldg(const cpx<float> *p)
{
    const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ cpx<double> ldg(const cpx<double> *p)
{
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    return {v.x, v.y};
}
// ------------------------------------------------------------------------------------------------
// constant multipliers.  In FP32 every constant of the step (twiddles, in-register DFT constants,
// sine pre-factors, kinetic and potential phase tables) is carried as an unevaluated sum hi + lo of
// two floats: the rounding of a constant is the same in every step and would otherwise accumulate
// coherently over 10^4 steps, while the rounding of data is random and grows only as a square root.
// In FP64 a constant is one double.
// ------------------------------------------------------------------------------------------------
template <typename T> struct Prec;
template <> struct Prec<double> {
    using C = cpx<double>; // complex constant
    using Rl = double;     // real constant
    static __host__ C make(double re, double im) { return {re, im}; }
    static __host__ Rl make_r(double v) { return v; }
    static __device__ __forceinline__ cpx<double> mul(cpx<double> x, C w) { return x * w; }
    static __device__ __forceinline__ C conj(C w) { return {w.x, -w.y}; }
    static __device__ __forceinline__ cpx<double> mul2(cpx<double> x, C w) { return x * w; }
    static __device__ __forceinline__ cpx<double> mulr(cpx<double> x, Rl s) { return scale(x, s); }
    static __device__ __forceinline__ C ld(const C *p) { return ldg(p); }
    static __device__ __forceinline__ Rl ldr(const Rl *p) { return __ldg(p); }
    static __device__ __forceinline__ C from_double(double re, double im) { return {re, im}; }
    // static potential factors (tables of exp(-i V_static dt/2), exp(-i V_static dt)): one double each
    using S = cpx<double>;
    static __host__ __device__ S make_s(double re, double im) { return {re, im}; }
    static __device__ __forceinline__ S ld_s(const S *p) { return ldg(p); }
    static __device__ __forceinline__ cpx<double> mul_s(cpx<double> x, S w) { return x * w; }
    static __device__ __forceinline__ S conj_s(S w) { return {w.x, -w.y}; }
};
template <> struct Prec<float> {
    struct alignas(16) C { float rh, ih, rl, il; };
    // The sine pre-factors keep their low parts: rounded to single FP32 they passed the paired
    // ensemble study (8.9e-6 / 6.6e-6 at N = 8192 / 4096) and ran 2.5-3.5% faster, but the same
    // rounding every step biased the no-jump norm by +1.3e-8 per step at N = 64.
    struct alignas(8) Rl { float h, l; };
    static __host__ C make(double re, double im)
    {
        const float rh = (float)re, ih = (float)im;
        return {rh, ih, (float)(re - (double)rh), (float)(im - (double)ih)};
    }
    static __host__ Rl make_r(double v)
    {
        const float h = (float)v;
        return {h, (float)(v - (double)h)};
    }
    static __device__ __forceinline__ cpx<float> mul(cpx<float> x, C w)
    {
        const float lr = fmaf(x.x, w.rl, -x.y * w.il), li = fmaf(x.x, w.il, x.y * w.rl);
        return {fmaf(x.x, w.rh, fmaf(-x.y, w.ih, lr)), fmaf(x.x, w.ih, fmaf(x.y, w.rh, li))};
    }
    // the same product as mul, in packed FP32x2 instructions (bit-identical results)
    static __device__ __forceinline__ cpx<float> mul2(cpx<float> x, C w)
    {
        const float2 xx = make_float2(x.x, x.x), yy = make_float2(-x.y, x.y);
        const float2 l = __ffma2_rn(xx, make_float2(w.rl, w.il), __fmul2_rn(yy, make_float2(w.il, w.rl)));
        const float2 r = __ffma2_rn(xx, make_float2(w.rh, w.ih), __ffma2_rn(yy, make_float2(w.ih, w.rh), l));
        return {r.x, r.y};
    }
    static __device__ __forceinline__ C conj(C w) { return {w.rh, -w.ih, w.rl, -w.il}; }
    static __device__ __forceinline__ cpx<float> mulr(cpx<float> x, Rl s)
    {
        return {fmaf(x.x, s.h, x.x * s.l), fmaf(x.y, s.h, x.y * s.l)};
    }
    static __device__ __forceinline__ C ld(const C *p)
    {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        return {v.x, v.y, v.z, v.w};
    }
    static __device__ __forceinline__ Rl ldr(const Rl *p)
    {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        return {v.x, v.y};
    }
    static __device__ __forceinline__ C from_double(double re, double im)
    {
        const float rh = (float)re, ih = (float)im;
        return {rh, ih, (float)(re - (double)rh), (float)(im - (double)ih)};
    }
    // The static potential factors are the one family of constants kept without low parts: the
    // paired FP32/FP64 study measured no loss from rounding them (ensemble errors 1.6e-6 / 1.1e-5 at
    // N = 4096 / 8192 against 2.6e-6 / 4.2e-6 with hi+lo; median norm error 6.7e-7 against 5.3e-7),
    // while their table is the one a trajectory reads per (colour, l) row -- half the bytes.
    using S = cpx<float>;
    static __host__ __device__ S make_s(double re, double im) { return {(float)re, (float)im}; }
    static __device__ __forceinline__ S ld_s(const S *p) { return ldg(p); }
    static __device__ __forceinline__ cpx<float> mul_s(cpx<float> x, S w)
    {
        return {fmaf(x.x, w.x, -x.y * w.y), fmaf(x.x, w.y, x.y * w.x)};
    }
    static __device__ __forceinline__ S conj_s(S w) { return {w.x, -w.y}; }
};

// a * (rh + i ih) with the constant's low parts (rl, il) in FP32 (PK: the packed product); plain
// product in FP64
template <typename T, bool PK = false> __device__ __forceinline__ cpx<T> mulk(cpx<T> a, double re, double im)
{
    if constexpr (sizeof(T) == 4) {
        const Prec<float>::C w{(float)re, (float)im, (float)(re - (double)(float)re), (float)(im - (double)(float)im)};
        return PK ? Prec<float>::mul2(a, w) : Prec<float>::mul(a, w);
    } else {
        return a * mk<T>(re, im);
    }
}
template <typename T> __device__ __forceinline__ T mulkr(T v, double c)
{
    if constexpr (sizeof(T) == 4) return fmaf(v, (float)c, v * (float)(c - (double)(float)c));
    else return v * c;
}

template <typename T> __device__ __forceinline__ double abs2d(cpx<T> a)
{
    return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}

// ------------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter (k,0,0,0), key = 64-bit seed.
// Waiting period k of a trajectory uses the four words of counter k: the threshold r from words
// 0 and 1 (53 bits), the angular-momentum draw u_l from word 2 and the colour draw u_c from word 3.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void philox10(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        if (i) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
}

struct Draws { double r, ul, uc; };

// the jump digest of a record: 32-bit FNV-1a over the little-endian bytes of (step, new l, new colour)
// of every jump in order
constexpr uint32_t DIGEST_BASIS = 2166136261u;
__host__ __device__ __forceinline__ uint32_t digest_word(uint32_t h, uint32_t w)
{
#pragma unroll
    for (int b = 0; b < 4; ++b) h = (h ^ ((w >> (8 * b)) & 255u)) * 16777619u;
    return h;
}
__host__ __device__ __forceinline__ uint32_t digest_jump(uint32_t h, int step, int l, int c)
{
    return digest_word(digest_word(digest_word(h, (uint32_t)step), (uint32_t)l), (uint32_t)c);
}

__device__ __forceinline__ Draws draws(unsigned long long seed, uint32_t k)
{
    uint32_t c0 = k, c1 = 0, c2 = 0, c3 = 0;
    philox10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    const unsigned long long w = ((unsigned long long)c1 << 32) | c0;
    Draws d;
    d.r = ((double)(w >> 11) + 0.5) * 0x1.0p-53;
    d.ul = ((double)c2 + 0.5) * 0x1.0p-32;
    d.uc = ((double)c3 + 0.5) * 0x1.0p-32;
    return d;
}

// ------------------------------------------------------------------------------------------------
// in-register DFTs of size 2, 4, 8, 16: X_k = sum_n x_n exp(-2 pi i n k / R), natural order in/out
// ------------------------------------------------------------------------------------------------
// x * exp(-2 pi i j/16) for a compile-time j (after unrolling the switch folds away); the constants
// cos(pi/8), sin(pi/8), sqrt(1/2) enter with their FP32 low parts in the FP32 form
template <typename T, bool PK = false> __device__ __forceinline__ cpx<T> tw16(cpx<T> a, int j)
{
    constexpr double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173, h = 0.70710678118654752440;
    switch (j & 15) {
    case 0: return a;
    case 1: return mulk<T, PK>(a, c1, -s1);
    case 2: return mk(mulkr<T>(a.x + a.y, h), mulkr<T>(a.y - a.x, h));
    case 3: return mulk<T, PK>(a, s1, -c1);
    case 4: return mul_mi(a);
    case 5: return mulk<T, PK>(a, -s1, -c1);
    case 6: return mk(mulkr<T>(a.y - a.x, h), mulkr<T>(-a.x - a.y, h));
    case 7: return mulk<T, PK>(a, -c1, -s1);
    case 8: return mk(-a.x, -a.y);
    case 9: return mulk<T, PK>(a, -c1, s1);
    case 10: return mk(mulkr<T>(-a.x - a.y, h), mulkr<T>(a.x - a.y, h));
    case 11: return mulk<T, PK>(a, -s1, c1);
    case 12: return mul_i(a);
    case 13: return mulk<T, PK>(a, s1, c1);
    case 14: return mk(mulkr<T>(a.x - a.y, h), mulkr<T>(a.x + a.y, h));
    default: return mulk<T, PK>(a, c1, s1);
    }
}

template <typename T> __device__ __forceinline__ void dft2(cpx<T> &a, cpx<T> &b)
{
    const cpx<T> t = a;
    a = t + b;
    b = t - b;
}

template <typename T> __device__ __forceinline__ void dft4(cpx<T> &x0, cpx<T> &x1, cpx<T> &x2, cpx<T> &x3)
{
    const cpx<T> a = x0 + x2, b = x0 - x2, c = x1 + x3, d = mul_mi(x1 - x3);
    x0 = a + c;
    x2 = a - c;
    x1 = b + d;
    x3 = b - d;
}

// DFT of R = R1*R2 points held at x[base + stride*n]: inner DFTs of size R1 over n1 (n = R2 n1 + n2),
// twiddles W_R^{n2 k1}, outer DFTs of size R2 over n2; output index k = k1 + R1 k2.
template <typename T, int R> struct DFT;

template <typename T> struct DFT<T, 1> {
    template <int S> __device__ __forceinline__ static void run(cpx<T> *) {}
};
template <typename T> struct DFT<T, 2> {
    template <int S> __device__ __forceinline__ static void run(cpx<T> *x) { dft2(x[0], x[S]); }
};
template <typename T> struct DFT<T, 4> {
    template <int S> __device__ __forceinline__ static void run(cpx<T> *x) { dft4(x[0], x[S], x[2 * S], x[3 * S]); }
};
template <typename T> struct DFT<T, 8> {
    template <int S> __device__ __forceinline__ static void run(cpx<T> *x)
    {
        // n = 2 n1 + n2: two DFT4 over n1, twiddle W8^{n2 k1}, four DFT2 over n2
        cpx<T> y[8];
#pragma unroll
        for (int n2 = 0; n2 < 2; ++n2) {
            cpx<T> a = x[(0 + n2) * S], b = x[(2 + n2) * S], c = x[(4 + n2) * S], d = x[(6 + n2) * S];
            dft4(a, b, c, d);
            y[n2 * 4 + 0] = a;
            y[n2 * 4 + 1] = tw16(b, 2 * n2 * 1);
            y[n2 * 4 + 2] = tw16(c, 2 * n2 * 2);
            y[n2 * 4 + 3] = tw16(d, 2 * n2 * 3);
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            cpx<T> a = y[k1], b = y[4 + k1];
            dft2(a, b);
            x[(k1)*S] = a;
            x[(k1 + 4) * S] = b;
        }
    }
};
template <typename T> struct DFT<T, 16> {
    template <int S> __device__ __forceinline__ static void run(cpx<T> *x)
    {
        // n = 4 n1 + n2: four DFT4 over n1, twiddle W16^{n2 k1}, four DFT4 over n2
        cpx<T> y[16];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            cpx<T> a = x[(0 + n2) * S], b = x[(4 + n2) * S], c = x[(8 + n2) * S], d = x[(12 + n2) * S];
            dft4(a, b, c, d);
            y[n2 * 4 + 0] = a;
            y[n2 * 4 + 1] = tw16(b, n2 * 1);
            y[n2 * 4 + 2] = tw16(c, n2 * 2);
            y[n2 * 4 + 3] = tw16(d, n2 * 3);
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            cpx<T> a = y[k1], b = y[4 + k1], c = y[8 + k1], d = y[12 + k1];
            dft4(a, b, c, d);
            x[(k1)*S] = a;
            x[(k1 + 4) * S] = b;
            x[(k1 + 8) * S] = c;
            x[(k1 + 12) * S] = d;
        }
    }
};

// ------------------------------------------------------------------------------------------------
// device records
// ------------------------------------------------------------------------------------------------
struct MediumDev {
    double A;       // T0^3 tau0, so T(tau_n)^3 = A / (tau0 + n dtau)  (kind 0)
    double tau0;    // fm/c: tau of step 0 (kind 1: the table's first tau)
    double dtau;    // dt * hbar c, fm/c per step
    double er[2];   // -kappa_c dt/2 per colour: the real exponent of the space kernel is er*T^3*r^2
    double ei[2];   // -gamma_c dt/2 per colour: the phase of the space kernel is ei*T^3*r^2
    double erj[2];  // er * dr^2: the real exponent is erj * T^3 * j^2 on grid point j
    double eij[2];  // ei * dr^2 / pi: the phase is pi * eij * T^3 * j^2
    int kfit;       // 0: constant kappa_hat, folded into er/erj; 1, 2, 3: er/erj are per unit kappa_hat
                    // and T^3 in the real exponent becomes kappa_hat(T) T^3 from lattice fit kfit
    int kind;       // 0 Bjorken; 1 tabulated: points [tab_off, tab_off + tab_len) of the profile store
    int tab_off, tab_len;
};

// T^3 at tau of a tabulated medium, p = its (tau, T) pairs: linear in T between the neighbouring
// points, the first/last T outside.  seg is the caller's segment index (p[seg].tau <= tau), moved
// forward only, so a trajectory walks its table once.
template <typename T> __device__ __forceinline__ T table_T3(const double *p, int len, T tau, int &seg)
{
    while (seg + 2 < len && tau >= (T)p[2 * (seg + 1)]) ++seg;
    const T t0 = (T)p[2 * seg], t1 = (T)p[2 * seg + 2], T0 = (T)p[2 * seg + 1], T1 = (T)p[2 * seg + 3];
    T f = (tau - t0) / (t1 - t0);
    f = f < (T)0 ? (T)0 : (f > (T)1 ? (T)1 : f);
    const T Tt = T0 + f * (T1 - T0);
    return Tt * Tt * Tt;
}

// the same from scratch (binary search), for kernels that do not carry a segment index
__device__ __forceinline__ double table_T3_at(const double *p, int len, double tau)
{
    int lo = 0, hi = len - 1;   // find the last point with tau_i <= tau, at most len - 2
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (p[2 * mid] <= tau) lo = mid;
        else hi = mid;
    }
    int seg = lo;
    return table_T3<double>(p, len, tau, seg);
}

// kappa_hat(T) T^3 given T^3: kfit 0 returns T^3 (kappa_hat is folded into the exponent's
// coefficient); kfit 1, 2, 3 multiply by the central, lower or upper lattice fit of the Munich
// potential (App. E), kappa_hat = 1 / (a x^{3/2} + b x + c x^{1/2} + d) with x = T / T_c,
// T_c = 0.155 GeV, evaluated in the working precision once per step.
template <typename T> __device__ __forceinline__ T kappa_T3(int kfit, T T3)
{
    if (kfit == 0) return T3;
    const T a = kfit == 1 ? (T)0.00397 : kfit == 2 ? (T)0.00712 : (T)0.00272;
    const T b = kfit == 1 ? (T)-0.08341 : kfit == 2 ? (T)-0.14262 : (T)-0.05854;
    const T c = kfit == 1 ? (T)0.98031 : kfit == 2 ? (T)1.55601 : (T)0.71513;
    const T d = kfit == 1 ? (T)-0.51889 : kfit == 2 ? (T)-0.80712 : (T)-0.38197;
    const T s = sqrt(cbrt(T3) * (T)(1.0 / 0.155));
    return T3 / (((a * s + b) * s + c) * s + d);
}

struct TrajDev {
    unsigned long long seed;
    int spec, medium, n_steps, group;
};

static_assert(sizeof(qtraj_obs) == 192, "qtraj_obs layout");
static_assert(sizeof(qtraj_trace_rec) == 80, "qtraj_trace_rec layout");

// Read-only context tables (device pointers) and scalars.
template <typename T> struct Tables {
    using C = typename Prec<T>::C;
    const C *W;                        // N twiddles exp(-2 pi i t / N)
    const C *WL;                       // last-pass twiddles W^(m g): sections [R][N/(2R)] for R = 16, 8, 4
    const C *KT;                       // N kinetic factors exp(-i T_kin(p_k) dt) * 2/N, k = 0..N-1
    const typename Prec<T>::Rl *sinpre; // N values sin(pi j / N)
    const typename Prec<T>::S *statV;  // [2][LTAB][N] exp(-i (V_coul + l(l+1)/(M r^2)) dt/2)
    const typename Prec<T>::S *statV2; // [2][LTAB][N] the same over a full step, exp(-i (...) dt)
    const double *eig;     // [NBASIS][N] Coulomb basis, discretely normalised
    const double *ic;      // initial states, discretely normalised: [n_spec][N] real, or
                           // [n_spec][N][2] (re, im) when ic_cplx (after a vacuum evolution)
    const double *ov0;     // [n_spec][NBASIS][2] initial overlaps
    const int *ov0_zero;   // [n_spec][NBASIS] structural zero of the initial overlap
    const int *spec_l;     // [n_spec]
    const int *spec_color; // [n_spec]
    const MediumDev *media;
    double dr, dt, M, p_os;
    double coul[2];        // coefficient of 1/r of the colour's Coulomb potential
    int max_jumps, l_cap, use_rmin;
    double r_max;
    int ic_cplx;
    const double *prof;    // profile store: (tau, T) pairs of the tabulated media
    double r1s;            // <1S|r|1S> on the grid (discrete), the unit of the summary's R
    // the isotropic KSU potential (potential = 1; App. E), see qtraj_params.potential:
    int potential;
    const T *phi_tab;      // (phi, h phi') at a = KSU_PHI_A0 + i h, i < KSU_PHI_NODES (h = 1/KSU_PHI_PER)
    const T *phi_ser;      // [KSU_PHI_SER][2]: the small-argument series of phi, coefficients of y^k
                           // (y = a^2) of the ln a part and of the rest (k = 1 ..)
    T ksu_a_dr;            // a / dr: the Coulomb part a/r = ksu_a_dr / j
    T ksu_sig_dr;          // sigma dr: the linear part sigma r = ksu_sig_dr j
    T ksu_two_sigma;       // 2 sigma
    T ksu_cap;             // V_vac(r_SB) = -a/r_SB + sigma r_SB
    T ksu_alpha0, ksu_b0, ksu_mu0sq;   // alpha_s(mu) = alpha0 / (1 + alpha0 b0 ln(mu^2 / mu0^2))
    T ksu_md2;             // F_mD^2 Nc (1 + N_F/6) pi C_F: m_D^2 = ksu_md2 T^2 alpha_s(2 pi T)
    T ksu_cf;              // C_F
    T ksu_dt;              // the step (GeV^-1) in the working precision
};
constexpr double KSU_PHI_A0 = 0.5, KSU_PHI_A1 = 40.0;
constexpr int KSU_PHI_PER = 256;                                   // nodes per unit of a
constexpr int KSU_PHI_NODES = (int)((KSU_PHI_A1 - KSU_PHI_A0) * KSU_PHI_PER) + 1;
constexpr int KSU_PHI_SER = 8;                                     // series terms (a < KSU_PHI_A0)

// per-launch arguments of both forms
struct LaunchArgs {
    const TrajDev *trajs;
    int n_traj;
    qtraj_obs *obs;         // per trajectory (main mode) or per group (no-jump mode)
    const qtraj_obs *group; // no-jump records read by the shortcut (main mode)
    int *counter;           // work counter (fused) -- zeroed before the launch
    int *status;            // bit 0: a non-finite norm was seen
    double *states;         // optional final states [n_traj][N] complex128
    int nojump;             // 1: no-jump mode (trajectory t = group t, never jumps)
    qtraj_trace_rec *trace; // per-step summary rows [trace_n][trace_cap] (traced kernel; off if trace_every 0)
    int *trace_cnt;         // rows written per traced trajectory
    int trace_every, trace_n, trace_cap;
    // fused form, one launch for the rMin shortcut: work items [0, n_groups) are the no-jump runs of
    // the groups (gtrajs -> gobs, then gready[g] = 1), items n_groups + t the trajectories.  A
    // trajectory fetched after its group's flag is set takes the shortcut; one fetched before runs
    // its whole medium, which gives the same record (the shortcut is exact) but counts its steps.
    const TrajDev *gtrajs;
    int n_groups;
    qtraj_obs *gobs;
    int *gready;
};

// static part of the half-step space kernel for (colour, l, j); rows beyond the table are
// evaluated in FP64 on the fly.  A jump moves l by one, and l(l+1) grows by 2 per jump on average
// (l -> l+1 with probability (l+1)/(2l+1)), so l >= 256 takes some 33,000 jumps.
template <typename T>
__device__ __forceinline__ typename Prec<T>::S static_factor(const Tables<T> &tb, int N, int c, int l, int j)
{
    if (l < LTAB) return Prec<T>::ld_s(&tb.statV[((size_t)c * LTAB + l) * N + j]);
    if (j == 0) return Prec<T>::make_s(0.0, 0.0);
    const double r = j * tb.dr;
    const double V = tb.coul[c] / r + (double)l * (l + 1) / (tb.M * r * r);
    double s, co;
    sincos(-V * tb.dt * 0.5, &s, &co);
    return Prec<T>::make_s(co, s);
}

// T-dependent part exp((er + i ei) T^3 r^2) of the half-step space kernel
__device__ __forceinline__ cpx<float> dyn_factor(float er, float ei, float r2)
{
    float s, c;
    sincosf(ei * r2, &s, &c);
    const float m = expf(er * r2);
    return mk(m * c, m * s);
}
__device__ __forceinline__ cpx<double> dyn_factor(double er, double ei, double r2)
{
    double s, c;
    sincos(ei * r2, &s, &c);
    const double m = exp(er * r2);
    return mk(m * c, m * s);
}

} // namespace qt
