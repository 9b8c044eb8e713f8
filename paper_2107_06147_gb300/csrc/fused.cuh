// fused.cuh -- the fused persistent trajectory kernel.
//
// One CTA evolves one trajectory at a time, through every step of its medium, and then fetches the
// next trajectory from a global work counter.  The wave function never leaves the SM: between the
// sine transforms it lives in one shared-memory buffer of N + N/R complex values; during a transform
// each thread holds 2R values in registers.
//
// One step (Sec. 3.3, steps 1-5) with T = T(tau_n) (Sec. 3.4, Bjorken):
//   x <- K_V(n) x        K_V = exp(-i V_eff dt/2) = static(c, l, r) * exp((er + i ei) T^3 r^2)
//   S = DST(x)           S_k = sum_j x_j sin(pi j k / N)
//   S <- K_T S           K_T = exp(-i T_kin(p_k) dt) * 2/N   (2/N = inverse DST scale)
//   x = DST(S)
//   x <- K_V(n) x, norm^2 = (L/N) sum |x_j|^2, jump if norm^2 <= r (Sec. 3.2.1, 3.4.3-3.4.4, 3.5)
// The end half-step of step n and the start half-step of step n+1 are applied as one factor
// static^2 * exp((er_n + er_{n+1}) r^2 + i (ei_n + ei_{n+1}) r^2); the norm after the end half-step is
// accumulated with the weights |K_V(n)|^2 = exp(2 er_n r^2) on the way.  On the rare steps that
// jump, the start half-step is turned into the new colour's and l's afterwards (all these factors are
// diagonal in r and commute with the jump's multiplication by r).
//
// The DST-I of the N-point complex vector f (f_0 = f_N = 0) is computed with one N-point complex FFT:
//   y_j = sin(pi j/N)(f_j + f_{N-j}) + (f_j - f_{N-j})/2,   Y = FFT_N(y),
//   S_{2k}   = (i/2)(Y_k - Y_{N-k}),
//   S_{2k+1} = S_{2k-1} + (Y_k + Y_{N-k})/2,  S_{-1} = -S_1    (a prefix sum over k < N/2).
// This equals the length-2N FFT of the odd extension (the paper's sine series with the wall at
// r = L) at half its arithmetic and memory.  In shared memory S is kept as S_{2k} at [k] and S_{2k+1}
// at [N/2 + k + k/R] (the padded "odd area").
//
// FFT: Stockham autosort with radices R (first pass), MID = N/R^2 in passes of <= 16, R (last).
// Thread g of G = N/(2R) owns butterflies b1 = g, b2 = N/R - g (g = 0: 0 and N/(2R)) of the first
// and last passes, i.e. the indices b + m N/R, m < R.  Those index sets are closed under j -> N - j,
// so the pre- and post-processing, which pair j with N - j, stay inside a thread's registers.
// Shared-memory addresses of the FFT passes are padded by one element every R.
#pragma once
#include "fused_launch.cuh"
#include "qtraj_device.cuh"

namespace qt {

// V selects the launch variant (fused_launch.cuh); variants 2 and 3 use radix 8 for N >= 1024:
// twice the threads per trajectory, half the registers per thread, one more FFT pass.

template <int N, int V = 0> struct FusedPlan {
    // radix 8 up to N = 2048 (passes 8, 16, 8 at N = 1024 and 8, 16, 2, 8 at 2048: +9% each over
    // radix 16's 16, 4, 16 and 16, 8, 16, whose short middle passes and small CTAs cost more
    // instructions per point), 16 above
    static constexpr int R = (N <= 32) ? 4 : (N <= 2048) ? 8 : (V == 2 || V == 3 ? 8 : 16);
    static constexpr int G = N / (2 * R);        // threads per trajectory
    static constexpr int NR = N / R;             // stride of a first/last-pass butterfly
    static constexpr int MID = N / (R * R);      // product of the middle radices
    static constexpr int M1 = MID >= 16 ? 16 : MID;
    static constexpr int M2 = MID / M1;          // 1, 2, 4, 8 or 16
    static constexpr int BUF = N + N / R + 8;    // padded FFT extent; also holds the E/odd layout
    // middle-pass twiddle tables in shared memory, row m holding W^(m k) for the k of every thread
    // (tw1: [M1][R] of W_{R M1}; tw2: [M2][R M1] of W_{R M1 M2}), so that a warp reads consecutive
    // entries.  (A flat table W^t read at t = m k with one pad entry every 8 met up to 7-way bank
    // conflicts at odd m -- 44% of the step's shared-memory conflicts at N = 4096.)
    static constexpr int TW1 = R * M1;
    static constexpr int TW2 = M2 > 1 ? R * M1 * M2 : 0;
    static_assert(N == R * M1 * M2 * R, "plan");
};


// ------------------------------------------------------------------------------------------------
// accumulators: FP32 forms accumulate sums of squares with compensated (cascaded) summation and
// combine partial sums in double-float (error-free transformations in FP32), so no FP64 instruction
// enters the step loop (GB300's FP64 pipe is narrow); FP64 forms accumulate in double.
// ------------------------------------------------------------------------------------------------
struct DF { float hi, lo; };

__device__ __forceinline__ DF two_sum(float a, float b)
{
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
// commutative bit for bit (two_sum is exact; a.lo + b.lo is added first), so xor-butterfly
// reductions leave the same value in every lane
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    DF s = two_sum(a.hi, b.hi);
    const float t = s.lo + (a.lo + b.lo);
    const float hi = s.hi + t;
    return {hi, t - (hi - s.hi)};
}

template <typename T> struct SqAcc;
template <> struct SqAcc<float> {
    DF v{0.f, 0.f};
    // v += w |a|^2 in plain FP32: a thread sums its ~N/G terms of one parity (16 at N = 4096), a
    // relative error of ~sqrt(16) x 6e-8 = 2.4e-7, random from step to step; the sums of the threads
    // are then combined in double-float.  The norm feeds only the waiting-time comparison and the
    // jump's renormalisation, and the FP32 state's own norm error is ~1e-6 per hundred steps, so a
    // compensated per-thread sum (as an earlier revision had) buys nothing the comparison can see.
    __device__ __forceinline__ void add_w(cpx<float> a, float w) { v.hi = fmaf(w, fmaf(a.x, a.x, a.y * a.y), v.hi); }
    __device__ __forceinline__ void shfl_add(unsigned mask, int off, int w)
    {
        DF o{__shfl_xor_sync(mask, v.hi, off, w), __shfl_xor_sync(mask, v.lo, off, w)};
        v = df_add(v, o);
    }
    __device__ __forceinline__ double value() const { return (double)v.hi + (double)v.lo; }
    __device__ __forceinline__ void merge(const SqAcc &o) { v = df_add(v, o.v); }
};
template <> struct SqAcc<double> {
    double v = 0.0;
    __device__ __forceinline__ void merge(const SqAcc &o) { v += o.v; }
    __device__ __forceinline__ void add_w(cpx<double> a, double w) { v = fma(w, fma(a.x, a.x, a.y * a.y), v); }
    __device__ __forceinline__ void shfl_add(unsigned mask, int off, int w) { v += __shfl_xor_sync(mask, v, off, w); }
    __device__ __forceinline__ double value() const { return v; }
};

// compensated complex value for the scan's carries between threads.  Chunk totals use cascaded
// summation (the TwoSum error terms are collected separately); carries between threads are
// double-float additions.  The rounding of a chunk total is added to every later odd coefficient
// (a step in k, energy growing with the number of coefficients after it): with plain FP32 chunk
// totals the no-jump FP32 norm drifted by +7e-9 per step at N = 1024 (against < 5e-9 compensated),
// so the 3% they would save at N = 4096 is not taken.
template <typename T> struct Carry;
template <> struct Carry<float> {
    DF re{0.f, 0.f}, im{0.f, 0.f};
    __device__ __forceinline__ void add(cpx<float> a)
    {
        const DF r = two_sum(re.hi, a.x), i = two_sum(im.hi, a.y);
        re = DF{r.hi, re.lo + r.lo};
        im = DF{i.hi, im.lo + i.lo};
    }
    __device__ __forceinline__ void add(const Carry &o) { re = df_add(re, o.re); im = df_add(im, o.im); }
    __device__ __forceinline__ cpx<float> plus(cpx<float> a) const   // this + a, one rounding of the sum
    {
        return mk((re.hi + a.x) + re.lo, (im.hi + a.y) + im.lo);
    }
    __device__ __forceinline__ Carry shfl_up(unsigned mask, int off, int w) const
    {
        Carry o;
        o.re = DF{__shfl_up_sync(mask, re.hi, off, w), __shfl_up_sync(mask, re.lo, off, w)};
        o.im = DF{__shfl_up_sync(mask, im.hi, off, w), __shfl_up_sync(mask, im.lo, off, w)};
        return o;
    }
};
template <> struct Carry<double> {
    double re = 0.0, im = 0.0;
    __device__ __forceinline__ void add(cpx<double> a) { re += a.x; im += a.y; }
    __device__ __forceinline__ void add(const Carry &o) { re += o.re; im += o.im; }
    __device__ __forceinline__ cpx<double> plus(cpx<double> a) const { return mk(re + a.x, im + a.y); }
    __device__ __forceinline__ Carry shfl_up(unsigned mask, int off, int w) const
    {
        Carry o;
        o.re = __shfl_up_sync(mask, re, off, w);
        o.im = __shfl_up_sync(mask, im, off, w);
        return o;
    }
};

template <int G> __device__ __forceinline__ unsigned lane_mask()
{
    return G >= 32 ? 0xffffffffu : ((1u << G) - 1u);
}

// combines per-warp totals (equal in every lane of a warp) across the G threads of a trajectory in a
// fixed order; red holds >= G/32 doubles
template <int G> __device__ __forceinline__ double cross_warp(double v, double *red)
{
    if constexpr (G > 32) {
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < G / 32; ++w) s += red[w];
        __syncthreads();
        return s;
    } else {
        return v;
    }
}

// sum over the G threads of a trajectory (deterministic order, one value in every thread)
template <int G> __device__ __forceinline__ double slot_sum(double v, double *red)
{
    constexpr int W = G < 32 ? G : 32;
    const unsigned mask = lane_mask<G>();
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off, W);
    if constexpr (G <= 32) v = __shfl_sync(mask, v, 0, W);
    return cross_warp<G>(v, red);
}

// squared norm over the G threads of a trajectory; FP32 forms reduce in double-float all the way and
// convert once, so no FP64 instruction is needed per thread beyond the final conversion
template <typename T, int G> __device__ __forceinline__ double slot_norm(SqAcc<T> acc, double *red)
{
    constexpr int W = G < 32 ? G : 32;
    const unsigned mask = lane_mask<G>();
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) acc.shfl_add(mask, off, W);
    if constexpr (sizeof(T) == 4) {
        DF v = acc.v;
        if constexpr (G <= 32) {
            v.hi = __shfl_sync(mask, v.hi, 0, W);
            v.lo = __shfl_sync(mask, v.lo, 0, W);
        } else {
            DF *fr = reinterpret_cast<DF *>(red);
            if ((threadIdx.x & 31) == 0) fr[threadIdx.x >> 5] = v;
            __syncthreads();
            v = fr[0];
#pragma unroll
            for (int w = 1; w < G / 32; ++w) v = df_add(v, fr[w]);
            __syncthreads();
        }
        return (double)v.hi + (double)v.lo;
    } else {
        double v = acc.value();
        if constexpr (G <= 32) v = __shfl_sync(mask, v, 0, W);
        return cross_warp<G>(v, red);
    }
}

// The norm sum as the step loop compares it with the waiting-time threshold: double-float in the FP32
// forms (so that no FP64 instruction -- a slow pipe on GB300 -- runs in every step), double in FP64.
template <typename T> struct NormSum { using type = double; };
template <> struct NormSum<float> { using type = DF; };

template <typename T, int G> __device__ __forceinline__ typename NormSum<T>::type slot_norm_sum(SqAcc<T> acc, double *red)
{
    if constexpr (sizeof(T) == 4) {
        constexpr int W = G < 32 ? G : 32;
        const unsigned mask = lane_mask<G>();
#pragma unroll
        for (int off = W / 2; off > 0; off >>= 1) acc.shfl_add(mask, off, W);
        DF v = acc.v;
        if constexpr (G <= 32) {
            v.hi = __shfl_sync(mask, v.hi, 0, W);
            v.lo = __shfl_sync(mask, v.lo, 0, W);
        } else {
            DF *fr = reinterpret_cast<DF *>(red);
            if ((threadIdx.x & 31) == 0) fr[threadIdx.x >> 5] = v;
            __syncthreads();
            v = fr[0];
#pragma unroll
            for (int w = 1; w < G / 32; ++w) v = df_add(v, fr[w]);
            __syncthreads();
        }
        return v;
    } else {
        return slot_norm<T, G>(acc, red);
    }
}

// The waiting-time threshold in the form of the norm sum it is compared with: r / dr (the norm is
// dr times the sum), as a normalised double-float in FP32 forms, computed in FP64 once per waiting
// period.  The comparisons are then exact on the double-float values.
template <typename T> struct Threshold;
template <> struct Threshold<double> {
    double thr, dr;
    __device__ void set(double r, double dr_) { thr = r; dr = dr_; }
    __device__ bool finite(double s) const { return isfinite(s * dr); }
    __device__ bool reached(double s) const { return s * dr <= thr; }
    __device__ bool near(double s, double eps) const { return fabs(s * dr - thr) < eps; }
};
template <> struct Threshold<float> {
    DF t;
    float eps_s;
    __device__ void set(double r, double dr)
    {
        const double q = r / dr;
        t.hi = (float)q;
        t.lo = (float)(q - (double)t.hi);
        eps_s = (float)(border_eps<float>() / dr);
    }
    __device__ bool finite(DF s) const { return isfinite(s.hi) && isfinite(s.lo); }
    __device__ bool reached(DF s) const { return s.hi < t.hi || (s.hi == t.hi && s.lo <= t.lo); }
    __device__ bool near(DF s, double) const { return fabsf((s.hi - t.hi) + (s.lo - t.lo)) < eps_s; }
};

// exp(x) and (cos, sin)(pi y): the pi-scaled form has no large-argument reduction path
__device__ __forceinline__ float k_exp(float x) { return expf(x); }
__device__ __forceinline__ double k_exp(double x) { return exp(x); }
__device__ __forceinline__ float k_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double k_expm1(double x) { return expm1(x); }

template <typename T> __device__ __noinline__ T table_T3_far(const double *p, int len, T tau, int *seg)
{
    int s = *seg;
    const T v = table_T3<T>(p, len, tau, s);
    *seg = s;
    return v;
}

// f1 = exp(a) exp(i pi y) - 1, the deviation from 1 of a dynamic factor, for a <= 0 (also returns
// exp(a) - 1).
// FP32: truncated Taylor series at 0 -- exp(a) - 1 to degree 8 for a >= -1/2 (truncation below
// |a|^9/9! <= 5.4e-9), sin(t) to degree 9 and cos(t) - 1 to degree 10 in t = pi y for |t| <= 1
// (truncation below 2.8e-8 and 2.1e-9) -- each accurate relative to the small quantity it returns;
// outside those ranges (large r, where |f1| is no longer small) the library functions.
// FP64: exp and sincospi; a rounding next to 1 is 1e-16 there and does not matter.
template <typename T> struct Dyn;
// the rare points outside the series' ranges, kept out of line so the hot loop stays small
static __device__ __noinline__ float em1_far(float a) { return expf(a) - 1.0f; }
static __device__ __noinline__ void dyn_far(float a, float y, float *em1, float *s, float *cm1)
{
    *em1 = expf(a) - 1.0f;
    float sh, ch;
    sincospif(0.5f * y, &sh, &ch);
    *s = 2.0f * sh * ch;
    *cm1 = -2.0f * sh * sh;
}

template <> struct Dyn<float> {
    static __device__ __forceinline__ void f1(float a, float y, float *fr, float *fi, float *e)
    {
        f1t(a, 3.14159265358979f * y, fr, fi, e);
    }
    // exp(a) - 1 alone (the phase-free factor), the same series and range as f1t
    static __device__ __forceinline__ float em1(float a)
    {
        if (a >= -0.5f) {
            float p = 1.0f / 40320.0f;
            p = fmaf(p, a, 1.0f / 5040.0f);
            p = fmaf(p, a, 1.0f / 720.0f);
            p = fmaf(p, a, 1.0f / 120.0f);
            p = fmaf(p, a, 1.0f / 24.0f);
            p = fmaf(p, a, 1.0f / 6.0f);
            p = fmaf(p, a, 0.5f);
            p = fmaf(p, a, 1.0f);
            return a * p;
        }
        return em1_far(a);
    }
    // the same from the phase t = pi y (the hot loop forms t directly; beyond the series' range y is
    // recomputed from t)
    static __device__ __forceinline__ void f1t(float a, float t, float *fr, float *fi, float *e)
    {
        float em1, s, cm1;
        if (a >= -0.5f && fabsf(t) <= 1.0f) {
            float p = 1.0f / 40320.0f;
            p = fmaf(p, a, 1.0f / 5040.0f);
            p = fmaf(p, a, 1.0f / 720.0f);
            p = fmaf(p, a, 1.0f / 120.0f);
            p = fmaf(p, a, 1.0f / 24.0f);
            p = fmaf(p, a, 1.0f / 6.0f);
            p = fmaf(p, a, 0.5f);
            p = fmaf(p, a, 1.0f);
            em1 = a * p;
            const float u = t * t;
            float ps = 1.0f / 362880.0f;
            ps = fmaf(ps, u, -1.0f / 5040.0f);
            ps = fmaf(ps, u, 1.0f / 120.0f);
            ps = fmaf(ps, u, -1.0f / 6.0f);
            ps = fmaf(ps, u, 1.0f);
            s = t * ps;
            float pc = -1.0f / 3628800.0f;
            pc = fmaf(pc, u, 1.0f / 40320.0f);
            pc = fmaf(pc, u, -1.0f / 720.0f);
            pc = fmaf(pc, u, 1.0f / 24.0f);
            pc = fmaf(pc, u, -0.5f);
            cm1 = u * pc;
        } else {
            dyn_far(a, t * 0.318309886183790672f, &em1, &s, &cm1);
        }
        const float mag = 1.0f + em1;
        *fr = fmaf(cm1, mag, em1);
        *fi = s * mag;
        *e = em1;
    }
    // both points of a pair at once in packed FP32x2 instructions, the same operations per component
    // as f1t / em1 (bit-identical); a pair with a point outside the series' range takes f1t per point
    static __device__ __forceinline__ void f1t2(float2 a, float2 t, float2 *fr, float2 *fi, float2 *e)
    {
        if (a.x >= -0.5f && a.y >= -0.5f && fabsf(t.x) <= 1.0f && fabsf(t.y) <= 1.0f) {
            float2 p = __ffma2_rn(make_float2(1.0f / 40320.0f, 1.0f / 40320.0f), a, make_float2(1.0f / 5040.0f, 1.0f / 5040.0f));
            p = __ffma2_rn(p, a, make_float2(1.0f / 720.0f, 1.0f / 720.0f));
            p = __ffma2_rn(p, a, make_float2(1.0f / 120.0f, 1.0f / 120.0f));
            p = __ffma2_rn(p, a, make_float2(1.0f / 24.0f, 1.0f / 24.0f));
            p = __ffma2_rn(p, a, make_float2(1.0f / 6.0f, 1.0f / 6.0f));
            p = __ffma2_rn(p, a, make_float2(0.5f, 0.5f));
            p = __ffma2_rn(p, a, make_float2(1.0f, 1.0f));
            const float2 em1 = __fmul2_rn(a, p);
            const float2 u = __fmul2_rn(t, t);
            float2 ps = __ffma2_rn(make_float2(1.0f / 362880.0f, 1.0f / 362880.0f), u, make_float2(-1.0f / 5040.0f, -1.0f / 5040.0f));
            ps = __ffma2_rn(ps, u, make_float2(1.0f / 120.0f, 1.0f / 120.0f));
            ps = __ffma2_rn(ps, u, make_float2(-1.0f / 6.0f, -1.0f / 6.0f));
            ps = __ffma2_rn(ps, u, make_float2(1.0f, 1.0f));
            const float2 s = __fmul2_rn(t, ps);
            float2 pc = __ffma2_rn(make_float2(-1.0f / 3628800.0f, -1.0f / 3628800.0f), u, make_float2(1.0f / 40320.0f, 1.0f / 40320.0f));
            pc = __ffma2_rn(pc, u, make_float2(-1.0f / 720.0f, -1.0f / 720.0f));
            pc = __ffma2_rn(pc, u, make_float2(1.0f / 24.0f, 1.0f / 24.0f));
            pc = __ffma2_rn(pc, u, make_float2(-0.5f, -0.5f));
            const float2 cm1 = __fmul2_rn(u, pc);
            const float2 mag = __fadd2_rn(make_float2(1.0f, 1.0f), em1);
            *fr = __ffma2_rn(cm1, mag, em1);
            *fi = __fmul2_rn(s, mag);
            *e = em1;
        } else {
            f1t(a.x, t.x, &fr->x, &fi->x, &e->x);
            f1t(a.y, t.y, &fr->y, &fi->y, &e->y);
        }
    }
    static __device__ __forceinline__ float2 em1_2(float2 a)
    {
        if (a.x >= -0.5f && a.y >= -0.5f) {
            float2 p = __ffma2_rn(make_float2(1.0f / 40320.0f, 1.0f / 40320.0f), a, make_float2(1.0f / 5040.0f, 1.0f / 5040.0f));
            p = __ffma2_rn(p, a, make_float2(1.0f / 720.0f, 1.0f / 720.0f));
            p = __ffma2_rn(p, a, make_float2(1.0f / 120.0f, 1.0f / 120.0f));
            p = __ffma2_rn(p, a, make_float2(1.0f / 24.0f, 1.0f / 24.0f));
            p = __ffma2_rn(p, a, make_float2(1.0f / 6.0f, 1.0f / 6.0f));
            p = __ffma2_rn(p, a, make_float2(0.5f, 0.5f));
            p = __ffma2_rn(p, a, make_float2(1.0f, 1.0f));
            return __fmul2_rn(a, p);
        }
        return make_float2(em1(a.x), em1(a.y));
    }
};
template <> struct Dyn<double> {
    static __device__ __forceinline__ void f1(double a, double y, double *fr, double *fi, double *e)
    {
        const double mag = exp(a);
        double s, c;
        sincospi(y, &s, &c);
        *fr = mag * c - 1.0;
        *fi = mag * s;
        *e = mag - 1.0;
    }
};
__device__ __forceinline__ void k_sincospi(float y, float *s, float *c) { sincospif(y, s, c); }
__device__ __forceinline__ void k_sincospi(double y, double *s, double *c) { sincospi(y, s, c); }

// static factor of a (colour, l) row beyond the table (l >= LTAB, some 33,000 jumps from l = 0),
// evaluated in FP64; span 1 = half step, 2 = full step
template <typename T>
__device__ __noinline__ typename Prec<T>::S static_far(double coul, double M, double dt, int l, double r, double span)
{
    const double V = coul / r + (double)l * (l + 1) / (M * r * r);
    double s, c;
    sincos(-V * dt * 0.5 * span, &s, &c);
    return Prec<T>::make_s(c, s);
}

// ------------------------------------------------------------------------------------------------
// the isotropic KSU potential (App. E): per-step scalars at one temperature and the per-point
// dynamic part V_R + a/r (the Cornell -a/r sits in the static factor) and V_I
// ------------------------------------------------------------------------------------------------
template <typename T> struct KsuT {
    T m;      // Debye mass m_D(T)
    T two_s;  // 2 sigma / m_D
    T gI;     // alpha_s(2 pi T) C_F T: V_I = -gI phi(m_D r)
};

__device__ __forceinline__ float k_log(float x) { return logf(x); }
__device__ __forceinline__ double k_log(double x) { return log(x); }
__device__ __forceinline__ float k_cbrt(float x) { return cbrtf(x); }
__device__ __forceinline__ double k_cbrt(double x) { return cbrt(x); }

template <typename T> __device__ __forceinline__ KsuT<T> ksu_at(const Tables<T> &tb, T T3)
{
    const T Tt = k_cbrt(T3);
    const T mu = (T)6.28318530717958647692 * Tt;
    const T as = tb.ksu_alpha0 / ((T)1 + tb.ksu_alpha0 * tb.ksu_b0 * k_log(mu * mu / tb.ksu_mu0sq));
    const T m = Tt * sqrt(tb.ksu_md2 * as);
    return {m, tb.ksu_two_sigma / m, as * tb.ksu_cf * Tt};
}

// phi(x) of V_I: the small-argument series below KSU_PHI_A0, cubic Hermite interpolation of the
// table up to KSU_PHI_A1, the asymptotic series 1 - sum_j (2j)! (2j+2) / x^(2j+2) above
template <typename T> __device__ __forceinline__ T ksu_phi(const Tables<T> &tb, T x)
{
    if (x < (T)KSU_PHI_A0) {
        const T y = x * x;
        T pl = (T)0, pc = (T)0;
#pragma unroll
        for (int k = KSU_PHI_SER - 1; k >= 0; --k) {
            pl = (pl + tb.phi_ser[2 * k]) * y;
            pc = (pc + tb.phi_ser[2 * k + 1]) * y;
        }
        return x > (T)0 ? -(pl * k_log(x) + pc) : (T)0;
    }
    if (x < (T)KSU_PHI_A1) {
        const T u = (x - (T)KSU_PHI_A0) * (T)KSU_PHI_PER;
        int i = (int)u;
        if (i > KSU_PHI_NODES - 2) i = KSU_PHI_NODES - 2;
        const T s = u - (T)i, s2 = s * s, s3 = s2 * s;
        const T *n = tb.phi_tab + 2 * i;
        const T h00 = (T)2 * s3 - (T)3 * s2 + (T)1, h10 = s3 - (T)2 * s2 + s, h01 = (T)3 * s2 - (T)2 * s3, h11 = s3 - s2;
        return h00 * n[0] + h10 * n[1] + h01 * n[2] + h11 * n[3];
    }
    const T q = (T)1 / (x * x);
    T p = (T)6706022400.0;
    p = fma(p, q, (T)43545600.0);
    p = fma(p, q, (T)403200.0);
    p = fma(p, q, (T)5760.0);
    p = fma(p, q, (T)144.0);
    p = fma(p, q, (T)8.0);
    p = fma(p, q, (T)2.0);
    return (T)1 - p * q;
}

// at grid point j > 0 and one temperature: vd = V_R + a/r (V_R = min(KMS, V_vac(r_SB))) and vi = V_I
template <typename T> __device__ __forceinline__ void ksu_point(const Tables<T> &tb, const KsuT<T> &k, T fj, T &vd, T &vi)
{
    const T aor = tb.ksu_a_dr / fj, r_sig = tb.ksu_sig_dr * fj;     // a/r, sigma r
    const T x = k.m * (fj * (T)tb.dr);
    const T e = exp(-x);
    // 1 - (1 + x) e^-x, by its series below 0.05 (the difference cancels there)
    T g;
    if (x < (T)0.05) {
        T p = (T)(-1.0 / 3991680.0);              // the terms (-1)^n (n-1) x^n / n!, n = 2 .. 11
        p = fma(p, x, (T)(1.0 / 403200.0));
        p = fma(p, x, (T)(-1.0 / 45360.0));
        p = fma(p, x, (T)(1.0 / 5760.0));
        p = fma(p, x, (T)(-1.0 / 840.0));
        p = fma(p, x, (T)(1.0 / 144.0));
        p = fma(p, x, (T)(-1.0 / 30.0));
        p = fma(p, x, (T)(1.0 / 8.0));
        p = fma(p, x, (T)(-1.0 / 3.0));
        p = fma(p, x, (T)0.5);
        g = p * x * x;
    } else {
        g = (T)1 - ((T)1 + x) * e;
    }
    vd = aor * g + k.two_s * ((T)1 - e) - r_sig * e;   // KMS + a/r
    if (vd - aor > tb.ksu_cap) vd = tb.ksu_cap + aor;  // the string-breaking cap
    vi = -k.gI * ksu_phi(tb, x);
}

// in-place DFT of RR values (natural order in); output k lands in slot operm(k); PK: packed products
template <typename T, int RR, bool PK = false> struct DFTI {
    static __device__ __forceinline__ constexpr int operm(int k)
    {
        if constexpr (RR == 16) return (k % 4) * 4 + k / 4;
        else if constexpr (RR == 8) return (k % 4) * 2 + k / 4;
        else return k;
    }
    static __device__ __forceinline__ void run(cpx<T> *x)
    {
        if constexpr (RR == 16) {
#pragma unroll
            for (int n2 = 0; n2 < 4; ++n2) {
                dft4(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);       // k1 of column n2 at slot n2 + 4 k1
                x[4 + n2] = tw16<T, PK>(x[4 + n2], n2 * 1);
                x[8 + n2] = tw16<T, PK>(x[8 + n2], n2 * 2);
                x[12 + n2] = tw16<T, PK>(x[12 + n2], n2 * 3);
            }
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) dft4(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
        } else if constexpr (RR == 8) {
#pragma unroll
            for (int n2 = 0; n2 < 2; ++n2) {
                dft4(x[n2], x[2 + n2], x[4 + n2], x[6 + n2]);        // k1 of column n2 at slot n2 + 2 k1
                x[2 + n2] = tw16<T, PK>(x[2 + n2], 2 * n2 * 1);
                x[4 + n2] = tw16<T, PK>(x[4 + n2], 2 * n2 * 2);
                x[6 + n2] = tw16<T, PK>(x[6 + n2], 2 * n2 * 3);
            }
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) dft2(x[2 * k1], x[2 * k1 + 1]);
        } else if constexpr (RR == 4) {
            dft4(x[0], x[1], x[2], x[3]);
        } else if constexpr (RR == 2) {
            dft2(x[0], x[1]);
        }
    }
};

// ------------------------------------------------------------------------------------------------
// the sine transform
// ------------------------------------------------------------------------------------------------
template <typename T, int N, int V> struct Fused {
    using P = FusedPlan<N, V>;
    using PR = Prec<T>;
    using C = typename Prec<T>::C;
    using RL = typename Prec<T>::Rl;
    static constexpr int R = P::R, G = P::G, NR = P::NR, E = 2 * R;
    // FP32 at N >= 8192: the hi+lo complex products (pass twiddles, kinetic factors, DFT constants) as
    // packed FP32x2 instructions -- +9% at N = 8192 and +12% at 16384 over the scalar products, which
    // stay faster at N <= 4096 (-6% at 4096 with the packed form); the results are bit-identical
    static constexpr bool PK = sizeof(T) == 4 && N >= 8192;
    using DR = DFTI<T, R, PK>;
    static __device__ __forceinline__ cpx<T> cmul(cpx<T> x, C w) { return PK ? PR::mul2(x, w) : PR::mul(x, w); }

    static __device__ __forceinline__ int pad(int j) { return j + j / R; }
    // E/odd layout of the transform's output (and of the state between transforms): S_{2k} at
    // even_pos(k), S_{2k+1} at odd_pos(k).  (An XOR swizzle of both areas, meant to spread the
    // even/odd lanes of the transform's load over all banks, measured 0.4-4.6% slower.)
    static __device__ __forceinline__ int even_pos(int k) { return k; }
    static __device__ __forceinline__ int odd_pos(int k) { return N / 2 + k + k / R; }
    static __device__ __forceinline__ int b_of(int g, int t) { return t == 0 ? (g == 0 ? 0 : g) : (g == 0 ? NR / 2 : NR - g); }
    // global index of register element e (first/last-pass layout)
    static __device__ __forceinline__ int idx(int g, int e) { return b_of(g, e / R) + (e % R) * NR; }
    // shared-memory position of S_j in the E/odd layout
    static __device__ __forceinline__ int s_pos(int j) { return (j & 1) ? odd_pos(j >> 1) : even_pos(j >> 1); }

    // y_j = s (f_j + f_{N-j}) + (f_j - f_{N-j})/2 for the pair (ea, eb) = (j, N-j)
    static __device__ __forceinline__ void pre_pair(cpx<T> *x, int ea, int eb, RL s)
    {
        const cpx<T> a = x[ea], b = x[eb];
        const cpx<T> sum = PR::mulr(a + b, s), dif = scale(a - b, (T)0.5);
        x[ea] = sum + dif;
        x[eb] = sum - dif;
    }

    static __device__ __forceinline__ void pre(cpx<T> *x, int g, const RL *sinpre)
    {
        if (g != 0) {
#pragma unroll
            for (int m = 0; m < R; ++m) pre_pair(x, m, R + (R - 1 - m), PR::ldr(&sinpre[g + m * NR]));
        } else {
            x[0] = mk<T>(0, 0);                                // j = 0
            x[R / 2] = scale(x[R / 2], (T)2);                  // j = N/2 pairs with itself, sin = 1
#pragma unroll
            for (int m = 1; m < R / 2; ++m) pre_pair(x, m, R - m, PR::ldr(&sinpre[m * NR]));
#pragma unroll
            for (int m = 0; m < R / 2; ++m) pre_pair(x, R + m, R + (R - 1 - m), PR::ldr(&sinpre[NR / 2 + m * NR]));
        }
    }

    // E_k = (i/2)(Y_k - Y_{N-k}) -> [k];  C_k = (Y_k + Y_{N-k})/2 (C_0 halved) -> odd area
    static __device__ __forceinline__ void post_pair(cpx<T> *buf, int k, cpx<T> A, cpx<T> B)
    {
        buf[even_pos(k)] = mul_i(scale(A - B, (T)0.5));
        buf[odd_pos(k)] = scale(A + B, (T)0.5);
    }

    // Y at index b_t + m NR is in register slot t R + operm(m) after the last pass
    static __device__ __forceinline__ cpx<T> Y(const cpx<T> *x, int t, int m) { return x[t * R + DR::operm(m)]; }

    static __device__ __forceinline__ void post(const cpx<T> *x, int g, cpx<T> *buf)
    {
        if (g != 0) {
#pragma unroll
            for (int m = 0; m < R; ++m) {
                if (m < R / 2) post_pair(buf, g + m * NR, Y(x, 0, m), Y(x, 1, R - 1 - m));
                else post_pair(buf, (NR - g) + (R - 1 - m) * NR, Y(x, 1, R - 1 - m), Y(x, 0, m));
            }
        } else {
            buf[even_pos(0)] = mk<T>(0, 0);
            buf[odd_pos(0)] = scale(Y(x, 0, 0), (T)0.5);      // S_1 = C_0 / 2 = Y_0 / 2
#pragma unroll
            for (int m = 1; m < R / 2; ++m) post_pair(buf, m * NR, Y(x, 0, m), Y(x, 0, R - m));
#pragma unroll
            for (int m = 0; m < R / 2; ++m) post_pair(buf, NR / 2 + m * NR, Y(x, 1, m), Y(x, 1, R - 1 - m));
        }
    }

    // inclusive prefix sum of the N/2 odd-area values: thread g owns the chunk k in [gR, gR + R).
    // Chunk totals and the carries between chunks are compensated (a rounding error there would reach
    // every later coefficient); the running sum inside a chunk is plain and only reaches its chunk.
    static __device__ __forceinline__ void scan(cpx<T> *buf, int g, Carry<T> *wtot)
    {
        constexpr int W = G < 32 ? G : 32;
        const unsigned mask = lane_mask<G>();
        cpx<T> v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = buf[odd_pos(g * R + q)];
        Carry<T> tot;
#pragma unroll
        for (int q = 0; q < R; ++q) tot.add(v[q]);
        const int lane = threadIdx.x & (W - 1);
        Carry<T> inc = tot;
#pragma unroll
        for (int off = 1; off < W; off <<= 1) {
            Carry<T> y = inc.shfl_up(mask, off, W);
            if (lane >= off) inc.add(y);
        }
        Carry<T> excl = inc.shfl_up(mask, 1, W);
        if (lane == 0) excl = Carry<T>();
        if constexpr (G > 32) {
            const int warp = threadIdx.x >> 5;
            if (lane == 31) wtot[warp] = inc;
            __syncthreads();
#pragma unroll 1
            for (int w = 0; w < warp; ++w) excl.add(wtot[w]);
        }
        cpx<T> run = mk<T>(0, 0);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            run = run + v[q];
            buf[odd_pos(g * R + q)] = excl.plus(run);
        }
    }

    // One middle pass (radix RM after PP points): butterfly i reads [i + m N/RM], multiplies by
    // W_{PP RM}^{m k} (k = i mod PP) and writes [(i - k) RM + k + m PP].  A thread's butterflies are
    // g + q G; when PP <= G they share k = g mod PP and so their twiddles, which are loaded once per m
    // (from tw, the table [RM][PP] of W_{PP RM}^{m k}).
    template <int RM, int PP>
    static __device__ __forceinline__ void mid_pass(cpx<T> *x, cpx<T> *buf, const C *tw, int g)
    {
        if constexpr (RM > 1) {
            constexpr int NB = N / RM, PER = E / RM;
            static_assert(PP <= G, "mid-pass twiddle sharing needs PP <= G");
            const int k = g & (PP - 1);
#pragma unroll
            for (int m = 0; m < RM; ++m) {
                C w{};
                if (m) w = tw_at(tw, m * PP + k);
#pragma unroll
                for (int q = 0; q < PER; ++q) {
                    cpx<T> v = buf[pad(g + q * G + m * NB)];
                    if (m) v = cmul(v, w);
                    x[q * RM + m] = v;
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int i = g + q * G;
                DFTI<T, RM, PK>::run(x + q * RM);
                const int base = (i - k) * RM + k;
#pragma unroll
                for (int m = 0; m < RM; ++m) buf[pad(base + m * PP)] = x[q * RM + DFTI<T, RM, PK>::operm(m)];
            }
            __syncthreads();
        }
    }

    // twiddle tables of the middle passes live in shared memory (FusedPlan: TW1, TW2); an FP32 entry
    // (hi+lo, 16 bytes) is one 16-byte load
    static __device__ __forceinline__ C tw_at(const C *tw, int i)
    {
        if constexpr (sizeof(T) == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(tw + i);
            return C{v.x, v.y, v.z, v.w};
        } else {
            return tw[i];
        }
    }

    // S (E/odd layout in buf), optionally times K_T, at the first-pass indices -> DST -> E/odd layout
    static __device__ __forceinline__ void dst(cpx<T> *x, cpx<T> *buf, const Tables<T> &tb, int g, Carry<T> *wtot,
                                               const C *tw1, const C *tw2, bool kinetic)
    {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int j = idx(g, e);
            cpx<T> v = buf[s_pos(j)];
            if (kinetic) v = cmul(v, PR::ld(&tb.KT[j]));
            x[e] = v;
        }
        __syncthreads();
        pre(x, g, tb.sinpre);
        // first pass (radix R, no twiddles): butterfly b -> [b R + k]
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            DR::run(x + t * R);
            const int b = b_of(g, t);
#pragma unroll
            for (int k = 0; k < R; ++k) buf[pad(b * R + k)] = x[t * R + DR::operm(k)];
        }
        __syncthreads();
        mid_pass<P::M1, R>(x, buf, tw1, g);
        mid_pass<P::M2, R * P::M1>(x, buf, tw2, g);
        // last pass (radix R, stride N/R): inputs [b + m NR], twiddle W^(m b).  For the mirror butterfly
        // b2 = NR - g, W^(m b2) = W_R^m conj(W^(m g)): one table load serves both (g = 0 pairs
        // 0 with NR/2, whose twiddles are loaded directly).
#pragma unroll
        for (int m = 0; m < R; ++m) {
            cpx<T> v1 = buf[pad(b_of(g, 0) + m * NR)];
            cpx<T> v2 = buf[pad(b_of(g, 1) + m * NR)];
            if (m) {
                // W^(m g): up to N = 2048 from the radix's compact [m][g] section (a warp reads
                // consecutive entries; measured +3% at N = 1024, +6.5% at 2048), above from the
                // strided W[m g] (the compact table measured 9% slower at N = 4096, 1% at 16384)
                const C w = N <= 2048 ? PR::ld(&tb.WL[(R == 16 ? 0 : R == 8 ? N / 2 : N) + m * G + g])
                                      : PR::ld(&tb.W[m * g]);
                v1 = cmul(v1, w);
                if (g != 0) {
                    v2 = tw16<T, PK>(cmul(v2, PR::conj(w)), m * (16 / R));
                } else {
                    v2 = cmul(v2, PR::ld(&tb.W[m * (NR / 2)]));
                }
            }
            x[m] = v1;
            x[R + m] = v2;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 2; ++t) DR::run(x + t * R);
        post(x, g, buf);
        __syncthreads();
        scan(buf, g, wtot);
        __syncthreads();
    }
};

// ------------------------------------------------------------------------------------------------
// pointwise work on the E/odd layout: thread g visits k = g, g + G, ... < N/2 and the two elements
// S_{2k} (at even_pos(k) = k) and S_{2k+1} (at odd_pos(k))
// ------------------------------------------------------------------------------------------------
template <typename T, int N, int V> struct Pointwise {
    using K = Fused<T, N, V>;
    static constexpr bool PD = sizeof(T) == 4 && N >= 2048 && N <= 8192;
    using PR = Prec<T>;
    using C = typename Prec<T>::C;
    static constexpr int G = K::G;

    using SC = typename Prec<T>::S;
    static __device__ __forceinline__ SC stat(const Tables<T> &tb, const SC *tab, int c, int l, int j, bool full)
    {
        if (l < LTAB) return PR::ld_s(&tab[((size_t)c * LTAB + l) * N + j]);
        if (j == 0) return PR::make_s(0.0, 0.0);
        return static_far<T>(tb.coul[c], tb.M, tb.dt, l, j * tb.dr, full ? 2.0 : 1.0);
    }

    // mode 0: x <- stat1 dyn_b x (the first half-step of a trajectory)
    // mode 1: x <- stat2 dyn_a dyn_b x; returns sum exp(2 er_a r^2) |x_old|^2 (end-of-step norm / dr)
    // mode 2: x <- stat1 dyn_a x; returns sum |x_new|^2
    // dyn = exp((er + i ei) r^2), er and ei multiplied by T^3.  The caller passes the summed
    // coefficients times dr^2 (phase / pi): A for the magnitude, B for the phase, D = (er_a - er_b) dr^2
    // for the norm weight; they are rounded once per step and multiply the exact j twice, so no
    // rounding that repeats identically every step enters the arguments.
    static __device__ typename NormSum<T>::type factor(cpx<T> *buf, const Tables<T> &tb, int g, int c, int l, int mode,
                                                       T A, T B, T D, double *red)
    {
        SqAcc<T> acc, acc_odd;   // even and odd j accumulate separately (two dependency chains)
        // a medium with gamma_hat = 0 has no dynamic phase (B = 0 exactly): the FP32 form then skips
        // the sine and cosine series, whose value would be exactly 0 -- the same arithmetic
        if (sizeof(T) == 4 && B == (T)0) factor_pts<false>(buf, tb, g, c, l, mode, A, B, D, acc, acc_odd);
        else factor_pts<true>(buf, tb, g, c, l, mode, A, B, D, acc, acc_odd);
        if (mode == 0) return {};
        acc.merge(acc_odd);
        return slot_norm_sum<T, G>(acc, red);
    }

    // The KSU counterpart of factor (same modes, same w + w f1 form): the dynamic exponent of the
    // half-step at temperature T is (V_I - i (V_R + a/r)) dt/2 at each point, evaluated per point;
    // ka, kb are the per-step scalars of T_n (the closing half-step) and T_{n+1} (the opening one).
    static __device__ typename NormSum<T>::type factor_ksu(cpx<T> *buf, const Tables<T> &tb, int g, int l, int mode,
                                                           const KsuT<T> &ka, const KsuT<T> &kb, double *red)
    {
        SqAcc<T> acc, acc_odd;
        const SC *tab = (mode == 1) ? tb.statV2 : tb.statV;
        const T hdt = (T)0.5 * tb.ksu_dt;
#pragma unroll 1
        for (int k = g; k < N / 2; k += G) {
#pragma unroll
            for (int par = 0; par < 2; ++par) {
                const int j = 2 * k + par;
                const int p = par ? K::odd_pos(k) : K::even_pos(k);
                const T fj = (T)j;
                T A = (T)0, t = (T)0, z = (T)0;
                if (j > 0) {
                    T vda = (T)0, via = (T)0, vdb = (T)0, vib = (T)0;
                    if (mode != 0) ksu_point<T>(tb, ka, fj, vda, via);
                    if (mode != 2) ksu_point<T>(tb, kb, fj, vdb, vib);
                    A = (via + vib) * hdt;
                    t = -(vda + vdb) * hdt;
                    z = (via - vib) * hdt;   // |K_V(n)|^2 = exp(A + z)
                }
                T f1r, f1i, em1;
                if constexpr (sizeof(T) == 4) Dyn<T>::f1t(A, t, &f1r, &f1i, &em1);
                else Dyn<T>::f1(A, t * (T)0.318309886183790671537767526745, &f1r, &f1i, &em1);
                const T mag = (T)1 + em1;
                cpx<T> v = buf[p];
                SqAcc<T> &ac = par ? acc_odd : acc;
                if (mode == 1) ac.add_w(v, mag * exp(z));
                const cpx<T> w = PR::mul_s(v, stat(tb, tab, 0, l, j, mode == 1));
                v = mk(w.x + (w.x * f1r - w.y * f1i), w.y + (w.x * f1i + w.y * f1r));
                if (mode == 2) ac.add_w(v, (T)1);
                buf[p] = v;
            }
        }
        if (mode == 0) return {};
        acc.merge(acc_odd);
        return slot_norm_sum<T, G>(acc, red);
    }

    template <bool phase>
    static __device__ __forceinline__ void factor_pts(cpx<T> *buf, const Tables<T> &tb, int g, int c, int l, int mode,
                                                      T A, T B, T D, SqAcc<T> &acc, SqAcc<T> &acc_odd)
    {
        const SC *tab = (mode == 1) ? tb.statV2 : tb.statV;
        const T Bpi = (T)3.14159265358979323846 * B;   // the phase coefficient: t = pi B j^2
#pragma unroll 2
        for (int k = g; k < N / 2; k += G) {
            // FP32 at N = 2048 .. 8192: the series of the pair (2k, 2k+1) in packed FP32x2 instructions
            // (bit-identical; +1.6% / +2.4% / +0.7% at N = 2048 / 4096 / 8192, -0.9% at 1024 and 16384)
            float2 F1R, F1I = make_float2(0.f, 0.f), EM1, Z;
            if constexpr (PD) {
                const float j0 = (float)(2 * k), j1 = (float)(2 * k + 1);
                const float2 j2 = __fmul2_rn(make_float2(j0, j1), make_float2(j0, j1));
                const float2 a2 = __fmul2_rn(make_float2(A, A), j2);
                if (phase) {
                    Dyn<float>::f1t2(a2, __fmul2_rn(make_float2(Bpi, Bpi), j2), &F1R, &F1I, &EM1);
                } else {
                    EM1 = Dyn<float>::em1_2(a2);
                    F1R = EM1;
                }
                Z = __fmul2_rn(make_float2(D, D), j2);
            }
#pragma unroll
            for (int par = 0; par < 2; ++par) {
                const int j = 2 * k + par;
                const int p = par ? K::odd_pos(k) : K::even_pos(k);
                const T fj = (T)j;
                // the dynamic factor exp(a) exp(i pi y) is close to 1 and changes little from step to
                // step; it is applied as w + w f1 with f1 its deviation from 1, evaluated so that the
                // rounding is relative to f1, not to 1 (a rounding of a value next to 1 would repeat
                // identically every step and add up)
                T f1r, f1i = (T)0, em1;
                T z = (T)0;
                if constexpr (PD) {
                    f1r = par ? F1R.y : F1R.x;
                    f1i = par ? F1I.y : F1I.x;
                    em1 = par ? EM1.y : EM1.x;
                    z = par ? Z.y : Z.x;
                } else if constexpr (sizeof(T) == 4) {
                    // j^2 is exact in FP32 up to N = 4096 (and rounded once above); the coefficients
                    // change every step, so no rounding of a, t or z repeats from step to step
                    const T j2 = fj * fj;
                    if (phase) {
                        Dyn<T>::f1t(A * j2, Bpi * j2, &f1r, &f1i, &em1);
                    } else {   // gamma_hat = 0: the phase is 0 and f1 = exp(a) - 1 exactly as f1t gives it
                        em1 = Dyn<T>::em1(A * j2);
                        f1r = em1;
                    }
                    z = D * j2;
                } else {
                    Dyn<T>::f1((A * fj) * fj, (B * fj) * fj, &f1r, &f1i, &em1);
                    z = (D * fj) * fj;
                }
                const T mag = (T)1 + em1;   // |exp(a)|, for the norm weight (working precision suffices)
                cpx<T> v = buf[p];
                SqAcc<T> &ac = par ? acc_odd : acc;
                if (mode == 1) {
                    // exp(2 er_a r^2) = mag * exp((er_a - er_b) r^2), the second factor 1 + z with
                    // |z| <~ 1e-4 (the temperature's change over one step): FP32 keeps the first order
                    // (z^2 / 2 < 1e-8 is below its rounding), FP64 the series to z^3
                    if constexpr (sizeof(T) == 4) ac.add_w(v, mag + mag * z);
                    else ac.add_w(v, mag * ((T)1 + z * ((T)1 + z * ((T)0.5 + z * (T)(1.0 / 6.0)))));
                }
                const cpx<T> w = PR::mul_s(v, stat(tb, tab, c, l, j, mode == 1));
                if constexpr (sizeof(T) == 4) {   // w + w f1, fused
                    v = phase ? mk(fmaf(w.x, f1r, fmaf(-w.y, f1i, w.x)), fmaf(w.y, f1r, fmaf(w.x, f1i, w.y)))
                              : mk(fmaf(w.x, f1r, w.x), fmaf(w.y, f1r, w.y));
                } else {
                    v = mk(w.x + (w.x * f1r - w.y * f1i), w.y + (w.x * f1i + w.y * f1r));
                }
                if (mode == 2) ac.add_w(v, (T)1);
                buf[p] = v;
            }
        }
    }

    static __device__ cpx<double> to_d(const typename Prec<double>::C &a) { return a; }
    static __device__ cpx<double> to_d(const typename Prec<float>::C &a)
    {
        return mk((double)a.rh + (double)a.rl, (double)a.ih + (double)a.il);
    }

    // A jump after the factor of mode 1 (more steps follow) or mode 2 (after the last step).
    // Returns sum r^2 |end-of-step state|^2 (/ dr); with mode 1 the end-of-step state is
    // exp(-er_b r^2) times the stored one.  With mode 1 it also turns the start half-step already
    // applied from (c, l) into (c2, l2): x <- conj(stat1(c,l)) stat1(c2,l2) exp(d_er r^2 + i d_ei r^2) x.
    // The coefficients come times dr^2 (the phase also / pi) and multiply j^2: w2 = -2 er_b dr^2,
    // A = d_er dr^2, B = d_ei dr^2 / pi.  A one-off factor, so working precision suffices.
    static __device__ double jump_turn(cpx<T> *buf, const Tables<T> &tb, int g, int c, int l, int c2, int l2,
                                       bool after_last, T w2, T A, T B, double *red)
    {
        const T dr2 = (T)(tb.dr * tb.dr);
        SqAcc<T> acc;
        for (int k = g; k < N / 2; k += G) {
            for (int par = 0; par < 2; ++par) {
                const int j = 2 * k + par;
                const int p = par ? K::odd_pos(k) : K::even_pos(k);
                const T fj = (T)j, j2 = fj * fj;
                cpx<T> v = buf[p];
                if (after_last) {
                    acc.add_w(v, dr2 * j2);
                } else {
                    acc.add_w(v, dr2 * j2 * k_exp(w2 * j2));
                    v = PR::mul_s(PR::mul_s(v, PR::conj_s(stat(tb, tb.statV, c, l, j, false))), stat(tb, tb.statV, c2, l2, j, false));
                    T sn, cs;
                    k_sincospi(B * j2, &sn, &cs);
                    const T m = k_exp(A * j2);
                    v = v * mk(m * cs, m * sn);
                    buf[p] = v;
                }
            }
        }
        return slot_norm<T, G>(acc, red);
    }

    // Per-step summary row of the end-of-step state e = stat1 exp(A j^2 + i pi B j^2) x, x the state
    // before the closing half-step (A = erj K3, B = eij T3 of the step): norm, <r>, overlaps, FP64
    // accumulation; thread 0 writes the row.  One pass for the norm and <r> and one per basis state
    // of the same l, so that few values stay live.  Only in the traced kernel (V = 4).
    static __device__ __forceinline__ cpx<double> end_value(const cpx<T> *buf, const Tables<T> &tb, int c, int l, int j,
                                                            int p, T A, T B)
    {
        const T fj = (T)j;
        T f1r, f1i, em1;
        Dyn<T>::f1((A * fj) * fj, (B * fj) * fj, &f1r, &f1i, &em1);
        const cpx<T> w = PR::mul_s(buf[p], stat(tb, tb.statV, c, l, j, false));
        return mk((double)(w.x + (w.x * f1r - w.y * f1i)), (double)(w.y + (w.x * f1i + w.y * f1r)));
    }

    static __device__ void trace_row(const cpx<T> *buf, const Tables<T> &tb, int g, int c, int l, T A, T B,
                                     double *red, qtraj_trace_rec *out, int step)
    {
        double n2 = 0.0, rr = 0.0;
        for (int k = g; k < N / 2; k += G)
            for (int par = 0; par < 2; ++par) {
                const int j = 2 * k + par;
                const cpx<double> e = end_value(buf, tb, c, l, j, par ? K::odd_pos(k) : K::even_pos(k), A, B);
                const double m2 = e.x * e.x + e.y * e.y;
                n2 += m2;
                rr += (double)j * tb.dr * m2;
            }
        n2 = slot_sum<G>(n2, red);
        rr = slot_sum<G>(rr, red);
        const double dr = tb.dr;
        if (g == 0) {
            out->step = step;
            out->color = c;
            out->l = l;
            out->flags = 0;
            out->norm2 = n2 * dr;
            out->r_ratio = (rr / n2) / tb.r1s;
        }
#pragma unroll 1
        for (int s = 0; s < NBASIS; ++s) {
            const int bl = s == 2 || s == 4 ? 1 : (s == 5 ? 2 : 0);
            double vr = 0.0, vi = 0.0;
            if (c == 0 && bl == l) {
                for (int k = g; k < N / 2; k += G)
                    for (int par = 0; par < 2; ++par) {
                        const int j = 2 * k + par;
                        const cpx<double> e = end_value(buf, tb, c, l, j, par ? K::odd_pos(k) : K::even_pos(k), A, B);
                        const double ph = tb.eig[(size_t)s * N + j];
                        vr += ph * e.x;
                        vi += ph * e.y;
                    }
                vr = slot_sum<G>(vr, red);
                vi = slot_sum<G>(vi, red);
            }
            if (g == 0) out->ov2[s] = (vr * vr + vi * vi) * dr / n2;
        }
    }

    // Undoes the start half-step applied by a mode-1 factor, x <- conj(stat1(c,l)) exp(A j^2 + i pi B j^2) x
    // with A = -er_b dr^2 and B = -ei_b dr^2 / pi: the end-of-step state of a trajectory that stops
    // at a jump cap.
    static __device__ void undo_start(cpx<T> *buf, const Tables<T> &tb, int g, int c, int l, T A, T B)
    {
        for (int k = g; k < N / 2; k += G) {
            for (int par = 0; par < 2; ++par) {
                const int j = 2 * k + par;
                const int p = par ? K::odd_pos(k) : K::even_pos(k);
                const T fj = (T)j, j2 = fj * fj;
                T sn, cs;
                k_sincospi(B * j2, &sn, &cs);
                const T m = k_exp(A * j2);
                buf[p] = PR::mul_s(buf[p], PR::conj_s(stat(tb, tb.statV, c, l, j, false))) * mk(m * cs, m * sn);
            }
        }
    }

    // x <- x * r_j * f
    static __device__ void scale_r(cpx<T> *buf, const Tables<T> &tb, int g, double f)
    {
        const T s = (T)(tb.dr * f);
        for (int k = g; k < N / 2; k += G) {
            for (int par = 0; par < 2; ++par) {
                const int j = 2 * k + par;
                const int p = par ? K::odd_pos(k) : K::even_pos(k);
                buf[p] = scale(buf[p], (T)j * s);
            }
        }
    }
};

// the ready flag of a group's no-jump record, with acquire semantics: the record written before the
// flag was released is visible after it
__device__ __forceinline__ int group_ready(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// a record written by another CTA of this launch, read past L1
__device__ __forceinline__ qtraj_obs load_obs_cg(const qtraj_obs *p)
{
    static_assert(sizeof(qtraj_obs) % 8 == 0, "qtraj_obs is a whole number of 8-byte words");
    qtraj_obs o;
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(p);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(&o);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(qtraj_obs) / 8); ++i) dst[i] = __ldcg(src + i);
    return o;
}

// One thread per CTA takes work items from the counter: a group's no-jump run (item < n_groups) or a
// trajectory; r0 < p_NoJump (once the group's record is ready, or from a previous launch's records)
// and r0 > r_max are resolved here without evolving.
template <typename T>
__device__ int fetch_trajectory(const Tables<T> &tb, const LaunchArgs &a)
{
    for (;;) {
        const int w = atomicAdd(a.counter, 1);
        if (w >= a.n_groups + a.n_traj) return -1;
        if (a.nojump || w < a.n_groups) return w;
        const int t = w - a.n_groups;
        const TrajDev d = a.trajs[t];
        const Draws dr0 = draws(d.seed, 0u);
        int flags = 0;
        bool have = false;   // p_NoJump known (its group's record is published), or no shortcut at all
        if (tb.use_rmin) {
            qtraj_obs gj;
            if (a.gready) {
                if (group_ready(a.gready + d.group)) {
                    gj = load_obs_cg(a.gobs + d.group);
                    have = true;
                }
            } else if (a.group) {
                gj = a.group[d.group];
                have = true;
            }
            if (have) {
                if (fabs(dr0.r - gj.norm2) < border_eps<T>()) flags |= QTRAJ_F_BORDERLINE;
                if (dr0.r < gj.norm2) {
                    qtraj_obs o = gj;
                    o.r0 = dr0.r;
                    o.n_steps_exec = 0;
                    o.flags = flags | QTRAJ_F_NOJUMP_SHORTCUT;
                    a.obs[t] = o;
                    continue;
                }
            }
        }
        // r0 > r_max is resolved only once r0 < p_NoJump is excluded; otherwise the kernel evolves it
        if (tb.potential == 0 && dr0.r > tb.r_max && (have || !tb.use_rmin)) {
            qtraj_obs o;
            for (int s = 0; s < NBASIS; ++s) { o.surv[s] = 0; o.ov_re[s] = 0; o.ov_im[s] = 0; }
            o.norm2 = 1.0;
            o.r0 = dr0.r;
            o.l = tb.spec_l[d.spec];
            o.color = tb.spec_color[d.spec];
            o.n_jumps = 0;
            o.n_steps_exec = 0;
            o.flags = flags | QTRAJ_F_RMAX;
            o.first_jump_step = -1;
            o.last_jump_step = -1;
            o.jump_digest = DIGEST_BASIS;
            a.obs[t] = o;
            continue;
        }
        return w;
    }
}

// Occupancy target of a kernel variant: variant 0 asks for 512 resident threads per SM in FP32
// (<= 128 registers; at N = 4096 four CTAs of 128 threads, measured 8% faster on GB300 than three at
// <= 168 registers once the static tables lost their low parts and the norm sums their compensation);
// variant 1 asks for 640 (<= 102 registers, at the price of more spills), variants 2 and 3 (radix 8)
// for 768 and 1024.  FP64 holds twice the state and takes what the compiler needs.
template <typename T, int N, int V> struct FusedBounds {
    static constexpr int G = FusedPlan<N, V>::G;
    static constexpr int THREADS = (V == 0 || V == 4 || V == 5) ? 512 : V == 1 ? 640 : V == 2 ? 768 : 1024;
    static constexpr int MB = THREADS / G > 32 ? 32 : (THREADS / G > 0 ? THREADS / G : 1);
    static constexpr int MIN_BLOCKS = sizeof(T) == 4 ? MB : 1;
};

template <typename T, int N, int V>
__global__ void __launch_bounds__(FusedPlan<N, V>::G, (FusedBounds<T, N, V>::MIN_BLOCKS)) fused_kernel(Tables<T> tb, LaunchArgs a)
{
    using K = Fused<T, N, V>;
    using PW = Pointwise<T, N, V>;
    constexpr int G = K::G, E = K::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T> *buf = reinterpret_cast<cpx<T> *>(smem_raw);
    using C = typename Prec<T>::C;
    using P = FusedPlan<N, V>;
    C *tw1 = reinterpret_cast<C *>(buf + P::BUF);
    C *tw2 = tw1 + P::TW1;
    Carry<T> *wtot = reinterpret_cast<Carry<T> *>(tw2 + P::TW2);
    double *red = reinterpret_cast<double *>(wtot + (G / 32 + 1));
    __shared__ int s_traj;
    // middle-pass twiddles, row m of a table holding W^(m k) for every k (tw1: [M1][R] of W_{R M1},
    // tw2: [M2][R M1] of W_{R M1 M2}, the second only with a second middle pass), built once per CTA
    for (int t = threadIdx.x; t < P::TW1; t += G)
        tw1[t] = Prec<T>::ld(&tb.W[(t / P::R) * (t % P::R) * (N / P::TW1)]);
    if (P::M2 > 1)
        for (int t = threadIdx.x; t < P::TW2; t += G)
            tw2[t] = Prec<T>::ld(&tb.W[(t / P::TW1) * (t % P::TW1) * (N / P::TW2)]);

    const int g = threadIdx.x;
    const double dr = tb.dr;
    cpx<T> x[E];

    for (;;) {
        if (g == 0) s_traj = fetch_trajectory(tb, a);
        __syncthreads();
        const int wk = s_traj;
        __syncthreads();
        if (wk < 0) break;
        const bool grp = wk < a.n_groups;     // a group's no-jump run of this launch
        const int t = grp ? wk : wk - a.n_groups;
        constexpr bool KSU = V == 5;           // the isotropic KSU potential: H_eff only, no jumps
        const bool nojump = a.nojump || grp || KSU;

        const TrajDev d = grp ? a.gtrajs[t] : a.trajs[t];
        const MediumDev md = tb.media[d.medium];
        int l = tb.spec_l[d.spec], c = tb.spec_color[d.spec];
        if (tb.ic_cplx) {
            const double *ic = tb.ic + (size_t)d.spec * 2 * N;
            for (int k = g; k < N / 2; k += G) {
                buf[K::even_pos(k)] = mk<T>((T)ic[4 * k], (T)ic[4 * k + 1]);
                buf[K::odd_pos(k)] = mk<T>((T)ic[4 * k + 2], (T)ic[4 * k + 3]);
            }
        } else {
            const double *ic = tb.ic + (size_t)d.spec * N;
            for (int k = g; k < N / 2; k += G) {
                buf[K::even_pos(k)] = mk<T>((T)ic[2 * k], (T)0);
                buf[K::odd_pos(k)] = mk<T>((T)ic[2 * k + 1], (T)0);
            }
        }
        uint32_t kdraw = 0;
        Draws dw = draws(d.seed, 0u);
        const double r0 = nojump ? 0.0 : dw.r;   // (no draw is used without jumps)
        Threshold<T> thr;
        thr.set(nojump ? -1.0 : dw.r, dr);
        int nj = 0, flags = 0, fj = -1, lj = -1, ended = 0, executed = 0;
        uint32_t digest = DIGEST_BASIS;
        // r0 > r_max reaches here only when its group's no-jump record was not yet published: the paper
        // resolves r0 < p_NoJump by the shortcut first and r0 > r_max only otherwise.  The trajectory
        // is evolved: if its norm never falls to r0 it is the no-jump run (= the shortcut's record); the
        // first trigger shows r0 >= p_NoJump (the norm only decreases), and it ends as r_max does.
        const bool rmax_pending = !nojump && !KSU && dw.r > tb.r_max;
        bool rmax_hit = false;
        const bool traced = V == 4 && !grp && a.trace_every > 0 && t < a.trace_n;
        int nrec = 0;
        const int ns = d.n_steps;
        // per-step scalars in the working precision: T^3 = A / (tau0 + n dtau)
        const T mA = (T)md.A, mtau0 = (T)md.tau0, mdtau = (T)md.dtau;
        const bool tabulated = md.kind == 1;
        int seg = 0;
        // T(tau_n)^3: Bjorken, or the table at tau_n = tau_1 + n dtau (out of line: rare, and inline it
        // would hold registers in the step loop)
        auto T3_of = [&](int n) -> T {
            return tabulated ? table_T3_far<T>(tb.prof + 2 * (size_t)md.tab_off, md.tab_len, mtau0 + (T)n * mdtau, &seg)
                             : mA / (mtau0 + (T)n * mdtau);
        };
        T T3b = T3_of(0);
        T K3b = kappa_T3<T>(md.kfit, T3b);   // kappa_hat(T) T^3 when kappa_hat follows a lattice fit
        KsuT<T> kb{};
        if constexpr (KSU) kb = ksu_at<T>(tb, T3b);
        if (ns > 0) {
            __syncthreads();
            if constexpr (KSU) PW::factor_ksu(buf, tb, g, l, 0, kb, kb, red);
            else PW::factor(buf, tb, g, c, l, 0, (T)md.erj[c] * K3b, (T)md.eij[c] * T3b, (T)0, red);
        }

        for (int n = 0; n < ns; ++n) {
            const T T3a = T3b, K3a = K3b;
            const bool last = (n + 1 == ns);
            T3b = T3_of(n + 1);
            K3b = kappa_T3<T>(md.kfit, T3b);
            __syncthreads();
#pragma unroll 1
            for (int h = 0; h < 2; ++h) K::dst(x, buf, tb, g, wtot, tw1, tw2, h == 1);
            executed = n + 1;
            const T erj = (T)md.erj[c], eij = (T)md.eij[c];
            if constexpr (V == 4) {   // the traced twin of variant 0: per-step summary rows
                if (traced && ((n + 1) % a.trace_every == 0 || last) && nrec < a.trace_cap) {
                    PW::trace_row(buf, tb, g, c, l, erj * K3a, eij * T3a, red,
                                  a.trace + (size_t)t * a.trace_cap + nrec, n + 1);
                    ++nrec;
                    __syncthreads();
                }
            }
            const T Tsum = last ? T3a : T3a + T3b, Ksum = last ? K3a : K3a + K3b;
            typename NormSum<T>::type n2s;   // norm^2 / dr
            if constexpr (KSU) {
                const KsuT<T> ka = kb;
                kb = ksu_at<T>(tb, T3b);
                n2s = PW::factor_ksu(buf, tb, g, l, last ? 2 : 1, ka, kb, red);
            } else {
                n2s = PW::factor(buf, tb, g, c, l, last ? 2 : 1, erj * Ksum, eij * Tsum,
                                 last ? (T)0 : erj * (K3a - K3b), red);
            }
            if (!thr.finite(n2s)) {
                flags |= QTRAJ_F_NONFINITE;
                ended = 1;
                if (g == 0) atomicOr(a.status, 1);
                break;
            }
            if (!nojump) {
                if (thr.near(n2s, border_eps<T>())) flags |= QTRAJ_F_BORDERLINE;
                const bool trig = thr.reached(n2s);
                if (trig && rmax_pending) {
                    rmax_hit = true;
                    ended = 1;
                    break;
                }
                if (trig) {
                    // a trajectory stopped by a cap keeps its end-of-step state
                    const bool cap_j = tb.max_jumps >= 0 && nj >= tb.max_jumps;
                    const int l_new = (dw.ul < (double)l / (2.0 * l + 1.0)) ? l - 1 : l + 1;
                    const int c_new = (c == 1 && dw.uc < tb.p_os) ? 0 : 1;
                    const bool cap_l = !cap_j && tb.l_cap >= 0 && l_new > tb.l_cap;
                    if (cap_j || cap_l) {
                        if (!last) {
                            __syncthreads();
                            PW::undo_start(buf, tb, g, c, l, -(T)md.erj[c] * K3b, -(T)md.eij[c] * T3b);
                        }
                        ended = 1;
                        if (cap_j) {
                            flags |= QTRAJ_F_MAXJUMPS;
                        } else {
                            flags |= QTRAJ_F_LCAP;
                            if (fj < 0) fj = n;
                            l = l_new; c = c_new; ++nj;
                            lj = n;
                            digest = digest_jump(digest, n, l, c);
                        }
                        break;
                    }
                    if (fj < 0) fj = n;
                    // r times the end-of-step state, renormalised; the start half-step already applied
                    // is turned into the new colour's and l's
                    __syncthreads();
                    const double dr2 = tb.dr * tb.dr, T3d = (double)T3b, K3d = (double)K3b;
                    const T w2 = last ? (T)0 : (T)(-2.0 * md.er[c] * K3d * dr2);
                    const T dA = last ? (T)0 : (T)((md.er[c_new] - md.er[c]) * K3d * dr2);
                    const T dB = last ? (T)0 : (T)((md.ei[c_new] - md.ei[c]) * T3d * dr2 * 0.31830988618379067154);
                    const double s = PW::jump_turn(buf, tb, g, c, l, c_new, l_new, last, w2, dA, dB, red) * dr;
                    const double f = 1.0 / sqrt(s);
                    __syncthreads();
                    PW::scale_r(buf, tb, g, f);
                    l = l_new; c = c_new; ++nj;
                    lj = n;
                    digest = digest_jump(digest, n, l, c);
                    ++kdraw;
                    dw = draws(d.seed, kdraw);
                    thr.set(dw.r, dr);
                }
            }
        }
        __syncthreads();

        // observables (FP64)
        double acc = 0.0;
        for (int k = g; k < N / 2; k += G) {
            const cpx<T> a0 = buf[K::even_pos(k)], a1 = buf[K::odd_pos(k)];
            acc += (double)a0.x * a0.x + (double)a0.y * a0.y + (double)a1.x * a1.x + (double)a1.y * a1.y;
        }
        const double n2 = slot_sum<G>(acc, red) * dr;
        double ovr[NBASIS], ovi[NBASIS];
        const int basis_l[NBASIS] = {0, 0, 1, 0, 1, 2};
#pragma unroll
        for (int s = 0; s < NBASIS; ++s) {
            ovr[s] = 0.0;
            ovi[s] = 0.0;
            if (ended || c != 0 || basis_l[s] != l) continue;
            const double *phi = tb.eig + (size_t)s * N;
            double pr = 0.0, pi = 0.0;
            for (int k = g; k < N / 2; k += G) {
                const cpx<T> a0 = buf[K::even_pos(k)], a1 = buf[K::odd_pos(k)];
                const double f0 = phi[2 * k], f1 = phi[2 * k + 1];
                pr += f0 * (double)a0.x + f1 * (double)a1.x;
                pi += f0 * (double)a0.y + f1 * (double)a1.y;
            }
            ovr[s] = slot_sum<G>(pr, red) * dr;
            ovi[s] = slot_sum<G>(pi, red) * dr;
        }
        if (a.states && !grp) {
            double *st = a.states + (size_t)t * N * 2;
            for (int k = g; k < N / 2; k += G) {
                const cpx<T> a0 = buf[K::even_pos(k)], a1 = buf[K::odd_pos(k)];
                st[4 * k] = (double)a0.x;
                st[4 * k + 1] = (double)a0.y;
                st[4 * k + 2] = (double)a1.x;
                st[4 * k + 3] = (double)a1.y;
            }
        }
        if (g == 0) {
            qtraj_obs o;
            const int sp = d.spec;
            for (int s = 0; s < NBASIS; ++s) {
                o.ov_re[s] = ovr[s];
                o.ov_im[s] = ovi[s];
                double sv = 0.0;
                if (!ended && c == 0 && basis_l[s] == l) {
                    // with jumps the estimator takes the normalised state; without (KSU) the norm lost
                    // to V_I is the dissociation, and the overlap is taken unnormalised
                    const double prob = (ovr[s] * ovr[s] + ovi[s] * ovi[s]) / (KSU ? 1.0 : n2);
                    if (tb.ov0_zero[sp * NBASIS + s]) sv = prob;
                    else {
                        const double a0 = tb.ov0[(sp * NBASIS + s) * 2], b0 = tb.ov0[(sp * NBASIS + s) * 2 + 1];
                        sv = prob / (a0 * a0 + b0 * b0);
                    }
                }
                o.surv[s] = sv;
            }
            o.norm2 = n2;
            o.r0 = r0;
            o.l = l;
            o.color = c;
            o.n_jumps = nj;
            o.n_steps_exec = executed;
            o.flags = flags;
            o.first_jump_step = fj;
            o.last_jump_step = lj;
            o.jump_digest = digest;
            if (rmax_hit) {   // the r_max record, with the steps that found r0 >= p_NoJump
                for (int s = 0; s < NBASIS; ++s) { o.surv[s] = 0; o.ov_re[s] = 0; o.ov_im[s] = 0; }
                o.norm2 = 1.0;
                o.l = tb.spec_l[d.spec];
                o.color = tb.spec_color[d.spec];
                o.flags = flags | QTRAJ_F_RMAX;
            }
            if (grp) {
                a.gobs[t] = o;
                __threadfence();              // the record before the flag that publishes it
                atomicExch(a.gready + t, 1);
            } else {
                a.obs[t] = o;
            }
            if (traced) a.trace_cnt[t] = nrec;
        }
        __syncthreads();
    }
}

// shared-memory bytes of one CTA
template <typename T, int N, int V> constexpr int fused_smem_bytes()
{
    using P = FusedPlan<N, V>;
    return P::BUF * (int)sizeof(cpx<T>) +
           (P::TW1 + P::TW2) *
               (int)sizeof(typename Prec<T>::C) +
           (P::G / 32 + 1) * (int)sizeof(Carry<T>) + (P::G / 32 + 1) * 8 + 16;
}

// Launches fused_kernel<T, N, V> as one persistent wave (SMs x resident CTAs, at most max_ctas when
// max_ctas > 0, at most one CTA per trajectory) after setting its shared-memory size; fills info
// (query_only: launches nothing).  Every instantiation unit dispatches its grid sizes to this helper.
template <typename T, int N, int V>
cudaError_t fused_go(const Tables<T> &tb, const LaunchArgs &a, int sm_count, int max_ctas, cudaStream_t s,
                     FusedInfo *info, bool query_only)
{
    auto k = fused_kernel<T, N, V>;
    constexpr int G = FusedPlan<N, V>::G;
    constexpr int smem = fused_smem_bytes<T, N, V>();
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, G, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (info) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, k);
        if (e != cudaSuccess) return e;
        info->G = G;
        info->R = FusedPlan<N, V>::R;
        info->smem = smem;
        info->ctas_per_sm = occ;
        info->regs = fa.numRegs;
    }
    const long work = (long)a.n_traj + a.n_groups;
    if (query_only || work <= 0) return cudaSuccess;
    long grid = (long)sm_count * occ;
    if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
    if (grid > work) grid = work;
    k<<<(int)grid, G, smem, s>>>(tb, a);
    return cudaGetLastError();
}

} // namespace qt
