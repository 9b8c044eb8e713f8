// fused.cuh -- the fused persistent trajectory kernel.
//
// One CTA evolves one trajectory at a time, through every step of its medium, and then fetches the
// next trajectory from a global work counter.  The wave function never leaves the SM: between steps
// it lives in registers (2R complex values per thread), and the sine transforms exchange data
// through one shared-memory buffer of N + N/(2R) complex values.
//
// One step (Sec. 3.3, steps 1-5) with T = T(tau_n) (Sec. 3.4, Bjorken):
//   x <- K_V x                     K_V = exp(-i V_eff dt/2): static table x exp((er + i ei) T^3 r^2)
//   S = DST(x)                     S_k = sum_j x_j sin(pi j k / N)
//   S <- K_T S                     K_T = exp(-i T_kin(p_k) dt) * 2/N   (2/N = inverse DST scale)
//   x = DST(S), x <- K_V x
//   norm^2 = (L/N) sum |x_j|^2 ; if norm^2 <= r: jump (Sec. 3.2.1, 3.4.3-3.4.4, 3.5)
//
// The DST-I of the N-point complex vector f (f_0 = f_N = 0) is computed with one N-point complex FFT:
//   y_j = sin(pi j/N)(f_j + f_{N-j}) + (f_j - f_{N-j})/2,   Y = FFT_N(y),
//   S_{2k}   = (i/2)(Y_k - Y_{N-k}),
//   S_{2k+1} = S_{2k-1} + (Y_k + Y_{N-k})/2,  S_{-1} = -S_1    (a prefix sum over k < N/2).
// This equals the length-2N FFT of the odd extension (the paper's "Fourier sine series" with the
// wall at r = L) at half its arithmetic and memory.
//
// FFT: Stockham autosort with radices R (first pass), MID = N/R^2 split in passes of <= 16, R (last).
// Thread g of G = N/(2R) owns butterflies b1 = g, b2 = N/R - g (g = 0: 0 and N/(2R)) of the first
// and last passes, i.e. the indices b + m N/R, m < R.  Those index sets are closed under j -> N - j,
// so the DST pre- and post-processing, which pair j with N - j, stay inside a thread's registers.
#pragma once
#include "qtraj_device.cuh"

namespace qt {

template <int N> struct FusedPlan {
    static constexpr int R = (N <= 32) ? 4 : (N <= 512) ? 8 : 16;
    static constexpr int G = N / (2 * R);        // threads per trajectory
    static constexpr int NR = N / R;             // stride of a first/last-pass butterfly
    static constexpr int MID = N / (R * R);      // product of the middle radices
    static constexpr int M1 = MID >= 16 ? 16 : MID;
    static constexpr int M2 = MID / M1;          // 1, 2 or 4
    static constexpr int SCAN_PAD = R + 1;       // padded chunk of the odd-coefficient scan
    static constexpr int BUF = N + N / (2 * R) + 8;
    static_assert(N == R * M1 * M2 * R, "plan");
};

// ------------------------------------------------------------------------------------------------
// accumulators: FP32 forms accumulate sums of squares in double-float (error-free transformations
// in FP32), so that norms carry FP64-level accuracy without using GB300's narrow FP64 pipe in the
// step loop; FP64 forms accumulate in double.
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
__device__ __forceinline__ DF df_add_sq(DF a, float v)   // a + v*v, the square split exactly
{
    const float p = v * v, e = fmaf(v, v, -p);
    DF s = two_sum(a.hi, p);
    const float t = s.lo + a.lo + e;
    const float hi = s.hi + t;
    return {hi, t - (hi - s.hi)};
}

template <typename T> struct SqAcc;
template <> struct SqAcc<float> {
    DF v{0.f, 0.f};
    __device__ __forceinline__ void add(cpx<float> a) { v = df_add_sq(df_add_sq(v, a.x), a.y); }
    __device__ __forceinline__ void shfl_add(unsigned mask, int off, int w)
    {
        DF o{__shfl_xor_sync(mask, v.hi, off, w), __shfl_xor_sync(mask, v.lo, off, w)};
        v = df_add(v, o);
    }
    __device__ __forceinline__ double value() const { return (double)v.hi + (double)v.lo; }
};
template <> struct SqAcc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(cpx<double> a) { v = fma(a.x, a.x, fma(a.y, a.y, v)); }
    __device__ __forceinline__ void shfl_add(unsigned mask, int off, int w) { v += __shfl_xor_sync(mask, v, off, w); }
    __device__ __forceinline__ double value() const { return v; }
};

// compensated complex prefix element for the odd-coefficient scan
template <typename T> struct ScanVal;
template <> struct ScanVal<float> {
    DF re{0.f, 0.f}, im{0.f, 0.f};
    __device__ __forceinline__ void add(cpx<float> a) { re = df_add(re, DF{a.x, 0.f}); im = df_add(im, DF{a.y, 0.f}); }
    __device__ __forceinline__ void add(const ScanVal &o) { re = df_add(re, o.re); im = df_add(im, o.im); }
    __device__ __forceinline__ cpx<float> plus(cpx<float> a) const   // (a + this) rounded once
    {
        const DF r = df_add(re, DF{a.x, 0.f}), i = df_add(im, DF{a.y, 0.f});
        return mk(r.hi + r.lo, i.hi + i.lo);
    }
    __device__ __forceinline__ ScanVal shfl_up(unsigned mask, int off, int w) const
    {
        ScanVal o;
        o.re = DF{__shfl_up_sync(mask, re.hi, off, w), __shfl_up_sync(mask, re.lo, off, w)};
        o.im = DF{__shfl_up_sync(mask, im.hi, off, w), __shfl_up_sync(mask, im.lo, off, w)};
        return o;
    }
};
template <> struct ScanVal<double> {
    double re = 0.0, im = 0.0;
    __device__ __forceinline__ void add(cpx<double> a) { re += a.x; im += a.y; }
    __device__ __forceinline__ void add(const ScanVal &o) { re += o.re; im += o.im; }
    __device__ __forceinline__ cpx<double> plus(cpx<double> a) const { return mk(a.x + re, a.y + im); }
    __device__ __forceinline__ ScanVal shfl_up(unsigned mask, int off, int w) const
    {
        ScanVal o;
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

// sum over the G threads of a trajectory (deterministic order)
template <int G> __device__ __forceinline__ double slot_sum(double v, double *red)
{
    constexpr int W = G < 32 ? G : 32;
    const unsigned mask = lane_mask<G>();
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off, W);
    if constexpr (G <= 32) v = __shfl_sync(mask, v, 0, W);   // one value for every lane
    return cross_warp<G>(v, red);
}

template <typename T, int G> __device__ __forceinline__ double slot_norm(SqAcc<T> acc, double *red)
{
    constexpr int W = G < 32 ? G : 32;
    const unsigned mask = lane_mask<G>();
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) acc.shfl_add(mask, off, W);
    double v = acc.value();
    if constexpr (G <= 32) v = __shfl_sync(mask, v, 0, W);
    return cross_warp<G>(v, red);
}

// ------------------------------------------------------------------------------------------------
// the kernel
// ------------------------------------------------------------------------------------------------
template <typename T, int N> struct Fused {
    using P = FusedPlan<N>;
    static constexpr int R = P::R, G = P::G, NR = P::NR, E = 2 * R;

    // global index of register element e (first/last-pass layout)
    static __device__ __forceinline__ int idx(int g, int e)
    {
        const int b = (e < R) ? (g == 0 ? 0 : g) : (g == 0 ? NR / 2 : NR - g);
        return b + (e % R) * NR;
    }

    // y_j = s (f_j + f_{N-j}) + (f_j - f_{N-j})/2 for the pair (ea, eb) = (j, N-j)
    using PR = Prec<T>;
    using RL = typename Prec<T>::Rl;

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

    // E_k = (i/2)(Y_k - Y_{N-k}) -> buf[k];  C_k = (Y_k + Y_{N-k})/2 (C_0 halved) -> odd area
    static __device__ __forceinline__ int odd_pos(int k) { return N / 2 + k + k / R; }

    static __device__ __forceinline__ void post_pair(cpx<T> *buf, int k, cpx<T> A, cpx<T> B)
    {
        buf[k] = mul_i(scale(A - B, (T)0.5));
        buf[odd_pos(k)] = scale(A + B, (T)0.5);
    }

    static __device__ __forceinline__ void post(const cpx<T> *x, int g, cpx<T> *buf)
    {
        if (g != 0) {
#pragma unroll
            for (int m = 0; m < R; ++m) {
                const int eb = R + (R - 1 - m);
                if (m < R / 2) post_pair(buf, g + m * NR, x[m], x[eb]);
                else post_pair(buf, (NR - g) + (R - 1 - m) * NR, x[eb], x[m]);
            }
        } else {
            buf[0] = mk<T>(0, 0);
            buf[odd_pos(0)] = scale(x[0], (T)0.5);             // S_1 = C_0 / 2 = Y_0 / 2
#pragma unroll
            for (int m = 1; m < R / 2; ++m) post_pair(buf, m * NR, x[m], x[R - m]);
#pragma unroll
            for (int m = 0; m < R / 2; ++m) post_pair(buf, NR / 2 + m * NR, x[R + m], x[R + (R - 1 - m)]);
        }
    }

    // inclusive prefix sum of the N/2 odd-area values: thread g owns k in [gR, gR + R)
    static __device__ __forceinline__ void scan(cpx<T> *buf, int g, ScanVal<T> *wtot)
    {
        constexpr int W = G < 32 ? G : 32;
        const unsigned mask = lane_mask<G>();
        cpx<T> *p = buf + N / 2 + g * P::SCAN_PAD;
        cpx<T> v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = p[q];
        ScanVal<T> run;                 // compensated chunk total
#pragma unroll
        for (int q = 0; q < R; ++q) run.add(v[q]);
        // exclusive scan of chunk totals across the trajectory's threads
        const int lane = threadIdx.x & (W - 1);
        ScanVal<T> inc = run;
#pragma unroll
        for (int off = 1; off < W; off <<= 1) {
            ScanVal<T> y = inc.shfl_up(mask, off, W);
            if (lane >= off) inc.add(y);
        }
        ScanVal<T> excl = inc.shfl_up(mask, 1, W);
        if (lane == 0) excl = ScanVal<T>();
        if constexpr (G > 32) {
            const int warp = threadIdx.x >> 5;
            if (lane == 31) wtot[warp] = inc;
            __syncthreads();
#pragma unroll 1
            for (int w = 0; w < warp; ++w) excl.add(wtot[w]);
        }
        // the chunk's running sum continues from the carried offset in compensated arithmetic, so
        // every output is rounded once
        ScanVal<T> acc = excl;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            acc.add(v[q]);
            p[q] = acc.plus(mk<T>(0, 0));
        }
    }

    // S_j from the DST output area: even j -> buf[j/2], odd j -> odd area
    static __device__ __forceinline__ cpx<T> s_at(const cpx<T> *buf, int j)
    {
        return (j & 1) ? buf[odd_pos(j >> 1)] : buf[j >> 1];
    }

    template <int RM, int PP>
    static __device__ __forceinline__ void mid_pass(cpx<T> *x, cpx<T> *buf, const typename Prec<T>::C *W, int g)
    {
        if constexpr (RM > 1) {
            constexpr int NB = N / RM, PER = E / RM;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int i = g + q * G, k = i & (PP - 1);
#pragma unroll
                for (int m = 0; m < RM; ++m) {
                    cpx<T> v = buf[i + m * NB];
                    if (m) v = PR::mul(v, PR::ld(&W[m * k * (N / (PP * RM))]));
                    x[q * RM + m] = v;
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int i = g + q * G, k = i & (PP - 1);
                DFT<T, RM>::template run<1>(x + q * RM);
                const int base = (i - k) * RM + k;
#pragma unroll
                for (int m = 0; m < RM; ++m) buf[base + m * PP] = x[q * RM + m];
            }
            __syncthreads();
        }
    }

    // x (first-pass layout, values f_j at idx(g, e)) -> DST output in buf (even/odd areas)
    static __device__ __forceinline__ void dst(cpx<T> *x, cpx<T> *buf, const Tables<T> &tb, int g, ScanVal<T> *wtot)
    {
        pre(x, g, tb.sinpre);
        // first pass (radix R, no twiddles): butterfly b -> buf[b R + m]
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            DFT<T, R>::template run<1>(x + t * R);
            const int b = (t == 0) ? (g == 0 ? 0 : g) : (g == 0 ? NR / 2 : NR - g);
#pragma unroll
            for (int m = 0; m < R; ++m) buf[b * R + m] = x[t * R + m];
        }
        __syncthreads();
        mid_pass<P::M1, R>(x, buf, tb.W, g);
        mid_pass<P::M2, R * P::M1>(x, buf, tb.W, g);
        // last pass (radix R, P = N/R): inputs buf[b + m NR], twiddle W^(m b), outputs stay in registers
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int b = (t == 0) ? (g == 0 ? 0 : g) : (g == 0 ? NR / 2 : NR - g);
#pragma unroll
            for (int m = 0; m < R; ++m) {
                cpx<T> v = buf[b + m * NR];
                if (m) v = PR::mul(v, PR::ld(&tb.W[m * b]));
                x[t * R + m] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 2; ++t) DFT<T, R>::template run<1>(x + t * R);
        post(x, g, buf);
        __syncthreads();
        scan(buf, g, wtot);
        __syncthreads();
    }

    // x <- K_V x for (colour, l) at T^3
    static __device__ __forceinline__ void space_kernel(cpx<T> *x, const Tables<T> &tb, int g, int c, int l, T er, T ei,
                                                        T dr)
    {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int j = idx(g, e);
            const T r = (T)j * dr;
            x[e] = PR::mul(x[e], static_factor<T>(tb, N, c, l, j)) * dyn_factor(er, ei, r * r);
        }
    }

    static __device__ __forceinline__ double norm2(const cpx<T> *x, double *red, double dr)
    {
        SqAcc<T> acc;
#pragma unroll
        for (int e = 0; e < E; ++e) acc.add(x[e]);
        return slot_norm<T, G>(acc, red) * dr;
    }
};

// one thread per CTA takes trajectories from the counter; r0 < p_NoJump and r0 > r_max are resolved
// here without evolving
template <typename T>
__device__ int fetch_trajectory(const Tables<T> &tb, const LaunchArgs &a)
{
    for (;;) {
        const int t = atomicAdd(a.counter, 1);
        if (t >= a.n_traj) return -1;
        if (a.nojump) return t;
        const TrajDev d = a.trajs[t];
        const Draws dr0 = draws(d.seed, 0u);
        int flags = 0;
        if (tb.use_rmin) {
            const qtraj_obs &gj = a.group[d.group];
            if (fabs(dr0.r - gj.norm2) < BORDER_EPS) flags |= QTRAJ_F_BORDERLINE;
            if (dr0.r < gj.norm2) {
                qtraj_obs o = gj;
                o.r0 = dr0.r;
                o.n_steps_exec = 0;
                o.flags = flags | QTRAJ_F_NOJUMP_SHORTCUT;
                a.obs[t] = o;
                continue;
            }
        }
        if (dr0.r > tb.r_max) {
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
            a.obs[t] = o;
            continue;
        }
        return t;
    }
}

template <typename T, int N>
__global__ void __launch_bounds__(FusedPlan<N>::G) fused_kernel(Tables<T> tb, LaunchArgs a)
{
    using K = Fused<T, N>;
    constexpr int R = K::R, G = K::G, E = K::E;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T> *buf = reinterpret_cast<cpx<T> *>(smem_raw);
    ScanVal<T> *wtot = reinterpret_cast<ScanVal<T> *>(buf + FusedPlan<N>::BUF);
    double *red = reinterpret_cast<double *>(wtot + (G / 32 + 1));
    __shared__ int s_traj;
    (void)R;

    const int g = threadIdx.x;
    const double dr = tb.dr;
    cpx<T> x[E];

    for (;;) {
        if (g == 0) s_traj = fetch_trajectory(tb, a);
        __syncthreads();
        const int t = s_traj;
        __syncthreads();
        if (t < 0) break;

        const TrajDev d = a.trajs[t];
        const MediumDev md = tb.media[d.medium];
        int l = tb.spec_l[d.spec], c = tb.spec_color[d.spec];
        const double *ic = tb.ic + (size_t)d.spec * N;
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = mk<T>((T)ic[K::idx(g, e)], (T)0);

        uint32_t kdraw = 0;
        Draws dw = draws(d.seed, 0u);
        const double r0 = a.nojump ? 0.0 : dw.r;
        double thr = a.nojump ? -1.0 : dw.r;
        int nj = 0, flags = 0, fj = -1, ended = 0, executed = 0;
        const int ns = d.n_steps;

        for (int n = 0; n < ns; ++n) {
            const double T3 = md.A / (md.tau0 + (double)n * md.dtau);
            const T er = (T)(md.er[c] * T3), ei = (T)(md.ei[c] * T3);
            K::space_kernel(x, tb, g, c, l, er, ei, (T)dr);
            K::dst(x, buf, tb, g, wtot);
            // kinetic step on the spectrum, back to registers
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = K::idx(g, e);
                x[e] = Prec<T>::mul(K::s_at(buf, j), Prec<T>::ld(&tb.KT[j]));
            }
            __syncthreads();
            K::dst(x, buf, tb, g, wtot);
#pragma unroll
            for (int e = 0; e < E; ++e) x[e] = K::s_at(buf, K::idx(g, e));
            __syncthreads();                           // buf is free for the next step
            K::space_kernel(x, tb, g, c, l, er, ei, (T)dr);
            executed = n + 1;

            const double n2 = K::norm2(x, red, dr);
            if (!isfinite(n2)) {
                flags |= QTRAJ_F_NONFINITE;
                ended = 1;
                if (g == 0) atomicOr(a.status, 1);
                break;
            }
            if (!a.nojump) {
                if (fabs(n2 - thr) < BORDER_EPS) flags |= QTRAJ_F_BORDERLINE;
                if (n2 <= thr) {
                    if (tb.max_jumps >= 0 && nj >= tb.max_jumps) {
                        flags |= QTRAJ_F_MAXJUMPS;
                        ended = 1;
                        break;
                    }
                    const int l_new = (dw.ul < (double)l / (2.0 * l + 1.0)) ? l - 1 : l + 1;
                    const int c_new = (c == 1 && dw.uc < tb.p_os) ? 0 : 1;
                    if (fj < 0) fj = n;
                    if (tb.l_cap >= 0 && l_new > tb.l_cap) {
                        flags |= QTRAJ_F_LCAP;
                        l = l_new; c = c_new; ++nj;
                        ended = 1;
                        break;
                    }
                    // psi <- r psi / ||r psi||
                    double s = 0.0;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const double rj = K::idx(g, e) * dr;
                        const double xr = (double)x[e].x * rj, xi = (double)x[e].y * rj;
                        s += xr * xr + xi * xi;
                    }
                    s = slot_sum<G>(s, red) * dr;
                    const double inv = 1.0 / sqrt(s);
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const double f = K::idx(g, e) * dr * inv;
                        x[e] = mk<T>((T)((double)x[e].x * f), (T)((double)x[e].y * f));
                    }
                    l = l_new; c = c_new; ++nj;
                    ++kdraw;
                    dw = draws(d.seed, kdraw);
                    thr = dw.r;
                }
            }
        }

        // observables (FP64)
        const double n2 = K::norm2(x, red, dr);
        double ovr[NBASIS], ovi[NBASIS];
#pragma unroll
        for (int s = 0; s < NBASIS; ++s) { ovr[s] = 0.0; ovi[s] = 0.0; }
        const int basis_l[NBASIS] = {0, 0, 1, 0, 1, 2};
        if (!ended && c == 0) {
#pragma unroll 1
            for (int s = 0; s < NBASIS; ++s) {
                if (basis_l[s] != l) continue;
                const double *phi = tb.eig + (size_t)s * N;
                double pr = 0.0, pi = 0.0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const double f = phi[K::idx(g, e)];
                    pr += f * (double)x[e].x;
                    pi += f * (double)x[e].y;
                }
                ovr[s] = slot_sum<G>(pr, red) * dr;
                ovi[s] = slot_sum<G>(pi, red) * dr;
            }
        }
        if (a.states) {
            double *st = a.states + (size_t)t * N * 2;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = K::idx(g, e);
                st[2 * j] = (double)x[e].x;
                st[2 * j + 1] = (double)x[e].y;
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
                    const double prob = (ovr[s] * ovr[s] + ovi[s] * ovi[s]) / n2;
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
            a.obs[t] = o;
        }
        __syncthreads();
    }
}

// shared-memory bytes of one CTA
template <typename T, int N> constexpr int fused_smem_bytes()
{
    return FusedPlan<N>::BUF * (int)sizeof(cpx<T>) + (FusedPlan<N>::G / 32 + 1) * (int)sizeof(ScanVal<T>) +
           (FusedPlan<N>::G / 32 + 1) * 8 + 16;
}

} // namespace qt
