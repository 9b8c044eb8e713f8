// plain.cu -- the plain per-step FP64 form: every time step is a sequence of separate kernels over
// the whole batch, with the wave functions in HBM between kernels:
//   space half-step + DST pre-processing -> FFT passes (global-memory Stockham, radix 4/2)
//   -> post-processing + prefix scan + kinetic factor + pre-processing -> FFT passes
//   -> post-processing + prefix scan + space half-step + norm -> waiting-time test / jump.
// It computes the same step as the fused kernel (Sec. 3.3, steps 1-5; the DST-I through one N-point
// FFT as described in fused.cuh) and is the baseline the fused forms are measured against.
#include "plain.cuh"

namespace qt {

namespace {

constexpr int PB = 256; // threads of the per-trajectory kernels

__device__ __forceinline__ double T3_of(const Tables<double> &tb, const MediumDev &m, int n)
{
    const double tau = m.tau0 + (double)n * m.dtau;
    if (m.kind == 1) return table_T3_at(tb.prof + 2 * (size_t)m.tab_off, m.tab_len, tau);
    return m.A / tau;
}

// K3 = kappa_T3(md.kfit, T3): the T^3 of the real exponent, times kappa_hat(T) for a fitted medium
__device__ __forceinline__ cpx<double> space_factor(const Tables<double> &tb, int N, const MediumDev &md, int c, int l,
                                                    int j, double T3, double K3)
{
    const double r = j * tb.dr;
    return static_factor<double>(tb, N, c, l, j) * dyn_factor(md.er[c] * K3, md.ei[c] * T3, r * r);
}

__device__ __forceinline__ bool running(const PlainState &s, const TrajDev &d, int n)
{
    return s.active && n < d.n_steps;
}

// block-wide sum of a double over PB threads, same value returned to every thread
__device__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < PB / 32; ++w) s += sh[w];
    __syncthreads();
    return s;
}

__global__ void plain_setup(Tables<double> tb, LaunchArgs a, PlainState *st, cpx<double> *psi, int N)
{
    const int b = blockIdx.x;
    __shared__ int s_active;
    const TrajDev d = a.trajs[b];
    if (threadIdx.x == 0) {
        PlainState s;
        const Draws dw = draws(d.seed, 0u);
        s.thr = a.nojump ? -1.0 : dw.r;
        s.ul = dw.ul;
        s.uc = dw.uc;
        s.r0 = a.nojump ? 0.0 : dw.r;
        s.l = tb.spec_l[d.spec];
        s.c = tb.spec_color[d.spec];
        s.nj = 0;
        s.fj = -1;
        s.flags = 0;
        s.active = 1;
        s.kdraw = 0;
        s.executed = 0;
        s.lj = -1;
        s.digest = DIGEST_BASIS;
        if (!a.nojump) {
            if (tb.use_rmin) {
                const qtraj_obs &gj = a.group[d.group];
                if (fabs(dw.r - gj.norm2) < BORDER_EPS) s.flags |= QTRAJ_F_BORDERLINE;
                if (dw.r < gj.norm2) {
                    qtraj_obs o = gj;
                    o.r0 = dw.r;
                    o.n_steps_exec = 0;
                    o.flags = s.flags | QTRAJ_F_NOJUMP_SHORTCUT;
                    a.obs[b] = o;
                    s.active = 0;
                }
            }
            if (s.active && dw.r > tb.r_max) {
                qtraj_obs o;
                for (int q = 0; q < NBASIS; ++q) { o.surv[q] = 0; o.ov_re[q] = 0; o.ov_im[q] = 0; }
                o.norm2 = 1.0;
                o.r0 = dw.r;
                o.l = s.l;
                o.color = s.c;
                o.n_jumps = 0;
                o.n_steps_exec = 0;
                o.flags = s.flags | QTRAJ_F_RMAX;
                o.first_jump_step = -1;
                o.last_jump_step = -1;
                o.jump_digest = DIGEST_BASIS;
                a.obs[b] = o;
                s.active = 0;
            }
        }
        if (s.active && d.n_steps == 0) s.active = 2;   // finalised by plain_finalize_empty
        st[b] = s;
        s_active = s.active;
    }
    __syncthreads();
    if (s_active) {
        if (tb.ic_cplx) {
            const double *ic = tb.ic + (size_t)d.spec * 2 * N;
            for (int j = threadIdx.x; j < N; j += blockDim.x) psi[(size_t)b * N + j] = mk(ic[2 * j], ic[2 * j + 1]);
        } else {
            const double *ic = tb.ic + (size_t)d.spec * N;
            for (int j = threadIdx.x; j < N; j += blockDim.x) psi[(size_t)b * N + j] = mk(ic[j], 0.0);
        }
    }
}

// start of step n: y = pre(K_V psi).  One thread per pair (q, N - q), q = 0..N/2.
__global__ void plain_space_pre(Tables<double> tb, LaunchArgs a, const PlainState *st, const cpx<double> *psi,
                                cpx<double> *y, int N, int n)
{
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int per = N / 2 + 1;
    const int b = (int)(gid / per), q = (int)(gid % per);
    if (b >= a.n_traj) return;
    const TrajDev d = a.trajs[b];
    const PlainState s = st[b];
    if (!running(s, d, n)) return;
    const MediumDev md = tb.media[d.medium];
    const double T3 = T3_of(tb, md, n), K3 = kappa_T3<double>(md.kfit, T3);
    const cpx<double> *p = psi + (size_t)b * N;
    cpx<double> *o = y + (size_t)b * N;
    if (q == 0) {
        o[0] = mk(0.0, 0.0);
    } else if (q == N / 2) {
        o[q] = scale(space_factor(tb, N, md, s.c, s.l, q, T3, K3) * p[q], 2.0);
    } else {
        const cpx<double> fa = space_factor(tb, N, md, s.c, s.l, q, T3, K3) * p[q];
        const cpx<double> fb = space_factor(tb, N, md, s.c, s.l, N - q, T3, K3) * p[N - q];
        const cpx<double> sum = scale(fa + fb, tb.sinpre[q]), dif = scale(fa - fb, 0.5);
        o[q] = sum + dif;
        o[N - q] = sum - dif;
    }
}


template <int RP>
__global__ void plain_fft_pass(const cpx<double> *in, cpx<double> *out, const cpx<double> *W, int N, int P,
                               LaunchArgs a, const PlainState *st, int n)
{
    const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int NB = N / RP;
    const int b = (int)(gid / NB), i = (int)(gid % NB);
    if (b >= a.n_traj) return;
    if (!running(st[b], a.trajs[b], n)) return;
    const int k = i & (P - 1);
    const cpx<double> *src = in + (size_t)b * N;
    cpx<double> v[RP];
#pragma unroll
    for (int m = 0; m < RP; ++m) {
        v[m] = src[i + m * NB];
        if (m) v[m] = v[m] * W[(long)m * k * (N / (P * RP))];
    }
    DFT<double, RP>::template run<1>(v);
    cpx<double> *dst = out + (size_t)b * N;
    const int base = (i - k) * RP + k;
#pragma unroll
    for (int m = 0; m < RP; ++m) dst[base + m * P] = v[m];
}

// post-processing of FFT output Y into the DST S (natural order, in S), the odd prefix scan, then
// mode 0: y = pre(K_T S) for the second transform; mode 1: psi = K_V S and its norm.
__global__ void __launch_bounds__(PB) plain_post(Tables<double> tb, LaunchArgs a, const PlainState *st,
                                                 const cpx<double> *Y, cpx<double> *S, cpx<double> *out, double *n2,
                                                 int N, int n, int mode)
{
    const int b = blockIdx.x;
    const TrajDev d = a.trajs[b];
    const PlainState s = st[b];
    if (!running(s, d, n)) return;
    __shared__ double shr[PB / 32];
    __shared__ double shc[2 * (PB / 32)];
    const cpx<double> *Yb = Y + (size_t)b * N;
    cpx<double> *Sb = S + (size_t)b * N;
    const int half = N / 2;
    for (int k = threadIdx.x; k < half; k += PB) {
        const cpx<double> A = Yb[k], B = Yb[(N - k) & (N - 1)];
        Sb[2 * k] = (k == 0) ? mk(0.0, 0.0) : mul_i(scale(A - B, 0.5));
        Sb[2 * k + 1] = (k == 0) ? scale(A, 0.5) : scale(A + B, 0.5);
    }
    __syncthreads();
    // inclusive scan of Sb[2k+1], k < N/2: thread chunk [t*ch, t*ch + ch)
    const int ch = (half + PB - 1) / PB;
    const int k0 = threadIdx.x * ch;
    double tr = 0.0, ti = 0.0;
    for (int q = 0; q < ch && k0 + q < half; ++q) {
        const cpx<double> v = Sb[2 * (k0 + q) + 1];
        tr += v.x;
        ti += v.y;
    }
    double ir = tr, ii = ti;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double yr = __shfl_up_sync(0xffffffffu, ir, off), yi = __shfl_up_sync(0xffffffffu, ii, off);
        if (lane >= off) { ir += yr; ii += yi; }
    }
    if (lane == 31) { shc[2 * warp] = ir; shc[2 * warp + 1] = ii; }
    __syncthreads();
    double er = ir - tr, ei = ii - ti;
    for (int w = 0; w < warp; ++w) { er += shc[2 * w]; ei += shc[2 * w + 1]; }
    for (int q = 0; q < ch && k0 + q < half; ++q) {
        const cpx<double> v = Sb[2 * (k0 + q) + 1];
        er += v.x;
        ei += v.y;
        Sb[2 * (k0 + q) + 1] = mk(er, ei);
    }
    __syncthreads();
    cpx<double> *ob = out + (size_t)b * N;
    if (mode == 0) {
        for (int q = threadIdx.x; q <= half; q += PB) {
            if (q == 0) {
                ob[0] = mk(0.0, 0.0);
            } else if (q == half) {
                ob[q] = scale(Sb[q] * tb.KT[q], 2.0);
            } else {
                const cpx<double> fa = Sb[q] * tb.KT[q], fb = Sb[N - q] * tb.KT[N - q];
                const cpx<double> sum = scale(fa + fb, tb.sinpre[q]), dif = scale(fa - fb, 0.5);
                ob[q] = sum + dif;
                ob[N - q] = sum - dif;
            }
        }
    } else {
        const MediumDev md = tb.media[d.medium];
        const double T3 = T3_of(tb, md, n), K3 = kappa_T3<double>(md.kfit, T3);
        double acc = 0.0;
        for (int j = threadIdx.x; j < N; j += PB) {
            const cpx<double> f = space_factor(tb, N, md, s.c, s.l, j, T3, K3) * Sb[j];
            ob[j] = f;
            acc = fma(f.x, f.x, fma(f.y, f.y, acc));
        }
        const double tot = block_sum(acc, shr);
        if (threadIdx.x == 0) n2[b] = tot * tb.dr;
    }
}

__device__ void plain_write_obs(const Tables<double> &tb, const LaunchArgs &a, int b, const TrajDev &d,
                                const PlainState &s, const cpx<double> *p, int N, int ended, double *sh)
{
    const int basis_l[NBASIS] = {0, 0, 1, 0, 1, 2};
    double acc = 0.0;
    for (int j = threadIdx.x; j < N; j += PB) acc = fma(p[j].x, p[j].x, fma(p[j].y, p[j].y, acc));
    const double n2 = block_sum(acc, sh) * tb.dr;
    double ovr[NBASIS], ovi[NBASIS];
    for (int q = 0; q < NBASIS; ++q) {
        ovr[q] = 0.0;
        ovi[q] = 0.0;
        if (ended || s.c != 0 || basis_l[q] != s.l) continue;
        const double *phi = tb.eig + (size_t)q * N;
        double pr = 0.0, pi = 0.0;
        for (int j = threadIdx.x; j < N; j += PB) {
            pr += phi[j] * p[j].x;
            pi += phi[j] * p[j].y;
        }
        ovr[q] = block_sum(pr, sh) * tb.dr;
        ovi[q] = block_sum(pi, sh) * tb.dr;
    }
    if (a.states) {
        double *out = a.states + (size_t)b * N * 2;
        for (int j = threadIdx.x; j < N; j += PB) {
            out[2 * j] = p[j].x;
            out[2 * j + 1] = p[j].y;
        }
    }
    if (threadIdx.x == 0) {
        qtraj_obs o;
        for (int q = 0; q < NBASIS; ++q) {
            o.ov_re[q] = ovr[q];
            o.ov_im[q] = ovi[q];
            double sv = 0.0;
            if (!ended && s.c == 0 && basis_l[q] == s.l) {
                const double prob = (ovr[q] * ovr[q] + ovi[q] * ovi[q]) / n2;
                if (tb.ov0_zero[d.spec * NBASIS + q]) sv = prob;
                else {
                    const double a0 = tb.ov0[(d.spec * NBASIS + q) * 2], b0 = tb.ov0[(d.spec * NBASIS + q) * 2 + 1];
                    sv = prob / (a0 * a0 + b0 * b0);
                }
            }
            o.surv[q] = sv;
        }
        o.norm2 = n2;
        o.r0 = s.r0;
        o.l = s.l;
        o.color = s.c;
        o.n_jumps = s.nj;
        o.n_steps_exec = s.executed;
        o.flags = s.flags;
        o.first_jump_step = s.fj;
        o.last_jump_step = s.lj;
        o.jump_digest = s.digest;
        a.obs[b] = o;
    }
}

// waiting-time test after step n, the jump, and the read-out after the last step (Sec. 3.5 item 4)
__global__ void __launch_bounds__(PB) plain_jump(Tables<double> tb, LaunchArgs a, PlainState *st, cpx<double> *psi,
                                                 const double *n2in, int N, int n)
{
    const int b = blockIdx.x;
    const TrajDev d = a.trajs[b];
    PlainState s = st[b];
    if (!running(s, d, n)) return;
    __shared__ double sh[PB / 32];
    cpx<double> *p = psi + (size_t)b * N;
    const double n2 = n2in[b];
    s.executed = n + 1;
    int ended = 0, jump = 0;
    int l_new = s.l, c_new = s.c;
    if (!isfinite(n2)) {
        s.flags |= QTRAJ_F_NONFINITE;
        ended = 1;
        if (threadIdx.x == 0) atomicOr(a.status, 1);
    } else if (!a.nojump) {
        if (fabs(n2 - s.thr) < BORDER_EPS) s.flags |= QTRAJ_F_BORDERLINE;
        if (n2 <= s.thr) {
            if (tb.max_jumps >= 0 && s.nj >= tb.max_jumps) {
                s.flags |= QTRAJ_F_MAXJUMPS;
                ended = 1;
            } else {
                l_new = (s.ul < (double)s.l / (2.0 * s.l + 1.0)) ? s.l - 1 : s.l + 1;
                c_new = (s.c == 1 && s.uc < tb.p_os) ? 0 : 1;
                if (s.fj < 0) s.fj = n;
                if (tb.l_cap >= 0 && l_new > tb.l_cap) {
                    s.flags |= QTRAJ_F_LCAP;
                    s.l = l_new;
                    s.c = c_new;
                    ++s.nj;
                    s.lj = n;
                    s.digest = digest_jump(s.digest, n, s.l, s.c);
                    ended = 1;
                } else {
                    jump = 1;
                }
            }
        }
    }
    if (jump) {
        double acc = 0.0;
        for (int j = threadIdx.x; j < N; j += PB) {
            const double rj = j * tb.dr;
            const cpx<double> v = scale(p[j], rj);
            p[j] = v;
            acc = fma(v.x, v.x, fma(v.y, v.y, acc));
        }
        const double tot = block_sum(acc, sh) * tb.dr;
        const double inv = 1.0 / sqrt(tot);
        for (int j = threadIdx.x; j < N; j += PB) p[j] = scale(p[j], inv);
        __syncthreads();
        s.l = l_new;
        s.c = c_new;
        ++s.nj;
        s.lj = n;
        s.digest = digest_jump(s.digest, n, s.l, s.c);
        ++s.kdraw;
        const Draws dw = draws(d.seed, (uint32_t)s.kdraw);
        s.thr = dw.r;
        s.ul = dw.ul;
        s.uc = dw.uc;
    }
    if (ended || n == d.n_steps - 1) {
        plain_write_obs(tb, a, b, d, s, p, N, ended, sh);
        s.active = 0;
    }
    if (threadIdx.x == 0) st[b] = s;
}

// trajectories whose medium has no step at all (T0 <= Tf) are read out unevolved
__global__ void __launch_bounds__(PB) plain_finalize_empty(Tables<double> tb, LaunchArgs a, PlainState *st,
                                                           const cpx<double> *psi, int N)
{
    const int b = blockIdx.x;
    PlainState s = st[b];
    if (s.active != 2) return;
    __shared__ double sh[PB / 32];
    plain_write_obs(tb, a, b, a.trajs[b], s, psi + (size_t)b * N, N, 0, sh);
    if (threadIdx.x == 0) { s.active = 0; st[b] = s; }
}

} // namespace

cudaError_t plain_run(const Tables<double> &tb, const LaunchArgs &a, int N, int max_steps, PlainBuffers buf,
                      cudaStream_t stream, int *launches)
{
    const int B = a.n_traj;
    if (B == 0) return cudaSuccess;
    int nl = 0;
    plain_setup<<<B, PB, 0, stream>>>(tb, a, buf.st, buf.psi, N);
    ++nl;
    plain_finalize_empty<<<B, PB, 0, stream>>>(tb, a, buf.st, buf.psi, N);
    ++nl;
    const long pairs = (long)B * (N / 2 + 1);
    const int pre_blocks = (int)((pairs + 255) / 256);
    int logn = 0;
    while ((1 << logn) < N) ++logn;
    for (int n = 0; n < max_steps; ++n) {
        for (int half = 0; half < 2; ++half) {
            if (half == 0) {
                plain_space_pre<<<pre_blocks, 256, 0, stream>>>(tb, a, buf.st, buf.psi, buf.y, N, n);
                ++nl;
            }
            // FFT of buf.y: passes of radix 4, then one of radix 2 if log2 N is odd; result ends in `res`
            cpx<double> *src = buf.y, *dst = buf.z;
            int P = 1, rem = logn;
            while (rem > 0) {
                const int rp = rem >= 2 ? 4 : 2;
                const long nb = (long)B * (N / rp);
                const int blocks = (int)((nb + 255) / 256);
                if (rp == 4) plain_fft_pass<4><<<blocks, 256, 0, stream>>>(src, dst, tb.W, N, P, a, buf.st, n);
                else plain_fft_pass<2><<<blocks, 256, 0, stream>>>(src, dst, tb.W, N, P, a, buf.st, n);
                ++nl;
                P *= rp;
                rem -= rp == 4 ? 2 : 1;
                cpx<double> *t = src;
                src = dst;
                dst = t;
            }
            // src holds Y.  Post-processing writes S to buf.s and then the next input: the second
            // transform's input into buf.y (Y is dead by then), or the new state into buf.psi.
            plain_post<<<B, PB, 0, stream>>>(tb, a, buf.st, src, buf.s, half == 0 ? buf.y : buf.psi, buf.n2, N, n,
                                             half);
            ++nl;
        }
        plain_jump<<<B, PB, 0, stream>>>(tb, a, buf.st, buf.psi, buf.n2, N, n);
        ++nl;
    }
    if (launches) *launches += nl;
    return cudaGetLastError();
}

} // namespace qt
