// tcdft.cu -- the 16-point DFT blocks of the sine transforms' radix-16 FFT passes (Sec. 3.3: the
// transforms dominate the step) on the tensor cores, measured against the CUDA cores.
//
// One CTA of 256 threads holds a batch of 256 columns of 16 complex FP32 points in shared memory
// (column c, point m at c*18 + m; two buffers) and applies `passes` passes y_c = (F/4) x_c, F the DFT
// matrix exp(-2 pi i m'm/16).  F/4 is a quarter of a unitary matrix times 4, so |y| = |x| and four
// passes give x back exactly in exact arithmetic.
//
//   method 0  CUDA cores: the fused kernel's DFT16 (radix 4 x 4, constants in hi+lo), then x 1/4;
//             one column per thread.
//   tensor-core forms: mma.sync m16n8k16 -> FP32 on the real form [Re -Im; Im Re] of F/4.  The matrix
//   is split into PA parts and the data into PB parts of the operand type, and the products A_j B_k
//   of part orders j + k <= MAXORD are accumulated, smallest first; each product is four MMAs
//   (Re Re, -Im Im, Im Re, Re Im) per 8 columns.
//   method 1  BF16X3: BF16, PA = PB = 2, three products (hi.hi + hi.lo + lo.hi);
//   method 2  BF16X9: BF16, PA = 4, PB = 3, nine products (matrix to ~2^-34, like the hi+lo constants);
//   method 3  FP16X3: FP16, PA = PB = 2, three products;
//   method 4  FP16X5: FP16, PA = 3, PB = 2, five products (matrix to ~2^-35).
//   FP16 forms scale every column by a power of two to a largest value in [2^14, 2^15) before the split
//   (the low parts stay normal), and store matrix part j times 2^(11 j) with its own accumulator, the
//   accumulators combined as acc_0 + 2^-11 acc_1 + 2^-22 acc_2.
// A warp takes tiles of 8 columns: lane (g, t) loads points 2t, 2t+1, 2t+8, 2t+9 of column g (the
// B fragment) and receives outputs g and g+8 of columns 2t and 2t+1 (the accumulator fragment).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <vector>

#include "api_internal.h"
#include "qtraj_device.cuh"

namespace {

constexpr int COLS = 256, PTS = 16, LD = 18, THREADS = 256, BUF = COLS * LD;

template <int METHOD> struct Form {
    static constexpr bool F16 = METHOD >= 3;
    static constexpr int PA = METHOD == 2 ? 4 : METHOD == 4 ? 3 : 2;
    static constexpr int PB = METHOD == 2 ? 3 : 2;
    static constexpr int MAXORD = METHOD == 2 ? 3 : METHOD == 4 ? 2 : 1;
    static constexpr int NACC = F16 ? PA : 1;   // accumulators: one per scaled matrix part (FP16)
};

// e^{-2 pi i k/16} in double from cos(pi/8), sin(pi/8), sqrt(1/2)
__device__ void w16(int k, double &re, double &im)
{
    constexpr double c1 = 0.92387953251128675613, s1 = 0.38268343236508977173, h = 0.70710678118654752440;
    const int q = k & 3, quad = (k >> 2) & 3;      // e^{-2 pi i q/16} = c - i s
    const double c = q == 0 ? 1.0 : q == 1 ? c1 : q == 2 ? h : s1;
    const double s = q == 0 ? 0.0 : q == 1 ? s1 : q == 2 ? h : c1;
    double r = c, i = -s;
    for (int n = 0; n < quad; ++n) {               // times e^{-i pi/2} = -i
        const double t = r;
        r = i;
        i = -t;
    }
    re = r;
    im = i;
}

template <bool F16> __device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    if constexpr (F16) {
        __half2 v = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&v);
    } else {
        __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&v);
    }
}
template <bool F16> __device__ __forceinline__ float2 unpack2(uint32_t u)
{
    if constexpr (F16) return __half22float2(*reinterpret_cast<__half2 *>(&u));
    else return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}
template <bool F16> __device__ __forceinline__ double round_part(double v)
{
    if constexpr (F16) return (double)__half2float(__double2half(v));
    else return (double)__bfloat162float(__double2bfloat16(v));
}

template <bool F16> __device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    if constexpr (F16)
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                     "{%0,%1,%2,%3};\n"
                     : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    else
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                     "{%0,%1,%2,%3};\n"
                     : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                     : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(127 + e) << 23); }   // |e| <= 126

template <int METHOD> __device__ __forceinline__ void tc_pass(const float2 *rd, float2 *wr, const uint32_t (&fr)[Form<METHOD>::PA][4],
                                                             const uint32_t (&fi)[Form<METHOD>::PA][4], int lane, int warp)
{
    using Fm = Form<METHOD>;
    constexpr bool F16 = Fm::F16;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
    for (int tile = 0; tile < COLS / 8 / (THREADS / 32); ++tile) {
        const int c0 = warp * (COLS / (THREADS / 32)) + tile * 8;
        const float4 lo = *reinterpret_cast<const float4 *>(rd + (c0 + g) * LD + 2 * t);
        const float4 hi = *reinterpret_cast<const float4 *>(rd + (c0 + g) * LD + 2 * t + 8);
        float xr[4] = {lo.x, lo.z, hi.x, hi.z}, xi[4] = {lo.y, lo.w, hi.y, hi.w};
        int e_in = 0, e_out0 = 0, e_out1 = 0;
        if constexpr (F16) {
            float amax = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) amax = fmaxf(amax, fmaxf(fabsf(xr[q]), fabsf(xi[q])));
            amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 1));
            amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 2));
            // amax in [2^E, 2^(E+1)), E = biased exponent - 127; scale to [2^14, 2^15)
            e_in = min(100, max(-100, 14 - ((int)((__float_as_uint(amax) >> 23) & 0xff) - 127)));
            const float s = pow2f(e_in);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                xr[q] *= s;
                xi[q] *= s;
            }
            e_out0 = __shfl_sync(0xffffffffu, e_in, 8 * t);       // a lane of column 2t
            e_out1 = __shfl_sync(0xffffffffu, e_in, 8 * t + 4);   // a lane of column 2t + 1
        }
        uint32_t br[Fm::PB][2], bi[Fm::PB][2], bn[Fm::PB][2];
#pragma unroll
        for (int k = 0; k < Fm::PB; ++k) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                br[k][h] = pack2<F16>(xr[2 * h], xr[2 * h + 1]);
                bi[k][h] = pack2<F16>(xi[2 * h], xi[2 * h + 1]);
                bn[k][h] = bi[k][h] ^ 0x80008000u;   // -Im x: both sign bits flipped
                if (k + 1 < Fm::PB) {                // the residuals, exact in FP32
                    const float2 ur = unpack2<F16>(br[k][h]), ui = unpack2<F16>(bi[k][h]);
                    xr[2 * h] -= ur.x;
                    xr[2 * h + 1] -= ur.y;
                    xi[2 * h] -= ui.x;
                    xi[2 * h + 1] -= ui.y;
                }
            }
        }
        float yr[Fm::NACC][4], yi[Fm::NACC][4];
#pragma unroll
        for (int a = 0; a < Fm::NACC; ++a)
#pragma unroll
            for (int q = 0; q < 4; ++q) yr[a][q] = yi[a][q] = 0.f;
#pragma unroll
        for (int s = Fm::MAXORD; s >= 0; --s)   // smallest products first
#pragma unroll
            for (int j = 0; j < Fm::PA; ++j) {
                const int k = s - j;
                if (k < 0 || k >= Fm::PB) continue;
                const int a = F16 ? j : 0;
                mma<F16>(yr[a], fr[j], br[k][0], br[k][1]);
                mma<F16>(yr[a], fi[j], bn[k][0], bn[k][1]);
                mma<F16>(yi[a], fi[j], br[k][0], br[k][1]);
                mma<F16>(yi[a], fr[j], bi[k][0], bi[k][1]);
            }
        float zr[4], zi[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if constexpr (F16) {
                float r = 0.f, i = 0.f;
#pragma unroll
                for (int a = Fm::NACC - 1; a >= 1; --a) {
                    r = fmaf(yr[a][q], pow2f(-11 * a), r);
                    i = fmaf(yi[a][q], pow2f(-11 * a), i);
                }
                const float us = pow2f(-((q & 1) ? e_out1 : e_out0));
                zr[q] = (yr[0][q] + r) * us;
                zi[q] = (yi[0][q] + i) * us;
            } else {
                zr[q] = yr[0][q];
                zi[q] = yi[0][q];
            }
        }
        // accumulator rows g (q = 0, 1) and g + 8 (q = 2, 3); columns 2t (q = 0, 2) and 2t + 1 (q = 1, 3)
        wr[(c0 + 2 * t) * LD + g] = make_float2(zr[0], zi[0]);
        wr[(c0 + 2 * t + 1) * LD + g] = make_float2(zr[1], zi[1]);
        wr[(c0 + 2 * t) * LD + g + 8] = make_float2(zr[2], zi[2]);
        wr[(c0 + 2 * t + 1) * LD + g + 8] = make_float2(zr[3], zi[3]);
    }
}

template <int METHOD>
__global__ void __launch_bounds__(THREADS) dft16_passes(const float2 *in, float2 *out, int passes)
{
    extern __shared__ __align__(16) float2 sm[];
    const float2 *src = in + (size_t)blockIdx.x * COLS * PTS;
    for (int i = threadIdx.x; i < COLS * PTS; i += THREADS) sm[(i / PTS) * LD + i % PTS] = src[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    using Fm = Form<METHOD>;
    static_assert(Fm::PB > 0 && Fm::MAXORD > 0 && Fm::NACC > 0 && (Fm::F16 || Fm::PA > 0), "form");
    uint32_t fr[Fm::PA][4], fi[Fm::PA][4];   // A fragments of the parts of Re F/4 and Im F/4
    if constexpr (METHOD != 0) {
        const int g = lane >> 2, t = lane & 3;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int row = (q & 1) ? g + 8 : g, col = (q & 2) ? 2 * t + 8 : 2 * t;
            float pr[2][Fm::PA], pi[2][Fm::PA];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                double vr, vi;
                w16(row * (col + e), vr, vi);
                vr *= 0.25;
                vi *= 0.25;
#pragma unroll
                for (int j = 0; j < Fm::PA; ++j) {   // part j, stored times 2^(11 j) in the FP16 forms
                    const double hr = round_part<Fm::F16>(Fm::F16 ? vr * (double)(1LL << (11 * j)) : vr);
                    const double hm = round_part<Fm::F16>(Fm::F16 ? vi * (double)(1LL << (11 * j)) : vi);
                    pr[e][j] = (float)hr;
                    pi[e][j] = (float)hm;
                    vr -= Fm::F16 ? hr / (double)(1LL << (11 * j)) : hr;
                    vi -= Fm::F16 ? hm / (double)(1LL << (11 * j)) : hm;
                }
            }
#pragma unroll
            for (int j = 0; j < Fm::PA; ++j) {
                fr[j][q] = pack2<Fm::F16>(pr[0][j], pr[1][j]);
                fi[j][q] = pack2<Fm::F16>(pi[0][j], pi[1][j]);
            }
        }
    }
    __syncthreads();

    for (int p = 0; p < passes; ++p) {
        const float2 *rd = sm + (p & 1) * BUF;
        float2 *wr = sm + ((p & 1) ^ 1) * BUF;
        if constexpr (METHOD == 0) {
            const int c = threadIdx.x;
            qt::cpx<float> x[PTS];
#pragma unroll
            for (int m = 0; m < PTS; m += 2) {
                const float4 v = *reinterpret_cast<const float4 *>(rd + c * LD + m);
                x[m] = qt::mk(v.x, v.y);
                x[m + 1] = qt::mk(v.z, v.w);
            }
            qt::DFT<float, 16>::template run<1>(x);
#pragma unroll
            for (int m = 0; m < PTS; m += 2)
                *reinterpret_cast<float4 *>(wr + c * LD + m) =
                    make_float4(0.25f * x[m].x, 0.25f * x[m].y, 0.25f * x[m + 1].x, 0.25f * x[m + 1].y);
        } else {
            tc_pass<METHOD>(rd, wr, fr, fi, lane, warp);
        }
        __syncthreads();
    }
    const float2 *fin = sm + (passes & 1) * BUF;
    float2 *dst = out + (size_t)blockIdx.x * COLS * PTS;
    for (int i = threadIdx.x; i < COLS * PTS; i += THREADS) dst[i] = fin[(i / PTS) * LD + i % PTS];
}

using KernelFn = void (*)(const float2 *, float2 *, int);

} // namespace

extern "C" qtraj_status qtraj_dft16_study(int method, int n_batches, int passes, const double *x_host, double *y_host,
                                         double *ms)
{
    qt::api_clear_error();
    if (method < 0 || method > 4 || n_batches <= 0 || passes < 0 || !x_host || !y_host || !ms)
        return qt::api_fail(QTRAJ_EINVAL, "method 0..4, n_batches > 0, passes >= 0 and the three buffers required");
    const size_t n = (size_t)n_batches * COLS * PTS;
    std::vector<float2> h(n);
    for (size_t i = 0; i < n; ++i) h[i] = make_float2((float)x_host[2 * i], (float)x_host[2 * i + 1]);
    float2 *d_in = nullptr, *d_out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    qtraj_status st = QTRAJ_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && st == QTRAJ_OK) st = qt::api_fail(QTRAJ_ECUDA, cudaGetErrorString(e));
        return st == QTRAJ_OK;
    };
    const int smem = 2 * BUF * (int)sizeof(float2);
    const KernelFn kernels[5] = {dft16_passes<0>, dft16_passes<1>, dft16_passes<2>, dft16_passes<3>, dft16_passes<4>};
    const KernelFn k = kernels[method];
    if (ok(cudaMalloc(&d_in, n * sizeof(float2))) && ok(cudaMalloc(&d_out, n * sizeof(float2))) &&
        ok(cudaMemcpy(d_in, h.data(), n * sizeof(float2), cudaMemcpyHostToDevice)) && ok(cudaEventCreate(&e0)) &&
        ok(cudaEventCreate(&e1)) && ok(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) {
        k<<<n_batches, THREADS, smem>>>(d_in, d_out, passes);   // warm-up
        if (ok(cudaGetLastError()) && ok(cudaEventRecord(e0))) {
            k<<<n_batches, THREADS, smem>>>(d_in, d_out, passes);
            if (ok(cudaGetLastError()) && ok(cudaEventRecord(e1)) && ok(cudaEventSynchronize(e1))) {
                float tms = 0.f;
                if (ok(cudaEventElapsedTime(&tms, e0, e1))) *ms = tms;
                if (ok(cudaMemcpy(h.data(), d_out, n * sizeof(float2), cudaMemcpyDeviceToHost)))
                    for (size_t i = 0; i < n; ++i) {
                        y_host[2 * i] = h[i].x;
                        y_host[2 * i + 1] = h[i].y;
                    }
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (d_in) cudaFree(d_in);
    if (d_out) cudaFree(d_out);
    return st;
}
