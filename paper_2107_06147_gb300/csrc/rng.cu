// rng.cu -- the device generator of the trajectory kernels exposed for checking: Philox4x32-10
// words for given (counter, key) pairs, and the three waiting-period uniforms of given (seed, k)
// pairs, computed by the same device functions the fused and plain forms call (qtraj_device.cuh).
#include <cuda_runtime.h>

#include "api_internal.h"
#include "qtraj_device.cuh"

namespace {

__global__ void philox_words(const uint32_t *ctr, const uint32_t *key, int n, uint32_t *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t c0 = ctr[4 * i], c1 = ctr[4 * i + 1], c2 = ctr[4 * i + 2], c3 = ctr[4 * i + 3];
        qt::philox10(c0, c1, c2, c3, key[2 * i], key[2 * i + 1]);
        out[4 * i] = c0;
        out[4 * i + 1] = c1;
        out[4 * i + 2] = c2;
        out[4 * i + 3] = c3;
    }
}

__global__ void period_draws(const uint64_t *seed, const uint32_t *k, int n, double *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const qt::Draws d = qt::draws(seed[i], k[i]);
        out[3 * i] = d.r;
        out[3 * i + 1] = d.ul;
        out[3 * i + 2] = d.uc;
    }
}

int grid_for(int n)
{
    const int b = (n + 255) / 256;
    return b < 1 ? 1 : (b > 4096 ? 4096 : b);
}

} // namespace

extern "C" qtraj_status qtraj_philox4x32_10(const uint32_t *d_ctr, const uint32_t *d_key, int n, uint32_t *d_out,
                                           void *stream)
{
    qt::api_clear_error();
    if (n < 0 || (n > 0 && (!d_ctr || !d_key || !d_out))) return qt::api_fail(QTRAJ_EINVAL, "null buffer or n < 0");
    if (n == 0) return QTRAJ_OK;
    philox_words<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(d_ctr, d_key, n, d_out);
    if (cudaGetLastError() != cudaSuccess) return qt::api_fail(QTRAJ_ECUDA, "philox launch failed");
    return QTRAJ_OK;
}

extern "C" qtraj_status qtraj_period_draws(const uint64_t *d_seed, const uint32_t *d_k, int n, double *d_out,
                                          void *stream)
{
    qt::api_clear_error();
    if (n < 0 || (n > 0 && (!d_seed || !d_k || !d_out))) return qt::api_fail(QTRAJ_EINVAL, "null buffer or n < 0");
    if (n == 0) return QTRAJ_OK;
    period_draws<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(d_seed, d_k, n, d_out);
    if (cudaGetLastError() != cudaSuccess) return qt::api_fail(QTRAJ_ECUDA, "draws launch failed");
    return QTRAJ_OK;
}
