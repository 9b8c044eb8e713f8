// fused_f32_b.cu -- float instantiations of the fused trajectory kernel for N in {2048, 4096}.
#include "fused.cuh"
#include "fused_launch.cuh"

namespace qt {
cudaError_t fused_launch_f32_c(int N, const Tables<float> &tb, const LaunchArgs &a, int sm_count, int max_ctas,
                             cudaStream_t s, FusedInfo *info, bool query_only, int variant);
namespace {
template <int N, int V>
cudaError_t go(const Tables<float> &tb, const LaunchArgs &a, int sm_count, int max_ctas, cudaStream_t s, FusedInfo *info,
               bool query_only)
{
    auto k = fused_kernel<float, N, V>;
    constexpr int G = FusedPlan<N, V>::G;
    constexpr int smem = fused_smem_bytes<float, N, V>();
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
    if (query_only || a.n_traj <= 0) return cudaSuccess;
    long grid = (long)sm_count * occ;
    if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
    if (grid > a.n_traj) grid = a.n_traj;
    k<<<(int)grid, G, smem, s>>>(tb, a);
    return cudaGetLastError();
}
} // namespace

cudaError_t fused_launch_f32_b(int N, const Tables<float> &tb, const LaunchArgs &a, int sm_count, int max_ctas,
                             cudaStream_t s, FusedInfo *info, bool query_only, int variant)
{
    if (a.trace_every > 0) variant = 0;   // the per-step summary runs the traced twin of variant 0
    switch (N) {
    case 2048:
        switch (variant) {
        case 1: return go<2048, 1>(tb, a, sm_count, max_ctas, s, info, query_only);
        case 2: return go<2048, 2>(tb, a, sm_count, max_ctas, s, info, query_only);
        case 3: return go<2048, 3>(tb, a, sm_count, max_ctas, s, info, query_only);
        default: return a.trace_every > 0 ? go<2048, 4>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : go<2048, 0>(tb, a, sm_count, max_ctas, s, info, query_only);
        }
    case 4096:
        switch (variant) {
        case 1: return go<4096, 1>(tb, a, sm_count, max_ctas, s, info, query_only);
        case 2: return go<4096, 2>(tb, a, sm_count, max_ctas, s, info, query_only);
        case 3: return go<4096, 3>(tb, a, sm_count, max_ctas, s, info, query_only);
        default: return a.trace_every > 0 ? go<4096, 4>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : go<4096, 0>(tb, a, sm_count, max_ctas, s, info, query_only);
        }
    default: return fused_launch_f32_c(N, tb, a, sm_count, max_ctas, s, info, query_only, variant);
    }
}

} // namespace qt
