// fused_f32_c.cu -- float instantiations of the fused trajectory kernel for N in {8192, 16384}.
#include "fused.cuh"
#include "fused_launch.cuh"

namespace qt {
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

cudaError_t fused_launch_f32_c(int N, const Tables<float> &tb, const LaunchArgs &a, int sm_count, int max_ctas,
                             cudaStream_t s, FusedInfo *info, bool query_only, int variant)
{
    if (a.trace_every > 0) variant = 0;   // the per-step summary runs the traced twin of variant 0
    switch (N) {
    case 8192: return a.trace_every > 0 ? go<8192, 4>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : go<8192, 0>(tb, a, sm_count, max_ctas, s, info, query_only);
    case 16384: return a.trace_every > 0 ? go<16384, 4>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : go<16384, 0>(tb, a, sm_count, max_ctas, s, info, query_only);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace qt
