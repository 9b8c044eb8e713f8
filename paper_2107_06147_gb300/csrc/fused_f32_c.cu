// fused_f32_c.cu -- float instantiations of the fused trajectory kernel for N in {8192, 16384}.
#include "fused.cuh"
#include "fused_launch.cuh"

namespace qt {

cudaError_t fused_launch_f32_c(int N, const Tables<float> &tb, const LaunchArgs &a, int sm_count, int max_ctas,
                             cudaStream_t s, FusedInfo *info, bool query_only, int variant)
{
    // the per-step summary runs the traced twin of variant 0, the KSU potential its own twin of it
    if (a.trace_every > 0 || tb.potential == 1) variant = 0;
    switch (N) {
    case 8192: return tb.potential == 1 ? fused_go<float, 8192, 5>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : a.trace_every > 0 ? fused_go<float, 8192, 4>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : fused_go<float, 8192, 0>(tb, a, sm_count, max_ctas, s, info, query_only);
    case 16384: return tb.potential == 1 ? fused_go<float, 16384, 5>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : a.trace_every > 0 ? fused_go<float, 16384, 4>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : fused_go<float, 16384, 0>(tb, a, sm_count, max_ctas, s, info, query_only);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace qt
