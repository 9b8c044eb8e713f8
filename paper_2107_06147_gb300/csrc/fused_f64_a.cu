// fused_f64_a.cu -- double instantiations of the fused trajectory kernel for N in {16, 32, 64, 128, 256, 512, 1024}.
#include "fused.cuh"
#include "fused_launch.cuh"

namespace qt {
cudaError_t fused_launch_f64_b(int N, const Tables<double> &tb, const LaunchArgs &a, int sm_count, int max_ctas,
                             cudaStream_t s, FusedInfo *info, bool query_only, int variant);

cudaError_t fused_launch_f64(int N, const Tables<double> &tb, const LaunchArgs &a, int sm_count, int max_ctas,
                             cudaStream_t s, FusedInfo *info, bool query_only, int variant)
{
    // the per-step summary runs the traced twin of variant 0, the KSU potential its own twin of it
    if (a.trace_every > 0 || tb.potential == 1) variant = 0;
    switch (N) {
    case 16: return tb.potential == 1 ? fused_go<double, 16, 5>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : a.trace_every > 0 ? fused_go<double, 16, 4>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : fused_go<double, 16, 0>(tb, a, sm_count, max_ctas, s, info, query_only);
    case 32: return tb.potential == 1 ? fused_go<double, 32, 5>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : a.trace_every > 0 ? fused_go<double, 32, 4>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : fused_go<double, 32, 0>(tb, a, sm_count, max_ctas, s, info, query_only);
    case 64: return tb.potential == 1 ? fused_go<double, 64, 5>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : a.trace_every > 0 ? fused_go<double, 64, 4>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : fused_go<double, 64, 0>(tb, a, sm_count, max_ctas, s, info, query_only);
    case 128: return tb.potential == 1 ? fused_go<double, 128, 5>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : a.trace_every > 0 ? fused_go<double, 128, 4>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : fused_go<double, 128, 0>(tb, a, sm_count, max_ctas, s, info, query_only);
    case 256: return tb.potential == 1 ? fused_go<double, 256, 5>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : a.trace_every > 0 ? fused_go<double, 256, 4>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : fused_go<double, 256, 0>(tb, a, sm_count, max_ctas, s, info, query_only);
    case 512: return tb.potential == 1 ? fused_go<double, 512, 5>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : a.trace_every > 0 ? fused_go<double, 512, 4>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : fused_go<double, 512, 0>(tb, a, sm_count, max_ctas, s, info, query_only);
    case 1024: return tb.potential == 1 ? fused_go<double, 1024, 5>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : a.trace_every > 0 ? fused_go<double, 1024, 4>(tb, a, sm_count, max_ctas, s, info, query_only)
                                  : fused_go<double, 1024, 0>(tb, a, sm_count, max_ctas, s, info, query_only);
    default: return fused_launch_f64_b(N, tb, a, sm_count, max_ctas, s, info, query_only, variant);
    }
}

} // namespace qt
