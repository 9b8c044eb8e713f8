// fused_launch.cuh -- host entry to the fused kernel instantiations (one per precision and N).
#pragma once
#include "qtraj_device.cuh"

namespace qt {

struct FusedInfo {
    int G, R, smem, ctas_per_sm, regs;
};

// Launches the fused kernel for grid size N (query_only: fills info and launches nothing).
// max_ctas bounds the persistent grid (0 = one full wave at the kernel's occupancy).  variant selects
// the occupancy target and radix (see FusedPlan, FusedBounds); variants 1-3 exist for FP32 N in
// {2048, 4096} and fall back to variant 0 elsewhere.
cudaError_t fused_launch_f32(int N, const Tables<float> &tb, const LaunchArgs &a, int sm_count, int max_ctas,
                             cudaStream_t s, FusedInfo *info, bool query_only, int variant);
cudaError_t fused_launch_f64(int N, const Tables<double> &tb, const LaunchArgs &a, int sm_count, int max_ctas,
                             cudaStream_t s, FusedInfo *info, bool query_only, int variant);

} // namespace qt
