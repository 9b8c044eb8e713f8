// plain.cuh -- interface of the plain per-step FP64 form (plain.cu).
#pragma once
#include "qtraj_device.cuh"

namespace qt {

// per-trajectory state of the plain form, kept in HBM between the kernels of a step
struct PlainState {
    double thr, ul, uc, r0; // current waiting-time threshold and jump draws; first threshold
    int l, c, nj, fj, flags, active, kdraw, executed, lj;
    uint32_t digest;   // jump digest (qtraj_obs.jump_digest)
};

struct PlainBuffers {
    cpx<double> *psi, *y, *z, *s; // [n_traj][N] each: state, FFT ping, FFT pong, DST output
    double *n2;                   // [n_traj]
    PlainState *st;               // [n_traj]
};

// Enqueues the whole evolution of a.n_traj trajectories (max_steps = longest medium) on `stream`.
cudaError_t plain_run(const Tables<double> &tb, const LaunchArgs &a, int N, int max_steps, PlainBuffers buf,
                      cudaStream_t stream, int *launches);

} // namespace qt
