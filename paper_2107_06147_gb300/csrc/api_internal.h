// api_internal.h -- library-internal entry points of api.cu used by the serving loop (serve.cu).
// Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include "qtraj.h"

namespace qt {
// Sets the calling thread's qtraj_last_error message and returns st.
qtraj_status api_fail(qtraj_status st, const char *msg);
void api_clear_error();
// Enqueues on `stream` the copy of the last evolve's records to host memory (pinned, so that the
// copy is asynchronous) and returns without waiting.
qtraj_status obs_to_host_async(qtraj_ctx *c, void *host, cudaStream_t stream);
// Grows the context's device media table and its pinned staging buffer for an evolve of n
// trajectories with up to n media now, so that such an evolve later neither frees nor allocates
// (either can wait for the whole device).
qtraj_status reserve_media(qtraj_ctx *c, int n);
// The validity rules qtraj_evolve applies to a medium; nullptr if valid, else the reason.
const char *medium_problem(const qtraj_medium &m);
} // namespace qt
