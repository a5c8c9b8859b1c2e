// serve.cuh -- what the serving loop (serve.cu) and the context (capi.cu) share.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <new>

#include "../../include/gb3fmm.h"

namespace gb3 {
struct Serve;
// the context's serving state (created on first use), parameters and device
Serve*& ctx_serve(fmm_ctx* ctx);
const fmm_params* ctx_params(fmm_ctx* ctx);
int ctx_device(fmm_ctx* ctx);
// record msg as the context's last error and return code
int ctx_fail(fmm_ctx* ctx, int code, const char* msg);
// stop the slots once the queue has drained, free their workspaces
void serve_destroy(Serve* s);
uint64_t serve_workspace_bytes(Serve* s);
}  // namespace gb3
