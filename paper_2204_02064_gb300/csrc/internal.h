// Host-side internals shared by the translation units of the library.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>

#include <cuda_runtime.h>

#include "perks.h"

struct perks_context {
    int device = 0;
    int sm_count = 0;
    int smem_optin = 0;        // max dynamic shared memory per block (opt-in)
    int smem_per_sm = 0;
    long long l2_bytes = 0;
    int cooperative = 0;
    long long timeout_ns = 2000000000LL;
    bool quiet = false;        // record no message (a stack context of an allocation-free call)
    std::string last_error = "no error";
};

namespace perks {

inline perks_status fail(perks_context *ctx, perks_status st, const char *fmt, ...) {
    if (!ctx || ctx->quiet) return st;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
    return st;
}

inline perks_status cuda_fail(perks_context *ctx, cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(ctx, PERKS_ERR_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
    if (e == cudaErrorCooperativeLaunchTooLarge)
        return fail(ctx, PERKS_ERR_LAUNCH_TOO_LARGE, "%s: %s", what, cudaGetErrorString(e));
    return fail(ctx, PERKS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define PERKS_CUDA(ctx, call)                                         \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return ::perks::cuda_fail(ctx, e_, #call); \
    } while (0)

// Sets the context's device current for the calling thread.
// Makes the context's device current and clears the runtime's last-error
// slot, so the launch checks of this call report this call's launches only
// (not an error some earlier, unrelated runtime call left behind).
inline perks_status use_device(perks_context *ctx) {
    PERKS_CUDA(ctx, cudaSetDevice(ctx->device));
    (void)cudaGetLastError();
    return PERKS_OK;
}

// Raises the dynamic shared memory limit of kernel `fn` on the context's
// device (which must be current) to the device's opt-in maximum less the
// kernel's static shared memory, and returns that budget in *budget.
// cudaFuncSetAttribute acts on the current device only, so the call is made
// once per (kernel, device) and recorded in a fixed-size table under a mutex
// (no heap use; safe from several host threads).
perks_status smem_optin(perks_context *ctx, const void *fn, int *budget);

inline size_t dtype_size(int dtype) {
    return dtype == PERKS_F64 ? 8 : dtype == PERKS_F32 ? 4 : 2;
}

}  // namespace perks
