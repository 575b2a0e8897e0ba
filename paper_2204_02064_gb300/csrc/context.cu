// Context entry points of the C ABI: device queries, error messages and the
// barrier time limit shared by every persistent launch.
#include "internal.h"

using namespace perks;

extern "C" perks_status perks_context_create(int device, perks_context **out) {
    if (!out) return PERKS_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return PERKS_ERR_INVALID_ARG;
    perks_context *ctx = new perks_context();
    ctx->device = device;
    cudaDeviceProp prop;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete ctx;
        return PERKS_ERR_CUDA;
    }
    ctx->sm_count = prop.multiProcessorCount;
    ctx->smem_optin = (int)prop.sharedMemPerBlockOptin;
    ctx->smem_per_sm = (int)prop.sharedMemPerMultiprocessor;
    ctx->l2_bytes = prop.l2CacheSize;
    ctx->cooperative = prop.cooperativeLaunch;
    if (!ctx->cooperative) {
        delete ctx;
        return PERKS_ERR_UNSUPPORTED;
    }
    *out = ctx;
    return PERKS_OK;
}

extern "C" perks_status perks_context_destroy(perks_context *ctx) {
    delete ctx;
    return PERKS_OK;
}

extern "C" const char *perks_last_error(const perks_context *ctx) {
    if (!ctx) return "NULL context";
    return ctx->last_error.c_str();
}

extern "C" perks_status perks_context_set_barrier_timeout(perks_context *ctx, int64_t limit_ns) {
    if (!ctx) return PERKS_ERR_INVALID_ARG;
    if (limit_ns < 0) return fail(ctx, PERKS_ERR_INVALID_ARG, "barrier timeout must be >= 0");
    ctx->timeout_ns = limit_ns;
    return PERKS_OK;
}

extern "C" perks_status perks_context_info(const perks_context *ctx, int32_t *sm_count,
                                           int32_t *smem_per_block, int64_t *l2_bytes) {
    if (!ctx) return PERKS_ERR_INVALID_ARG;
    if (sm_count) *sm_count = ctx->sm_count;
    if (smem_per_block) *smem_per_block = ctx->smem_optin;
    if (l2_bytes) *l2_bytes = ctx->l2_bytes;
    return PERKS_OK;
}
