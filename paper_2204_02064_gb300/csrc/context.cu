// Context entry points of the C ABI: device queries, error messages and the
// barrier time limit shared by every persistent launch.
#include <mutex>

#include "common.cuh"
#include "internal.h"

using namespace perks;

namespace perks {

struct OptinRecord {
    const void *fn;
    int static_smem;
    unsigned long long devices;  // bit d: the limit is raised on device d
};
static constexpr int kOptinSlots = 2048;
static OptinRecord g_optin[kOptinSlots];
static int g_optin_used = 0;
static std::mutex g_optin_mutex;

perks_status smem_optin(perks_context *ctx, const void *fn, int *budget) {
    std::lock_guard<std::mutex> lock(g_optin_mutex);
    OptinRecord *rec = nullptr;
    for (int i = 0; i < g_optin_used; ++i)
        if (g_optin[i].fn == fn) { rec = &g_optin[i]; break; }
    int static_smem;
    if (rec) {
        static_smem = rec->static_smem;
    } else {
        cudaFuncAttributes fa;
        PERKS_CUDA(ctx, cudaFuncGetAttributes(&fa, fn));
        static_smem = (int)fa.sharedSizeBytes;
        if (g_optin_used < kOptinSlots) {
            rec = &g_optin[g_optin_used++];
            rec->fn = fn;
            rec->static_smem = static_smem;
            rec->devices = 0;
        }
    }
    const int b = ctx->smem_optin - static_smem;
    const bool known = rec && ctx->device < 64 && (rec->devices >> ctx->device & 1ull);
    if (!known) {
        PERKS_CUDA(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, b));
        // every persistent kernel wants the largest shared-memory share of the SM
        PERKS_CUDA(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared));
        if (rec && ctx->device < 64) rec->devices |= 1ull << ctx->device;
    }
    *budget = b;
    return PERKS_OK;
}

}  // namespace perks

namespace {

// `iterations` grid barriers and nothing else: the per-step synchronisation
// cost of a persistent kernel with this grid.
__global__ void barrier_bench_kernel(unsigned long long *counter, DevError *err, int iterations, long long timeout_ns) {
    unsigned long long epoch = 0;
    for (int i = 0; i < iterations; ++i)
        if (!grid_barrier(counter, gridDim.x, epoch, err, timeout_ns)) return;
}

// Eight independent fused multiply-add chains per thread, `iters` long: with
// 32 warps per SM enough FMAs are in flight to keep the FP64 pipe busy, so
// the rate measured is the pipe's throughput.  b < 1 and c keep every value
// bounded; the sums are written out so that no chain is dead code.
__global__ void __launch_bounds__(256) fp64_fma_kernel(double *out, int iters, double b, double c) {
    const double s = 1e-9 * (threadIdx.x + 1);
    double a0 = s, a1 = 2 * s, a2 = 3 * s, a3 = 4 * s, a4 = 5 * s, a5 = 6 * s, a6 = 7 * s, a7 = 8 * s;
    for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
        a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}

// Random gathers from an L2-resident vector (cache-global loads, as the
// row-vector SpMV issues them): eight independent linear-congruential index
// streams per thread keep loads in flight; the sums are written out.
template <typename T>
__global__ void __launch_bounds__(256) gather_kernel(const T *__restrict__ x, unsigned mask, int iters, T *out) {
    unsigned h[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k] = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 40503u * (k + 1);
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            h[k] = h[k] * 1664525u + 1013904223u;
            acc[k] += __ldcg(x + ((h[k] >> 7) & mask));
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
}

}  // namespace

extern "C" perks_status perks_gather_benchmark(perks_context *ctx, int32_t log2_elems, int32_t elem_bytes,
                                               int32_t iterations, double *gathers_per_s) {
    if (!ctx) return PERKS_ERR_INVALID_ARG;
    if (log2_elems < 10 || log2_elems > 28 || (elem_bytes != 4 && elem_bytes != 8) || iterations < 1 ||
        !gathers_per_s)
        return fail(ctx, PERKS_ERR_INVALID_ARG, "gather_benchmark: bad arguments");
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    const int threads = 256, blocks = 4 * ctx->sm_count;
    const size_t n = (size_t)1 << log2_elems;
    void *x = nullptr, *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&x, n * elem_bytes);
    if (e == cudaSuccess) e = cudaMemset(x, 0, n * elem_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)elem_bytes * threads * blocks);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up (and fills L2)
        e = cudaEventRecord(e0);
        if (elem_bytes == 8)
            gather_kernel<double><<<blocks, threads>>>((const double *)x, (unsigned)(n - 1), iterations,
                                                       (double *)out);
        else
            gather_kernel<float><<<blocks, threads>>>((const float *)x, (unsigned)(n - 1), iterations,
                                                      (float *)out);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (x) cudaFree(x);
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gather_benchmark");
    *gathers_per_s = 8.0 * (double)iterations * threads * blocks / (ms * 1e-3);
    return PERKS_OK;
}

extern "C" perks_status perks_fp64_fma_benchmark(perks_context *ctx, int32_t iterations, double *tflops) {
    if (!ctx) return PERKS_ERR_INVALID_ARG;
    if (iterations < 1 || !tflops) return fail(ctx, PERKS_ERR_INVALID_ARG, "fp64_fma_benchmark: bad arguments");
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    const int threads = 256, blocks = 4 * ctx->sm_count;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(double) * threads * blocks);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
        if (e == cudaSuccess) e = cudaEventRecord(e0);
        fp64_fma_kernel<<<blocks, threads>>>(out, iterations, 0.9999999, 1e-7);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fp64_fma_benchmark");
    const double flop = 2.0 * 8.0 * (double)iterations * threads * blocks;
    *tflops = flop / (ms * 1e-3) / 1e12;
    return PERKS_OK;
}

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

extern "C" perks_status perks_barrier_benchmark(perks_context *ctx, int32_t blocks, int32_t threads,
                                                int32_t iterations, double *us_per_barrier) {
    if (!ctx) return PERKS_ERR_INVALID_ARG;
    if (blocks < 1 || threads < 32 || threads > 1024 || iterations < 1 || !us_per_barrier)
        return fail(ctx, PERKS_ERR_INVALID_ARG, "barrier_benchmark: bad arguments");
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    int per_sm = 0;
    PERKS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, barrier_bench_kernel, threads, 0));
    if ((long long)per_sm * ctx->sm_count < blocks)
        return fail(ctx, PERKS_ERR_LAUNCH_TOO_LARGE, "barrier_benchmark: %d blocks are not co-resident", blocks);
    unsigned long long *counter = nullptr;
    DevError *err = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&counter, sizeof(*counter));
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(*err));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    DevError h{};
    long long tmo = ctx->timeout_ns;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
        e = cudaMemset(counter, 0, sizeof(*counter));
        if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(*err));
        void *args[] = {&counter, &err, &iterations, &tmo};
        if (e == cudaSuccess) e = cudaEventRecord(e0);
        if (e == cudaSuccess) e = cudaLaunchCooperativeKernel((const void *)barrier_bench_kernel, dim3(blocks),
                                                             dim3(threads), args, 0, nullptr);
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(h), cudaMemcpyDeviceToHost);
    }
    if (counter) cudaFree(counter);
    if (err) cudaFree(err);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "barrier_benchmark");
    if (h.code) return fail(ctx, h.code, "barrier_benchmark: barrier wait timed out");
    *us_per_barrier = 1e3 * ms / iterations;
    return PERKS_OK;
}
