// Device helpers shared by the persistent kernels: asynchronous global->shared
// copies, the bounded grid barrier and small numeric utilities.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "perks.h"

namespace perks {

// ------------------------------------------------------------------ storage

template <typename T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

template <typename T> __device__ __forceinline__ typename AccOf<T>::type to_acc(T v) {
    return static_cast<typename AccOf<T>::type>(v);
}
template <> __device__ __forceinline__ float to_acc<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}
template <typename T> __device__ __forceinline__ T from_acc(typename AccOf<T>::type v) {
    return static_cast<T>(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

// ------------------------------------------------------------- async copies

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// cp.async of one 4-, 8- or 16-byte element: 16-byte copies bypass L1
// (.cg); smaller ones can only use .ca.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem_dst, const void *gmem_src) {
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
    if constexpr (BYTES == 16) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem_dst)),
                     "l"(gmem_src)
                     : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(smem_dst)),
                     "l"(gmem_src), "n"(BYTES)
                     : "memory");
    }
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ------------------------------------------------------------- grid barrier

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_gpu(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_gpu_add(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Device-side error record: word 0 = error code (0 = none), word 1 = the
// block that first failed, word 2 = the barrier epoch at which it failed.
struct DevError {
    int code;
    int block;
    int epoch;
    int pad;
};

__device__ __forceinline__ unsigned long long ld_relaxed_gpu_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acquire_gpu() {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

// Grid-wide barrier over `nblocks` co-resident blocks (a cooperative launch
// guarantees co-residency).  `counter` is a monotone 64-bit arrival count,
// zeroed before the launch; the e-th barrier (e = 1, 2, ...) completes when
// the count reaches e * nblocks.  After __syncthreads, thread 0 arrives with
// a gpu-scope release reduction (cumulative over the block's writes ordered
// before it by the bar.sync), polls with relaxed loads and, once the count is
// reached, issues one acquire fence; the closing __syncthreads orders every
// thread's later accesses after it.  No full (sc) fence is needed.  The wait
// is bounded by `timeout_ns` of %globaltimer: on expiry (or when another
// block has already failed) the block records BARRIER_TIMEOUT and the call
// returns false in every thread, so the caller leaves its loop and the whole
// grid winds down without hanging.
__device__ __forceinline__ bool grid_barrier(unsigned long long *counter, unsigned nblocks,
                                             unsigned long long &epoch, DevError *err,
                                             long long timeout_ns) {
    __shared__ int s_fail;
    __syncthreads();
    if (threadIdx.x == 0) {
        int fail = 0;
        ++epoch;
        const unsigned long long target = epoch * (unsigned long long)nblocks;
        red_release_gpu_add(counter, 1ull);
        if (ld_relaxed_gpu_u64(counter) < target) {
            const uint64_t t0 = global_timer_ns();
            unsigned spins = 0;
            for (;;) {
                if (timeout_ns == 0) {  // test hook: give up at the first wait
                    if (atomicCAS(&err->code, 0, PERKS_ERR_BARRIER_TIMEOUT) == 0) {
                        err->block = blockIdx.x;
                        err->epoch = (int)epoch;
                    }
                    fail = 1;
                    break;
                }
                if (ld_relaxed_gpu_u64(counter) >= target) break;
                if ((++spins & 255u) == 0) {
                    if (ld_relaxed_gpu(&err->code) != 0) { fail = 1; break; }
                    if ((long long)(global_timer_ns() - t0) > timeout_ns) {
                        if (atomicCAS(&err->code, 0, PERKS_ERR_BARRIER_TIMEOUT) == 0) {
                            err->block = blockIdx.x;
                            err->epoch = (int)epoch;
                        }
                        fail = 1;
                        break;
                    }
                }
            }
        }
        fence_acquire_gpu();
        s_fail = fail;
    }
    __syncthreads();
    return s_fail == 0;
}

// ----------------------------------------------------------- warp reductions

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace perks
