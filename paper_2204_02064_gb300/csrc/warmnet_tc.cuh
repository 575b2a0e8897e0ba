// Tensor-core (tcgen05) 3x3 convolution, 32 -> 32 channels, bf16 activations
// (NCHW), fp32 accumulation in tensor memory: the two inner layers of the
// warm-start network, as an implicit GEMM.
//
// A tile is 128 consecutive pixels of one image in row-major order (it may
// span several short rows, so no MMA row is wasted on grids narrower than 128
// pixels; pixels past the image's end are zero rows).  For each of the 9 taps
// the tile's input window (128 pixels x 32 channels, shifted by the tap's
// offset times the dilation, zero outside the image) is the A operand
// (M = 128, K = 32) and the tap's weights W[:, :, tap] the B operand
// (N = 32, K = 32); D[128 x 32] += A_tap B_tap^T over the 9 taps and two
// K = 16 steps is 18 tcgen05.mma (kind::f16, bf16 x bf16 -> fp32) issued by
// one thread, accumulating in 32 TMEM columns.  The epilogue reads the
// accumulator back with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31, i.e.
// pixels 32w..32w+31), adds the bias, applies ReLU and stores bf16.
//
// Operands sit in shared memory in the canonical no-swizzle K-major layout:
// 8-row x 16-byte core matrices, the core matrix of rows 8i..8i+7 and
// channels 8j..8j+7 at byte offset (i * 4 + j) * 128, so the descriptor's
// leading-dimension offset (next core matrix along K) is 128 bytes and its
// stride offset (next 8-row group) 512 bytes; the second K = 16 step starts
// 256 bytes further.  Waits on the MMA-completion mbarrier are bounded; every
// exit path frees the TMEM it allocated.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace perks {

constexpr int kTcPix = 128;                       // pixels per tile (MMA M)
constexpr int kTcC = 32;                          // channels (MMA N and K)
constexpr int kTcTapBytes = kTcPix * kTcC * 2;    // 8 KB: one tap's A operand
constexpr int kTcWBytes = kTcC * kTcC * 2;        // 2 KB: one tap's B operand
constexpr int kTcThreads = 128;

__host__ __device__ constexpr size_t tc_conv_smem() {
    return 9 * (size_t)kTcTapBytes + 9 * (size_t)kTcWBytes + 16;
}

// Byte offset of element (row, k) in a no-swizzle K-major operand with K = 32.
__device__ __forceinline__ int tc_off(int row, int k) {
    return ((row >> 3) * 4 + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);            // start address
    d |= (uint64_t)((128 >> 4) & 0x3FFF) << 16;       // leading byte offset: next core matrix along K
    d |= (uint64_t)((512 >> 4) & 0x3FFF) << 32;       // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                           // descriptor version (tcgen05)
    // base offset 0, leading-offset mode 0, layout type 0 = no swizzle
    return d;
}

// kind::f16 instruction descriptor: D fp32, A and B bf16, both K-major,
// N = 32, M = 128.
__host__ __device__ constexpr uint32_t tc_idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcC >> 3) << 17) | ((uint32_t)(kTcPix >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool tc_wait(unsigned long long *bar, unsigned parity, DevError *err) {
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_timer_ns() - t0 > 1000000000ull) {  // 1 s: the MMAs of one tile take microseconds
            if (err && atomicCAS(&err->code, 0, PERKS_ERR_BARRIER_TIMEOUT) == 0) err->block = blockIdx.x;
            return false;
        }
    }
}

// out[img][co][y][x] = relu(bias[co] + sum_{ci, tap} w[co][ci][tap] in[img][ci][y + dy][x + dx])
// for all images; w is the fp32 layer weight array [32][32][9].
__global__ void __launch_bounds__(kTcThreads, 1) tc_conv32_kernel(const __nv_bfloat16 *__restrict__ in,
                                                                const float *__restrict__ w,
                                                                const float *__restrict__ bias,
                                                                __nv_bfloat16 *__restrict__ out, int nimg, int H,
                                                                int W, int dil, DevError *err) {
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *sa = smem;                                  // 9 taps x 8 KB
    unsigned char *sb = smem + 9 * kTcTapBytes;                // 9 taps x 2 KB
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(sb + 9 * kTcWBytes);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // B operands (weights) once per block, converted to bf16
    for (int e = tid; e < 9 * kTcC * kTcC; e += blockDim.x) {
        const int tap = e / (kTcC * kTcC), n = (e / kTcC) % kTcC, k = e % kTcC;
        *reinterpret_cast<__nv_bfloat16 *>(sb + tap * kTcWBytes + tc_off(n, k)) =
            __float2bfloat16_rn(w[(n * kTcC + k) * 9 + tap]);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = tc_idesc();

    const long long plane = (long long)H * W;
    const long long tiles_img = (plane + kTcPix - 1) / kTcPix;
    const long long ntiles = (long long)nimg * tiles_img;
    unsigned parity = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int img = (int)(t / tiles_img);
        const long long p0 = (t % tiles_img) * kTcPix;  // first pixel of the tile in its image
        // A operands: pixel p0 + tid of the tile, all 32 channels, 9 taps
        const long long pm = p0 + tid;
        const bool valid = pm < plane;
        const int y = valid ? (int)(pm / W) : 0, x = valid ? (int)(pm % W) : 0;
        const __nv_bfloat16 *inb = in + (long long)img * kTcC * plane;
#pragma unroll 1
        for (int tap = 0; tap < 9; ++tap) {
            const int yy = y + (tap / 3 - 1) * dil, xx = x + (tap % 3 - 1) * dil;
            const bool inside = valid && yy >= 0 && yy < H && xx >= 0 && xx < W;
            unsigned char *dst = sa + tap * kTcTapBytes;
#pragma unroll
            for (int kg = 0; kg < 4; ++kg) {
                __align__(16) __nv_bfloat16 v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    v[j] = inside ? inb[(long long)(kg * 8 + j) * plane + (long long)yy * W + xx] : __float2bfloat16_rn(0.f);
                *reinterpret_cast<uint4 *>(dst + tc_off(tid, kg * 8)) = *reinterpret_cast<const uint4 *>(v);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            uint32_t acc = 0;
            for (int tap = 0; tap < 9; ++tap)
                for (int ks = 0; ks < 2; ++ks) {
                    const uint64_t ad = tc_smem_desc(smem_u32(sa + tap * kTcTapBytes + ks * 256));
                    const uint64_t bd = tc_smem_desc(smem_u32(sb + tap * kTcWBytes + ks * 256));
                    tc_mma(tmem, ad, bd, idesc, acc);
                    acc = 1;
                }
            tc_commit(bar);
        }
        ok = tc_wait(bar, parity, err);
        parity ^= 1u;
        ok = __syncthreads_and(ok) != 0;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(tmem + ((uint32_t)(warp * 32) << 16)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const long long pe = p0 + warp * 32 + lane;  // TMEM lane = pixel of the tile
        if (pe < plane) {
            __nv_bfloat16 *ob = out + (long long)img * kTcC * plane + pe;
#pragma unroll
            for (int c = 0; c < kTcC; ++c) {
                const float v = fmaxf(__uint_as_float(r[c]) + bias[c], 0.f);
                ob[(long long)c * plane] = __float2bfloat16_rn(v);
            }
        }
        // the next tile's operand stores and MMAs come after every thread's read of D
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
}

}  // namespace perks
