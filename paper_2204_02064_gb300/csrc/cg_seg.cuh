// Column-segmented SpMV for the persistent CG (the SPMV_SEG kind).
//
// A CSR SpMV with uniformly scattered columns is bound by its gathers: every
// x[col] touches a different cache line, and an SM's L1 serves about one
// line per clock.  Here each block keeps the vector it multiplies in SHARED
// memory, one column segment of kSegWidth entries at a time, brought in by a
// bulk asynchronous copy (cp.async.bulk, completion on an mbarrier) into one
// of two buffers while the other is consumed; the gathers then hit shared
// memory.  This is the PERKS idea of serving the solver's operands from
// on-chip memory (Sec. 4.3.2), applied to the vector rather than to A.
//
// Layout, built once per operator on the GPU (seg_* kernels in cg.cu):
// block g owns rows [part_row[g], part_row[g+1]); thread t of the block owns
// the rows r = part_row[g] + t + k * kCgThreads (slot k); for every block g
// and segment s the nonzeros of (g, s) are stored thread by thread, each
// thread's run ordered by slot then column.  Per nonzero: the value (fp64,
// plus an fp32 copy for the fp32 inner solves), the column offset within the
// segment (u16) and the slot (u8); per (g, s): the start of each warp's runs
// (u32) and every thread's run length (u8).  A row's products are summed in
// column order -- the order of a sequential CSR row sum -- into its shared
// memory accumulator, so the result does not depend on the segmentation.
#pragma once

#include "common.cuh"

namespace perks {

constexpr int kSegWidth = 8192;      // columns per segment
constexpr int kSegMaxRows = 8192;    // rows per block (shared-memory accumulators)
constexpr int kSegWarps = 512 / 32;  // warps per block (kCgThreads = 512)

struct SegArgs {
    int nseg;
    const double *val;
    const float *val32;
    const unsigned short *col;   // column - s * kSegWidth
    const unsigned char *slot;   // row slot k
    const unsigned *wbase;       // [G][nseg][kSegWarps + 1]
    const unsigned char *count;  // [G][nseg][kCgThreads]
};

// Dynamic shared memory of the SEG kernel: two segment buffers (fp64 size),
// the row accumulators, the reduction scratch and two mbarriers.
__host__ __device__ constexpr size_t seg_smem_bytes() {
    return 2 * (size_t)kSegWidth * sizeof(double) + (size_t)kSegMaxRows * sizeof(double) + 64 * sizeof(double) +
           2 * sizeof(unsigned long long);
}

// ------------------------------------------------------------ mbarrier / bulk copy

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// One bulk copy global -> shared, `bytes` a multiple of 16, both addresses
// 16-byte aligned; completion is counted on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Waits for phase `parity` of `bar`, for at most timeout_ns of %globaltimer;
// false (and the error recorded) if it did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity, DevError *err,
                                                  long long timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((long long)(global_timer_ns() - t0) > (timeout_ns > 0 ? timeout_ns : 1000000000LL)) {
            if (atomicCAS(&err->code, 0, PERKS_ERR_BARRIER_TIMEOUT) == 0) {
                err->block = blockIdx.x;
                err->epoch = -2;
            }
            return false;
        }
    }
}

struct SegState {
    unsigned long long *bar;  // [2] in shared memory
    unsigned parity;          // bit b: phase parity expected next on bar[b]
};

// Starts the copy of segment s of `vin` (n entries) into buffer `b`.
template <typename V>
__device__ __forceinline__ void seg_issue(const V *vin, int n, int s, V *buf, unsigned long long *bar) {
    const int c0 = s * kSegWidth;
    const int cnt = min(kSegWidth, n - c0);
    const unsigned bytes = (unsigned)((cnt * (int)sizeof(V) + 15) & ~15);  // vectors carry >= 16 bytes of padding
    mbar_arrive_expect_tx(bar, bytes);
    bulk_copy_g2s(buf, vin + c0, bytes, bar);
}

// vout[r] = sum_j A[r][j] vin[j] for the block's rows; returns the block's
// share of <dotv, vout> (0 if dotv is null), summed over the block.  False
// in `ok` if a segment copy did not complete in time.
template <typename V>
__device__ double spmv_seg(const SegArgs &sg, int n, int r0, int r1, const V *__restrict__ gval,
                           const V *__restrict__ vin, V *__restrict__ vout, const V *dotv, unsigned char *smem,
                           SegState &st, double *red, DevError *err, long long timeout_ns, bool &ok) {
    V *xb0 = reinterpret_cast<V *>(smem);
    V *xb1 = reinterpret_cast<V *>(smem + (size_t)kSegWidth * sizeof(double));
    V *ys = reinterpret_cast<V *>(smem + 2 * (size_t)kSegWidth * sizeof(double));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nrows = r1 - r0;
    const int g = blockIdx.x;
    for (int i = tid; i < nrows; i += blockDim.x) ys[i] = V(0);
    __syncthreads();  // ys cleared; the previous call's reads of both buffers are done
    if (tid == 0) {
        asm volatile("fence.proxy.async;" ::: "memory");
        seg_issue<V>(vin, n, 0, xb0, &st.bar[0]);
    }
    ok = true;
    for (int s = 0; s < sg.nseg; ++s) {
        const int b = s & 1;
        V *xs = b ? xb1 : xb0;
        if (tid == 0 && s + 1 < sg.nseg) seg_issue<V>(vin, n, s + 1, b ? xb0 : xb1, &st.bar[b ^ 1]);
        const unsigned par = (st.parity >> b) & 1u;
        const bool landed = mbar_wait_bounded(&st.bar[b], par, err, timeout_ns);
        st.parity ^= 1u << b;
        if (__syncthreads_or(!landed)) {
            // a copy did not land in time: wait (bounded) for the one still in
            // flight, then give up; the caller sees ok = false
            if (tid == 0 && s + 1 < sg.nseg) mbar_wait_bounded(&st.bar[b ^ 1], (st.parity >> (b ^ 1)) & 1u, err, timeout_ns);
            ok = false;
            break;
        }
        const long long gs = (long long)g * sg.nseg + s;
        const int cnt = sg.count[gs * blockDim.x + tid];
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        unsigned e = sg.wbase[gs * (kSegWarps + 1) + warp] + (unsigned)(incl - cnt);
        const unsigned e1 = e + (unsigned)cnt;
        for (; e < e1; ++e) {
            const int k = __ldcs(sg.slot + e);
            const int c = __ldcs(sg.col + e);
            V *y = ys + tid + k * (int)blockDim.x;
            *y = fma(__ldcs(gval + e), xs[c], *y);
        }
        __syncthreads();  // buffer b consumed before iteration s+1 refills it with segment s+2
        if (tid == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    double dot = 0.0;
    for (int i = tid; i < nrows; i += blockDim.x) {
        const V y = ys[i];
        vout[r0 + i] = y;
        if (dotv) dot = fma((double)dotv[r0 + i], (double)y, dot);
    }
    __syncthreads();
    return block_sum(dot, red);
}

}  // namespace perks
