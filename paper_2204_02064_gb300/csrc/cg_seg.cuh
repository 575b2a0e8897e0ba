// Column-segmented SpMV for the persistent CG (the SPMV_SEG kind).
//
// A CSR SpMV with uniformly scattered columns is bound by its gathers: every
// x[col] touches a different cache line, and an SM's L1 serves about one
// line per clock.  Here each block holds the vector it multiplies in SHARED
// memory, one column segment of kSegWidth entries at a time, together with
// the block's nonzeros of that segment; both are brought in by bulk
// asynchronous copies (cp.async.bulk, completion on an mbarrier) into one of
// two buffers while the other is consumed, so the gathers and every operand
// of the inner loop are shared-memory accesses.  This is the PERKS idea of
// serving the solver's operands from on-chip memory (Sec. 4.3.2), applied to
// the vector the SpMV gathers from.
//
// Layout, built once per operator on the GPU (seg_* kernels in cg.cu):
// block g owns rows [part_row[g], part_row[g+1]); warp w of the block owns
// the rows whose local index is w modulo kSegWarps.  The nonzeros of block g
// in segment s form a tile, starting at a multiple of 8 entries, ordered by
// owning warp, then row, then column; per nonzero: the value (fp64, plus an
// fp32 copy for the fp32 inner solves), the column offset within the segment
// (u16) and the local row (u16); per tile: its start and the start of each
// warp's run (kSegWarps + 1 u16, padded to 48 bytes).  Diagonal entries stay
// out of the tiles (a block's own rows would crowd the segments holding its
// diagonal) and are applied last, per row.  Lanes of a warp take consecutive
// nonzeros; nonzeros of one row that share a 32-wide chunk are applied in lane
// order, so every row is summed in column order of its off-diagonal entries,
// then its diagonal, whatever the segmentation.
#pragma once

#include "common.cuh"

namespace perks {

__device__ __forceinline__ double block_sum(double v, double *red);

constexpr int kSegWidth = 4096;      // columns per segment
constexpr int kSegMaxRows = 8192;    // rows per block (shared-memory accumulators)
constexpr int kSegWarps = 512 / 32;  // warps per block (kCgThreads = 512)
constexpr int kSegCap = 2048;        // nonzeros per tile (one block, one segment)
constexpr int kSegOfsPad = 24;       // u16 per tile of warp offsets (48 bytes)

struct SegArgs {
    int nseg;
    const double *val;
    const float *val32;
    const unsigned short *col;   // column - s * kSegWidth
    const unsigned short *row;   // row - part_row[g]
    const unsigned *tile_off;    // [G][nseg] first nonzero of the tile (multiple of 8)
    const unsigned short *wofs;  // [G][nseg][kSegOfsPad] warp run starts within the tile, [kSegWarps] = length
    const double *diag;          // [n] diagonal entries (kept out of the tiles)
    const float *diag32;
};

// Shared memory of one segment buffer (sized for fp64) and of the SEG kernel.
__host__ __device__ constexpr size_t seg_buf_bytes() {
    return (size_t)kSegWidth * 8 + (size_t)kSegCap * 8 + (size_t)kSegCap * 2 * 2 + kSegOfsPad * 2;
}
__host__ __device__ constexpr size_t seg_smem_bytes() {
    return 2 * seg_buf_bytes() + (size_t)kSegMaxRows * sizeof(double) + 64 * sizeof(double) +
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

template <typename V> struct SegBuf {
    V *x;
    V *val;
    unsigned short *col, *row, *wofs;
};

template <typename V> __device__ __forceinline__ SegBuf<V> seg_buf(unsigned char *smem, int b) {
    unsigned char *p = smem + (size_t)b * seg_buf_bytes();
    SegBuf<V> s;
    s.x = reinterpret_cast<V *>(p);
    s.val = reinterpret_cast<V *>(p + (size_t)kSegWidth * 8);
    s.col = reinterpret_cast<unsigned short *>(p + (size_t)kSegWidth * 8 + (size_t)kSegCap * 8);
    s.row = s.col + kSegCap;
    s.wofs = s.row + kSegCap;
    return s;
}

__device__ __forceinline__ unsigned round16(unsigned b) { return (b + 15u) & ~15u; }

// Starts the copies of segment s (vector slice and the block's tile) into
// buffer `dst`, all counted on `bar`.
template <typename V>
__device__ __forceinline__ void seg_issue(const SegArgs &sg, const V *gval, const V *vin, int n, int s,
                                          const SegBuf<V> &dst, unsigned long long *bar) {
    const int c0 = s * kSegWidth;
    const int cnt = min(kSegWidth, n - c0);
    const long long t = (long long)blockIdx.x * sg.nseg + s;
    const unsigned off = __ldg(sg.tile_off + t);
    const unsigned len = __ldg(sg.wofs + t * kSegOfsPad + kSegWarps);
    const unsigned len8 = (len + 7u) & ~7u;
    const unsigned bx = round16((unsigned)cnt * sizeof(V));  // vectors carry >= 16 bytes of padding
    const unsigned bv = len8 * sizeof(V), bi = len8 * 2u, bo = kSegOfsPad * 2u;
    mbar_arrive_expect_tx(bar, bx + bv + 2 * bi + bo);
    bulk_copy_g2s(dst.x, vin + c0, bx, bar);
    if (len8) {
        bulk_copy_g2s(dst.val, gval + off, bv, bar);
        bulk_copy_g2s(dst.col, sg.col + off, bi, bar);
        bulk_copy_g2s(dst.row, sg.row + off, bi, bar);
    }
    bulk_copy_g2s(dst.wofs, sg.wofs + t * kSegOfsPad, bo, bar);
}

template <typename V> __device__ __forceinline__ const V *seg_diag(const SegArgs &g);
template <> __device__ __forceinline__ const double *seg_diag<double>(const SegArgs &g) { return g.diag; }
template <> __device__ __forceinline__ const float *seg_diag<float>(const SegArgs &g) { return g.diag32; }

// vout[r] = sum_j A[r][j] vin[j] for the block's rows; returns the block's
// share of <dotv, vout> (0 if dotv is null), summed over the block.  `ok` is
// false if a copy did not complete in time (the error is recorded).
template <typename V>
__device__ double spmv_seg(const SegArgs &sg, int n, int r0, int r1, const V *__restrict__ gval,
                           const V *__restrict__ vin, V *__restrict__ vout, const V *dotv, unsigned char *smem,
                           SegState &st, double *red, DevError *err, long long timeout_ns, bool &ok) {
    V *ys = reinterpret_cast<V *>(smem + 2 * seg_buf_bytes());
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nrows = r1 - r0;
    for (int i = tid; i < nrows; i += blockDim.x) ys[i] = V(0);
    __syncthreads();  // ys cleared; the previous call's reads of both buffers are done
    if (tid == 0) {
        asm volatile("fence.proxy.async;" ::: "memory");
        seg_issue<V>(sg, gval, vin, n, 0, seg_buf<V>(smem, 0), &st.bar[0]);
    }
    ok = true;
    for (int s = 0; s < sg.nseg; ++s) {
        const int b = s & 1;
        if (tid == 0 && s + 1 < sg.nseg) seg_issue<V>(sg, gval, vin, n, s + 1, seg_buf<V>(smem, b ^ 1), &st.bar[b ^ 1]);
        // warp-uniform outcome, so the warp-wide collectives below see full warps
        const bool landed = __all_sync(0xffffffffu, mbar_wait_bounded(&st.bar[b], (st.parity >> b) & 1u, err,
                                                                        timeout_ns));
        st.parity ^= 1u << b;
        const SegBuf<V> B = seg_buf<V>(smem, b);
        if (landed) {
            const int e0 = B.wofs[warp], e1 = B.wofs[warp + 1];
            for (int c = e0; c < e1; c += 32) {
                const int e = c + lane;
                const bool act = e < e1;
                const unsigned amask = __ballot_sync(0xffffffffu, act);
                if (act) {
                    const int row = B.row[e];
                    const V prod_v = B.val[e];
                    const V xv = B.x[B.col[e]];
                    const unsigned grp = __match_any_sync(amask, row);
                    if (grp == (1u << lane)) {
                        ys[row] = fma(prod_v, xv, ys[row]);
                    } else {
                        // nonzeros of one row within this chunk: apply in lane order
                        const int rank = __popc(grp & ((1u << lane) - 1u));
                        const int n_in = __popc(grp);
                        for (int q = 0; q < n_in; ++q) {
                            if (rank == q) ys[row] = fma(prod_v, xv, ys[row]);
                            __syncwarp(grp);
                        }
                    }
                }
                __syncwarp();  // this chunk's updates are visible to the next chunk's lanes
            }
        }
        if (__syncthreads_or(!landed)) {
            // a copy did not land in time: wait (bounded) for the one still in
            // flight, then give up
            if (tid == 0 && s + 1 < sg.nseg)
                mbar_wait_bounded(&st.bar[b ^ 1], (st.parity >> (b ^ 1)) & 1u, err, timeout_ns);
            ok = false;
            break;
        }
        if (tid == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    const V *dg = seg_diag<V>(sg);
    double dot = 0.0;
    for (int i = tid; i < nrows; i += blockDim.x) {
        const V y = fma(dg[r0 + i], vin[r0 + i], ys[i]);
        vout[r0 + i] = y;
        if (dotv) dot = fma((double)dotv[r0 + i], (double)y, dot);
    }
    __syncthreads();
    return block_sum(dot, red);
}

}  // namespace perks
