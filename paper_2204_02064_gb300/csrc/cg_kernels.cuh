// Conjugate gradient as a persistent kernel (Sec. 2.2.2 algorithm, Sec. 4.3
// PERKS port).
//
// SpMV is merge-based (Merrill & Garland, SC'16, as Sec. 4.3.1 adopts): the
// CSR matrix is viewed as a merge of the row-end offsets with the nonzero
// indices; a diagonal search splits that merge path evenly.  Two levels, as
// Sec. 4.3.2 describes: (1) block level -- computed ONCE per operator by
// cg_partition_kernel, snapped to row boundaries so no row straddles two
// blocks, and cut into tiles of kTile path items whose start coordinates are
// stored in global memory and cached in shared memory for the whole solve;
// (2) thread level -- a diagonal search inside each staged tile in shared
// memory, kIpt items per thread, partial rows fixed up through shared memory
// in a fixed order (deterministic).
//
// Each tile's values, column indices and row ends are staged into shared
// memory with cp.async, kCgBufs buffers deep so that kCgBufs-1 tiles stream
// in while one is computed; when a block's whole range fits, its tiles stay
// in shared memory across iterations (the PERKS cache of A).  The gathered
// vector entries x[col] are staged next to them, so each nonzero costs one
// fused multiply-add in the walk (GB300's fp64 pipe issues only 2 per clock
// per SM, so the product is not formed separately).
//
// The CG recurrence, dot products and axpys are fused in the same
// persistent loop with three grid barriers per iteration; grid-wide sums are
// taken in a fixed order by every block, so all blocks take identical
// decisions (convergence, breakdown) without further communication.
#pragma once

#include <cstring>

#include "common.cuh"
#include "cg_seg.cuh"

namespace perks {

constexpr int kCgThreads = 512;
constexpr int kCgIpt = 4;
constexpr int kCgTile = kCgThreads * kCgIpt;  // merge-path items per tile
constexpr int kCgMaxTiles = 2048;              // tiles per block
constexpr int kCgBufs = 4;                     // tile buffers in shared memory (3 tiles in flight)

enum CgMode : int { CGK_FP64 = 0, CGK_FP32_IR = 1, CGK_SPMV = 3 };

struct CgResult {
    int status;
    int iterations;
    int outer;
    int pad;
    double true_rr;
    double bb;
};

struct CgArgs {
    int n;
    long long nnz;
    const int *rowptr;
    const int *col;
    const double *val;
    const float *val32;
    const int *part_row;     // G+1 row boundaries
    const int *part_ntiles;  // G
    const int2 *part_tiles;  // G x (kCgMaxTiles+1): (local rows, local nonzeros) at each tile start
    const double *b;
    double *x, *r, *p, *q;
    float *r32, *p32, *q32, *d32;
    double *part;            // 2 x G block partial sums
    double *trace;
    int trace_cap;
    CgResult *res;
    double rtol;
    int max_iter;
    int max_restarts;
    double inner_rtol;
    int mode;
    int allow_cache;
    int spmv_kind;           // 0: row-vector SpMV (default), 1: thread-level merge walk, 2: column-segmented
    int vcache;              // row-vector kind, vectors kept in shared memory: 0 none, 1 r (r32), 2 x, r, q (r32, d32, q32)
    int vcache_rows;         // rows of the largest block (capacity of each cached vector)
    const double *spmv_in;
    double *spmv_out;
    SegArgs seg;             // column-segmented layout (spmv_kind 2)
    unsigned long long *bar;
    DevError *err;
    long long timeout_ns;
};

// ------------------------------------------------------------ merge search

// Rows fully consumed at merge diagonal d of the path merging the row ends
// re(i) (i < nrows, non-decreasing) with the nonzero indices 0..nnz-1.
template <class RowEnd>
__device__ __forceinline__ int merge_search(long long d, int nrows, long long nnz, RowEnd re) {
    long long lo = d - nnz > 0 ? d - nnz : 0;
    long long hi = d < nrows ? d : nrows;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if ((long long)re((int)mid) <= d - mid - 1) lo = mid + 1;
        else hi = mid;
    }
    return (int)lo;
}

// Block-level partition: block b of `G` gets rows [part_row[b], part_row[b+1])
// and tiles of kTile items of its local merge path.
__global__ void cg_partition_kernel(const int *__restrict__ rowptr, int n, long long nnz, int G,
                                    int *part_row, int *part_ntiles, int2 *part_tiles, int *overflow) {
    __shared__ int s_r[2];
    const int b = blockIdx.x;
    if (threadIdx.x < 2) {
        const int bb = b + threadIdx.x;
        int row;
        if (bb >= G) row = n;
        else {
            const long long d = (long long)bb * ((long long)n + nnz) / G;
            row = merge_search(d, n, nnz, [&](int i) { return (long long)rowptr[i + 1]; });
        }
        s_r[threadIdx.x] = row;
        if (threadIdx.x == 0) part_row[b] = row;
        if (b == G - 1 && threadIdx.x == 1) part_row[G] = n;
    }
    __syncthreads();
    const int r0 = s_r[0], r1 = s_r[1];
    const int jb = rowptr[r0];
    const int rows = r1 - r0;
    const long long lnz = (long long)rowptr[r1] - jb;
    const long long items = rows + lnz;
    const int T = (int)((items + kCgTile - 1) / kCgTile);
    if (threadIdx.x == 0) {
        part_ntiles[b] = T;
        if (T > kCgMaxTiles) atomicExch(overflow, 1);
    }
    if (T > kCgMaxTiles) return;
    for (int u = threadIdx.x; u <= T; u += blockDim.x) {
        const long long d = u == T ? items : (long long)u * kCgTile;
        const int x = merge_search(d, rows, lnz,
                                   [&](int i) { return (long long)rowptr[r0 + i + 1] - jb; });
        part_tiles[(long long)b * (kCgMaxTiles + 1) + u] = make_int2(x, (int)(d - x));
    }
}

// ----------------------------------------------------------- shared memory

template <typename V> struct TileBuf {
    V *val;
    int *col;
    int *re;  // re[0] = start of the tile's first row, re[v+1] = end of its v-th row
};

struct CgSmem {
    int2 *tiles;    // kCgMaxTiles+1
    int2 *coord;    // kCgThreads+1
    int *crow;      // kCgThreads
    double *cval;   // kCgThreads
    double *prod;   // kCgTile
    double *red;    // 32
    double *tc_val; // 2
    int *tc_row;    // 2
    unsigned char *bufs;
};

__host__ __device__ constexpr size_t cg_buf_bytes() {
    return (size_t)kCgTile * 8 + (size_t)kCgTile * 4 + (size_t)(kCgTile + 4) * 4;
}
__host__ __device__ constexpr size_t cg_fixed_bytes() {
    return (size_t)(kCgMaxTiles + 1) * 8 + (size_t)(kCgThreads + 1) * 8 + (size_t)kCgThreads * 4 +
           (size_t)kCgThreads * 8 + (size_t)kCgTile * 8 + 32 * 8 + 16 + 16 + 64;
}
__host__ __device__ constexpr size_t cg_smem_bytes() { return cg_fixed_bytes() + kCgBufs * cg_buf_bytes(); }

__device__ __forceinline__ CgSmem carve_cg_smem(unsigned char *base) {
    CgSmem s;
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char *p = base + o; o += (bytes + 15) & ~size_t(15); return p; };
    s.bufs = take(kCgBufs * cg_buf_bytes());
    s.prod = reinterpret_cast<double *>(take((size_t)kCgTile * 8));
    s.cval = reinterpret_cast<double *>(take((size_t)kCgThreads * 8));
    s.red = reinterpret_cast<double *>(take(32 * 8));
    s.tc_val = reinterpret_cast<double *>(take(16));
    s.tiles = reinterpret_cast<int2 *>(take((size_t)(kCgMaxTiles + 1) * 8));
    s.coord = reinterpret_cast<int2 *>(take((size_t)(kCgThreads + 1) * 8));
    s.crow = reinterpret_cast<int *>(take((size_t)kCgThreads * 4));
    s.tc_row = reinterpret_cast<int *>(take(16));
    return s;
}

template <typename V> __device__ __forceinline__ TileBuf<V> tile_buf(const CgSmem &s, int i) {
    unsigned char *b = s.bufs + (size_t)i * cg_buf_bytes();
    TileBuf<V> t;
    t.val = reinterpret_cast<V *>(b);
    t.col = reinterpret_cast<int *>(b + (size_t)kCgTile * 8);
    t.re = reinterpret_cast<int *>(b + (size_t)kCgTile * 12);
    return t;
}

// Per-block view of its slice of the matrix (kept in registers).
struct CgSlice {
    int r0, r1;  // rows
    int jb;      // first nonzero
    int T;       // tiles
    bool cached; // all tiles resident in shared memory
};

// Stage tile u (CTA-local coordinates from s.tiles) into buffer `tb`.
template <typename V, bool ASYNC>
__device__ __forceinline__ void stage_tile(const CgArgs &a, const CgSmem &s, const CgSlice &sl, int u,
                                           const V *gval, TileBuf<V> tb) {
    const int2 c0 = s.tiles[u], c1 = s.tiles[u + 1];
    const int nr = c1.x - c0.x, nzt = c1.y - c0.y;
    const long long j0 = (long long)sl.jb + c0.y;
    for (int v = threadIdx.x; v < nzt; v += blockDim.x) {
        if (ASYNC) {
            cp_async<sizeof(V)>(tb.val + v, gval + j0 + v);
            cp_async<4>(tb.col + v, a.col + j0 + v);
        } else {
            tb.val[v] = gval[j0 + v];
            tb.col[v] = a.col[j0 + v];
        }
    }
    // re[0..nr+1]: row starts/ends of rows c0.x .. c0.x+nr (CTA-local nonzero index)
    for (int v = threadIdx.x; v <= nr + 1; v += blockDim.x) {
        const int row = sl.r0 + c0.x + v;  // re[v] = start of row (c0.x + v)
        if (row > sl.r1) tb.re[v] = 0x7fffffff;
        else if (ASYNC) cp_async<4>(tb.re + v, a.rowptr + row);
        else tb.re[v] = a.rowptr[row];
    }
}

// Block-wide sum in a fixed order; result valid in every thread.
__device__ __forceinline__ double block_sum(double v, double *red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
        t = warp_sum(t);
        if (l == 0) red[0] = t;
    }
    __syncthreads();
    t = red[0];
    __syncthreads();
    return t;
}

// Sum of the G block partials part[0..G), in a fixed order, by every block.
__device__ __forceinline__ double grid_sum(const double *part, int G, double *red) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (w == 0) {
        double t = 0.0;
        for (int i = l; i < G; i += 32) t += __ldcg(part + i);
        t = warp_sum(t);
        if (l == 0) red[1] = t;
    }
    __syncthreads();
    const double r = red[1];
    __syncthreads();
    return r;
}

// q = A v over the block's rows (merge-path SpMV); returns the block's
// partial of sum_rows dotv[row] * q[row] (0 if dotv is null), summed in
// double, valid in every thread.  V is the value / vector type; the row sums
// accumulate in V.
template <typename V>
__device__ double spmv_block(const CgArgs &a, const CgSmem &s, const CgSlice &sl, const V *gval,
                             const V *__restrict__ vin, V *__restrict__ vout, const V *dotv) {
    const int tid = threadIdx.x;
    double dot = 0.0;
    if (tid == 0) { s.tc_row[0] = -1; s.tc_val[0] = 0.0; }
    const bool cached = sl.cached;
    if (!cached) {
#pragma unroll
        for (int k = 0; k < kCgBufs - 1; ++k) {
            if (k < sl.T) stage_tile<V, true>(a, s, sl, k, gval, tile_buf<V>(s, k));
            cp_async_commit();
        }
    }
    for (int u = 0; u < sl.T; ++u) {
        const TileBuf<V> tb = tile_buf<V>(s, cached ? u : (u % kCgBufs));
        if (!cached) {
            const int un = u + kCgBufs - 1;
            if (un < sl.T) stage_tile<V, true>(a, s, sl, un, gval, tile_buf<V>(s, un % kCgBufs));
            cp_async_commit();
            cp_async_wait<kCgBufs - 1>();
        }
        __syncthreads();  // (A) tile u staged; carry-in visible
        const int2 c0 = s.tiles[u], c1 = s.tiles[u + 1];
        const int nr = c1.x - c0.x, nzt = c1.y - c0.y;
        const int items = nr + nzt;
        // gather the vector entries of the tile's nonzeros (coalesced over the tile)
        V *xv = reinterpret_cast<V *>(s.prod);
        for (int v = tid; v < nzt; v += blockDim.x) xv[v] = __ldcg(vin + tb.col[v]);
        const int d0 = min(tid * kCgIpt, items);
        const int d1 = min(d0 + kCgIpt, items);
        // thread-level merge search in shared memory: rows consumed at d0
        const long long jt = (long long)sl.jb + c0.y;  // global index of the tile's first nonzero
        const int x0 = merge_search(d0, nr, nzt, [&](int i) { return (long long)tb.re[i + 1] - jt; });
        __syncthreads();  // (B) gathers visible
        const int y0 = d0 - x0;
        // walk the path: j is the global nonzero index, tb.re holds global row starts
        int i = x0;
        long long j = jt + y0;
        const bool partial_start = j > tb.re[i];
        V acc = V(0);
        bool has_def = false;
        V def_val = V(0);
        for (int it = d0; it < d1; ++it) {
            if (j < tb.re[i + 1]) {
                const int v = (int)(j - jt);
                acc = fma(tb.val[v], xv[v], acc);
                ++j;
            } else {
                const int row = sl.r0 + c0.x + i;
                if (i == x0 && partial_start) {
                    has_def = true;
                    def_val = acc;
                } else {
                    vout[row] = acc;
                    if (dotv) dot = fma((double)dotv[row], (double)acc, dot);
                }
                acc = V(0);
                ++i;
            }
        }
        s.crow[tid] = i;
        s.cval[tid] = (double)acc;
        __syncthreads();  // (C)
        const int tcr = s.tc_row[u & 1];
        const double tcv = s.tc_val[u & 1];
        if (has_def) {
            double tot = (double)def_val;
            int kk = tid - 1;
            while (kk >= 0 && s.crow[kk] == x0) { tot += s.cval[kk]; --kk; }
            if (kk < 0 && x0 == 0 && tcr == c0.x) tot += tcv;
            const int row = sl.r0 + c0.x + x0;
            const V vt = (V)tot;
            vout[row] = vt;
            if (dotv) dot += (double)dotv[row] * (double)vt;
        }
        if (tid == blockDim.x - 1) {
            const int rl = s.crow[tid];
            double tot = 0.0;
            int kk = tid;
            while (kk >= 0 && s.crow[kk] == rl) { tot += s.cval[kk]; --kk; }
            if (kk < 0 && rl == 0 && tcr == c0.x) tot += tcv;
            s.tc_row[(u + 1) & 1] = c0.x + rl;
            s.tc_val[(u + 1) & 1] = tot;
        }
    }
    cp_async_wait_all();
    __syncthreads();
    return block_sum(dot, s.red);
}

// Row-vector SpMV over the block's merge-path row range: sub-warps of kSub
// lanes take kRowsPer consecutive rows each (a warp covers 32/kSub*kRowsPer
// consecutive rows, so its loads are contiguous); the rows advance in
// lockstep so their loads are independent and in flight together; each lane
// strides over a row's nonzeros with direct coalesced loads and one fused
// multiply-add per nonzero; the sub-warp sums by shuffles.  On GB300 this
// costs ~8 instructions per nonzero against ~20 for the thread-level merge
// walk; the block-level merge-path partition still balances the blocks.
// A DFMA costs a whole warp issue on GB300's FP64 pipe (2 lanes per clock
// per SM) however many lanes it has active, so the layout keeps warp
// instructions dense: 8 lanes per row and two rows per sub-warp, the steps
// a warp runs end at its longest row (full passes of kU steps, then passes of
// 4, 2 and 1 for the remainder), and the two rows' partial sums are reduced together (one exchange hands each half of
// the sub-warp one row, so 3 additions cover both rows instead of 6).
// Measured (n = 2^20, 36.7 M nonzeros): the lone fp64 SpMV 218 us with the
// first, unpipelined 4-lane layout; 179 us with 8 lanes, one row and 8
// steps of loads in flight.
constexpr int kSub = 8;
constexpr int kRowsPer = 2;
// steps of both rows whose loads are in flight together in a full pass
// (fp64 4, fp32 6: within the persistent kernel's 64 registers)
template <typename V> __host__ __device__ constexpr int full_pass_steps() { return sizeof(V) == 8 ? 4 : 6; }

// UU steps of both rows of a sub-warp: all their column indices and values
// are loaded first, then all the gathers are issued, then the FMAs run (each
// row's terms still in order), so the pass waits for one HBM load and one L2
// gather instead of UU of each.
template <int UU, typename V>
__device__ __forceinline__ void spmv_pass(const int *__restrict__ col, const V *__restrict__ gval,
                                          const V *__restrict__ vin, const int (&jb)[kRowsPer],
                                          const int (&je)[kRowsPer], int u, V (&acc)[kRowsPer]) {
    int cj[UU][kRowsPer];
    V vv[UU][kRowsPer], xv[UU][kRowsPer];
#pragma unroll
    for (int q = 0; q < UU; ++q)
#pragma unroll
        for (int k = 0; k < kRowsPer; ++k) {
            const int j = jb[k] + u + q * kSub;
            const bool in = j < je[k];
            cj[q][k] = in ? __ldcs(col + j) : -1;
            vv[q][k] = in ? __ldcs(gval + j) : V(0);
        }
#pragma unroll
    for (int q = 0; q < UU; ++q)
#pragma unroll
        for (int k = 0; k < kRowsPer; ++k) xv[q][k] = cj[q][k] >= 0 ? __ldcg(vin + cj[q][k]) : V(0);
#pragma unroll
    for (int q = 0; q < UU; ++q)
#pragma unroll
        for (int k = 0; k < kRowsPer; ++k)
            if (cj[q][k] >= 0) acc[k] = fma(vv[q][k], xv[q][k], acc[k]);
}

template <typename V>
__device__ double spmv_block_vec(const CgArgs &a, const CgSlice &sl, const V *__restrict__ gval,
                                 const V *__restrict__ vin, V *__restrict__ vout, const V *dotv, double *red,
                                 V *vout_s) {
    static_assert(kRowsPer == 2 && kSub == 8, "the reduction below pairs two rows over eight lanes");
    constexpr int kU = full_pass_steps<V>();
    const int lane = threadIdx.x & (kSub - 1);
    const int sub = threadIdx.x / kSub;
    const int nsub = blockDim.x / kSub;
    const unsigned mask = 0xffffffffu;
    double dot = 0.0;
    const int stride = nsub * kRowsPer;
    for (int base = sl.r0; base < sl.r1; base += stride) {
        const int row0 = base + sub * kRowsPer;
        int jb[kRowsPer], je[kRowsPer];
        V acc[kRowsPer];
        int longest = 0;
#pragma unroll
        for (int k = 0; k < kRowsPer; ++k) {
            const int r = row0 + k;
            jb[k] = r < sl.r1 ? __ldg(a.rowptr + r) + lane : 0;
            je[k] = r < sl.r1 ? __ldg(a.rowptr + r + 1) : 0;
            acc[k] = V(0);
            longest = max(longest, je[k] - jb[k] + lane);
        }
        // steps any lane of this warp still needs (uniform across the warp)
        const int wlong = __reduce_max_sync(mask, longest);
        // full passes of kU steps, then the remainder in passes of 4, 2 and 1:
        // no step issues FMAs that no lane of the warp needs
        int u = 0;
        for (; u + kSub * kU <= wlong; u += kSub * kU) spmv_pass<kU>(a.col, gval, vin, jb, je, u, acc);
        if (kU > 4 && u + kSub * 4 <= wlong) {
            spmv_pass<4>(a.col, gval, vin, jb, je, u, acc);
            u += 4 * kSub;
        }
        if (kU > 2 && u + kSub * 2 <= wlong) {
            spmv_pass<2>(a.col, gval, vin, jb, je, u, acc);
            u += 2 * kSub;
        }
        for (; u < wlong; u += kSub) spmv_pass<1>(a.col, gval, vin, jb, je, u, acc);
        // lanes 0-3 of the sub-warp keep row 0, lanes 4-7 row 1: each sends
        // the other row's partial across and adds the one it receives, then
        // the four lanes of each half sum their row
        const bool hi = (lane & 4) != 0;
        V v = hi ? acc[1] : acc[0];
        v += __shfl_xor_sync(mask, hi ? acc[0] : acc[1], 4, kSub);
        v += __shfl_xor_sync(mask, v, 2, kSub);
        v += __shfl_xor_sync(mask, v, 1, kSub);
        if ((lane & 3) == 0) {
            const int r = row0 + (hi ? 1 : 0);
            if (r < sl.r1) {
                if (vout_s) vout_s[r - sl.r0] = v;  // the block's own rows, kept on chip
                else vout[r] = v;
                if (dotv) dot = fma((double)dotv[r], (double)v, dot);
            }
        }
    }
    __syncthreads();
    return block_sum(dot, red);
}

template <typename V>
__device__ __forceinline__ double spmv_any(const CgArgs &a, const CgSmem &s, const CgSlice &sl, const V *gval,
                                           const V *vin, V *vout, const V *dotv, V *vout_s) {
    if (a.spmv_kind == 0 && !sl.cached) return spmv_block_vec<V>(a, sl, gval, vin, vout, dotv, s.red, vout_s);
    if (s.bufs == nullptr) return 0.0;  // row-vector kernel: never reached (spmv_kind is 0)
    return spmv_block<V>(a, s, sl, gval, vin, vout, dotv);
}

template <typename V> __device__ __forceinline__ const V *seg_vals(const SegArgs &g);
template <> __device__ __forceinline__ const double *seg_vals<double>(const SegArgs &g) { return g.val; }
template <> __device__ __forceinline__ const float *seg_vals<float>(const SegArgs &g) { return g.val32; }

// The SpMV of kernel kind KIND (0 row-vector, 1 merge walk, 2 column-segmented).
// vout_s (row-vector kind only): the block's rows of the result go there,
// indexed from the block's first row, instead of to vout.
template <int KIND, typename V>
__device__ __forceinline__ double spmv_k(const CgArgs &a, const CgSmem &s, const CgSlice &sl, const V *gval,
                                         const V *vin, V *vout, const V *dotv, unsigned char *smem, SegState &st,
                                         V *vout_s = nullptr) {
    if constexpr (KIND == 2) {
        bool ok;
        return spmv_seg<V>(a.seg, a.n, sl.r0, sl.r1, seg_vals<V>(a.seg), vin, vout, dotv, smem, st, s.red, a.err,
                           a.timeout_ns, ok);
    } else {
        return spmv_any<V>(a, s, sl, gval, vin, vout, dotv, KIND == 0 ? vout_s : nullptr);
    }
}

__device__ __forceinline__ bool cg_sync(const CgArgs &a, unsigned long long &epoch) {
    return grid_barrier(a.bar, gridDim.x, epoch, a.err, a.timeout_ns);
}

// Shared memory of the row-vector kernel: the reduction scratch, followed
// (vector cache on) by kCgVcacheBytesPerRow bytes per row of the largest
// block: x, r and q in fp64, or r32, d32 and q32 for the fp32 inner solves.
constexpr size_t kCgRowvecSmem = 1024;
constexpr size_t kCgVcacheBytesPerRow = 3 * sizeof(double);

// Persistent CG (mode FP64 / FP32_IR) or a single SpMV (mode SPMV).
// ROWVEC: row-vector SpMV only, 1 KB of shared memory and at most 64
// registers, so two blocks share an SM (twice the loads in flight); otherwise
// the merge-based SpMV with its staged tiles, one block per SM.
template <int KIND>
__global__ void __launch_bounds__(kCgThreads, KIND == 0 ? 2 : 1) perks_cg_kernel(const __grid_constant__ CgArgs a) {
    constexpr bool ROWVEC = KIND != 1;  // no merge-walk tiles in shared memory
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CgSmem s;
    SegState st;
    st.bar = nullptr;
    st.parity = 0;
    if constexpr (KIND == 0) {
        std::memset(&s, 0, sizeof(s));
        s.red = reinterpret_cast<double *>(smem_raw);
    } else if constexpr (KIND == 2) {
        std::memset(&s, 0, sizeof(s));
        s.red = reinterpret_cast<double *>(smem_raw + 2 * seg_buf_bytes() + (size_t)kSegMaxRows * sizeof(double));
        st.bar = reinterpret_cast<unsigned long long *>(s.red + 64);
        if (threadIdx.x == 0) {
            mbar_init(&st.bar[0], 1);
            mbar_init(&st.bar[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    } else {
        s = carve_cg_smem(smem_raw);
    }
    const int G = gridDim.x, blk = blockIdx.x, tid = threadIdx.x;
    unsigned long long epoch = 0;

    CgSlice sl;
    sl.r0 = a.part_row[blk];
    sl.r1 = a.part_row[blk + 1];
    sl.jb = a.rowptr[sl.r0];
    sl.T = a.part_ntiles[blk];
    sl.cached = false;
    if constexpr (!ROWVEC) {
        for (int u = tid; u <= sl.T; u += blockDim.x)
            s.tiles[u] = a.part_tiles[(long long)blk * (kCgMaxTiles + 1) + u];
        __syncthreads();
        sl.cached = a.allow_cache && a.mode == CGK_FP64 && sl.T <= kCgBufs;
    }
    if (sl.cached) {
        for (int u = 0; u < sl.T; ++u) stage_tile<double, false>(a, s, sl, u, a.val, tile_buf<double>(s, u));
        __syncthreads();
    }

    if (a.mode == CGK_SPMV) {
        spmv_k<KIND, double>(a, s, sl, a.val, a.spmv_in, a.spmv_out, nullptr, smem_raw, st);
        return;
    }

    double *part0 = a.part, *part1 = a.part + G;
    const double *b = a.b;
    double *x = a.x, *r = a.r, *p = a.p, *q = a.q;

    // Vector cache (row-vector kind; the paper's caching of r, Sec. 4.3.2):
    // vectors only this block touches stay in shared memory for the whole
    // solve -- level 1: r (r32 in the fp32 inner solves); level 2: x, r, q
    // (r32, d32, q32).  p (p32), gathered by every block, stays in global
    // memory.  A cached x goes back to global memory before each
    // true-residual SpMV (which gathers it) and at the end.
    const bool vr64 = KIND == 0 && a.vcache >= 1 && a.mode == CGK_FP64;
    const bool vc64 = KIND == 0 && a.vcache >= 2 && a.mode == CGK_FP64;
    const bool vr32 = KIND == 0 && a.vcache >= 1 && a.mode == CGK_FP32_IR;
    const bool vc32 = KIND == 0 && a.vcache >= 2 && a.mode == CGK_FP32_IR;
    const int cap = a.vcache_rows;
    double *rs = reinterpret_cast<double *>(smem_raw + kCgRowvecSmem);
    double *xs = rs + cap, *qs = xs + cap;
    float *r32s = reinterpret_cast<float *>(smem_raw + kCgRowvecSmem);
    float *d32s = r32s + cap, *q32s = d32s + cap;
    const int r0 = sl.r0;
    auto X = [&](int i) -> double & { return vc64 ? xs[i - r0] : x[i]; };
    auto R = [&](int i) -> double & { return vr64 ? rs[i - r0] : r[i]; };
    auto Q = [&](int i) -> double & { return vc64 ? qs[i - r0] : q[i]; };
    auto put_x = [&]() {  // cached x -> global x (own rows)
        if (vc64)
            for (int i = sl.r0 + tid; i < sl.r1; i += blockDim.x) x[i] = xs[i - r0];
    };

    // ---- r0 = b - A x0, ||b||^2
    if (vc64)
        for (int i = sl.r0 + tid; i < sl.r1; i += blockDim.x) xs[i - r0] = x[i];
    spmv_k<KIND, double>(a, s, sl, a.val, x, q, nullptr, smem_raw, st, vc64 ? qs : nullptr);
    double bb_p = 0.0, rr_p = 0.0;
    for (int i = sl.r0 + tid; i < sl.r1; i += blockDim.x) {
        const double ri = b[i] - Q(i);
        R(i) = ri;
        p[i] = ri;
        bb_p += b[i] * b[i];
        rr_p += ri * ri;
    }
    bb_p = block_sum(bb_p, s.red);
    rr_p = block_sum(rr_p, s.red);
    if (tid == 0) { part0[blk] = bb_p; part1[blk] = rr_p; }
    if (!cg_sync(a, epoch)) return;
    const double bb = grid_sum(part0, G, s.red);
    double rr = grid_sum(part1, G, s.red);
    const double tol2 = a.rtol * a.rtol * bb;
    if (!cg_sync(a, epoch)) return;  // partials read before they are reused

    int status = PERKS_ERR_NOT_CONVERGED;
    int it = 0, outer = 0;

    if (a.mode == CGK_FP64) {
        for (int restart = 0;; ++restart) {
            if (rr <= tol2) { status = PERKS_OK; break; }
            bool converged = false;
            while (it < a.max_iter) {
                // A: q = A p, <p, q>
                const double pq_p = spmv_k<KIND, double>(a, s, sl, a.val, p, q, p, smem_raw, st, vc64 ? qs : nullptr);
                if (tid == 0) part0[blk] = pq_p;
                if (!cg_sync(a, epoch)) return;
                // B: alpha; x += alpha p; r -= alpha q; <r, r>
                const double pq = grid_sum(part0, G, s.red);
                if (!(pq > 0.0) || !isfinite(pq)) { status = PERKS_ERR_BREAKDOWN; break; }
                const double alpha = rr / pq;
                double rn_p = 0.0;
                for (int i = sl.r0 + tid; i < sl.r1; i += blockDim.x) {
                    X(i) = fma(alpha, p[i], X(i));
                    const double ri = fma(-alpha, Q(i), R(i));
                    R(i) = ri;
                    rn_p += ri * ri;
                }
                rn_p = block_sum(rn_p, s.red);
                if (tid == 0) part1[blk] = rn_p;
                if (!cg_sync(a, epoch)) return;
                // C: beta; p = r + beta p
                const double rr_new = grid_sum(part1, G, s.red);
                const double beta = rr_new / rr;
                if (blk == 0 && tid == 0 && it < a.trace_cap) {
                    a.trace[3 * it + 0] = alpha;
                    a.trace[3 * it + 1] = beta;
                    a.trace[3 * it + 2] = rr_new;
                }
                for (int i = sl.r0 + tid; i < sl.r1; i += blockDim.x) p[i] = fma(beta, p[i], R(i));
                rr = rr_new;
                ++it;
                if (!cg_sync(a, epoch)) return;
                if (rr <= tol2) { converged = true; break; }
            }
            if (status == PERKS_ERR_BREAKDOWN) break;
            // C5: true residual in fp64 (the SpMV gathers x from global memory)
            if (vc64) {
                put_x();
                if (!cg_sync(a, epoch)) return;
            }
            spmv_k<KIND, double>(a, s, sl, a.val, x, q, nullptr, smem_raw, st, vc64 ? qs : nullptr);
            double tr_p = 0.0;
            for (int i = sl.r0 + tid; i < sl.r1; i += blockDim.x) {
                const double ri = b[i] - Q(i);
                R(i) = ri;
                tr_p += ri * ri;
            }
            tr_p = block_sum(tr_p, s.red);
            if (tid == 0) part0[blk] = tr_p;
            if (!cg_sync(a, epoch)) return;
            rr = grid_sum(part0, G, s.red);
            if (rr <= tol2) { status = PERKS_OK; break; }
            if (!converged || restart >= a.max_restarts) break;
            for (int i = sl.r0 + tid; i < sl.r1; i += blockDim.x) p[i] = R(i);
            ++outer;
            if (!cg_sync(a, epoch)) return;
        }
        put_x();
    } else {  // CGK_FP32_IR
        float *r32 = a.r32, *p32 = a.p32, *q32 = a.q32, *d32 = a.d32;
        auto R32 = [&](int i) -> float & { return vr32 ? r32s[i - r0] : r32[i]; };
        auto D32 = [&](int i) -> float & { return vc32 ? d32s[i - r0] : d32[i]; };
        auto Q32 = [&](int i) -> float & { return vc32 ? q32s[i - r0] : q32[i]; };
        for (;;) {
            // outer: rr holds ||b - A x||^2 (fp64); r holds the residual
            if (rr <= tol2) { status = PERKS_OK; break; }
            if (outer >= a.max_restarts || it >= a.max_iter) break;
            double r0_p = 0.0;
            for (int i = sl.r0 + tid; i < sl.r1; i += blockDim.x) {
                const float ri = (float)r[i];
                R32(i) = ri;
                p32[i] = ri;
                D32(i) = 0.0f;
                r0_p += (double)ri * (double)ri;
            }
            r0_p = block_sum(r0_p, s.red);
            if (tid == 0) part0[blk] = r0_p;
            if (!cg_sync(a, epoch)) return;
            double irr = grid_sum(part0, G, s.red);
            const double itol2 = a.inner_rtol * a.inner_rtol * irr;
            if (!cg_sync(a, epoch)) return;
            while (it < a.max_iter) {
                const double pq_p =
                    spmv_k<KIND, float>(a, s, sl, a.val32, p32, q32, p32, smem_raw, st, vc32 ? q32s : nullptr);
                if (tid == 0) part0[blk] = pq_p;
                if (!cg_sync(a, epoch)) return;
                const double pq = grid_sum(part0, G, s.red);
                if (!(pq > 0.0) || !isfinite(pq)) { status = PERKS_ERR_BREAKDOWN; break; }
                const float alpha = (float)(irr / pq);
                double rn_p = 0.0;
                for (int i = sl.r0 + tid; i < sl.r1; i += blockDim.x) {
                    D32(i) = fmaf(alpha, p32[i], D32(i));
                    const float ri = fmaf(-alpha, Q32(i), R32(i));
                    R32(i) = ri;
                    rn_p += (double)ri * (double)ri;
                }
                rn_p = block_sum(rn_p, s.red);
                if (tid == 0) part1[blk] = rn_p;
                if (!cg_sync(a, epoch)) return;
                const double rr_new = grid_sum(part1, G, s.red);
                const float beta = (float)(rr_new / irr);
                for (int i = sl.r0 + tid; i < sl.r1; i += blockDim.x) p32[i] = fmaf(beta, p32[i], R32(i));
                irr = rr_new;
                ++it;
                if (!cg_sync(a, epoch)) return;
                if (irr <= itol2) break;
            }
            if (status == PERKS_ERR_BREAKDOWN) break;
            // x += d (fp64), then the fp64 residual of the refined x
            for (int i = sl.r0 + tid; i < sl.r1; i += blockDim.x) x[i] += (double)D32(i);
            ++outer;
            if (!cg_sync(a, epoch)) return;
            spmv_k<KIND, double>(a, s, sl, a.val, x, q, nullptr, smem_raw, st);
            double tr_p = 0.0;
            for (int i = sl.r0 + tid; i < sl.r1; i += blockDim.x) {
                const double ri = b[i] - q[i];
                r[i] = ri;
                tr_p += ri * ri;
            }
            tr_p = block_sum(tr_p, s.red);
            if (tid == 0) part0[blk] = tr_p;
            if (!cg_sync(a, epoch)) return;
            rr = grid_sum(part0, G, s.red);
            if (!cg_sync(a, epoch)) return;
        }
    }
    if (blk == 0 && tid == 0) {
        a.res->status = status;
        a.res->iterations = it;
        a.res->outer = outer;
        a.res->true_rr = rr;
        a.res->bb = bb;
    }
}

}  // namespace perks
