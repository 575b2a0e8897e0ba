// Host side of the CG solver: operator creation (device copies, the fp32
// value copy, the merge-path partition computed once), the persistent solve,
// the multi-launch baseline and the C ABI entry points perks_csr_* / perks_cg_*.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cg_kernels.cuh"
#include "internal.h"

using namespace perks;

namespace {

// ---------------------------------------------------- multi-launch baseline
// One launch per CG phase (SpMV + <p,q>; alpha and the x/r update + <r,r>;
// beta and the p update), scalars kept on the device, convergence polled by
// the host every kPoll iterations.  Same SpMV and reductions as the
// persistent kernel, so the two differ only in how the loop is driven.

struct MultiState {
    double rr[2];
    double bb;
    double tol2;
    double pq;
    int done;     // 1 = converged / out of iterations, 2 = breakdown
    int iters;
};

constexpr int kPoll = 8;

__device__ __forceinline__ CgSlice load_slice(const CgArgs &a, const CgSmem &s) {
    CgSlice sl;
    const int blk = blockIdx.x;
    sl.r0 = a.part_row[blk];
    sl.r1 = a.part_row[blk + 1];
    sl.jb = a.rowptr[sl.r0];
    sl.T = a.part_ntiles[blk];
    sl.cached = false;
    for (int u = threadIdx.x; u <= sl.T; u += blockDim.x)
        s.tiles[u] = a.part_tiles[(long long)blk * (kCgMaxTiles + 1) + u];
    __syncthreads();
    return sl;
}

// q = A v; part[blk] = <dotv, q> over the block's rows
__global__ void __launch_bounds__(kCgThreads, 1) cg_multi_spmv(const __grid_constant__ CgArgs a,
                                                             const double *v, double *q,
                                                             const double *dotv, double *part,
                                                             const MultiState *ms) {
    if (ms && ms->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CgSmem s = carve_cg_smem(smem_raw);
    const CgSlice sl = load_slice(a, s);
    const double d = spmv_any<double>(a, s, sl, a.val, v, q, dotv, nullptr);
    if (threadIdx.x == 0 && part) part[blockIdx.x] = d;
}

// r = b - q, p = r; partials of <b,b> and <r,r>
__global__ void __launch_bounds__(kCgThreads) cg_multi_init(const __grid_constant__ CgArgs a) {
    __shared__ double red[32];
    const int blk = blockIdx.x;
    const int r0 = a.part_row[blk], r1 = a.part_row[blk + 1];
    double bb = 0.0, rr = 0.0;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const double ri = a.b[i] - a.q[i];
        a.r[i] = ri;
        a.p[i] = ri;
        bb += a.b[i] * a.b[i];
        rr += ri * ri;
    }
    bb = block_sum(bb, red);
    rr = block_sum(rr, red);
    if (threadIdx.x == 0) { a.part[blk] = bb; a.part[gridDim.x + blk] = rr; }
}

__global__ void __launch_bounds__(kCgThreads) cg_multi_init2(const __grid_constant__ CgArgs a, MultiState *ms) {
    __shared__ double red[32];
    const double bb = grid_sum(a.part, gridDim.x, red);
    const double rr = grid_sum(a.part + gridDim.x, gridDim.x, red);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ms->bb = bb;
        ms->tol2 = a.rtol * a.rtol * bb;
        ms->rr[0] = rr;
        ms->iters = 0;
        ms->done = rr <= ms->tol2 ? 1 : 0;
    }
}

// iteration k, phase B: alpha = rr/pq; x += alpha p; r -= alpha q
__global__ void __launch_bounds__(kCgThreads) cg_multi_update1(const __grid_constant__ CgArgs a, int k,
                                                            MultiState *ms) {
    if (ms->done) return;
    __shared__ double red[32];
    const int blk = blockIdx.x;
    const double pq = grid_sum(a.part, gridDim.x, red);
    if (!(pq > 0.0) || !isfinite(pq)) {
        if (blk == 0 && threadIdx.x == 0) ms->pq = pq;
        return;  // update2 sees pq and stops
    }
    const double alpha = ms->rr[k & 1] / pq;
    const int r0 = a.part_row[blk], r1 = a.part_row[blk + 1];
    double rn = 0.0;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        a.x[i] = fma(alpha, a.p[i], a.x[i]);
        const double ri = fma(-alpha, a.q[i], a.r[i]);
        a.r[i] = ri;
        rn += ri * ri;
    }
    rn = block_sum(rn, red);
    if (threadIdx.x == 0) a.part[gridDim.x + blk] = rn;
    if (blk == 0 && threadIdx.x == 0) ms->pq = pq;
}

// iteration k, phase C: beta; p = r + beta p; convergence flag
__global__ void __launch_bounds__(kCgThreads) cg_multi_update2(const __grid_constant__ CgArgs a, int k,
                                                            MultiState *ms) {
    if (ms->done) return;
    __shared__ double red[32];
    const int blk = blockIdx.x;
    const double pq = ms->pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
        if (blk == 0 && threadIdx.x == 0) ms->done = 2;
        return;
    }
    const double rr = ms->rr[k & 1];
    const double rr_new = grid_sum(a.part + gridDim.x, gridDim.x, red);
    const double beta = rr_new / rr;
    const int r0 = a.part_row[blk], r1 = a.part_row[blk + 1];
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) a.p[i] = fma(beta, a.p[i], a.r[i]);
    if (blk == 0 && threadIdx.x == 0) {
        if (k < a.trace_cap) {
            a.trace[3 * k + 0] = rr / pq;
            a.trace[3 * k + 1] = beta;
            a.trace[3 * k + 2] = rr_new;
        }
        ms->rr[(k + 1) & 1] = rr_new;
        ms->iters = k + 1;
        if (rr_new <= ms->tol2 || k + 1 >= a.max_iter) ms->done = 1;
    }
}

// true residual r = b - q (q = A x); partial <r,r>
__global__ void __launch_bounds__(kCgThreads) cg_multi_resid(const __grid_constant__ CgArgs a) {
    __shared__ double red[32];
    const int blk = blockIdx.x;
    const int r0 = a.part_row[blk], r1 = a.part_row[blk + 1];
    double rr = 0.0;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const double ri = a.b[i] - a.q[i];
        a.r[i] = ri;
        rr += ri * ri;
    }
    rr = block_sum(rr, red);
    if (threadIdx.x == 0) a.part[blk] = rr;
}

// restart from the true residual: p = r, rr = <r,r>, done = 0 if above tol
__global__ void __launch_bounds__(kCgThreads) cg_multi_restart(const __grid_constant__ CgArgs a, int k,
                                                            MultiState *ms, CgResult *res) {
    __shared__ double red[32];
    const int blk = blockIdx.x;
    const double rr = grid_sum(a.part, gridDim.x, red);
    const bool ok = rr <= ms->tol2;
    const int r0 = a.part_row[blk], r1 = a.part_row[blk + 1];
    if (!ok)
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) a.p[i] = a.r[i];
    if (blk == 0 && threadIdx.x == 0) {
        res->true_rr = rr;
        res->bb = ms->bb;
        res->status = ok ? 0 : (ms->done == 2 ? PERKS_ERR_BREAKDOWN : PERKS_ERR_NOT_CONVERGED);
        res->iterations = ms->iters;
        ms->rr[k & 1] = rr;
    }
}

__global__ void cg_multi_clear_done(MultiState *ms) { ms->done = 0; }

__global__ void check_columns(const int *__restrict__ col, long long nnz, int n, int *bad) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nnz; i += (long long)gridDim.x * blockDim.x)
        if (col[i] < 0 || col[i] >= n) { atomicExch(bad, 1); return; }
}

__global__ void cast_to_f32(const double *__restrict__ v, float *__restrict__ o, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        o[i] = (float)v[i];
}

// ------------------------------------------- column-segmented SpMV layout

// Thread (g, w) walks the rows of block g owned by warp w (local index = w
// mod kSegWarps) in increasing order, and each row's nonzeros in column order,
// so the nonzeros of every (block, segment, warp) bucket are visited in the
// order the layout stores them.  Pass 0 counts, pass 1 scatters.
template <int PASS>
__global__ void seg_walk_kernel(const int *__restrict__ rowptr, const int *__restrict__ col,
                                const double *__restrict__ val, const int *__restrict__ part_row, int G, int nseg,
                                unsigned *cnt, const unsigned *tile_off, const unsigned short *wofs,
                                double *sval, float *sval32, unsigned short *scol, unsigned short *srow,
                                double *sdiag, float *sdiag32) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= G * kSegWarps) return;
    const int g = t / kSegWarps, w = t % kSegWarps;
    const int r0 = part_row[g], r1 = part_row[g + 1];
    for (int rl = w; rl < r1 - r0; rl += kSegWarps) {
        const int r = r0 + rl;
        double dsum = 0.0;
        for (int j = rowptr[r]; j < rowptr[r + 1]; ++j) {
            const int c = col[j];
            if (c == r) {  // diagonal: kept per row, applied after the segments
                dsum += val[j];
                continue;
            }
            const int sg = c / kSegWidth;
            const long long tile = (long long)g * nseg + sg;
            unsigned *cur = cnt + tile * kSegWarps + w;
            if (PASS == 0) {
                ++*cur;
            } else {
                const unsigned pos = tile_off[tile] + wofs[tile * kSegOfsPad + w] + (*cur)++;
                sval[pos] = val[j];
                sval32[pos] = (float)val[j];
                scol[pos] = (unsigned short)(c - sg * kSegWidth);
                srow[pos] = (unsigned short)rl;
            }
        }
        if (PASS == 1) {
            sdiag[r] = dsum;
            sdiag32[r] = (float)dsum;
        }
    }
}

// Tile lengths, warp offsets and tile starts (each rounded up to 8 nonzeros
// so every slice of the layout starts on a 16-byte boundary); one block.
__global__ void seg_tiles_kernel(const unsigned *cnt, long long ntiles, unsigned short *wofs, unsigned *tile_off,
                                 unsigned long long *total, unsigned *max_len) {
    __shared__ unsigned long long s_sum[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const long long per = (ntiles + nt - 1) / nt;
    const long long t0 = tid * per, t1 = min(ntiles, t0 + per);
    unsigned long long local = 0;
    unsigned mx = 0;
    for (long long t = t0; t < t1; ++t) {
        unsigned acc = 0;
        for (int w = 0; w < kSegWarps; ++w) {
            const unsigned c = cnt[t * kSegWarps + w];
            wofs[t * kSegOfsPad + w] = (unsigned short)min(acc, 65535u);
            acc += c;
        }
        wofs[t * kSegOfsPad + kSegWarps] = (unsigned short)min(acc, 65535u);
        for (int w = kSegWarps + 1; w < kSegOfsPad; ++w) wofs[t * kSegOfsPad + w] = 0;
        mx = max(mx, acc);
        local += (acc + 7u) & ~7u;
    }
    s_sum[tid] = local;
    __syncthreads();
    if (tid == 0) {
        unsigned long long run = 0;
        for (int i = 0; i < nt; ++i) {
            const unsigned long long v = s_sum[i];
            s_sum[i] = run;
            run += v;
        }
        *total = run;
    }
    __syncthreads();
    unsigned long long off = s_sum[tid];
    for (long long t = t0; t < t1; ++t) {
        tile_off[t] = (unsigned)min(off, 0xFFFFFFFFull);
        off += (wofs[t * kSegOfsPad + kSegWarps] + 7u) & ~7u;
    }
    atomicMax(max_len, mx);
}

}  // namespace

struct perks_op {
    perks_context *ctx = nullptr;
    int device = 0;  // for destroy, which may come after the context is gone
    int n = 0;
    long long nnz = 0;
    int G = 0;
    int *rowptr = nullptr, *col = nullptr;
    double *val = nullptr;
    float *val32 = nullptr;
    int *part_row = nullptr, *part_ntiles = nullptr;   // merge kernel: G blocks
    int2 *part_tiles = nullptr;
    int G2 = 0;                                         // row-vector kernel: G2 blocks
    int *part_row2 = nullptr, *part_ntiles2 = nullptr;
    int max_rows2 = 0;                                  // rows of the largest row-vector block
    size_t smem_vc = 0;                                 // row-vector kernel's shared memory with the vector cache
    bool vcache_ok = false;                             // the cache fits with G2 blocks co-resident
    int vcache_level = 0;                               // perks_op_set_vector_cache
    int2 *part_tiles2 = nullptr;
    // column-segmented SpMV: G blocks (part_row), layout built on first use
    bool seg_built = false;
    int nseg = 0;
    double *sval = nullptr;
    float *sval32 = nullptr;
    unsigned short *scol = nullptr, *srow = nullptr, *swofs = nullptr;
    unsigned *stile_off = nullptr;
    double *sdiag = nullptr;
    float *sdiag32 = nullptr;
    double *b = nullptr, *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr;
    float *r32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;
    double *part = nullptr;
    double *trace = nullptr;
    int trace_cap = 0;
    CgResult *res = nullptr;
    MultiState *ms = nullptr;
    int *ms_done_host = nullptr;  // pinned
    unsigned long long *bar = nullptr;
    DevError *err = nullptr;
    bool configured = false;
    int spmv_kind = 0;
    int last_mode = 0;
    int last_status = 0;
    perks_status last_launch = 0;
};

namespace {

template <typename T> perks_status dalloc(perks_context *ctx, T **p, size_t count) {
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T) + 16);
    if (e != cudaSuccess) { *p = nullptr; return cuda_fail(ctx, e, "cudaMalloc"); }
    return PERKS_OK;
}

void free_op(perks_op *op) {
    void *ptrs[] = {op->rowptr, op->col, op->val, op->val32, op->part_row, op->part_ntiles,
                    op->part_tiles, op->part_row2, op->part_ntiles2, op->part_tiles2, op->b, op->x, op->r, op->p, op->q, op->r32, op->p32,
                    op->q32, op->d32, op->part, op->trace, op->res, op->ms, op->bar, op->err,
                    op->sval, op->sval32, op->scol, op->srow, op->swofs, op->stile_off, op->sdiag, op->sdiag32};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (op->ms_done_host) cudaFreeHost(op->ms_done_host);
}

CgArgs make_args(perks_op *op, double rtol, int max_iter, int mode, double inner_rtol) {
    CgArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n = op->n;
    a.nnz = op->nnz;
    a.rowptr = op->rowptr;
    a.col = op->col;
    a.val = op->val;
    a.val32 = op->val32;
    const bool rv = op->spmv_kind == PERKS_SPMV_ROWVEC;
    a.part_row = rv ? op->part_row2 : op->part_row;  // merge and segmented kinds: G blocks
    a.part_ntiles = rv ? op->part_ntiles2 : op->part_ntiles;
    a.part_tiles = rv ? op->part_tiles2 : op->part_tiles;
    a.b = op->b;
    a.x = op->x; a.r = op->r; a.p = op->p; a.q = op->q;
    a.r32 = op->r32; a.p32 = op->p32; a.q32 = op->q32; a.d32 = op->d32;
    a.part = op->part;
    a.trace = op->trace;
    a.trace_cap = op->trace_cap;
    a.res = op->res;
    a.rtol = rtol;
    a.max_iter = max_iter;
    a.max_restarts = mode == CGK_FP32_IR ? 64 : 8;
    a.inner_rtol = inner_rtol;
    a.mode = mode;
    a.allow_cache = 1;
    a.spmv_kind = op->spmv_kind;
    a.vcache = rv && op->vcache_ok && mode != CGK_SPMV ? op->vcache_level : 0;
    a.vcache_rows = op->max_rows2;
    a.seg.nseg = op->nseg;
    a.seg.val = op->sval;
    a.seg.val32 = op->sval32;
    a.seg.col = op->scol;
    a.seg.row = op->srow;
    a.seg.tile_off = op->stile_off;
    a.seg.wofs = op->swofs;
    a.seg.diag = op->sdiag;
    a.seg.diag32 = op->sdiag32;
    a.bar = op->bar;
    a.err = op->err;
    a.timeout_ns = op->ctx->timeout_ns;
    return a;
}

perks_status configure(perks_op *op) {
    if (op->configured) return PERKS_OK;
    perks_context *ctx = op->ctx;
    const int smem = (int)cg_smem_bytes();
    PERKS_CUDA(ctx, cudaFuncSetAttribute((const void *)perks_cg_kernel<1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    PERKS_CUDA(ctx, cudaFuncSetAttribute((const void *)perks_cg_kernel<2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)seg_smem_bytes()));
    PERKS_CUDA(ctx, cudaFuncSetAttribute((const void *)cg_multi_spmv,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    PERKS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)perks_cg_kernel<1>,
                                                                  kCgThreads, smem));
    if (per_sm < 1 || per_sm * ctx->sm_count < op->G)
        return fail(ctx, PERKS_ERR_LAUNCH_TOO_LARGE, "CG kernel of %d blocks is not co-resident", op->G);
    int per_sm2 = 0;
    PERKS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, (const void *)perks_cg_kernel<0>,
                                                                  kCgThreads, kCgRowvecSmem));
    if (per_sm2 < 1 || per_sm2 * ctx->sm_count < op->G2)
        return fail(ctx, PERKS_ERR_LAUNCH_TOO_LARGE, "CG kernel of %d blocks is not co-resident", op->G2);
    // vector cache: on when the largest block's rows fit with all G2 blocks co-resident
    op->smem_vc = kCgRowvecSmem + (((size_t)op->max_rows2 * kCgVcacheBytesPerRow + 15) & ~size_t(15));
    op->vcache_ok = false;
    // (the attribute is per function, shared by every operator: set to the
    // device limit less the kernel's static shared memory; each launch passes
    // its own size)
    cudaFuncAttributes fa0;
    PERKS_CUDA(ctx, cudaFuncGetAttributes(&fa0, (const void *)perks_cg_kernel<0>));
    const int dyn_max = ctx->smem_optin - (int)fa0.sharedSizeBytes;
    if (op->smem_vc <= (size_t)dyn_max &&
        cudaFuncSetAttribute((const void *)perks_cg_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             dyn_max) == cudaSuccess) {
        int per_vc = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_vc, (const void *)perks_cg_kernel<0>, kCgThreads,
                                                          op->smem_vc) == cudaSuccess)
            op->vcache_ok = per_vc * ctx->sm_count >= op->G2;
    }
    (void)cudaGetLastError();
    int per_sm3 = 0;
    PERKS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm3, (const void *)perks_cg_kernel<2>,
                                                                  kCgThreads, seg_smem_bytes()));
    if (per_sm3 < 1 || per_sm3 * ctx->sm_count < op->G)
        return fail(ctx, PERKS_ERR_LAUNCH_TOO_LARGE, "CG kernel of %d blocks is not co-resident", op->G);
    op->configured = true;
    return PERKS_OK;
}

// Shared memory of the row-vector kernel at vector-cache level `level`.
size_t rowvec_smem(const perks_op *op, int level) {
    if (level <= 0) return kCgRowvecSmem;
    const size_t per_row = level == 1 ? sizeof(double) : kCgVcacheBytesPerRow;
    return kCgRowvecSmem + (((size_t)op->max_rows2 * per_row + 15) & ~size_t(15));
}

perks_status launch_persistent(perks_op *op, const CgArgs &a, cudaStream_t s) {
    perks_context *ctx = op->ctx;
    PERKS_CUDA(ctx, cudaMemsetAsync(op->bar, 0, sizeof(unsigned long long), s));
    PERKS_CUDA(ctx, cudaMemsetAsync(op->err, 0, sizeof(DevError), s));
    void *args[] = {(void *)&a};
    if (op->spmv_kind == PERKS_SPMV_ROWVEC)
        PERKS_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)perks_cg_kernel<0>, dim3(op->G2),
                                                    dim3(kCgThreads), args, rowvec_smem(op, a.vcache), s));
    else if (op->spmv_kind == PERKS_SPMV_SEG)
        PERKS_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)perks_cg_kernel<2>, dim3(op->G),
                                                    dim3(kCgThreads), args, seg_smem_bytes(), s));
    else
        PERKS_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)perks_cg_kernel<1>, dim3(op->G),
                                                    dim3(kCgThreads), args, cg_smem_bytes(), s));
    return PERKS_OK;
}

perks_status solve_multi(perks_op *op, CgArgs a, cudaStream_t s) {
    perks_context *ctx = op->ctx;
    const dim3 grid(op->spmv_kind == PERKS_SPMV_ROWVEC ? op->G2 : op->G), block(kCgThreads);
    const size_t smem = cg_smem_bytes();
    a.trace_cap = op->trace_cap;
    cg_multi_spmv<<<grid, block, smem, s>>>(a, op->x, op->q, nullptr, nullptr, nullptr);
    cg_multi_init<<<grid, block, 0, s>>>(a);
    cg_multi_init2<<<grid, block, 0, s>>>(a, op->ms);
    PERKS_CUDA(ctx, cudaGetLastError());
    int k = 0;
    for (int restart = 0; restart <= 8; ++restart) {
        while (k < a.max_iter) {
            for (int j = 0; j < kPoll && k < a.max_iter; ++j, ++k) {
                cg_multi_spmv<<<grid, block, smem, s>>>(a, op->p, op->q, op->p, op->part, op->ms);
                cg_multi_update1<<<grid, block, 0, s>>>(a, k, op->ms);
                cg_multi_update2<<<grid, block, 0, s>>>(a, k, op->ms);
            }
            PERKS_CUDA(ctx, cudaGetLastError());
            PERKS_CUDA(ctx, cudaMemcpyAsync(op->ms_done_host, &op->ms->done, sizeof(int),
                                            cudaMemcpyDeviceToHost, s));
            PERKS_CUDA(ctx, cudaStreamSynchronize(s));
            if (*op->ms_done_host) break;
        }
        // the loop may have run up to kPoll no-op iterations past convergence; k
        // is only used for the scalar slot parity, read back from ms->iters
        int iters = 0;
        PERKS_CUDA(ctx, cudaMemcpy(&iters, &op->ms->iters, sizeof(int), cudaMemcpyDeviceToHost));
        k = iters;
        cg_multi_spmv<<<grid, block, smem, s>>>(a, op->x, op->q, nullptr, nullptr, nullptr);
        cg_multi_resid<<<grid, block, 0, s>>>(a);
        cg_multi_restart<<<grid, block, 0, s>>>(a, k, op->ms, op->res);
        PERKS_CUDA(ctx, cudaGetLastError());
        CgResult r;
        PERKS_CUDA(ctx, cudaMemcpyAsync(&r, op->res, sizeof(r), cudaMemcpyDeviceToHost, s));
        PERKS_CUDA(ctx, cudaStreamSynchronize(s));
        if (r.status != PERKS_ERR_NOT_CONVERGED || k >= a.max_iter) break;
        int done = 0;
        PERKS_CUDA(ctx, cudaMemcpy(&done, &op->ms->done, sizeof(int), cudaMemcpyDeviceToHost));
        if (done == 2) break;
        cg_multi_clear_done<<<1, 1, 0, s>>>(op->ms);
    }
    return PERKS_OK;
}

perks_status read_result(perks_op *op, cudaStream_t s, perks_cg_stats *stats) {
    perks_context *ctx = op->ctx;
    PERKS_CUDA(ctx, cudaStreamSynchronize(s));
    DevError e{};
    PERKS_CUDA(ctx, cudaMemcpy(&e, op->err, sizeof(e), cudaMemcpyDeviceToHost));
    CgResult r{};
    PERKS_CUDA(ctx, cudaMemcpy(&r, op->res, sizeof(r), cudaMemcpyDeviceToHost));
    perks_status st = r.status;
    if (e.code != 0) st = e.code;
    if (stats) {
        stats->iterations = r.iterations;
        stats->outer_iterations = r.outer;
        stats->true_rel_residual = r.bb > 0 ? sqrt(r.true_rr / r.bb) : sqrt(r.true_rr);
        stats->status = st;
        stats->grid_blocks = op->spmv_kind == PERKS_SPMV_ROWVEC ? op->G2 : op->G;
        stats->threads_per_block = kCgThreads;
        const double vbytes = op->last_mode == PERKS_CG_FP32_IR ? 4.0 : 8.0;
        // A (values + column indices + row pointers) once, the gathered vector
        // once, and the vector updates: q, x, r, p read/written per iteration.
        // With the vector cache, x (d), r and q stay on chip: p's gather,
        // its read in the update and its read and write in the direction remain.
        const int lvl = op->spmv_kind == PERKS_SPMV_ROWVEC && op->vcache_ok &&
                                op->last_mode != PERKS_CG_FP64_MULTI ? op->vcache_level : 0;
        // per element: p gathered 1, q written 1 and read 1, x (d) 2, r 2 in
        // the update, p 2 and r 1 in the direction (less what stays on chip)
        const double vec_terms = lvl == 2 ? 4.0 : lvl == 1 ? 7.0 : 10.0;
        stats->bytes_per_iteration = op->nnz * (vbytes + 4.0) + 4.0 * (op->n + 1.0) + vbytes * op->n * vec_terms;
        if (stats->trace && stats->trace_len > 0) {
            const int k = std::min(std::min(stats->trace_len, op->trace_cap), r.iterations);
            if (k > 0)
                PERKS_CUDA(ctx, cudaMemcpy(stats->trace, op->trace, 3 * sizeof(double) * k,
                                           cudaMemcpyDeviceToHost));
        }
    }
    op->last_status = st;
    if (st == PERKS_ERR_BARRIER_TIMEOUT)
        return fail(ctx, st, "CG: grid barrier wait timed out (block %d, barrier %d)", e.block, e.epoch);
    if (st == PERKS_ERR_NOT_CONVERGED)
        return fail(ctx, st, "CG: not converged after %d iterations (true rel. residual %.3e)",
                    r.iterations, r.bb > 0 ? sqrt(r.true_rr / r.bb) : sqrt(r.true_rr));
    if (st == PERKS_ERR_BREAKDOWN) return fail(ctx, st, "CG: breakdown (<p, Ap> <= 0 or not finite)");
    return st;
}

}  // namespace

// ======================================================================= ABI

namespace {

// Builds the column-segmented layout (once per operator).  UNSUPPORTED when a
// block has more rows than its shared-memory accumulators hold or a tile
// more nonzeros than a segment buffer.
perks_status build_seg(perks_op *op) {
    if (op->seg_built) return PERKS_OK;
    perks_context *ctx = op->ctx;
    const int G = op->G;
    std::vector<int> pr((size_t)G + 1);
    PERKS_CUDA(ctx, cudaMemcpy(pr.data(), op->part_row, sizeof(int) * ((size_t)G + 1), cudaMemcpyDeviceToHost));
    for (int g = 0; g < G; ++g)
        if (pr[g + 1] - pr[g] > kSegMaxRows)
            return fail(ctx, PERKS_ERR_UNSUPPORTED,
                        "segmented SpMV: block %d has %d rows (at most %d)", g, pr[g + 1] - pr[g], kSegMaxRows);
    const int nseg = (op->n + kSegWidth - 1) / kSegWidth;
    const long long ntiles = (long long)G * nseg;
    unsigned *cnt = nullptr, *max_len = nullptr;
    unsigned long long *total = nullptr;
    perks_status rc = PERKS_OK;
    auto cleanup = [&]() {
        if (cnt) cudaFree(cnt);
        if (max_len) cudaFree(max_len);
        if (total) cudaFree(total);
    };
    if ((rc = dalloc(ctx, &cnt, (size_t)ntiles * kSegWarps)) || (rc = dalloc(ctx, &max_len, 1)) ||
        (rc = dalloc(ctx, &total, 1)) || (rc = dalloc(ctx, &op->swofs, (size_t)ntiles * kSegOfsPad)) ||
        (rc = dalloc(ctx, &op->stile_off, (size_t)ntiles))) {
        cleanup();
        return rc;
    }
    cudaError_t e = cudaMemset(cnt, 0, sizeof(unsigned) * (size_t)ntiles * kSegWarps);
    if (e == cudaSuccess) e = cudaMemset(max_len, 0, sizeof(unsigned));
    const int threads = G * kSegWarps;
    if (e == cudaSuccess) {
        seg_walk_kernel<0><<<(threads + 127) / 128, 128>>>(op->rowptr, op->col, op->val, op->part_row, G, nseg, cnt,
                                                           nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                           nullptr, nullptr);
        seg_tiles_kernel<<<1, 1024>>>(cnt, ntiles, op->swofs, op->stile_off, total, max_len);
        e = cudaGetLastError();
    }
    unsigned long long tot = 0;
    unsigned mx = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&tot, total, sizeof(tot), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&mx, max_len, sizeof(mx), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(ctx, e, "segmented SpMV layout"); }
    if (mx > (unsigned)kSegCap || tot >= 0xFFFFFFF0ull) {
        cleanup();
        return fail(ctx, PERKS_ERR_UNSUPPORTED, "segmented SpMV: a tile holds %u nonzeros (at most %d)", mx, kSegCap);
    }
    const size_t ne = (size_t)tot + 8;
    if ((rc = dalloc(ctx, &op->sval, ne)) || (rc = dalloc(ctx, &op->sval32, ne)) || (rc = dalloc(ctx, &op->scol, ne)) ||
        (rc = dalloc(ctx, &op->srow, ne)) || (rc = dalloc(ctx, &op->sdiag, (size_t)op->n)) ||
        (rc = dalloc(ctx, &op->sdiag32, (size_t)op->n))) {
        cleanup();
        return rc;
    }
    e = cudaMemset(op->sval, 0, sizeof(double) * ne);
    if (e == cudaSuccess) e = cudaMemset(op->sval32, 0, sizeof(float) * ne);
    if (e == cudaSuccess) e = cudaMemset(op->scol, 0, sizeof(unsigned short) * ne);
    if (e == cudaSuccess) e = cudaMemset(op->srow, 0, sizeof(unsigned short) * ne);
    if (e == cudaSuccess) e = cudaMemset(cnt, 0, sizeof(unsigned) * (size_t)ntiles * kSegWarps);
    if (e == cudaSuccess) {
        seg_walk_kernel<1><<<(threads + 127) / 128, 128>>>(op->rowptr, op->col, op->val, op->part_row, G, nseg, cnt,
                                                           op->stile_off, op->swofs, op->sval, op->sval32, op->scol,
                                                           op->srow, op->sdiag, op->sdiag32);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cleanup();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "segmented SpMV layout");
    op->nseg = nseg;
    op->seg_built = true;
    return PERKS_OK;
}

}  // namespace

extern "C" perks_status perks_csr_create(perks_context *ctx, int32_t n, int64_t nnz, const int32_t *rowptr,
                                         const int32_t *col, const double *val, int on_device,
                                         perks_op **out) {
    if (!ctx) return PERKS_ERR_INVALID_ARG;
    if (!out || !rowptr || (nnz > 0 && (!col || !val)))
        return fail(ctx, PERKS_ERR_INVALID_ARG, "csr_create: NULL argument");
    *out = nullptr;
    if (n < 1 || nnz < 0 || nnz > INT32_MAX)
        return fail(ctx, PERKS_ERR_INVALID_ARG, "csr_create: n must be >= 1 and 0 <= nnz < 2^31");
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    perks_op *op = new perks_op();
    op->ctx = ctx;
    op->device = ctx->device;
    op->n = n;
    op->nnz = nnz;
    op->G = ctx->sm_count;
    op->trace_cap = 4096;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
#define OPCHK(x)                    \
    do {                            \
        perks_status r_ = (x);      \
        if (r_) { free_op(op); delete op; return r_; } \
    } while (0)
#define OPCUDA(x)                                               \
    do {                                                        \
        cudaError_t e_ = (x);                                   \
        if (e_ != cudaSuccess) { free_op(op); delete op; return cuda_fail(ctx, e_, #x); } \
    } while (0)
    OPCHK(dalloc(ctx, &op->rowptr, (size_t)n + 1));
    OPCHK(dalloc(ctx, &op->col, (size_t)nnz));
    OPCHK(dalloc(ctx, &op->val, (size_t)nnz));
    OPCHK(dalloc(ctx, &op->val32, (size_t)nnz));
    OPCUDA(cudaMemcpy(op->rowptr, rowptr, sizeof(int) * ((size_t)n + 1), kind));
    if (nnz > 0) {
        OPCUDA(cudaMemcpy(op->col, col, sizeof(int) * (size_t)nnz, kind));
        OPCUDA(cudaMemcpy(op->val, val, sizeof(double) * (size_t)nnz, kind));
        cast_to_f32<<<1024, 256>>>(op->val, op->val32, nnz);
        OPCUDA(cudaGetLastError());
    }
    // basic structural check of the row pointers (host copy, once)
    std::vector<int> rp((size_t)n + 1);
    OPCUDA(cudaMemcpy(rp.data(), op->rowptr, sizeof(int) * ((size_t)n + 1), cudaMemcpyDeviceToHost));
    if (rp[0] != 0 || rp[n] != nnz) {
        free_op(op); delete op;
        return fail(ctx, PERKS_ERR_INVALID_ARG, "csr_create: rowptr[0] must be 0 and rowptr[n] == nnz");
    }
    for (int i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) {
            free_op(op); delete op;
            return fail(ctx, PERKS_ERR_INVALID_ARG, "csr_create: rowptr decreases at row %d", i);
        }
    {
        int *bad = nullptr;
        OPCHK(dalloc(ctx, &bad, 1));
        OPCUDA(cudaMemset(bad, 0, sizeof(int)));
        if (nnz > 0) check_columns<<<1024, 256>>>(op->col, nnz, n, bad);
        int hb = 0;
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpy(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost);
        cudaFree(bad);
        OPCUDA(e);
        if (hb) {
            free_op(op); delete op;
            return fail(ctx, PERKS_ERR_INVALID_ARG, "csr_create: column index outside [0, n)");
        }
    }
    const int G = op->G;
    op->G2 = 2 * ctx->sm_count;
    const int G2 = op->G2;
    OPCHK(dalloc(ctx, &op->part_row, (size_t)G + 1));
    OPCHK(dalloc(ctx, &op->part_ntiles, (size_t)G));
    OPCHK(dalloc(ctx, &op->part_tiles, (size_t)G * (kCgMaxTiles + 1)));
    OPCHK(dalloc(ctx, &op->part_row2, (size_t)G2 + 1));
    OPCHK(dalloc(ctx, &op->part_ntiles2, (size_t)G2));
    OPCHK(dalloc(ctx, &op->part_tiles2, (size_t)G2 * (kCgMaxTiles + 1)));
    int *overflow = nullptr;
    OPCHK(dalloc(ctx, &overflow, 1));
    OPCUDA(cudaMemset(overflow, 0, sizeof(int)));
    cg_partition_kernel<<<G, 256>>>(op->rowptr, n, nnz, G, op->part_row, op->part_ntiles, op->part_tiles,
                                    overflow);
    cg_partition_kernel<<<G2, 256>>>(op->rowptr, n, nnz, G2, op->part_row2, op->part_ntiles2, op->part_tiles2,
                                     overflow);
    OPCUDA(cudaGetLastError());
    {
        std::vector<int> pr((size_t)G2 + 1);
        OPCUDA(cudaMemcpy(pr.data(), op->part_row2, sizeof(int) * ((size_t)G2 + 1), cudaMemcpyDeviceToHost));
        for (int g = 0; g < G2; ++g) op->max_rows2 = std::max(op->max_rows2, pr[g + 1] - pr[g]);
    }
    int ov = 0;
    OPCUDA(cudaMemcpy(&ov, overflow, sizeof(int), cudaMemcpyDeviceToHost));
    cudaFree(overflow);
    if (ov) {
        free_op(op); delete op;
        return fail(ctx, PERKS_ERR_UNSUPPORTED, "csr_create: matrix too large (more than %d tiles per block)",
                    kCgMaxTiles);
    }
    OPCHK(dalloc(ctx, &op->b, (size_t)n));
    OPCHK(dalloc(ctx, &op->x, (size_t)n));
    OPCHK(dalloc(ctx, &op->r, (size_t)n));
    OPCHK(dalloc(ctx, &op->p, (size_t)n));
    OPCHK(dalloc(ctx, &op->q, (size_t)n));
    OPCHK(dalloc(ctx, &op->r32, (size_t)n));
    OPCHK(dalloc(ctx, &op->p32, (size_t)n));
    OPCHK(dalloc(ctx, &op->q32, (size_t)n));
    OPCHK(dalloc(ctx, &op->d32, (size_t)n));
    OPCHK(dalloc(ctx, &op->part, (size_t)2 * std::max(G, G2)));
    OPCHK(dalloc(ctx, &op->trace, (size_t)3 * op->trace_cap));
    OPCHK(dalloc(ctx, &op->res, 1));
    OPCHK(dalloc(ctx, &op->ms, 1));
    OPCHK(dalloc(ctx, &op->bar, 1));
    OPCHK(dalloc(ctx, &op->err, 1));
    OPCUDA(cudaMallocHost((void **)&op->ms_done_host, sizeof(int)));
    OPCUDA(cudaMemset(op->res, 0, sizeof(CgResult)));
    OPCUDA(cudaMemset(op->err, 0, sizeof(DevError)));
    OPCHK(configure(op));
    OPCUDA(cudaDeviceSynchronize());
#undef OPCHK
#undef OPCUDA
    *out = op;
    return PERKS_OK;
}

extern "C" perks_status perks_op_destroy(perks_op *op) {
    if (!op) return PERKS_OK;
    cudaSetDevice(op->device);
    free_op(op);
    delete op;
    return PERKS_OK;
}

extern "C" perks_status perks_csr_spmv(perks_op *op, const double *x, double *y, perks_stream stream) {
    if (!op) return PERKS_ERR_INVALID_ARG;
    if (!x || !y) return fail(op->ctx, PERKS_ERR_INVALID_ARG, "csr_spmv: NULL vector");
    perks_status rc = use_device(op->ctx);
    if (rc) return rc;
    CgArgs a = make_args(op, 0.0, 0, CGK_SPMV, 0.0);
    a.spmv_in = x;
    a.spmv_out = y;
    if (op->spmv_kind == PERKS_SPMV_SEG) {
        // the segment copies read whole 16-byte units: stage x into a padded vector
        PERKS_CUDA(op->ctx, cudaMemcpyAsync(op->p, x, sizeof(double) * (size_t)op->n, cudaMemcpyDeviceToDevice,
                                            (cudaStream_t)stream));
        a.spmv_in = op->p;
    }
    return launch_persistent(op, a, (cudaStream_t)stream);
}

extern "C" perks_status perks_cg_solve(perks_op *op, const double *b, double *x, double rtol, int32_t max_iter,
                                       int32_t mode, double inner_rtol, int on_device, perks_stream stream,
                                       perks_cg_stats *stats) {
    if (!op) return PERKS_ERR_INVALID_ARG;
    perks_context *ctx = op->ctx;
    if (!b || !x) return fail(ctx, PERKS_ERR_INVALID_ARG, "cg_solve: NULL b or x");
    if (!(rtol >= 0.0) || max_iter < 0) return fail(ctx, PERKS_ERR_INVALID_ARG, "cg_solve: bad rtol/max_iter");
    if (mode != PERKS_CG_FP64 && mode != PERKS_CG_FP32_IR && mode != PERKS_CG_FP64_MULTI)
        return fail(ctx, PERKS_ERR_INVALID_ARG, "cg_solve: unknown mode %d", mode);
    if (mode == PERKS_CG_FP32_IR && !(inner_rtol >= 0.0 && inner_rtol < 1.0))
        return fail(ctx, PERKS_ERR_INVALID_ARG, "cg_solve: inner_rtol must be in [0, 1)");
    if (mode == PERKS_CG_FP32_IR && inner_rtol == 0.0) {
        // automatic: two refinement steps of sqrt(rtol) each reach rtol;
        // fp32 inner solves stall near 1e-6, so no tighter than that
        inner_rtol = std::min(0.1, std::max(1e-6, std::sqrt(rtol)));
    }
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = sizeof(double) * (size_t)op->n;
    const cudaMemcpyKind in_kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind out_kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    PERKS_CUDA(ctx, cudaMemcpyAsync(op->b, b, vb, in_kind, s));
    PERKS_CUDA(ctx, cudaMemcpyAsync(op->x, x, vb, in_kind, s));
    PERKS_CUDA(ctx, cudaMemsetAsync(op->res, 0, sizeof(CgResult), s));
    PERKS_CUDA(ctx, cudaMemsetAsync(op->err, 0, sizeof(DevError), s));
    op->last_mode = mode;
    if (mode == PERKS_CG_FP64_MULTI) {
        CgArgs a = make_args(op, rtol, max_iter, CGK_FP64, inner_rtol);
        rc = solve_multi(op, a, s);
    } else {
        CgArgs a = make_args(op, rtol, max_iter, mode == PERKS_CG_FP64 ? CGK_FP64 : CGK_FP32_IR, inner_rtol);
        rc = launch_persistent(op, a, s);
    }
    if (rc) return rc;
    PERKS_CUDA(ctx, cudaMemcpyAsync(x, op->x, vb, out_kind, s));
    if (!stats) return PERKS_OK;
    return read_result(op, s, stats);
}

extern "C" perks_status perks_cg_last_result(perks_op *op, perks_stream stream, perks_cg_stats *stats) {
    if (!op) return PERKS_ERR_INVALID_ARG;
    perks_status rc = use_device(op->ctx);
    if (rc) return rc;
    perks_cg_stats local{};
    return read_result(op, (cudaStream_t)stream, stats ? stats : &local);
}

extern "C" perks_status perks_op_set_vector_cache(perks_op *op, int32_t level) {
    if (!op) return PERKS_ERR_INVALID_ARG;
    if (level < 0 || level > 2) return fail(op->ctx, PERKS_ERR_INVALID_ARG, "op_set_vector_cache: level 0, 1 or 2");
    op->vcache_level = level;
    return PERKS_OK;
}

extern "C" int32_t perks_op_vector_cache_active(const perks_op *op) {
    return op && op->vcache_ok && op->spmv_kind == PERKS_SPMV_ROWVEC ? op->vcache_level : 0;
}

extern "C" perks_status perks_op_set_spmv(perks_op *op, int32_t kind) {
    if (!op) return PERKS_ERR_INVALID_ARG;
    if (kind != PERKS_SPMV_ROWVEC && kind != PERKS_SPMV_MERGE && kind != PERKS_SPMV_SEG)
        return fail(op->ctx, PERKS_ERR_INVALID_ARG, "op_set_spmv: unknown kind %d", kind);
    if (kind == PERKS_SPMV_SEG) {
        perks_status rc = use_device(op->ctx);
        if (rc) return rc;
        rc = build_seg(op);
        if (rc) return rc;
    }
    op->spmv_kind = kind;
    return PERKS_OK;
}
