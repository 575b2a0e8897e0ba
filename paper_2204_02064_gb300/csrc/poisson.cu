// Batched variable-coefficient Poisson: -div(k grad u) = f on nx*ny grids
// (5-point finite volumes, h = 1, face coefficient = harmonic mean of the two
// cells' k, Dirichlet 0 through a ghost cell carrying the boundary cell's k),
// solved by CG (the Sec. 2.2.2 recurrence) as ONE persistent launch.
//
// Problems are independent, so the batch needs no grid barrier: each block
// (or group of C blocks) owns one problem at a time, pulling problems from an
// atomic counter, keeps its scalars and partial sums on chip and runs that
// problem's whole CG loop -- SpMV (matrix-free, from precomputed face
// coefficients), dot products and axpys.  With C = 1 the reductions are
// block-level only.  With C > 1 the problem's rows are split over the group's
// blocks, which meet at a bounded barrier of their own after each p update
// and in each dot product (block sums added in rank order, so every block of
// the group takes the same decisions): a batch ends with its hardest problem
// running alone, and a group runs it C times faster.  The true residual is
// recomputed in fp64 on exit and CG restarts while it is above tolerance.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"
#include "common.cuh"

using namespace perks;

namespace {

constexpr int kPoiThreads = 256;
constexpr int kPoiMaxGroup = 8;  // blocks per problem, at most

struct PoissonArgs {
    int nx, ny, nprob;
    long long n;                 // cells per problem
    const double *fx;            // [prob][ny][nx+1] x-face coefficients
    const double *fy;            // [prob][ny+1][nx] y-face coefficients
    const double *dg;            // [prob][n] diagonal: (fw + fe) + (fs + fn) of each cell
    const double *b;             // [prob][n]
    double *x, *r, *p, *q;       // [prob][n]
    double rtol;
    int max_iter;
    int max_restarts;
    int *queue;                  // next problem to take
    int *iters;                  // [prob] recurrence iterations
    double *true_rel;            // [prob] ||b - A x|| / ||b||
    int *status;                 // [prob]
    int group;                   // blocks per problem (C)
    unsigned long long *gbar;    // [groups] barrier counter of each block group
    int *gprob;                  // [groups] problem taken by each group
    double *gpart;               // [groups][2][C] block sums, double-buffered
    DevError *err;
    long long timeout_ns;
};

__global__ void poisson_faces_kernel(const double *__restrict__ k, int nx, int ny, long long total_cells,
                                     double *fx, double *fy) {
    // one thread per face; x-faces: (nx+1)*ny per problem, y-faces: nx*(ny+1)
    const long long nfx = (long long)(nx + 1) * ny, nfy = (long long)nx * (ny + 1);
    const long long nprob = total_cells / ((long long)nx * ny);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nprob * (nfx + nfy); t += stride) {
        const long long pb = t / (nfx + nfy), u = t % (nfx + nfy);
        const double *kp = k + pb * (long long)nx * ny;
        if (u < nfx) {
            const int j = (int)(u / (nx + 1)), i = (int)(u % (nx + 1));
            double f;
            if (i == 0) f = kp[(long long)j * nx];
            else if (i == nx) f = kp[(long long)j * nx + nx - 1];
            else {
                const double a = kp[(long long)j * nx + i - 1], c = kp[(long long)j * nx + i];
                f = 2.0 * a * c / (a + c);
            }
            fx[pb * nfx + u] = f;
        } else {
            const long long v = u - nfx;
            const int j = (int)(v / nx), i = (int)(v % nx);
            double f;
            if (j == 0) f = kp[i];
            else if (j == ny) f = kp[(long long)(ny - 1) * nx + i];
            else {
                const double a = kp[(long long)(j - 1) * nx + i], c = kp[(long long)j * nx + i];
                f = 2.0 * a * c / (a + c);
            }
            fy[pb * nfy + v] = f;
        }
    }
}

// Diagonal of every cell, (fw + fe) + (fs + fn), computed once: the matvec
// then needs one multiply and four fused multiply-adds per cell (the FP64
// pipe, not HBM, bounds this CG on GB300).
__global__ void poisson_diag_kernel(const double *__restrict__ fx, const double *__restrict__ fy, int nx, int ny,
                                    long long total_cells, double *dg) {
    const long long n = (long long)nx * ny;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total_cells;
         t += (long long)gridDim.x * blockDim.x) {
        const long long pb = t / n, c = t % n;
        const int j = (int)(c / nx), i = (int)(c % nx);
        const double *fxp = fx + pb * (long long)(nx + 1) * ny;
        const double *fyp = fy + pb * (long long)nx * (ny + 1);
        const double fw = fxp[(long long)j * (nx + 1) + i], fe = fxp[(long long)j * (nx + 1) + i + 1];
        const double fs = fyp[(long long)j * nx + i], fn = fyp[(long long)(j + 1) * nx + i];
        dg[t] = (fw + fe) + (fs + fn);
    }
}

// (A v)_c for cell c = (i, j) of one problem.
__device__ __forceinline__ double apply_cell(const double *__restrict__ fxp, const double *__restrict__ fyp,
                                             const double *__restrict__ dgp, const double *__restrict__ v, int nx,
                                             int ny, int i, int j) {
    const long long c = (long long)j * nx + i;
    const double fw = fxp[(long long)j * (nx + 1) + i], fe = fxp[(long long)j * (nx + 1) + i + 1];
    const double fs = fyp[(long long)j * nx + i], fn = fyp[(long long)(j + 1) * nx + i];
    const double vc = v[c];
    double acc = dgp[c] * vc;
    if (i > 0) acc = fma(-fw, v[c - 1], acc);
    if (i + 1 < nx) acc = fma(-fe, v[c + 1], acc);
    if (j > 0) acc = fma(-fs, v[c - nx], acc);
    if (j + 1 < ny) acc = fma(-fn, v[c + nx], acc);
    return acc;
}

// (A v) for kRows consecutive cells (i, j0..j0+kRows-1) of one column, with
// each value loaded once (v down the column, faces once per row) and the same
// arithmetic, in the same order, as apply_cell.  Rows at or beyond ny are
// skipped.
template <int K>
__device__ __forceinline__ void apply_column(const double *__restrict__ fxp, const double *__restrict__ fyp,
                                             const double *__restrict__ dgp, const double *__restrict__ v, int nx,
                                             int ny, int i, int j0, double (&out)[K], double (&vc)[K]) {
    double col[K + 2];
    double fyv[K + 1];
#pragma unroll
    for (int u = -1; u <= K; ++u) {
        const int j = j0 + u;
        col[u + 1] = (j >= 0 && j < ny) ? v[(long long)j * nx + i] : 0.0;
    }
#pragma unroll
    for (int u = 0; u <= K; ++u) {
        const int j = j0 + u;
        fyv[u] = (j <= ny) ? __ldg(fyp + (long long)j * nx + i) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < K; ++u) {
        const int j = j0 + u;
        if (j < ny) {
            const long long c = (long long)j * nx + i;
            const double *fr = fxp + (long long)j * (nx + 1) + i;
            const double fw = __ldg(fr), fe = __ldg(fr + 1);
            const double fs = fyv[u], fn = fyv[u + 1];
            const double vcen = col[u + 1];
            double acc = __ldg(dgp + c) * vcen;
            if (i > 0) acc = fma(-fw, v[c - 1], acc);
            if (i + 1 < nx) acc = fma(-fe, v[c + 1], acc);
            if (j > 0) acc = fma(-fs, col[u], acc);
            if (j + 1 < ny) acc = fma(-fn, col[u + 2], acc);
            out[u] = acc;
            vc[u] = vcen;
        }
    }
}

__device__ __forceinline__ double bsum(double v, double *red) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
        t = warp_sum(t);
        if (l == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// Row-blocked traversal: each thread takes cell column i of kRows rows at a
// time, so the loads of kRows independent cells (and their neighbours) are in
// flight together instead of one row's worth per memory round trip.
constexpr int kRows = 4;
// Linear traversal unroll for the vector updates.
constexpr int kLin = 2;

// r = b - A x over the whole problem; returns this thread's partial <r,r>
// (and <b,b> through bb); optionally p = r.
template <bool SET_P, int ROWS>
__device__ __forceinline__ double residual_pass(const double *__restrict__ fxp, const double *__restrict__ fyp,
                                                const double *__restrict__ dgp,
                                                const double *__restrict__ b, const double *__restrict__ x,
                                                double *__restrict__ r, double *__restrict__ p, int nx, int ny,
                                                int jb, int je, double &bb) {
    double rr = 0.0;
    for (int j0 = jb; j0 < je; j0 += ROWS)
        for (int i = threadIdx.x; i < nx; i += blockDim.x) {
            double rv[ROWS], bv[ROWS], xc[ROWS];
            apply_column<ROWS>(fxp, fyp, dgp, x, nx, ny, i, j0, rv, xc);
#pragma unroll
            for (int u = 0; u < ROWS; ++u) {
                const int j = j0 + u;
                if (j < ny) {
                    const long long c = (long long)j * nx + i;
                    bv[u] = __ldg(b + c);
                    rv[u] = bv[u] - rv[u];
                }
            }
#pragma unroll
            for (int u = 0; u < ROWS; ++u) {
                const int j = j0 + u;
                if (j < ny) {
                    const long long c = (long long)j * nx + i;
                    r[c] = rv[u];
                    if (SET_P) p[c] = rv[u];
                    bb = fma(bv[u], bv[u], bb);
                    rr = fma(rv[u], rv[u], rr);
                }
            }
        }
    return rr;
}

// Rows [jb, je) of a problem owned by block `rank` of a group of C: row
// blocks of ROWS rows split evenly.
template <int ROWS>
__device__ __forceinline__ void group_rows(int ny, int C, int rank, int &jb, int &je) {
    const int nrb = (ny + ROWS - 1) / ROWS;
    jb = min(ny, (int)((long long)nrb * rank / C) * ROWS);
    je = min(ny, (int)((long long)nrb * (rank + 1) / C) * ROWS);
}

template <int NT, int MINB, int ROWS, int LIN, bool GROUP>
__global__ void __launch_bounds__(NT, MINB) perks_poisson_cg_kernel(const __grid_constant__ PoissonArgs a) {
    __shared__ double red[33];
    __shared__ int s_prob;
    const int nx = a.nx, ny = a.ny;
    const long long n = a.n;
    const int C = GROUP ? a.group : 1;
    const int g = blockIdx.x / C, rank = blockIdx.x % C;
    int jb = 0, je = ny;
    if (GROUP) group_rows<ROWS>(ny, C, rank, jb, je);
    const long long cb = (long long)jb * nx, ce = (long long)je * nx;
    unsigned long long epoch = 0;
    int nred = 0;
    // the group's sum of a per-thread value: block sums, then the group's
    // block sums in rank order (the same value in every block); false if the
    // group barrier gave up
    auto gsum = [&](double v, double &out) -> bool {
        v = bsum(v, red);
        if (!GROUP) { out = v; return true; }
        double *slot = a.gpart + ((long long)g * 2 + (nred & 1)) * C;
        ++nred;
        if (threadIdx.x == 0) slot[rank] = v;
        if (!grid_barrier(a.gbar + g, C, epoch, a.err, a.timeout_ns)) return false;
        double t = 0.0;
        for (int i = 0; i < C; ++i) t += __ldcg(slot + i);
        out = t;
        return true;
    };
    for (;;) {
        if (GROUP) {
            if (rank == 0 && threadIdx.x == 0) a.gprob[g] = atomicAdd(a.queue, 1);
            if (!grid_barrier(a.gbar + g, C, epoch, a.err, a.timeout_ns)) return;
            if (threadIdx.x == 0) s_prob = __ldcg(a.gprob + g);
        } else {
            if (threadIdx.x == 0) s_prob = atomicAdd(a.queue, 1);
        }
        __syncthreads();
        const int pb = s_prob;
        __syncthreads();
        if (pb >= a.nprob) break;
        const double *__restrict__ fxp = a.fx + (long long)pb * (nx + 1) * ny;
        const double *__restrict__ fyp = a.fy + (long long)pb * nx * (ny + 1);
        const double *__restrict__ dgp = a.dg + (long long)pb * n;
        const double *__restrict__ b = a.b + pb * n;
        double *__restrict__ x = a.x + pb * n;
        double *__restrict__ r = a.r + pb * n;
        double *__restrict__ p = a.p + pb * n;
        double *__restrict__ q = a.q + pb * n;
        // r = b - A x, p = r
        double bb = 0.0, rr;
        const double rr_own = residual_pass<true, ROWS>(fxp, fyp, dgp, b, x, r, p, nx, ny, jb, je, bb);
        if (!gsum(bb, bb) || !gsum(rr_own, rr)) return;
        const double tol2 = a.rtol * a.rtol * bb;
        int it = 0, status = PERKS_ERR_NOT_CONVERGED;
        for (int restart = 0;; ++restart) {
            if (rr <= tol2) { status = PERKS_OK; break; }
            bool converged = false;
            while (it < a.max_iter) {
                // q = A p, <p, q>
                double pq = 0.0;
                for (int j0 = jb; j0 < je; j0 += ROWS)
                    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                        double qv[ROWS], pv[ROWS];
                        apply_column<ROWS>(fxp, fyp, dgp, p, nx, ny, i, j0, qv, pv);
#pragma unroll
                        for (int u = 0; u < ROWS; ++u) {
                            const int j = j0 + u;
                            if (j < je) {
                                q[(long long)j * nx + i] = qv[u];
                                pq = fma(pv[u], qv[u], pq);
                            }
                        }
                    }
                if (!gsum(pq, pq)) return;
                if (!(pq > 0.0) || !isfinite(pq)) { status = PERKS_ERR_BREAKDOWN; break; }
                const double alpha = rr / pq;
                // x += alpha p, r -= alpha q, <r, r>
                double rn = 0.0;
                for (long long c0 = cb + threadIdx.x; c0 < ce; c0 += (long long)blockDim.x * LIN) {
                    double xv[LIN], rv[LIN], pv[LIN], qv[LIN];
#pragma unroll
                    for (int u = 0; u < LIN; ++u) {
                        const long long c = c0 + (long long)u * blockDim.x;
                        if (c < ce) { xv[u] = x[c]; rv[u] = r[c]; pv[u] = p[c]; qv[u] = q[c]; }
                    }
#pragma unroll
                    for (int u = 0; u < LIN; ++u) {
                        const long long c = c0 + (long long)u * blockDim.x;
                        if (c < ce) {
                            x[c] = fma(alpha, pv[u], xv[u]);
                            const double ri = fma(-alpha, qv[u], rv[u]);
                            r[c] = ri;
                            rn = fma(ri, ri, rn);
                        }
                    }
                }
                if (!gsum(rn, rn)) return;
                const double beta = rn / rr;
                // p = r + beta p
                for (long long c0 = cb + threadIdx.x; c0 < ce; c0 += (long long)blockDim.x * LIN) {
                    double rv[LIN], pv[LIN];
#pragma unroll
                    for (int u = 0; u < LIN; ++u) {
                        const long long c = c0 + (long long)u * blockDim.x;
                        if (c < ce) { rv[u] = r[c]; pv[u] = p[c]; }
                    }
#pragma unroll
                    for (int u = 0; u < LIN; ++u) {
                        const long long c = c0 + (long long)u * blockDim.x;
                        if (c < ce) p[c] = fma(beta, pv[u], rv[u]);
                    }
                }
                if (GROUP) {  // the next SpMV reads the neighbouring blocks' edge rows of p
                    if (!grid_barrier(a.gbar + g, C, epoch, a.err, a.timeout_ns)) return;
                } else {
                    __syncthreads();
                }
                rr = rn;
                ++it;
                if (rr <= tol2) { converged = true; break; }
            }
            if (status == PERKS_ERR_BREAKDOWN) break;
            double bdum = 0.0;
            const double rt = residual_pass<true, ROWS>(fxp, fyp, dgp, b, x, r, p, nx, ny, jb, je, bdum);
            if (!gsum(rt, rr)) return;
            if (rr <= tol2) { status = PERKS_OK; break; }
            if (!converged || restart >= a.max_restarts) break;
        }
        if (rank == 0 && threadIdx.x == 0) {
            a.iters[pb] = it;
            a.true_rel[pb] = bb > 0 ? sqrt(rr / bb) : sqrt(rr);
            a.status[pb] = status;
        }
        __syncthreads();
    }
}

// x <- alpha x per problem with alpha = <x, b> / <x, A x>: of all multiples
// of the guess, the one closest to the solution in the A-norm (the energy
// norm CG minimises), so a warm start scaled this way starts CG no farther
// from the solution, in that norm, than a zero start.  Left unchanged where
// <x, A x> is not positive and finite (x = 0, for one).
template <int NT, int ROWS>
__global__ void __launch_bounds__(NT, 1) poisson_scale_guess_kernel(const __grid_constant__ PoissonArgs a,
                                                                   const double *__restrict__ bv,
                                                                   double *__restrict__ xv) {
    __shared__ double red[33];
    const int nx = a.nx, ny = a.ny;
    const long long n = a.n;
    for (int pb = blockIdx.x; pb < a.nprob; pb += gridDim.x) {
        const double *__restrict__ fxp = a.fx + (long long)pb * (nx + 1) * ny;
        const double *__restrict__ fyp = a.fy + (long long)pb * nx * (ny + 1);
        const double *__restrict__ dgp = a.dg + (long long)pb * n;
        const double *__restrict__ b = bv + pb * n;
        double *__restrict__ x = xv + pb * n;
        double xax = 0.0, xb = 0.0;
        for (int j0 = 0; j0 < ny; j0 += ROWS)
            for (int i = threadIdx.x; i < nx; i += blockDim.x) {
                double ax[ROWS], xc[ROWS];
                apply_column<ROWS>(fxp, fyp, dgp, x, nx, ny, i, j0, ax, xc);
#pragma unroll
                for (int u = 0; u < ROWS; ++u) {
                    const int j = j0 + u;
                    if (j < ny) {
                        xax = fma(xc[u], ax[u], xax);
                        xb = fma(xc[u], __ldg(b + (long long)j * nx + i), xb);
                    }
                }
            }
        xax = bsum(xax, red);
        xb = bsum(xb, red);
        if (xax > 0.0 && isfinite(xax) && isfinite(xb)) {
            const double alpha = xb / xax;
            for (long long c = threadIdx.x; c < n; c += blockDim.x) x[c] *= alpha;
        }
        __syncthreads();
    }
}

// y = A v for every problem (one launch; for tests).
__global__ void poisson_apply_kernel(const __grid_constant__ PoissonArgs a, const double *v, double *y) {
    const long long total = (long long)a.nprob * a.n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long pb = t / a.n, c = t % a.n;
        const double *fxp = a.fx + pb * (a.nx + 1) * a.ny;
        const double *fyp = a.fy + pb * a.nx * (a.ny + 1);
        y[t] = apply_cell(fxp, fyp, a.dg + pb * a.n, v + pb * a.n, a.nx, a.ny, (int)(c % a.nx), (int)(c / a.nx));
    }
}

}  // namespace

struct perks_poisson {
    perks_context *ctx = nullptr;
    int device = 0;  // for destroy, which may come after the context is gone
    int nx = 0, ny = 0, nprob = 0;
    long long n = 0;
    double *fx = nullptr, *fy = nullptr, *dg = nullptr, *b = nullptr, *x = nullptr, *r = nullptr, *p = nullptr,
           *q = nullptr;
    int *queue = nullptr, *iters = nullptr, *status = nullptr;
    double *true_rel = nullptr;
    int block_threads = 512;  // 512 (one block per SM; measured faster) or 256 (two per SM)
    int rows_per_pass = 1;    // 1 (64 registers, 32 warps per SM; measured faster) or kRows (128, 16 warps)
    int group = 0;            // blocks per problem (0: automatic)
    unsigned long long *gbar = nullptr;
    int *gprob = nullptr;
    double *gpart = nullptr;
    DevError *err = nullptr;
    int max_groups = 0;
};

namespace {
void free_poisson(perks_poisson *P) {
    void *ptrs[] = {P->fx, P->fy, P->dg, P->b, P->x, P->r, P->p, P->q, P->queue, P->iters, P->status, P->true_rel,
                    P->gbar, P->gprob, P->gpart, P->err};
    for (void *v : ptrs) if (v) cudaFree(v);
}

// Blocks per problem: as set, or automatically, for problems of 64K cells
// and more, 8 blocks (two per SM, one row per pass) or 4 (one per SM, 4
// rows per pass), and 1 for smaller problems (whose iterations are too short
// to pay for the group barriers).  A batch of 256 problems of 512^2 to 1e-8:
// 4 rows per pass 20.2 s with one block per problem, 16.4 s with 2, 15.9 s
// with 4 or 8; one row per pass 16.3 s with 2, 13.5 s with 4, 13.4 s with 8.
int effective_group(const perks_poisson *P) {
    if (P->group > 0) return P->group;
    if (P->n < 65536) return 1;
    return P->rows_per_pass == 1 ? 8 : 4;
}

PoissonArgs poisson_args(perks_poisson *P) {
    PoissonArgs a;
    std::memset(&a, 0, sizeof(a));
    a.nx = P->nx; a.ny = P->ny; a.nprob = P->nprob; a.n = P->n;
    a.fx = P->fx; a.fy = P->fy; a.dg = P->dg; a.b = P->b; a.x = P->x; a.r = P->r; a.p = P->p; a.q = P->q;
    a.queue = P->queue; a.iters = P->iters; a.true_rel = P->true_rel; a.status = P->status;
    a.group = effective_group(P); a.gbar = P->gbar; a.gprob = P->gprob; a.gpart = P->gpart; a.err = P->err;
    a.timeout_ns = P->ctx->timeout_ns;
    return a;
}
}  // namespace

extern "C" perks_status perks_poisson_create(perks_context *ctx, int32_t nx, int32_t ny, int32_t nprob,
                                             const double *k, int on_device, perks_poisson **out) {
    if (!ctx) return PERKS_ERR_INVALID_ARG;
    if (!out || !k || nx < 1 || ny < 1 || nprob < 1)
        return fail(ctx, PERKS_ERR_INVALID_ARG, "poisson_create: bad arguments");
    *out = nullptr;
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    auto *P = new perks_poisson();
    P->ctx = ctx;
    P->device = ctx->device;
    P->nx = nx; P->ny = ny; P->nprob = nprob;
    P->n = (long long)nx * ny;
    const size_t vb = sizeof(double) * (size_t)P->n * nprob;
    const size_t fxb = sizeof(double) * (size_t)(nx + 1) * ny * nprob;
    const size_t fyb = sizeof(double) * (size_t)nx * (ny + 1) * nprob;
    double *kd = nullptr;
    cudaError_t e = cudaSuccess;
    void **bufs[] = {(void **)&P->b, (void **)&P->x, (void **)&P->r, (void **)&P->p, (void **)&P->q, (void **)&P->dg};
    for (void **bp : bufs) if (e == cudaSuccess) e = cudaMalloc(bp, vb);
    if (e == cudaSuccess) e = cudaMalloc(&P->fx, fxb);
    if (e == cudaSuccess) e = cudaMalloc(&P->fy, fyb);
    if (e == cudaSuccess) e = cudaMalloc(&P->queue, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&P->iters, sizeof(int) * nprob);
    if (e == cudaSuccess) e = cudaMalloc(&P->status, sizeof(int) * nprob);
    if (e == cudaSuccess) e = cudaMalloc(&P->true_rel, sizeof(double) * nprob);
    P->max_groups = 2 * ctx->sm_count;  // at most two blocks per SM
    if (e == cudaSuccess) e = cudaMalloc(&P->gbar, sizeof(unsigned long long) * P->max_groups);
    if (e == cudaSuccess) e = cudaMalloc(&P->gprob, sizeof(int) * P->max_groups);
    if (e == cudaSuccess) e = cudaMalloc(&P->gpart, sizeof(double) * 2 * kPoiMaxGroup * P->max_groups);
    if (e == cudaSuccess) e = cudaMalloc(&P->err, sizeof(DevError));
    if (e == cudaSuccess && !on_device) {
        e = cudaMalloc(&kd, vb);
        if (e == cudaSuccess) e = cudaMemcpy(kd, k, vb, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        if (kd) cudaFree(kd);
        free_poisson(P);
        delete P;
        return cuda_fail(ctx, e, "poisson_create");
    }
    poisson_faces_kernel<<<1024, 256>>>(on_device ? k : kd, nx, ny, P->n * nprob, P->fx, P->fy);
    poisson_diag_kernel<<<1024, 256>>>(P->fx, P->fy, nx, ny, P->n * nprob, P->dg);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (kd) cudaFree(kd);
    if (e != cudaSuccess) { free_poisson(P); delete P; return cuda_fail(ctx, e, "poisson_create: faces"); }
    *out = P;
    return PERKS_OK;
}

extern "C" perks_status perks_poisson_destroy(perks_poisson *P) {
    if (!P) return PERKS_OK;
    cudaSetDevice(P->device);
    free_poisson(P);
    delete P;
    return PERKS_OK;
}

extern "C" perks_status perks_poisson_apply(perks_poisson *P, const double *v, double *y, perks_stream stream) {
    if (!P) return PERKS_ERR_INVALID_ARG;
    if (!v || !y) return fail(P->ctx, PERKS_ERR_INVALID_ARG, "poisson_apply: NULL vector");
    perks_status rc = use_device(P->ctx);
    if (rc) return rc;
    poisson_apply_kernel<<<1024, 256, 0, (cudaStream_t)stream>>>(poisson_args(P), v, y);
    PERKS_CUDA(P->ctx, cudaGetLastError());
    return PERKS_OK;
}

extern "C" perks_status perks_poisson_scale_guess(perks_poisson *P, const double *b, double *x,
                                                  perks_stream stream) {
    if (!P) return PERKS_ERR_INVALID_ARG;
    if (!b || !x) return fail(P->ctx, PERKS_ERR_INVALID_ARG, "poisson_scale_guess: NULL vector");
    perks_status rc = use_device(P->ctx);
    if (rc) return rc;
    const int grid = std::max(1, std::min(P->nprob, P->ctx->sm_count));
    poisson_scale_guess_kernel<512, kRows><<<grid, 512, 0, (cudaStream_t)stream>>>(poisson_args(P), b, x);
    PERKS_CUDA(P->ctx, cudaGetLastError());
    return PERKS_OK;
}

extern "C" perks_status perks_poisson_solve(perks_poisson *P, const double *b, double *x, double rtol,
                                            int32_t max_iter, perks_stream stream, perks_poisson_stats *stats) {
    if (!P) return PERKS_ERR_INVALID_ARG;
    perks_context *ctx = P->ctx;
    if (!b || !x || !(rtol >= 0) || max_iter < 0) return fail(ctx, PERKS_ERR_INVALID_ARG, "poisson_solve: bad arguments");
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t vb = sizeof(double) * (size_t)P->n * P->nprob;
    PERKS_CUDA(ctx, cudaMemcpyAsync(P->b, b, vb, cudaMemcpyDeviceToDevice, s));
    PERKS_CUDA(ctx, cudaMemcpyAsync(P->x, x, vb, cudaMemcpyDeviceToDevice, s));
    PERKS_CUDA(ctx, cudaMemsetAsync(P->queue, 0, sizeof(int), s));
    PoissonArgs a = poisson_args(P);
    a.rtol = rtol;
    a.max_iter = max_iter;
    a.max_restarts = 8;
    const int C = effective_group(P);
    const bool grouped = C > 1;
    const void *kern;
    if (P->rows_per_pass == 1)  // two 512-thread blocks per SM, one row per pass
        kern = grouped ? (const void *)perks_poisson_cg_kernel<512, 2, 1, 1, true>
                       : (const void *)perks_poisson_cg_kernel<512, 2, 1, 1, false>;
    else if (P->block_threads == 512)
        kern = grouped ? (const void *)perks_poisson_cg_kernel<512, 1, kRows, kLin, true>
                       : (const void *)perks_poisson_cg_kernel<512, 1, kRows, kLin, false>;
    else
        kern = grouped ? (const void *)perks_poisson_cg_kernel<kPoiThreads, 2, kRows, kLin, true>
                       : (const void *)perks_poisson_cg_kernel<kPoiThreads, 2, kRows, kLin, false>;
    int per_sm = 0;
    PERKS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, P->block_threads, 0));
    if (per_sm < 1) return fail(ctx, PERKS_ERR_LAUNCH_TOO_LARGE, "poisson_solve: kernel cannot be resident");
    void *kargs[] = {(void *)&a};
    int grid;
    if (!grouped) {
        grid = std::max(1, std::min(P->nprob, per_sm * ctx->sm_count));
        PERKS_CUDA(ctx, cudaLaunchKernel(kern, dim3(grid), dim3(P->block_threads), kargs, 0, s));
    } else {
        // groups wait on one another's blocks: every block resident (cooperative launch)
        const int groups = std::min({P->nprob, per_sm * ctx->sm_count / C, P->max_groups});
        if (groups < 1) return fail(ctx, PERKS_ERR_LAUNCH_TOO_LARGE, "poisson_solve: group larger than the GPU");
        grid = groups * C;
        PERKS_CUDA(ctx, cudaMemsetAsync(P->gbar, 0, sizeof(unsigned long long) * groups, s));
        PERKS_CUDA(ctx, cudaMemsetAsync(P->err, 0, sizeof(DevError), s));
        PERKS_CUDA(ctx, cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(P->block_threads), kargs, 0, s));
    }
    PERKS_CUDA(ctx, cudaMemcpyAsync(x, P->x, vb, cudaMemcpyDeviceToDevice, s));
    if (!stats) return PERKS_OK;
    PERKS_CUDA(ctx, cudaStreamSynchronize(s));
    int32_t *it_out = stats->iterations;
    double *tr_out = stats->true_rel_residual;
    const int32_t cap = stats->capacity;
    std::memset(stats, 0, sizeof(*stats));
    stats->iterations = it_out;
    stats->true_rel_residual = tr_out;
    stats->capacity = cap;
    stats->problems = P->nprob;
    stats->grid_blocks = grid;
    int *it = new int[P->nprob];
    int *st = new int[P->nprob];
    double *tr = new double[P->nprob];
    cudaMemcpy(it, P->iters, sizeof(int) * P->nprob, cudaMemcpyDeviceToHost);
    cudaMemcpy(st, P->status, sizeof(int) * P->nprob, cudaMemcpyDeviceToHost);
    cudaMemcpy(tr, P->true_rel, sizeof(double) * P->nprob, cudaMemcpyDeviceToHost);
    perks_status worst = PERKS_OK;
    long long sum_it = 0;
    for (int i = 0; i < P->nprob; ++i) {
        sum_it += it[i];
        stats->max_iterations = std::max(stats->max_iterations, it[i]);
        stats->max_true_rel_residual = std::max(stats->max_true_rel_residual, tr[i]);
        if (st[i] != PERKS_OK && worst == PERKS_OK) worst = st[i];
        if (stats->iterations && i < stats->capacity) {
            stats->iterations[i] = it[i];
            if (stats->true_rel_residual) stats->true_rel_residual[i] = tr[i];
        }
    }
    stats->mean_iterations = (double)sum_it / P->nprob;
    delete[] it;
    delete[] st;
    delete[] tr;
    if (grouped) {
        DevError de{};
        PERKS_CUDA(ctx, cudaMemcpy(&de, P->err, sizeof(DevError), cudaMemcpyDeviceToHost));
        if (de.code != 0)
            return fail(ctx, de.code, "poisson_solve: a block group's barrier gave up (block %d)", de.block);
    }
    if (worst != PERKS_OK) return fail(ctx, worst, "poisson_solve: a problem did not converge (status %d)", worst);
    return PERKS_OK;
}

extern "C" perks_status perks_poisson_set_group(perks_poisson *P, int32_t blocks) {
    if (!P) return PERKS_ERR_INVALID_ARG;
    if (blocks != 0 && blocks != 1 && blocks != 2 && blocks != 4 && blocks != 8)
        return fail(P->ctx, PERKS_ERR_INVALID_ARG, "poisson_set_group: 0 (automatic), 1, 2, 4 or 8 blocks");
    P->group = blocks;
    return PERKS_OK;
}

extern "C" perks_status perks_poisson_set_rows_per_pass(perks_poisson *P, int32_t rows) {
    if (!P) return PERKS_ERR_INVALID_ARG;
    if (rows != 1 && rows != kRows)
        return fail(P->ctx, PERKS_ERR_INVALID_ARG, "poisson_set_rows_per_pass: 1 or %d", kRows);
    P->rows_per_pass = rows;
    return PERKS_OK;
}

extern "C" perks_status perks_poisson_set_block_threads(perks_poisson *P, int32_t threads) {
    if (!P) return PERKS_ERR_INVALID_ARG;
    if (threads != 256 && threads != 512)
        return fail(P->ctx, PERKS_ERR_INVALID_ARG, "poisson_set_block_threads: 256 or 512");
    P->block_threads = threads;
    return PERKS_OK;
}
