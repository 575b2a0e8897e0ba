// Batched persistent stencils: many 2-D domains of uneven size, each with
// its own stencil (2d5pt, 2d9pt, 2d25pt, 2ds9pt), stepped together in ONE
// cooperative launch with one grid barrier per step.
//
// Each domain is cut into row tiles; a planner spreads the tiles of all
// domains over the blocks (longest-processing-time-first on a per-tile cost
// from the performance model of Sec. 5.2, i.e. a static work queue), and
// gives each block's tiles shared-memory cache rows from what its ring leaves
// free (the PERKS cache split, Sec. 4.1.3).  The autotuner searches the tile
// granularity and tile-width cap, first by that model and then by timing
// the best candidates on the GPU.  Every tile of a block is processed by the
// vectorised stencil step (stencil_vec.cuh) in turn; its cached rows stay in
// shared memory for the whole run.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"
#include "stencil_registry.h"
#include "stencil_vec.cuh"

using namespace perks;

namespace {

constexpr int kBatchThreads = 256;
constexpr int kBatchMaxR = 2;

struct BatchTile {
    int dom;    // domain index
    int tile;   // tile index within the domain's (ntx x 1 x ntz) grid
    int zs;     // cached rows of this tile in shared memory
    int smc_off;  // element offset of its cache in the block's cache area
};

struct BatchArgs {
    const PersistentArgs *doms;  // per-domain kernel arguments
    const int *dom_shape;        // ShapeId per domain
    const BatchTile *tiles;
    const int *block_first;      // G+1 offsets into tile_list
    const int *tile_list;        // tiles of each block
    long long ring_elems;        // elements reserved for the plane ring
    long long steps;
    unsigned long long *bar;
    DevError *err;
    long long timeout_ns;
};

// Loads the arguments of tile q's domain into shared memory and sets its
// cache rows; returns the tile.
__device__ __forceinline__ BatchTile load_tile(const BatchArgs &b, int q, PersistentArgs *s_args) {
    const BatchTile t = b.tiles[b.tile_list[q]];
    const int *src = reinterpret_cast<const int *>(b.doms + t.dom);
    int *dst = reinterpret_cast<int *>(s_args);
    constexpr int words = (int)(sizeof(PersistentArgs) / 4);
    __syncthreads();  // previous tile done with s_args
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    if (threadIdx.x == 0) s_args->zs = t.zs;
    __syncthreads();
    return t;
}

template <typename T, class SH, int V, int D>
__device__ __forceinline__ void batch_prologue(const PersistentArgs &a, const BatchTile &t, T *smc) {
    VecOf<T, V> regc[1];
    const VecPlan tp = make_vec_plan<SH, V, false>(a, t.tile);
    vec_prologue<T, SH, V, 0>(a, tp, smc + t.smc_off, regc);
}

template <typename T, class SH, int V, int D>
__device__ __forceinline__ void batch_step(const PersistentArgs &a, const BatchTile &t, long long k, bool last,
                                           T *ring, T *smc) {
    VecOf<T, V> regc[1];
    const VecPlan tp = make_vec_plan<SH, V, false>(a, t.tile);
    vec_step<T, SH, V, 0, D, false>(a, tp, k, last, 0, ring, smc + t.smc_off, regc);
    cp_async_wait_all();
}

template <typename T, int V, int D>
__global__ void __launch_bounds__(kBatchThreads, 1) perks_batch_kernel(const __grid_constant__ BatchArgs b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) PersistentArgs s_args;
    T *ring = reinterpret_cast<T *>(smem_raw);
    T *smc = ring + b.ring_elems;
    const int q0 = b.block_first[blockIdx.x], q1 = b.block_first[blockIdx.x + 1];
    unsigned long long epoch = 0;

    for (int q = q0; q < q1; ++q) {
        const BatchTile t = load_tile(b, q, &s_args);
        switch (b.dom_shape[t.dom]) {
        case SH_2D5: batch_prologue<T, S2d5, V, D>(s_args, t, smc); break;
        case SH_2D9: batch_prologue<T, S2d9, V, D>(s_args, t, smc); break;
        case SH_2D25: batch_prologue<T, S2d25, V, D>(s_args, t, smc); break;
        default: batch_prologue<T, S2ds9, V, D>(s_args, t, smc); break;
        }
    }
    if (!grid_barrier(b.bar, gridDim.x, epoch, b.err, b.timeout_ns)) return;
    for (long long k = 0; k < b.steps; ++k) {
        const bool last = (k + 1 == b.steps);
        for (int q = q0; q < q1; ++q) {
            const BatchTile t = load_tile(b, q, &s_args);
            switch (b.dom_shape[t.dom]) {
            case SH_2D5: batch_step<T, S2d5, V, D>(s_args, t, k, last, ring, smc); break;
            case SH_2D9: batch_step<T, S2d9, V, D>(s_args, t, k, last, ring, smc); break;
            case SH_2D25: batch_step<T, S2d25, V, D>(s_args, t, k, last, ring, smc); break;
            default: batch_step<T, S2ds9, V, D>(s_args, t, k, last, ring, smc); break;
            }
        }
        if (!last) {
            if (!grid_barrier(b.bar, gridDim.x, epoch, b.err, b.timeout_ns)) break;
        }
    }
    cp_async_wait_all();
}

// ------------------------------------------------------------- strip kernel
//
// Column-strip streaming: the batch's work is cut into items (domain, strip
// of 32 vectors = 32 V cells, range of rows) and a static
// longest-processing-time-first assignment gives every WARP its items.  A
// warp streams its item's input rows through a private ring of D row slots
// in shared memory (16-byte cp.async per lane, plus two halo cells on each
// side from the neighbouring strips), keeps the 2R + 1 rows the stencil
// reads in registers, and writes each output row with one 16-byte store per
// lane.  Halo cells come straight from the previous step's field, which
// nobody writes during the step, so warps never wait for each other inside a
// step: the only synchronisation is the grid barrier between steps.  Nothing
// is cached between steps (D_cache = 0): each step reads and writes every
// cell once, which is the HBM roofline of a domain set larger than the
// on-chip memory (171 MB of fp32 for the 64-domain workload).

struct StripItem {
    int dom;
    int x0;      // first cell of the strip (a multiple of 32 V)
    int z0, z1;  // output rows [z0, z1)
};

struct StripArgs {
    const PersistentArgs *doms;  // per-domain extents, weights, boundary, field[2]
    const int *dom_shape;
    const StripItem *items;      // items in warp order
    const int *warp_first;       // nwarps + 1 offsets into items
    long long steps;
    unsigned long long *bar;
    DevError *err;
    long long timeout_ns;
};

constexpr int kStripThreads = 256;
constexpr int kStripDepth = 8;   // ring rows per warp (16 measured slower: longer ring fill per item)

template <typename T, int V>
__host__ __device__ constexpr int strip_row_cells() { return 32 * V + 2 * V; }  // V pad cells on each side

// One item: output rows z0..z1-1 of the strip at x0.
template <typename T, class SH, int V, int D>
__device__ __forceinline__ void strip_item(const PersistentArgs &a, const StripItem it, int src, T *ring, int lane) {
    using A = typename ScalarOps<T>::A;
    using VT = VecOf<T, V>;
    constexpr int R = SH::R;
    constexpr int W = 2 * R + 1;
    constexpr int ROW = strip_row_cells<T, V>();
    static_assert(R <= 2 && D > 2 * R, "strip ring depth");
    const T *in = static_cast<const T *>(a.field[src]);
    T *out = static_cast<T *>(a.field[src ^ 1]);
    const int X = a.X, Z = a.Z;
    const int xl = it.x0 + lane * V;
    const bool own = xl < X;
    const T bnd = ScalarOps<T>::bnd(a);
    A w[SH::NPTS];
#pragma unroll
    for (int i = 0; i < SH::NPTS; ++i) w[i] = ScalarOps<T>::w(a, i);
    const int rfirst = it.z0 - R, rlast = it.z1 - 1 + R;

    // row r into ring slot (r - rfirst) % D; one cp.async group per row
    auto issue = [&](int r) {
        T *dst = ring + ((r - rfirst) % D) * ROW;
        const bool rin = r >= 0 && r < Z && r <= rlast;
        const long long rb = (long long)r * X;
        if (rin && own) cp_async<16>(dst + V + lane * V, in + rb + xl);
        else set_vec<T, V>(dst + V + lane * V, bnd);
        if (lane == 0) {
            if (rin && it.x0 >= 2) cp_async<2 * sizeof(T)>(dst + V - 2, in + rb + it.x0 - 2);
            else { dst[V - 2] = bnd; dst[V - 1] = bnd; }
        }
        if (lane == 31) {
            const int xr = it.x0 + 32 * V;
            if (rin && xr + 2 <= X) cp_async<2 * sizeof(T)>(dst + V + 32 * V, in + rb + xr);
            else { dst[V + 32 * V] = bnd; dst[V + 32 * V + 1] = bnd; }
        }
        cp_async_commit();
    };
    // the lane's cells -2 .. V+1 of row r (from its ring slot), in the accumulator type
    auto fetch = [&](int r, A (&row)[V + 4]) {
        cp_async_wait<D - 1>();
        __syncwarp();
        const T *p = ring + ((r - rfirst) % D) * ROW + V + lane * V;
        const VT c = *reinterpret_cast<const VT *>(p);
        const PairOf<T> l = *reinterpret_cast<const PairOf<T> *>(p - 2);
        const PairOf<T> h = *reinterpret_cast<const PairOf<T> *>(p + V);
        row[0] = to_acc(l.v[0]);
        row[1] = to_acc(l.v[1]);
#pragma unroll
        for (int j = 0; j < V; ++j) row[2 + j] = to_acc(c.v[j]);
        row[V + 2] = to_acc(h.v[0]);
        row[V + 3] = to_acc(h.v[1]);
        __syncwarp();  // every lane has read the slot before it is refilled
        issue(r + D);
    };

    for (int j = 0; j < D; ++j) issue(rfirst + j);
    A win[W][V + 4];
    // the first 2R rows of the window: rows z0-R .. z0+R-1 in slots 0 .. 2R-1
    static_for<0, 2 * R>([&](auto JI) { fetch(rfirst + decltype(JI)::value, win[decltype(JI)::value]); });
    // output row z reads window slots (z - rfirst + k) % W, k = 0..2R; the loop
    // advances W rows per turn so that every slot index is a constant
    for (int zb = it.z0; zb < it.z1; zb += W) {
        static_for<0, W>([&](auto PI) {
            constexpr int p = decltype(PI)::value;
            const int z = zb + p;
            if (z < it.z1) {
                fetch(z + R, win[(p + 2 * R) % W]);
                VT o;
                A acc[V];
                if constexpr (std::is_same<A, float>::value && V % 2 == 0) {
                    // fp32: a term whose x offset is even updates two cells
                    // with one packed fma (__ffma2_rn rounds each lane as
                    // fmaf does; the two cells sit in an aligned register
                    // pair of the window row), an odd offset one cell at a
                    // time; every cell adds its terms in table order from 0
                    float2 acc2[V / 2];
#pragma unroll
                    for (int q = 0; q < V / 2; ++q) acc2[q] = make_float2(0.f, 0.f);
                    static_for<0, SH::NPTS>([&](auto II) {
                        constexpr int i = decltype(II)::value;
                        constexpr int slot = (p + R + SH::dz(i)) % W;
                        constexpr int dx = SH::dx(i);
                        if constexpr (dx % 2 == 0) {
                            const float2 w2 = make_float2(w[i], w[i]);
#pragma unroll
                            for (int q = 0; q < V / 2; ++q)
                                acc2[q] = __ffma2_rn(w2, make_float2(win[slot][2 + 2 * q + dx], win[slot][3 + 2 * q + dx]),
                                                     acc2[q]);
                        } else {
#pragma unroll
                            for (int q = 0; q < V / 2; ++q) {
                                acc2[q].x = fmaf(w[i], win[slot][2 + 2 * q + dx], acc2[q].x);
                                acc2[q].y = fmaf(w[i], win[slot][3 + 2 * q + dx], acc2[q].y);
                            }
                        }
                    });
#pragma unroll
                    for (int q = 0; q < V / 2; ++q) {
                        acc[2 * q] = acc2[q].x;
                        acc[2 * q + 1] = acc2[q].y;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < V; ++q) acc[q] = A(0);
                    static_for<0, SH::NPTS>([&](auto II) {
                        constexpr int i = decltype(II)::value;
                        constexpr int slot = (p + R + SH::dz(i)) % W;
#pragma unroll
                        for (int q = 0; q < V; ++q) acc[q] = fma(w[i], win[slot][2 + q + SH::dx(i)], acc[q]);
                    });
                }
                if constexpr (std::is_same<T, __nv_bfloat16>::value) {
                    __nv_bfloat162 *o2 = reinterpret_cast<__nv_bfloat162 *>(&o);
#pragma unroll
                    for (int q = 0; q < V / 2; ++q) o2[q] = __floats2bfloat162_rn(acc[2 * q], acc[2 * q + 1]);
                } else {
#pragma unroll
                    for (int q = 0; q < V; ++q) o.v[q] = from_acc<T>(acc[q]);
                }
                if (own) *reinterpret_cast<VT *>(out + (long long)z * X + xl) = o;
            }
        });
    }
    cp_async_wait_all();
    __syncwarp();
}

template <typename T, int V>
__global__ void __launch_bounds__(kStripThreads, sizeof(T) == 8 ? 1 : 2)
    perks_batch_strip_kernel(const __grid_constant__ StripArgs b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int D = kStripDepth;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *ring = reinterpret_cast<T *>(smem_raw) + (long long)warp * D * strip_row_cells<T, V>();
    const int gw = blockIdx.x * (kStripThreads / 32) + warp;
    const int i0 = b.warp_first[gw], i1 = b.warp_first[gw + 1];
    unsigned long long epoch = 0;
    for (long long k = 0; k < b.steps; ++k) {
        const int src = (int)(k & 1);
        for (int q = i0; q < i1; ++q) {
            const StripItem it = b.items[q];
            const PersistentArgs &a = b.doms[it.dom];
            switch (b.dom_shape[it.dom]) {
            case SH_2D5: strip_item<T, S2d5, V, D>(a, it, src, ring, lane); break;
            case SH_2D9: strip_item<T, S2d9, V, D>(a, it, src, ring, lane); break;
            case SH_2D25: strip_item<T, S2d25, V, D>(a, it, src, ring, lane); break;
            default: strip_item<T, S2ds9, V, D>(a, it, src, ring, lane); break;
            }
        }
        if (k + 1 < b.steps) {
            if (!grid_barrier(b.bar, gridDim.x, epoch, b.err, b.timeout_ns)) return;
        }
    }
}

using StripFn = void (*)(StripArgs);

using BatchFn = void (*)(BatchArgs);

struct BatchKernel {
    int dtype;
    int v, d;
    BatchFn fn;
};

std::vector<BatchKernel> &batch_kernels() {
    static std::vector<BatchKernel> k = {
        {PERKS_F64, 2, 8, perks_batch_kernel<double, 2, 8>},
        {PERKS_F32, 4, 12, perks_batch_kernel<float, 4, 12>},
        {PERKS_BF16, 8, 16, perks_batch_kernel<__nv_bfloat16, 8, 16>},
    };
    return k;
}

// Strip kernels (column-strip streaming), by storage type.
StripFn strip_kernel(int dtype) {
    if (dtype == PERKS_F32) return perks_batch_strip_kernel<float, 4>;
    if (dtype == PERKS_F64) return perks_batch_strip_kernel<double, 2>;
    return nullptr;
}

int shape_id_2d(const perks_stencil_desc &d, double *kw) {
    // canonical 2-D shapes the batched kernel compiles
    struct Cand { int id; int r; bool box; };
    const Cand cands[] = {{SH_2D5, 1, false}, {SH_2D9, 1, true}, {SH_2D25, 2, true}, {SH_2DS9, 2, false}};
    for (const Cand &c : cands) {
        const int W = 2 * c.r + 1;
        const int npts = c.box ? W * W : 1 + 4 * c.r;
        if (d.ndim != 2 || d.npts != npts || d.radius != c.r) continue;
        unsigned char used[PERKS_MAX_POINTS] = {};
        bool ok = true;
        for (int i = 0; i < npts && ok; ++i) {
            int ux, uy;
            if (c.box) { ux = i % W - c.r; uy = i / W - c.r; }
            else if (i == 0) { ux = 0; uy = 0; }
            else {
                const int k = i - 1, dd = k / 4 + 1, a = (k % 4) / 2, sg = (k % 2 == 0) ? -1 : 1;
                ux = a == 0 ? sg * dd : 0;
                uy = a == 1 ? sg * dd : 0;
            }
            int found = -1;
            for (int j = 0; j < d.npts; ++j)
                if (!used[j] && d.offsets[3 * j] == ux && d.offsets[3 * j + 1] == uy && d.offsets[3 * j + 2] == 0) {
                    found = j;
                    break;
                }
            if (found < 0) ok = false;
            else { used[found] = 1; kw[i] = d.weights[found]; }
        }
        if (ok) return c.id;
    }
    return -1;
}

int ceil_div(int a, int b) { return (a + b - 1) / b; }

}  // namespace

struct perks_batch {
    perks_context *ctx = nullptr;
    int device = 0;  // for destroy, which may come after the context is gone
    int dtype = PERKS_F32;
    int es = 4;
    int ndom = 0;
    std::vector<perks_stencil_desc> desc;
    std::vector<int> shape;
    std::vector<std::vector<double>> kw;
    std::vector<void *> field[2];
    std::vector<int> cur;         // current buffer per domain (all equal after runs)
    std::vector<void *> faces[2];
    std::vector<size_t> faces_bytes;
    unsigned long long *bar = nullptr;
    DevError *err = nullptr;
    // plan
    double granularity = 1.0;     // target tile cells = granularity * total / G
    int width_cap = 0;            // max tile width (cells), 0 = kernel limit
    bool tuned = false;
    // device tables of the current plan
    PersistentArgs *d_doms = nullptr;
    int *d_shape = nullptr;
    BatchTile *d_tiles = nullptr;
    int *d_block_first = nullptr;
    int *d_tile_list = nullptr;
    size_t cap_tiles = 0;
    // host view of the plan
    int blocks = 0;
    int ntiles = 0;
    int max_tiles_per_block = 0;
    long long smem = 0;
    long long ring_elems = 0;
    long long cached_cells = 0;
    long long halo_cells = 0;
    double predicted_ms_per_step = 0.0;
    std::vector<PersistentArgs> h_doms;
    std::vector<perks_stencil *> per_step;  // baseline objects, one per domain
    // kernel choice: PERKS_BATCH_RING (tiles of rows through a plane ring) or
    // PERKS_BATCH_STRIP (column strips streamed by single warps)
    int kernel = PERKS_BATCH_RING;
    int strip_rows = 0;            // strip kernel: output rows per item (0 = automatic)
    StripItem *d_items = nullptr;
    int *d_warp_first = nullptr;
    size_t cap_items = 0, cap_warps = 0;
    int strip_blocks = 0;          // grid of the current strip plan (0: none)
    int nitems = 0, max_items_per_warp = 0;
    long long strip_halo = 0, strip_smem = 0;
    std::vector<PersistentArgs> h_sdoms;
    PersistentArgs *d_sdoms = nullptr;
};

namespace {

BatchKernel *batch_kernel(perks_batch *b) {
    for (BatchKernel &k : batch_kernels())
        if (k.dtype == b->dtype) return &k;
    return nullptr;
}

struct PlanOut {
    std::vector<PersistentArgs> doms;
    std::vector<BatchTile> tiles;
    std::vector<int> block_first, tile_list;
    long long ring_elems = 0, smem = 0, cached = 0, halo = 0;
    int max_tiles = 0;
    double predicted = 0.0;  // ms per step (model)
};

// Plans tiles, assignment and cache split for a granularity and width cap.
perks_status plan_batch(perks_batch *b, BatchKernel &k, double granularity, int width_cap, PlanOut &o) {
    int smem_budget = 0;  // dynamic shared memory per block on this device (limit raised once per device)
    {
        const perks_status rc = smem_optin(b->ctx, (const void *)k.fn, &smem_budget);
        if (rc) return rc;
    }
    perks_context *ctx = b->ctx;
    const int G = ctx->sm_count;  // one block per SM
    const int V = k.v;
    const int es = b->es;
    const int S = vec_slots<kBatchMaxR, 0>() + k.d;
    const int HX = std::max(V, 2);
    const int maxw = std::min(width_cap > 0 ? width_cap : kBatchThreads * V, kBatchThreads * V);
    long long total = 0;
    for (const auto &d : b->desc) total += d.nx * d.ny;
    const double target = std::max(1.0, granularity * (double)total / G);
    o.doms.assign(b->ndom, PersistentArgs{});
    o.tiles.clear();
    int txmax_all = 0;
    for (int i = 0; i < b->ndom; ++i) {
        const auto &d = b->desc[i];
        const int X = (int)d.nx, Z = (int)d.ny;
        const int XU = X / V;
        const int R = d.radius;
        int ntx = std::max(1, ceil_div(X, maxw));
        const long long cells = (long long)X * Z;
        int ntiles = std::max(1, (int)std::lround(cells / target));
        ntiles = std::max(ntiles, ntx);
        int ntz = std::max(1, ntiles / ntx);
        ntz = std::min(ntz, std::max(1, Z / std::max(R, 1)));
        while (ntx > 1 && (XU / ntx) * V < 2) --ntx;
        PersistentArgs &a = o.doms[i];
        std::memset(&a, 0, sizeof(a));
        a.X = X; a.Y = 1; a.Z = Z;
        a.XY = X;
        a.ntx = ntx; a.nty = 1; a.ntz = ntz;
        a.txmax = ceil_div(XU, ntx) * V;
        a.tymax = 1;
        a.tzmax = ceil_div(Z, ntz);
        a.PW = a.txmax + 2 * HX;
        a.plane = a.PW;
        a.ncol = a.txmax;
        a.steps = 0;
        a.boundary = d.boundary;
        a.boundary_f = (float)d.boundary;
        for (int j = 0; j < kMaxKernelPoints && j < (int)b->kw[i].size(); ++j) {
            a.w[j] = b->kw[i][j];
            a.wf[j] = (float)b->kw[i][j];
        }
        a.face_plane = (long long)a.tzmax * a.tymax;
        txmax_all = std::max(txmax_all, a.txmax);
        for (int t = 0; t < ntx * ntz; ++t) o.tiles.push_back(BatchTile{i, t, 0, 0});
    }
    o.ring_elems = (long long)S * (txmax_all + 2 * HX);
    o.ring_elems = (o.ring_elems + 15) & ~15ll;
    const long long ring_bytes = o.ring_elems * es;
    if (ring_bytes > smem_budget) return fail(ctx, PERKS_ERR_UNSUPPORTED, "batch: ring exceeds shared memory");

    // per-tile geometry and model cost (Sec. 5.2: bytes / per-SM bandwidth,
    // plus a pipeline fill per tile visit)
    const double bw_sm = 6.8e12 / G;           // bytes/s per SM
    const double row_fill_s = 1.0e-6;          // ring fill latency per tile visit
    std::vector<double> cost(o.tiles.size());
    std::vector<int> tw(o.tiles.size()), th(o.tiles.size());
    for (size_t q = 0; q < o.tiles.size(); ++q) {
        const PersistentArgs &a = o.doms[o.tiles[q].dom];
        const int ti = o.tiles[q].tile % a.ntx, tk = o.tiles[q].tile / a.ntx;
        int x0, txu, z0, tz;
        split_axis(a.X / V, a.ntx, ti, x0, txu);
        split_axis(a.Z, a.ntz, tk, z0, tz);
        tw[q] = txu * V;
        th[q] = tz;
        cost[q] = 2.0 * tw[q] * th[q] * es / bw_sm + row_fill_s;
    }
    // longest-processing-time-first assignment
    std::vector<int> order(o.tiles.size());
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<double> load(G, 0.0);
    std::vector<std::vector<int>> per_block(G);
    for (int q : order) {
        const int bb = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        per_block[bb].push_back(q);
        load[bb] += cost[q];
    }
    // cache rows: each block fills its free shared memory with rows of its tiles
    o.block_first.assign(G + 1, 0);
    o.tile_list.clear();
    long long max_cache = 0;
    o.cached = 0;
    o.halo = 0;
    double makespan = 0.0;
    for (int bb = 0; bb < G; ++bb) {
        o.block_first[bb] = (int)o.tile_list.size();
        long long free_elems = (smem_budget - ring_bytes) / es;
        long long off = 0;
        double t_block = 0.0;
        for (int q : per_block[bb]) {
            const PersistentArgs &a = o.doms[o.tiles[q].dom];
            const int R = b->desc[o.tiles[q].dom].radius;
            const long long row = a.ncol;
            int zs = (int)std::min<long long>(th[q], std::max<long long>(0, (free_elems - off) / row));
            o.tiles[q].zs = zs;
            o.tiles[q].smc_off = (int)off;
            off += (long long)zs * row;
            o.cached += (long long)zs * tw[q];
            const int ti = o.tiles[q].tile % a.ntx;
            const int nfx = (ti > 0) + (ti + 1 < a.ntx);
            const long long halo = 2LL * (nfx * R * th[q] + 2 * R * tw[q]);
            o.halo += halo;
            t_block += (2.0 * (double)(th[q] - zs) * tw[q] + halo) * es / bw_sm + row_fill_s;
            o.tile_list.push_back(q);
        }
        max_cache = std::max(max_cache, off);
        o.max_tiles = std::max(o.max_tiles, (int)per_block[bb].size());
        makespan = std::max(makespan, t_block);
    }
    o.block_first[G] = (int)o.tile_list.size();
    o.smem = ring_bytes + max_cache * es;
    o.predicted = makespan * 1e3;
    return PERKS_OK;
}

perks_status upload_plan(perks_batch *b, const PlanOut &o) {
    perks_context *ctx = b->ctx;
    const int G = ctx->sm_count;
    if (o.tiles.size() > b->cap_tiles) {
        if (b->d_tiles) cudaFree(b->d_tiles);
        if (b->d_tile_list) cudaFree(b->d_tile_list);
        b->d_tiles = nullptr;
        b->d_tile_list = nullptr;
        PERKS_CUDA(ctx, cudaMalloc(&b->d_tiles, o.tiles.size() * sizeof(BatchTile)));
        PERKS_CUDA(ctx, cudaMalloc(&b->d_tile_list, o.tiles.size() * sizeof(int)));
        b->cap_tiles = o.tiles.size();
    }
    if (!b->d_doms) PERKS_CUDA(ctx, cudaMalloc(&b->d_doms, b->ndom * sizeof(PersistentArgs)));
    if (!b->d_shape) PERKS_CUDA(ctx, cudaMalloc(&b->d_shape, b->ndom * sizeof(int)));
    if (!b->d_block_first) PERKS_CUDA(ctx, cudaMalloc(&b->d_block_first, (G + 1) * sizeof(int)));
    // faces per domain: [tile][side][z] pairs
    b->h_doms = o.doms;
    for (int i = 0; i < b->ndom; ++i) {
        PersistentArgs &a = b->h_doms[i];
        const size_t need = (size_t)a.ntx * a.ntz * 2 * a.face_plane * 2 * b->es;
        if (need > b->faces_bytes[i]) {
            for (int p = 0; p < 2; ++p) {
                if (b->faces[p][i]) cudaFree(b->faces[p][i]);
                b->faces[p][i] = nullptr;
                PERKS_CUDA(ctx, cudaMalloc(&b->faces[p][i], need));
            }
            b->faces_bytes[i] = need;
        }
        a.faces[0] = b->faces[0][i];
        a.faces[1] = b->faces[1][i];
    }
    PERKS_CUDA(ctx, cudaMemcpy(b->d_shape, b->shape.data(), b->ndom * sizeof(int), cudaMemcpyHostToDevice));
    PERKS_CUDA(ctx, cudaMemcpy(b->d_tiles, o.tiles.data(), o.tiles.size() * sizeof(BatchTile),
                               cudaMemcpyHostToDevice));
    PERKS_CUDA(ctx, cudaMemcpy(b->d_tile_list, o.tile_list.data(), o.tile_list.size() * sizeof(int),
                               cudaMemcpyHostToDevice));
    PERKS_CUDA(ctx, cudaMemcpy(b->d_block_first, o.block_first.data(), (G + 1) * sizeof(int),
                               cudaMemcpyHostToDevice));
    b->blocks = G;
    b->ntiles = (int)o.tiles.size();
    b->max_tiles_per_block = o.max_tiles;
    b->smem = o.smem;
    b->ring_elems = o.ring_elems;
    b->cached_cells = o.cached;
    b->halo_cells = o.halo;
    b->predicted_ms_per_step = o.predicted;
    return PERKS_OK;
}

// Strip plan: items of `rows` output rows (0: as many as give every warp
// about one item's worth of rows), longest-processing-time-first over the
// warps of a co-resident grid.  Item cost = rows read (its rows plus 2R of
// halo) x (1 + points / 25): the stream of rows, plus the stencil's FMAs.
perks_status plan_strips(perks_batch *b, int rows) {
    perks_context *ctx = b->ctx;
    StripFn fn = strip_kernel(b->dtype);
    if (!fn) return fail(ctx, PERKS_ERR_UNSUPPORTED, "batch: no strip kernel for this dtype");
    const int V = (int)(16 / b->es);
    const int W = 32 * V;
    const size_t smem = (size_t)(kStripThreads / 32) * kStripDepth * (32 * V + 2 * V) * b->es;
    int budget = 0;
    perks_status rc = smem_optin(ctx, (const void *)fn, &budget);
    if (rc) return rc;
    int per_sm = 0;
    PERKS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, kStripThreads, smem));
    if (per_sm < 1) return fail(ctx, PERKS_ERR_LAUNCH_TOO_LARGE, "batch strip kernel is not resident");
    const int G = per_sm * ctx->sm_count;
    const int nwarps = G * (kStripThreads / 32);
    long long total_rows = 0;
    for (const auto &d : b->desc) total_rows += (long long)ceil_div((int)d.nx, W) * d.ny;
    const int target = rows > 0 ? rows : (int)std::min<long long>(1024, std::max<long long>(8, total_rows / nwarps));
    std::vector<StripItem> items;
    std::vector<double> cost;
    long long halo = 0;
    for (int i = 0; i < b->ndom; ++i) {
        const int X = (int)b->desc[i].nx, Z = (int)b->desc[i].ny, R = b->desc[i].radius;
        const int nseg = std::max(1, (int)std::lround((double)Z / target));
        for (int x0 = 0; x0 < X; x0 += W)
            for (int sgi = 0; sgi < nseg; ++sgi) {
                int z0, nz;
                split_axis(Z, nseg, sgi, z0, nz);
                items.push_back(StripItem{i, x0, z0, z0 + nz});
                cost.push_back((double)(nz + 2 * R) * (1.0 + b->desc[i].npts / 25.0));
                halo += 2LL * R * std::min(W, X - x0) + 4LL * (nz + 2 * R);
            }
    }
    // LPT: the costliest item to the least loaded warp
    std::vector<int> order(items.size());
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<std::pair<double, int>> heap;  // (load, warp), min-heap
    heap.reserve(nwarps);
    for (int w = 0; w < nwarps; ++w) heap.push_back({0.0, w});
    auto cmp = [](const std::pair<double, int> &x, const std::pair<double, int> &y) { return x.first > y.first; };
    std::make_heap(heap.begin(), heap.end(), cmp);
    std::vector<std::vector<int>> per_warp(nwarps);
    for (int q : order) {
        std::pop_heap(heap.begin(), heap.end(), cmp);
        auto &top = heap.back();
        per_warp[top.second].push_back(q);
        top.first += cost[q];
        std::push_heap(heap.begin(), heap.end(), cmp);
    }
    std::vector<StripItem> sorted;
    std::vector<int> first(nwarps + 1, 0);
    int maxw = 0;
    for (int w = 0; w < nwarps; ++w) {
        first[w] = (int)sorted.size();
        for (int q : per_warp[w]) sorted.push_back(items[q]);
        maxw = std::max(maxw, (int)per_warp[w].size());
    }
    first[nwarps] = (int)sorted.size();
    if (sorted.size() > b->cap_items) {
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        PERKS_CUDA(ctx, cudaMalloc(&b->d_items, sorted.size() * sizeof(StripItem)));
        b->cap_items = sorted.size();
    }
    if ((size_t)nwarps + 1 > b->cap_warps) {
        if (b->d_warp_first) cudaFree(b->d_warp_first);
        b->d_warp_first = nullptr;
        PERKS_CUDA(ctx, cudaMalloc(&b->d_warp_first, (nwarps + 1) * sizeof(int)));
        b->cap_warps = (size_t)nwarps + 1;
    }
    PERKS_CUDA(ctx, cudaMemcpy(b->d_items, sorted.data(), sorted.size() * sizeof(StripItem), cudaMemcpyHostToDevice));
    PERKS_CUDA(ctx, cudaMemcpy(b->d_warp_first, first.data(), (nwarps + 1) * sizeof(int), cudaMemcpyHostToDevice));
    if (!b->d_sdoms) PERKS_CUDA(ctx, cudaMalloc(&b->d_sdoms, b->ndom * sizeof(PersistentArgs)));
    if (!b->d_shape) PERKS_CUDA(ctx, cudaMalloc(&b->d_shape, b->ndom * sizeof(int)));
    PERKS_CUDA(ctx, cudaMemcpy(b->d_shape, b->shape.data(), b->ndom * sizeof(int), cudaMemcpyHostToDevice));
    b->h_sdoms.assign(b->ndom, PersistentArgs{});
    for (int i = 0; i < b->ndom; ++i) {
        PersistentArgs &a = b->h_sdoms[i];
        std::memset(&a, 0, sizeof(a));
        a.X = (int)b->desc[i].nx; a.Y = 1; a.Z = (int)b->desc[i].ny;
        a.XY = a.X;
        a.boundary = b->desc[i].boundary;
        a.boundary_f = (float)b->desc[i].boundary;
        for (int j = 0; j < kMaxKernelPoints && j < (int)b->kw[i].size(); ++j) {
            a.w[j] = b->kw[i][j];
            a.wf[j] = (float)b->kw[i][j];
        }
    }
    b->strip_blocks = G;
    b->nitems = (int)sorted.size();
    b->max_items_per_warp = maxw;
    b->strip_halo = halo;
    b->strip_smem = (long long)smem;
    return PERKS_OK;
}

perks_status launch_strips(perks_batch *b, long long steps, cudaStream_t s) {
    perks_context *ctx = b->ctx;
    if (b->strip_blocks == 0) {
        perks_status rc = plan_strips(b, b->strip_rows);
        if (rc) return rc;
    }
    for (int i = 0; i < b->ndom; ++i) {
        PersistentArgs &a = b->h_sdoms[i];
        a.field[0] = b->field[b->cur[i]][i];
        a.field[1] = b->field[b->cur[i] ^ 1][i];
        a.steps = steps;
    }
    PERKS_CUDA(ctx, cudaMemcpyAsync(b->d_sdoms, b->h_sdoms.data(), b->ndom * sizeof(PersistentArgs),
                                    cudaMemcpyHostToDevice, s));
    PERKS_CUDA(ctx, cudaMemsetAsync(b->bar, 0, sizeof(unsigned long long), s));
    PERKS_CUDA(ctx, cudaMemsetAsync(b->err, 0, sizeof(DevError), s));
    StripArgs args;
    args.doms = b->d_sdoms;
    args.dom_shape = b->d_shape;
    args.items = b->d_items;
    args.warp_first = b->d_warp_first;
    args.steps = steps;
    args.bar = b->bar;
    args.err = b->err;
    args.timeout_ns = ctx->timeout_ns;
    void *kargs[] = {&args};
    PERKS_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)strip_kernel(b->dtype), dim3(b->strip_blocks),
                                                dim3(kStripThreads), kargs, (size_t)b->strip_smem, s));
    if (steps & 1)
        for (int i = 0; i < b->ndom; ++i) b->cur[i] ^= 1;
    return PERKS_OK;
}

perks_status ensure_plan(perks_batch *b) {
    BatchKernel *k = batch_kernel(b);
    if (!k) return fail(b->ctx, PERKS_ERR_UNSUPPORTED, "batch: no kernel for this dtype");
    if (b->blocks > 0) return PERKS_OK;
    PlanOut o;
    perks_status rc = plan_batch(b, *k, b->granularity, b->width_cap, o);
    if (rc) return rc;
    return upload_plan(b, o);
}

perks_status launch_batch(perks_batch *b, long long steps, cudaStream_t s) {
    perks_context *ctx = b->ctx;
    perks_status rc = ensure_plan(b);
    if (rc) return rc;
    BatchKernel *k = batch_kernel(b);
    for (int i = 0; i < b->ndom; ++i) {
        PersistentArgs &a = b->h_doms[i];
        a.field[0] = b->field[b->cur[i]][i];
        a.field[1] = b->field[b->cur[i] ^ 1][i];
        a.steps = steps;
        a.timeout_ns = ctx->timeout_ns;
    }
    PERKS_CUDA(ctx, cudaMemcpyAsync(b->d_doms, b->h_doms.data(), b->ndom * sizeof(PersistentArgs),
                                    cudaMemcpyHostToDevice, s));
    PERKS_CUDA(ctx, cudaMemsetAsync(b->bar, 0, sizeof(unsigned long long), s));
    PERKS_CUDA(ctx, cudaMemsetAsync(b->err, 0, sizeof(DevError), s));
    int per_sm = 0;
    PERKS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k->fn, kBatchThreads,
                                                                  b->smem));
    if (per_sm < 1) return fail(ctx, PERKS_ERR_LAUNCH_TOO_LARGE, "batch kernel is not resident");
    BatchArgs args;
    args.doms = b->d_doms;
    args.dom_shape = b->d_shape;
    args.tiles = b->d_tiles;
    args.block_first = b->d_block_first;
    args.tile_list = b->d_tile_list;
    args.ring_elems = b->ring_elems;
    args.steps = steps;
    args.bar = b->bar;
    args.err = b->err;
    args.timeout_ns = ctx->timeout_ns;
    void *kargs[] = {&args};
    PERKS_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)k->fn, dim3(b->blocks), dim3(kBatchThreads), kargs,
                                                (size_t)b->smem, s));
    if (steps & 1)
        for (int i = 0; i < b->ndom; ++i) b->cur[i] ^= 1;
    return PERKS_OK;
}

// Baseline: every domain advanced by its own one-launch-per-step kernel
// (one stencil object per domain, created on first use and kept).
perks_status launch_batch_per_step(perks_batch *b, long long steps, cudaStream_t s) {
    perks_context *ctx = b->ctx;
    if (b->per_step.empty()) {
        b->per_step.assign(b->ndom, nullptr);
        for (int i = 0; i < b->ndom; ++i) {
            perks_status rc = perks_stencil_create(ctx, &b->desc[i], &b->per_step[i]);
            if (rc) return rc;
        }
    }
    perks_status rc = PERKS_OK;
    for (int i = 0; i < b->ndom && !rc; ++i) rc = perks_stencil_set_field(b->per_step[i], b->field[b->cur[i]][i], 1, s);
    for (long long k = 0; k < steps && !rc; ++k)
        for (int i = 0; i < b->ndom && !rc; ++i) rc = perks_stencil_run(b->per_step[i], 1, PERKS_PER_STEP, s, nullptr);
    for (int i = 0; i < b->ndom && !rc; ++i) rc = perks_stencil_get_field(b->per_step[i], b->field[b->cur[i]][i], 1, s);
    return rc;
}

}  // namespace

// ======================================================================= ABI

extern "C" perks_status perks_batch_create(perks_context *ctx, int32_t ndom, const perks_stencil_desc *descs,
                                           perks_batch **out) {
    if (!ctx) return PERKS_ERR_INVALID_ARG;
    if (!descs || !out || ndom < 1) return fail(ctx, PERKS_ERR_INVALID_ARG, "batch_create: bad arguments");
    *out = nullptr;
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    const int dtype = descs[0].dtype;
    auto *b = new perks_batch();
    b->ctx = ctx;
    b->device = ctx->device;
    b->dtype = dtype;
    b->es = (int)dtype_size(dtype);
    b->ndom = ndom;
    BatchKernel *k = nullptr;
    for (BatchKernel &kk : batch_kernels())
        if (kk.dtype == dtype) k = &kk;
    if (!k) { delete b; return fail(ctx, PERKS_ERR_UNSUPPORTED, "batch_create: dtype %d", dtype); }
    for (int i = 0; i < ndom; ++i) {
        const perks_stencil_desc &d = descs[i];
        std::vector<double> kw(kMaxKernelPoints, 0.0);
        const int id = shape_id_2d(d, kw.data());
        if (d.dtype != dtype || d.ndim != 2 || d.nz != 1 || d.nx < 1 || d.ny < 1 || id < 0) {
            delete b;
            return fail(ctx, PERKS_ERR_UNSUPPORTED,
                        "batch_create: domain %d must be 2-D, same dtype, shape 2d5pt/2d9pt/2d25pt/2ds9pt", i);
        }
        if (d.nx % k->v != 0 || d.nx < 2 * k->v || d.ny < 2 * d.radius) {
            delete b;
            return fail(ctx, PERKS_ERR_UNSUPPORTED, "batch_create: domain %d nx must be a multiple of %d", i, k->v);
        }
        b->desc.push_back(d);
        b->shape.push_back(id);
        b->kw.push_back(kw);
    }
    b->kernel = strip_kernel(dtype) ? PERKS_BATCH_STRIP : PERKS_BATCH_RING;
    for (int p = 0; p < 2; ++p) b->field[p].assign(ndom, nullptr), b->faces[p].assign(ndom, nullptr);
    b->faces_bytes.assign(ndom, 0);
    b->cur.assign(ndom, 0);
    for (int i = 0; i < ndom; ++i)
        for (int p = 0; p < 2; ++p) {
            cudaError_t e = cudaMalloc(&b->field[p][i], (size_t)descs[i].nx * descs[i].ny * b->es);
            if (e != cudaSuccess) { perks_batch_destroy(b); return cuda_fail(ctx, e, "batch_create: cudaMalloc"); }
        }
    if (cudaMalloc(&b->bar, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&b->err, sizeof(DevError)) != cudaSuccess) {
        perks_batch_destroy(b);
        return fail(ctx, PERKS_ERR_OUT_OF_MEMORY, "batch_create: cudaMalloc");
    }
    *out = b;
    return PERKS_OK;
}

extern "C" perks_status perks_batch_destroy(perks_batch *b) {
    if (!b) return PERKS_OK;
    cudaSetDevice(b->device);
    for (int p = 0; p < 2; ++p) {
        for (void *q : b->field[p]) if (q) cudaFree(q);
        for (void *q : b->faces[p]) if (q) cudaFree(q);
    }
    void *ptrs[] = {b->bar, b->err, b->d_doms, b->d_shape, b->d_tiles, b->d_block_first, b->d_tile_list,
                    b->d_items, b->d_warp_first, b->d_sdoms};
    for (void *q : ptrs) if (q) cudaFree(q);
    for (perks_stencil *st : b->per_step) perks_stencil_destroy(st);
    delete b;
    return PERKS_OK;
}

extern "C" perks_status perks_batch_set_field(perks_batch *b, int32_t dom, const void *src, int src_on_device,
                                              perks_stream stream) {
    if (!b) return PERKS_ERR_INVALID_ARG;
    if (dom < 0 || dom >= b->ndom || !src) return fail(b->ctx, PERKS_ERR_INVALID_ARG, "batch_set_field: bad domain");
    perks_status rc = use_device(b->ctx);
    if (rc) return rc;
    const size_t bytes = (size_t)b->desc[dom].nx * b->desc[dom].ny * b->es;
    PERKS_CUDA(b->ctx, cudaMemcpyAsync(b->field[b->cur[dom]][dom], src, bytes,
                                       src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                       (cudaStream_t)stream));
    return PERKS_OK;
}

extern "C" perks_status perks_batch_get_field(perks_batch *b, int32_t dom, void *dst, int dst_on_device,
                                              perks_stream stream) {
    if (!b) return PERKS_ERR_INVALID_ARG;
    if (dom < 0 || dom >= b->ndom || !dst) return fail(b->ctx, PERKS_ERR_INVALID_ARG, "batch_get_field: bad domain");
    perks_status rc = use_device(b->ctx);
    if (rc) return rc;
    const size_t bytes = (size_t)b->desc[dom].nx * b->desc[dom].ny * b->es;
    PERKS_CUDA(b->ctx, cudaMemcpyAsync(dst, b->field[b->cur[dom]][dom], bytes,
                                       dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                       (cudaStream_t)stream));
    return PERKS_OK;
}

static void fill_batch_stats(const perks_batch *b, long long steps, perks_batch_stats *o) {
    std::memset(o, 0, sizeof(*o));
    o->steps = steps;
    o->grid_blocks = b->blocks;
    o->tiles = b->ntiles;
    o->max_tiles_per_block = b->max_tiles_per_block;
    o->smem_bytes_per_block = b->smem;
    long long cells = 0;
    for (const auto &d : b->desc) cells += d.nx * d.ny;
    o->cells = cells;
    o->cached_cells = b->cached_cells;
    o->halo_cells_per_step = b->halo_cells;
    o->granularity = b->granularity;
    o->width_cap = b->width_cap;
    o->predicted_ms_per_step = b->predicted_ms_per_step;
    o->kernel = b->kernel;
    o->strip_rows = b->strip_rows;
    if (b->kernel == PERKS_BATCH_STRIP) {
        o->grid_blocks = b->strip_blocks;
        o->tiles = b->nitems;
        o->max_tiles_per_block = b->max_items_per_warp;
        o->smem_bytes_per_block = b->strip_smem;
        o->cached_cells = 0;
        o->halo_cells_per_step = b->strip_halo;
        o->predicted_ms_per_step = 0.0;
    }
    const double S = b->es;
    o->algorithmic_bytes = steps > 0 ? S * (2.0 * steps * (double)(cells - o->cached_cells) +
                                            2.0 * o->cached_cells + (double)steps * o->halo_cells_per_step)
                                     : 0.0;
}

extern "C" perks_status perks_batch_run(perks_batch *b, int64_t steps, int32_t variant, perks_stream stream,
                                        perks_batch_stats *opt_out) {
    if (!b) return PERKS_ERR_INVALID_ARG;
    perks_context *ctx = b->ctx;
    if (steps < 0 || (variant != PERKS_PERSISTENT && variant != PERKS_PER_STEP))
        return fail(ctx, PERKS_ERR_INVALID_ARG, "batch_run: bad steps or variant");
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const bool strip = b->kernel == PERKS_BATCH_STRIP;
    if (steps > 0) {
        rc = variant == PERKS_PERSISTENT ? (strip ? launch_strips(b, steps, s) : launch_batch(b, steps, s))
                                         : launch_batch_per_step(b, steps, s);
        if (rc) return rc;
    } else {
        rc = strip ? (b->strip_blocks ? PERKS_OK : plan_strips(b, b->strip_rows)) : ensure_plan(b);
        if (rc) return rc;
    }
    if (opt_out) {
        fill_batch_stats(b, steps, opt_out);
        PERKS_CUDA(ctx, cudaStreamSynchronize(s));
        DevError e{};
        PERKS_CUDA(ctx, cudaMemcpy(&e, b->err, sizeof(e), cudaMemcpyDeviceToHost));
        if (e.code != 0) return fail(ctx, e.code, "batch: grid barrier wait timed out");
    }
    return PERKS_OK;
}

extern "C" perks_status perks_batch_autotune(perks_batch *b, int64_t probe_steps, perks_stream stream,
                                             perks_batch_stats *chosen) {
    if (!b) return PERKS_ERR_INVALID_ARG;
    perks_context *ctx = b->ctx;
    if (probe_steps < 0) return fail(ctx, PERKS_ERR_INVALID_ARG, "batch_autotune: probe_steps < 0");
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    BatchKernel *k = batch_kernel(b);
    b->blocks = 0;
    rc = ensure_plan(b);  // configures the kernel
    if (rc) return rc;
    // 1. model: rank candidate (granularity, width cap) pairs
    struct Cand { double g; int cap; double pred; };
    std::vector<Cand> cands;
    const double gs[] = {0.25, 0.5, 1.0, 2.0};
    const int caps[] = {0, 512, 256};
    for (double g : gs)
        for (int cap : caps) {
            if (cap > 0 && cap >= kBatchThreads * k->v) continue;
            PlanOut o;
            if (plan_batch(b, *k, g, cap, o) == PERKS_OK) cands.push_back({g, cap, o.predicted});
        }
    if (cands.empty()) return fail(ctx, PERKS_ERR_UNSUPPORTED, "batch_autotune: no feasible plan");
    std::sort(cands.begin(), cands.end(), [](const Cand &x, const Cand &y) { return x.pred < y.pred; });
    // 2. time the best model candidates on the GPU (the field is saved and restored)
    Cand best = cands[0];
    int best_strip_rows = -1;  // >= 0: the strip kernel with items of that height won
    if (probe_steps > 0) {
        cudaStream_t s = (cudaStream_t)stream;
        std::vector<void *> saved(b->ndom, nullptr);
        for (int i = 0; i < b->ndom; ++i) {
            const size_t bytes = (size_t)b->desc[i].nx * b->desc[i].ny * b->es;
            PERKS_CUDA(ctx, cudaMalloc(&saved[i], bytes));
            PERKS_CUDA(ctx, cudaMemcpyAsync(saved[i], b->field[b->cur[i]][i], bytes, cudaMemcpyDeviceToDevice, s));
        }
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best_ms = 1e30f;
        const size_t ntry = std::min<size_t>(cands.size(), 4);
        for (size_t c = 0; c < ntry && !rc; ++c) {
            b->granularity = cands[c].g;
            b->width_cap = cands[c].cap;
            b->blocks = 0;
            PlanOut o;
            rc = plan_batch(b, *k, cands[c].g, cands[c].cap, o);
            if (!rc) rc = upload_plan(b, o);
            if (!rc) rc = launch_batch(b, 1, s);  // warm-up
            cudaEventRecord(e0, s);
            if (!rc) rc = launch_batch(b, probe_steps, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (!rc && ms < best_ms) { best_ms = ms; best = cands[c]; }
        }
        // the strip kernel, with items of several heights
        if (!rc && strip_kernel(b->dtype)) {
            for (int rows : {0, 32, 64, 128, 256}) {
                b->strip_blocks = 0;
                rc = plan_strips(b, rows);
                if (rc) break;
                rc = launch_strips(b, 1, s);  // warm-up
                cudaEventRecord(e0, s);
                if (!rc) rc = launch_strips(b, probe_steps, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rc) break;
                if (ms < best_ms) { best_ms = ms; best_strip_rows = rows; }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (int i = 0; i < b->ndom; ++i) {
            const size_t bytes = (size_t)b->desc[i].nx * b->desc[i].ny * b->es;
            cudaMemcpyAsync(b->field[b->cur[i]][i], saved[i], bytes, cudaMemcpyDeviceToDevice, s);
        }
        cudaStreamSynchronize(s);
        for (void *q : saved) cudaFree(q);
        if (rc) return rc;
    }
    b->granularity = best.g;
    b->width_cap = best.cap;
    b->blocks = 0;
    rc = ensure_plan(b);
    if (rc) return rc;
    b->strip_blocks = 0;
    if (best_strip_rows >= 0) {
        b->kernel = PERKS_BATCH_STRIP;
        b->strip_rows = best_strip_rows;
        rc = plan_strips(b, best_strip_rows);
        if (rc) return rc;
    } else if (probe_steps > 0) {
        b->kernel = PERKS_BATCH_RING;
    }
    b->tuned = true;
    if (chosen) fill_batch_stats(b, 0, chosen);
    return PERKS_OK;
}

extern "C" perks_status perks_batch_set_plan(perks_batch *b, double granularity, int32_t width_cap) {
    if (!b) return PERKS_ERR_INVALID_ARG;
    if (!(granularity > 0) || width_cap < 0)
        return fail(b->ctx, PERKS_ERR_INVALID_ARG, "batch_set_plan: granularity > 0, width_cap >= 0");
    b->granularity = granularity;
    b->width_cap = width_cap;
    b->blocks = 0;
    b->kernel = PERKS_BATCH_RING;
    return PERKS_OK;
}

extern "C" perks_status perks_batch_set_kernel(perks_batch *b, int32_t kernel, int32_t strip_rows) {
    if (!b) return PERKS_ERR_INVALID_ARG;
    if ((kernel != PERKS_BATCH_RING && kernel != PERKS_BATCH_STRIP) || strip_rows < 0)
        return fail(b->ctx, PERKS_ERR_INVALID_ARG, "batch_set_kernel: kernel RING or STRIP, strip_rows >= 0");
    if (kernel == PERKS_BATCH_STRIP && !strip_kernel(b->dtype))
        return fail(b->ctx, PERKS_ERR_UNSUPPORTED, "batch_set_kernel: no strip kernel for this dtype");
    b->kernel = kernel;
    b->strip_rows = strip_rows;
    b->strip_blocks = 0;
    return PERKS_OK;
}
