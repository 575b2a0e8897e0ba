// Host side of the stencil solver: shape matching, the persistent-kernel
// planner (tile decomposition and register/shared-memory cache split, sized
// to the device's SMs and shared memory), launches and the C ABI entry
// points perks_stencil_*.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "stencil_registry.h"
#include "stencil_tile.cuh"

using namespace perks;

namespace {

// ------------------------------------------------------------ shape table

struct ShapeInfo {
    int ndim, radius;
    bool box;
    int npts;
    const char *name;
};

template <class SH> ShapeInfo shape_info(const char *name) {
    return ShapeInfo{SH::NDIM, SH::R, SH::BOX, SH::NPTS, name};
}

constexpr int kNumShapes = SH_COUNT;

const ShapeInfo &shape_by_id(int id) {
    static const ShapeInfo table[kNumShapes] = {
        shape_info<S2d5>("2d5pt"),   shape_info<S3d7>("3d7pt"),  shape_info<S2d9>("2d9pt"),
        shape_info<S2d25>("2d25pt"), shape_info<S2ds9>("2ds9pt"), shape_info<S3d27>("3d27pt"),
        shape_info<S3d13>("3d13pt"), shape_info<S3d19>("poisson"), shape_info<S2d13>("2d13pt"),
        shape_info<S2d17>("2d17pt")};
    return table[id];
}

int shape_uoff(int id, int i, int axis) {
    switch (id) {
    case 0: return S2d5::uoff(i, axis);
    case 1: return S3d7::uoff(i, axis);
    case 2: return S2d9::uoff(i, axis);
    case 3: return S2d25::uoff(i, axis);
    case 4: return S2ds9::uoff(i, axis);
    case 5: return S3d27::uoff(i, axis);
    case 6: return S3d13::uoff(i, axis);
    case 7: return S3d19::uoff(i, axis);
    case 8: return S2d13::uoff(i, axis);
    default: return S2d17::uoff(i, axis);
    }
}

// ------------------------------------------------------- kernel registry

constexpr int kPrefetch = 4;

template <typename T, class SH, int NT, int ZR>
KernelEntry entry(int dtype, int shape) {
    KernelEntry e;
    e.dtype = dtype;
    e.shape = shape;
    e.per_step = false;
    e.fn = perks_stencil_kernel<T, SH, NT, ZR, kPrefetch>;
    e.nt = NT;
    e.zr = ZR;
    e.d = kPrefetch;
    e.v = 1;
    return e;
}

std::vector<KernelEntry> build_registry() {
    std::vector<KernelEntry> table;
    {
        // scalar kernels: any x extent (fp64 / fp32)
        table.push_back(entry<double, S2d5, 256, 0>(PERKS_F64, SH_2D5));
        table.push_back(entry<double, S2d5, 256, 16>(PERKS_F64, SH_2D5));
        table.push_back(entry<float, S2d5, 256, 0>(PERKS_F32, SH_2D5));
        table.push_back(entry<float, S2d5, 256, 16>(PERKS_F32, SH_2D5));
        table.push_back(entry<double, S3d7, 1024, 0>(PERKS_F64, SH_3D7));
        table.push_back(entry<float, S3d7, 1024, 0>(PERKS_F32, SH_3D7));
        table.push_back(entry<double, S2d9, 256, 0>(PERKS_F64, SH_2D9));
        table.push_back(entry<float, S2d9, 256, 0>(PERKS_F32, SH_2D9));
        table.push_back(entry<double, S2d25, 256, 0>(PERKS_F64, SH_2D25));
        table.push_back(entry<float, S2d25, 256, 0>(PERKS_F32, SH_2D25));
        table.push_back(entry<double, S2ds9, 256, 0>(PERKS_F64, SH_2DS9));
        table.push_back(entry<float, S2ds9, 256, 0>(PERKS_F32, SH_2DS9));
        table.push_back(entry<double, S3d27, 1024, 0>(PERKS_F64, SH_3D27));
        table.push_back(entry<float, S3d27, 1024, 0>(PERKS_F32, SH_3D27));
        table.push_back(entry<double, S3d13, 1024, 0>(PERKS_F64, SH_3D13));
        table.push_back(entry<float, S3d13, 1024, 0>(PERKS_F32, SH_3D13));
        table.push_back(entry<double, S3d19, 1024, 0>(PERKS_F64, SH_3D19));
        table.push_back(entry<float, S3d19, 1024, 0>(PERKS_F32, SH_3D19));
        // vectorised kernels: x extent a multiple of V (16-byte vectors)
        register_vec_f64_core(table);
        register_vec_f64_box2d(table);
        register_vec_f64_box3d(table);
        register_vec_f32_core(table);
        register_vec_f32_box2d(table);
        register_vec_f32_box3d(table);
        register_vec_bf16_core(table);
        register_vec_bf16_box2d(table);
        register_vec_bf16_box3d(table);
        register_vec_f64_poisson(table);
        register_vec_f32_poisson(table);
        register_vec_bf16_poisson(table);
        register_vec_star2d_hi(table);
    }
    return table;
}

std::vector<KernelEntry> &registry() {
    static std::vector<KernelEntry> table = build_registry();  // built once, thread-safe
    return table;
}

std::vector<TileKernelEntry> &tile_registry() {
    static std::vector<TileKernelEntry> table = [] {
        std::vector<TileKernelEntry> t;
        register_tile_kernels(t);
        return t;
    }();
    return table;
}

// Planes per block barrier preferred by default where both variants exist.
constexpr int kDefaultPlanesPerBarrier = 2;

// Picks a kernel: the vectorised one when the x extent allows 16-byte
// vectors (unless the plan asks for the scalar kernel), the scalar one
// otherwise; with or without the register cache as requested.
KernelEntry *find_kernel(int dtype, int shape, bool want_reg, bool per_step, int X, bool allow_vec,
                         int want_p = 0, int want_nt = 0) {
    KernelEntry *best = nullptr;
    const int pref_p = want_p > 0 ? want_p : kDefaultPlanesPerBarrier;
    for (KernelEntry &e : registry()) {
        if (e.dtype != dtype || e.shape != shape || e.per_step != per_step) continue;
        if (want_nt > 0 && e.nt != want_nt) continue;
        if (e.v > 1 && (!allow_vec || X % e.v != 0)) continue;
        if (want_p > 0 && e.v > 1 && e.p != want_p) continue;
        auto score = [&](const KernelEntry &k) {
            return (k.v > 1 ? 4 : 0) + ((k.zr > 0) == want_reg ? 2 : 0) + (k.p == pref_p ? 1 : 0);
        };
        if (!best || score(e) > score(*best)) best = &e;
    }
    return best;
}

struct Plan {
    KernelEntry *k = nullptr;
    int ntx = 0, nty = 0, ntz = 0;
    int txmax = 0, tymax = 0, tzmax = 0;
    int PW = 0, PH = 0, plane = 0, ncol = 0;
    int zs = 0;
    long long smem = 0;
    int blocks = 0;
    bool balanced = false;     // cache-free body: equal shares of the ntx x nty columns' planes per block
    long long cached_cells = 0;
    long long halo_cells = 0;  // per step
    // resident-tile kernel (the whole tile in shared memory): tiles ntx x nty x ntz of
    // tx x tymax x tzmax cells at most
    bool resident = false;
    TileKernelEntry *tk = nullptr;
    int tx = 0, PP = 0, XGS = 0, groups = 0, chunks = 0, per_plane = 0;
    long long FS = 0;
};

}  // namespace

struct perks_stencil {
    perks_context *ctx = nullptr;
    int device = 0;  // for destroy, which may come after the context is gone
    perks_stencil_desc desc{};
    int es = 8;
    int X = 0, Y = 0, Z = 0;         // internal orientation (persistent kernel)
    int uX = 0, uY = 0, uZ = 0;      // user orientation (per-step kernel)
    long long cells = 0;
    void *field[2] = {nullptr, nullptr};
    int cur = 0;
    void *faces[2] = {nullptr, nullptr};
    size_t faces_bytes = 0;
    unsigned long long *bar = nullptr;
    DevError *err = nullptr;
    int shape_id = -1;
    double kw[kMaxKernelPoints] = {};
    bool has_plan = false;
    perks_stencil_plan plan{};
    unsigned long long *trace = nullptr;  // optional step trace of the persistent kernel
    int trace_steps = 0, trace_blocks = 0, trace_grid = 0;
    void *tfaces[2] = {nullptr, nullptr};  // resident-tile kernel: face buffers by step parity
    size_t tfaces_bytes = 0;
    bool no_resident = false;             // plan the plane-streaming kernel only
};

namespace {

int match_shape(const perks_stencil_desc &d, double *kw) {
    for (int id = 0; id < kNumShapes; ++id) {
        const ShapeInfo &s = shape_by_id(id);
        if (s.ndim != d.ndim || s.npts != d.npts || s.radius != d.radius) continue;
        bool ok = true;
        std::vector<int> used(d.npts, 0);
        for (int i = 0; i < s.npts && ok; ++i) {
            int found = -1;
            for (int j = 0; j < d.npts; ++j) {
                if (!used[j] && d.offsets[3 * j] == shape_uoff(id, i, 0) &&
                    d.offsets[3 * j + 1] == shape_uoff(id, i, 1) &&
                    d.offsets[3 * j + 2] == shape_uoff(id, i, 2)) {
                    found = j;
                    break;
                }
            }
            if (found < 0) ok = false;
            else { used[found] = 1; kw[i] = d.weights[found]; }
        }
        if (ok) return id;
    }
    return -1;
}

int ceil_div(int a, int b) { return (a + b - 1) / b; }

int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Plan of the resident-tile kernel: the tiling (one block per SM at most)
// whose tiles fit in shared memory with their ghost cells and that needs the
// fewest plane slots per thread and step.  Modelled cost of a step, in units
// of one 16-byte vector handled by one thread: slots * threads (dummy slots
// of uneven segments included) + half a slot per block barrier + the ghost
// vectors copied in.  Tiles split x exactly into rows of 1..32 vectors (a
// warp holds whole rows), y and z into nearly equal parts.
perks_status make_tile_plan(perks_stencil *st, Plan &pl) {
    perks_context *ctx = st->ctx;
    if (st->shape_id != SH_2D5 && st->shape_id != SH_3D7)
        return fail(ctx, PERKS_ERR_UNSUPPORTED, "resident-tile kernel: compiled for the 2d5pt and 3d7pt stencils only");
    const bool fixed = st->has_plan && st->plan.reserved[2] == PERKS_KERNEL_RESIDENT;
    const int want_nt = fixed ? st->plan.reserved[3] : 0;
    const int want_r = fixed ? st->plan.reg_cache : 0;  // resident plans: rows per thread (0 = any)
    const int fx = fixed ? st->plan.tiles_x : 0, fy = fixed ? st->plan.tiles_y : 0, fz = fixed ? st->plan.tiles_z : 0;
    const int GY = shape_by_id(st->shape_id).ndim == 3 ? 1 : 0;
    const int X = st->X, Y = st->Y, Z = st->Z, es = st->es;
    const int maxG = ctx->sm_count;
    double best = 1e300;
    Plan bp;
    long long best_smem = 0;
    for (TileKernelEntry &e : tile_registry()) {
        if (e.dtype != st->desc.dtype || e.shape != st->shape_id) continue;
        if ((want_nt > 0 && e.nt != want_nt) || (want_r > 0 && e.r != want_r)) continue;
        const int V = e.v;
        if (X % V != 0) continue;
        int budget = 0;
        const perks_status rc = smem_optin(ctx, (const void *)e.fn, &budget);
        if (rc) return rc;
        const int XV = X / V;
        for (int ntx = 1; ntx <= XV; ++ntx) {
            if ((fx > 0 && ntx != fx) || XV % ntx != 0) continue;
            const int nvx = XV / ntx, tx = nvx * V;
            if (nvx > 32 || 32 % nvx != 0) continue;
            for (int nty = 1; nty <= Y && ntx * nty <= maxG; ++nty) {
                if (fy > 0 && nty != fy) continue;
                const int tymax = ceil_div(Y, nty);
                if (fy == 0 && nty > 1 && tymax == ceil_div(Y, nty - 1)) continue;  // same tiles, more of them
                const int P = nvx * ceil_div(tymax, e.r);
                if (P > e.nt) continue;
                const int G = e.nt / P;
                const int ntz = fz > 0 ? fz : std::min(Z, maxG / (ntx * nty));
                if (ntz < 1 || ntz > Z || (long long)ntx * nty * ntz > maxG) continue;
                const int tzmax = ceil_div(Z, ntz);
                const int XGS = round_up(tzmax * tymax, V);
                const int PP = (tymax + 2 * GY) * tx;
                const long long smem = ((long long)(tzmax + 2) * PP + 2LL * XGS) * es;
                if (smem > budget) continue;
                const int L = ceil_div(tzmax, G), C = ceil_div(L, e.m);
                const double ghosts = 2.0 * tymax * nvx + (GY ? 2.0 * tzmax * nvx : 0.0) + 2.0 * XGS / V;
                const double cost = (double)C * e.m * e.nt + 0.5 * C * e.nt + ghosts;
                if (cost < best) {
                    best = cost;
                    bp.tk = &e;
                    bp.ntx = ntx; bp.nty = nty; bp.ntz = ntz;
                    bp.tx = tx; bp.txmax = tx; bp.tymax = tymax; bp.tzmax = tzmax;
                    bp.PP = PP; bp.XGS = XGS; bp.groups = G; bp.chunks = C; bp.per_plane = P;
                    best_smem = smem;
                }
            }
        }
    }
    if (!bp.tk)
        return fail(ctx, PERKS_ERR_UNSUPPORTED,
                    "resident-tile kernel: no tiling of %dx%dx%d fits shared memory on %d blocks", X, Y, Z, maxG);
    bp.resident = true;
    bp.blocks = bp.ntx * bp.nty * bp.ntz;
    bp.smem = best_smem;
    bp.FS = 2LL * bp.XGS + 2LL * bp.tzmax * bp.tx + 2LL * bp.tymax * bp.tx;
    int per_sm = 0;
    PERKS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)bp.tk->fn, bp.tk->nt,
                                                                  (size_t)bp.smem));
    if ((long long)per_sm * ctx->sm_count < bp.blocks)
        return fail(ctx, PERKS_ERR_LAUNCH_TOO_LARGE, "resident-tile kernel: %d blocks are not co-resident", bp.blocks);
    // halo cells written + read per step
    long long halo = 0;
    for (int t = 0; t < bp.blocks; ++t) {
        const int ti = t % bp.ntx, tj = (t / bp.ntx) % bp.nty, tk = t / (bp.ntx * bp.nty);
        int y0, ty, z0, tz;
        split_axis(Y, bp.nty, tj, y0, ty);
        split_axis(Z, bp.ntz, tk, z0, tz);
        const int nfx = (ti > 0) + (ti + 1 < bp.ntx), nfy = (tj > 0) + (tj + 1 < bp.nty);
        const int nfz = (tk > 0) + (tk + 1 < bp.ntz);
        halo += 2LL * ((long long)nfx * ty * tz + (GY ? (long long)nfy * bp.tx * tz : 0) + (long long)nfz * bp.tx * ty);
    }
    bp.cached_cells = st->cells;
    bp.halo_cells = halo;
    bp.plane = 0;
    bp.zs = bp.tzmax;
    pl = bp;
    return PERKS_OK;
}

perks_status make_plan(perks_stencil *st, Plan &pl, bool per_step = false) {
    perks_context *ctx = st->ctx;
    // The resident-tile kernel when it is asked for, or by default (no plan)
    // when every tile of the domain fits in shared memory.
    const int kind = st->has_plan ? st->plan.reserved[2] : PERKS_KERNEL_AUTO;
    if (!per_step && !st->no_resident && st->shape_id >= 0 &&
        (kind == PERKS_KERNEL_RESIDENT || (!st->has_plan && kind == PERKS_KERNEL_AUTO))) {
        const std::string saved_msg = ctx->last_error;
        const perks_status rc = make_tile_plan(st, pl);
        if (rc == PERKS_OK || kind == PERKS_KERNEL_RESIDENT) return rc;
        ctx->last_error = saved_msg;
    }
    if (st->shape_id < 0)
        return fail(ctx, PERKS_ERR_UNSUPPORTED,
                    "persistent kernel: offsets do not match a compiled shape "
                    "(2d5pt, 2ds9pt, 2d9pt, 2d25pt, 2d13pt, 2d17pt, 3d7pt, 3d13pt, 3d27pt, poisson)");
    const ShapeInfo &sh = shape_by_id(st->shape_id);
    bool want_reg = true, allow_vec = true;
    int want_p = 0, want_nt = 0;
    if (st->has_plan) {
        want_reg = st->plan.reg_cache != 0;
        allow_vec = st->plan.reserved[0] == 0;  // reserved[0] = 1 forces the scalar kernel
        want_p = st->plan.reserved[1];          // planes per barrier (0 = automatic)
        want_nt = per_step ? 0 : st->plan.reserved[3];  // threads per block (0 = automatic)
    }
    // A persistent plan that caches nothing runs the cache-free kernel body
    // (the per-step one) for all steps in one cooperative launch, with the
    // grid barrier between steps: the launch overhead goes, nothing is added
    // per plane.
    const bool body_per_step = per_step || (st->has_plan && st->plan.reg_cache == 0 &&
                                            st->plan.smem_cache_planes == 0 && allow_vec);
    KernelEntry *kp = find_kernel(st->desc.dtype, st->shape_id, want_reg, body_per_step, st->X, allow_vec, want_p,
                                  want_nt);
    if (!kp && want_p > 0)
        kp = find_kernel(st->desc.dtype, st->shape_id, want_reg, body_per_step, st->X, allow_vec, 0, want_nt);
    if (!kp && body_per_step && !per_step)  // no vectorised cache-free body for this extent
        kp = find_kernel(st->desc.dtype, st->shape_id, want_reg, false, st->X, allow_vec, want_p, want_nt);
    if (!kp && !per_step)  // shapes compiled with the cache-free body only (radius 3, 4)
        kp = find_kernel(st->desc.dtype, st->shape_id, want_reg, true, st->X, allow_vec, 0, want_nt);
    if (!kp && want_nt > 0)
        return fail(ctx, PERKS_ERR_UNSUPPORTED, "no plane-streaming kernel with %d threads for this dtype/shape",
                    want_nt);
    per_step = per_step || (kp && kp->per_step);
    if (!kp)
        return fail(ctx, PERKS_ERR_UNSUPPORTED,
                    "no %s kernel for this dtype/shape/extent (bf16 needs nx divisible by 8)",
                    per_step ? "per-step" : "persistent");
    KernelEntry &k = *kp;
    const bool balanced = st->has_plan && st->plan.balanced != 0;
    if (balanced && !(k.per_step && k.v > 1))
        return fail(ctx, PERKS_ERR_UNSUPPORTED,
                    "balanced shares need the cache-free vector body (reg_cache = 0, smem_cache_planes = 0)");
    int smem_budget = 0;
    {
        perks_status rc = smem_optin(ctx, (const void *)k.fn, &smem_budget);
        if (rc) return rc;
    }
    // the 256-thread cache-free bodies run two blocks per SM: each block's ring
    // takes at most half of the SM's shared memory
    if (k.per_step && k.v > 1 && k.nt <= 256 && k.shape == SH_3D7)
        smem_budget = std::min(smem_budget, ctx->smem_per_sm / 2 - 4096);
    const int R = sh.radius;
    const int RX = R, RY = sh.ndim == 3 ? R : 0, RZ = R;
    const int S = k.v > 1 ? 2 * RZ + k.p + k.d : 2 * RZ + 1 + k.d;  // ring slots (vector kernel: P planes per barrier)
    const int es = st->es;
    const int V = k.v;
    int HX = RX;  // ring pad columns on each side (vector kernel: a multiple of V, >= 2 and >= the radius)
    if (V > 1)
        for (HX = std::max(V, 2); HX < RX; HX += V) {}
    int per_sm = 0;
    PERKS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k.fn, k.nt,
                                                                  smem_budget));
    if (per_sm < 1)
        return fail(ctx, PERKS_ERR_LAUNCH_TOO_LARGE, "persistent kernel cannot be resident");
    const int maxG = per_sm * ctx->sm_count;

    const int X = st->X, Y = st->Y, Z = st->Z;
    const int XU = X / V;  // x extent in units of V cells
    double best = 1e300;
    Plan bp;
    const int fx_lo = st->has_plan && st->plan.tiles_x > 0 ? st->plan.tiles_x : 1;
    const int fx_hi = st->has_plan && st->plan.tiles_x > 0 ? st->plan.tiles_x : std::min(XU, 512);
    const int fy_lo = st->has_plan && st->plan.tiles_y > 0 ? st->plan.tiles_y : 1;
    const int fy_hi = st->has_plan && st->plan.tiles_y > 0 ? st->plan.tiles_y : std::min(Y, 512);
    for (int ntx = fx_lo; ntx <= fx_hi; ++ntx) {
        const int txmax = ceil_div(XU, ntx) * V, txmin = (XU / ntx) * V;
        if (txmin < std::max(RX, 1) || (V > 1 && txmin < 2)) break;
        if (txmax / V > k.nt) continue;
        for (int nty = fy_lo; nty <= fy_hi; ++nty) {
            const int tymax = ceil_div(Y, nty), tymin = Y / nty;
            if (tymin < std::max(RY, 1)) break;
            if ((long long)(txmax / V) * tymax > k.nt) continue;
            const int nring = V > 1 ? 2 * RY * (txmax / V) + (sh.box ? 4 * RY : 0) + 2 * tymax
                                    : 2 * RY * (txmax + (sh.box ? 2 * RX : 0)) + 2 * RX * tymax;
            if (nring > k.nt) continue;
            const int PW = txmax + 2 * HX, PH = tymax + 2 * RY;
            const long long ring_bytes = (long long)S * PW * PH * es;
            if (ring_bytes > smem_budget) continue;
            int ntz;
            if (balanced) ntz = 1;
            else if (st->has_plan && st->plan.tiles_z > 0) ntz = st->plan.tiles_z;
            else ntz = std::min(Z / std::max(RZ, 1), maxG / (ntx * nty));
            if (ntz < 1 || (long long)ntx * nty * ntz > maxG) continue;
            if (Z / ntz < std::max(RZ, 1)) continue;
            // planes per block: a tile's depth, or a balanced share (which may
            // be cut once more where it crosses into the next column)
            const int tzmax = balanced ? (int)(((long long)ntx * nty * Z + maxG - 1) / maxG) : ceil_div(Z, ntz);
            if (balanced && tzmax < 4 * std::max(RZ, 1)) continue;  // shares too thin for their z-halos
            const double vol = (double)txmax * tymax * tzmax;
            const double cost = vol * (1.0 + 2.0 * RX / txmax + (RY ? 2.0 * RY / tymax : 0.0) +
                                       (balanced ? 4.0 : 2.0) * RZ / tzmax) +
                                (txmax < 32 ? vol * 0.25 : 0.0);
            if (cost < best) {
                best = cost;
                bp.ntx = ntx; bp.nty = nty; bp.ntz = ntz;
                bp.txmax = txmax; bp.tymax = tymax; bp.tzmax = tzmax;
                bp.PW = PW; bp.PH = PH;
            }
        }
    }
    if (bp.ntx == 0)
        return fail(ctx, PERKS_ERR_UNSUPPORTED,
                    "persistent kernel: no tile decomposition of %dx%dx%d fits %d blocks of %d threads "
                    "(%d per SM with %d bytes of shared memory each)",
                    X, Y, Z, maxG, k.nt, per_sm, smem_budget);
    bp.k = &k;
    bp.plane = bp.PW * bp.PH;
    bp.ncol = bp.txmax * bp.tymax;
    bp.balanced = balanced;
    bp.blocks = balanced ? maxG : bp.ntx * bp.nty * bp.ntz;
    const long long ring_bytes = (long long)S * bp.plane * es;
    long long zs = (smem_budget - ring_bytes) / ((long long)bp.ncol * es);
    zs = std::min<long long>(zs, std::max(0, bp.tzmax - k.zr));
    if (st->has_plan && st->plan.smem_cache_planes >= 0) zs = std::min<long long>(zs, st->plan.smem_cache_planes);
    if (per_step) zs = 0;
    bp.zs = (int)std::max<long long>(0, zs);
    bp.smem = ring_bytes + (long long)bp.zs * bp.ncol * es;

    // cached cells and halo cells per step, tile by tile
    long long cached = 0, halo = 0;
    for (int t = 0; t < bp.ntx * bp.nty * bp.ntz; ++t) {
        const int ti = t % bp.ntx, tj = (t / bp.ntx) % bp.nty, tk = t / (bp.ntx * bp.nty);
        int x0, tx, y0, ty, z0, tz;
        split_axis(XU, bp.ntx, ti, x0, tx);
        tx *= V;
        split_axis(Y, bp.nty, tj, y0, ty);
        split_axis(Z, bp.ntz, tk, z0, tz);
        const int zc = per_step ? 0 : std::min(tz, k.zr + bp.zs);
        cached += (long long)zc * tx * ty;
        const int nfx = (ti > 0) + (ti + 1 < bp.ntx);
        const int nfy = (tj > 0) + (tj + 1 < bp.nty);
        const int nfz = (tk > 0) + (tk + 1 < bp.ntz);
        // written: x-faces (transposed), y-shell and z-shell of cached planes; read: the same halos
        const long long wx = (long long)nfx * RX * ty * tz;
        const long long wy = (long long)nfy * RY * tx * zc;
        const long long wz = (long long)nfz * RZ * tx * ty;
        halo += 2 * (wx + wy + wz);
    }
    if (balanced) {
        // z-halos at the share boundaries that fall inside a column
        const long long L = (long long)bp.ntx * bp.nty * Z;
        for (int b = 1; b < bp.blocks; ++b) {
            const long long cut = L * b / bp.blocks;
            if (cut % Z != 0) halo += 2LL * 2 * RZ * bp.txmax * bp.tymax;
        }
    }
    bp.cached_cells = cached;
    bp.halo_cells = halo;
    if (!st->has_plan && !per_step && cached < st->cells) {
        // Default plan when the caches cannot hold the whole domain: the
        // cache-free body for all steps in one launch.  Measured on GB300,
        // caching a part of a domain (3-D 384^3 in fp64/fp32/bf16, 2-D 4096^2)
        // costs more in bookkeeping than the re-reads it saves.
        const perks_stencil_plan saved_plan = st->plan;
        const std::string saved_msg = ctx->last_error;
        st->has_plan = true;
        st->plan = perks_stencil_plan{};
        st->plan.reg_cache = 0;
        st->plan.smem_cache_planes = 0;
        Plan cf;
        const perks_status r2 = make_plan(st, cf, false);
        st->has_plan = false;
        st->plan = saved_plan;
        if (r2 == PERKS_OK) {
            pl = cf;
            return PERKS_OK;
        }
        ctx->last_error = saved_msg;  // no cache-free plan: keep the cached one
    }
    pl = bp;
    return PERKS_OK;
}

void fill_stats(const perks_stencil *st, const Plan *pl, long long steps, int variant,
                perks_run_stats *o) {
    std::memset(o, 0, sizeof(*o));
    o->steps = steps;
    o->variant = variant;
    o->cells = st->cells;
    const double S = st->es;
    if (variant == PERKS_PERSISTENT && pl && pl->resident) {
        o->kernel = PERKS_KERNEL_RESIDENT;
        o->grid_blocks = pl->blocks;
        o->threads_per_block = pl->tk->nt;
        o->tiles_x = pl->ntx; o->tiles_y = pl->nty; o->tiles_z = pl->ntz;
        o->reg_cache_planes = pl->tk->r;  // rows per thread (their plane window lives in registers)
        o->smem_cache_planes = pl->tzmax;
        o->prefetch_planes = 0;
        o->planes_per_sync = pl->tk->m;
        o->smem_bytes_per_block = pl->smem;
        o->cached_cells = st->cells;
        o->halo_cells_per_step = pl->halo_cells;
        o->algorithmic_bytes = steps > 0 ? S * (2.0 * (double)st->cells + (double)steps * pl->halo_cells) : 0.0;
    } else if (variant == PERKS_PERSISTENT && pl) {
        o->kernel = PERKS_KERNEL_STREAMING;
        o->planes_per_sync = pl->k->p;
        o->grid_blocks = pl->blocks;
        o->threads_per_block = pl->k->nt;
        o->tiles_x = pl->ntx; o->tiles_y = pl->nty; o->tiles_z = pl->ntz;
        o->reg_cache_planes = pl->k->zr;
        o->smem_cache_planes = pl->zs;
        o->prefetch_planes = pl->k->d;
        o->smem_bytes_per_block = pl->smem;
        o->cached_cells = pl->cached_cells;
        o->halo_cells_per_step = pl->halo_cells;
        const double dun = (double)(st->cells - pl->cached_cells);
        o->algorithmic_bytes = steps > 0 ? S * (2.0 * steps * dun + 2.0 * pl->cached_cells +
                                                (double)steps * pl->halo_cells) : 0.0;
    } else {
        o->kernel = PERKS_KERNEL_PER_STEP;
        o->threads_per_block = 256;
        o->algorithmic_bytes = S * 2.0 * (double)steps * (double)st->cells;
    }
}

perks_status ensure_tile_buffers(perks_stencil *st, const Plan &pl) {
    perks_context *ctx = st->ctx;
    const size_t need = (size_t)pl.blocks * (size_t)pl.FS * st->es;
    if (need > st->tfaces_bytes) {
        for (int i = 0; i < 2; ++i) {
            if (st->tfaces[i]) cudaFree(st->tfaces[i]);
            st->tfaces[i] = nullptr;
        }
        st->tfaces_bytes = 0;
        for (int i = 0; i < 2; ++i) PERKS_CUDA(ctx, cudaMalloc(&st->tfaces[i], need));
        st->tfaces_bytes = need;
    }
    if (!st->bar) PERKS_CUDA(ctx, cudaMalloc(&st->bar, sizeof(unsigned long long)));
    if (!st->err) PERKS_CUDA(ctx, cudaMalloc(&st->err, sizeof(DevError)));
    return PERKS_OK;
}

// One cooperative launch of the resident-tile kernel: reads field[cur] before
// the first step, writes field[cur ^ (steps & 1)] after the last (the same
// buffer when steps is even: every block has read its tile before any block
// passes the first grid barrier).
perks_status run_resident(perks_stencil *st, long long steps, cudaStream_t s, const Plan &pl) {
    perks_context *ctx = st->ctx;
    perks_status rc = ensure_tile_buffers(st, pl);
    if (rc) return rc;
    TileArgs a;
    std::memset(&a, 0, sizeof(a));
    a.X = st->X; a.Y = st->Y; a.Z = st->Z;
    a.XY = (long long)st->X * st->Y;
    a.ntx = pl.ntx; a.nty = pl.nty; a.ntz = pl.ntz;
    a.tx = pl.tx; a.tymax = pl.tymax; a.tzmax = pl.tzmax;
    a.PP = pl.PP; a.XGS = pl.XGS; a.FS = pl.FS;
    a.groups = pl.groups; a.chunks = pl.chunks; a.per_plane = pl.per_plane;
    a.lognv = 0;
    while ((pl.tx / pl.tk->v) >> a.lognv > 1) ++a.lognv;
    a.steps = steps;
    a.boundary = st->desc.boundary;
    a.boundary_f = (float)st->desc.boundary;
    for (int i = 0; i < kMaxKernelPoints; ++i) { a.w[i] = st->kw[i]; a.wf[i] = (float)st->kw[i]; }
    a.in = st->field[st->cur];
    a.out = st->field[st->cur ^ (int)(steps & 1)];
    a.faces[0] = st->tfaces[0];
    a.faces[1] = st->tfaces[1];
    a.bar = st->bar;
    a.err = st->err;
    a.timeout_ns = ctx->timeout_ns;
    if (st->trace && pl.blocks <= st->trace_blocks) {
        a.trace = st->trace;
        a.trace_steps = st->trace_steps;
        st->trace_grid = pl.blocks;
        PERKS_CUDA(ctx, cudaMemsetAsync(st->trace, 0, sizeof(unsigned long long) * 2 * (size_t)(st->trace_steps + 1) *
                                                          st->trace_blocks, s));
    }
    PERKS_CUDA(ctx, cudaMemsetAsync(st->bar, 0, sizeof(unsigned long long), s));
    PERKS_CUDA(ctx, cudaMemsetAsync(st->err, 0, sizeof(DevError), s));
    void *args[] = {&a};
    PERKS_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)pl.tk->fn, dim3(pl.blocks), dim3(pl.tk->nt), args,
                                                (size_t)pl.smem, s));
    if (steps & 1) st->cur ^= 1;
    return PERKS_OK;
}

perks_status ensure_persistent_buffers(perks_stencil *st, const Plan &pl) {
    perks_context *ctx = st->ctx;
    const int RX = shape_by_id(st->shape_id).radius;
    const int width = pl.k->v > 1 ? 2 : RX;  // vector kernels store x-edges as pairs of cells
    const size_t need = (size_t)pl.blocks * 2 * width * pl.tzmax * pl.tymax * st->es;
    if (need > st->faces_bytes) {
        for (int i = 0; i < 2; ++i) {
            if (st->faces[i]) cudaFree(st->faces[i]);
            st->faces[i] = nullptr;
        }
        st->faces_bytes = 0;
        for (int i = 0; i < 2; ++i) PERKS_CUDA(ctx, cudaMalloc(&st->faces[i], need));
        st->faces_bytes = need;
    }
    if (!st->bar) PERKS_CUDA(ctx, cudaMalloc(&st->bar, sizeof(unsigned long long)));
    if (!st->err) PERKS_CUDA(ctx, cudaMalloc(&st->err, sizeof(DevError)));
    return PERKS_OK;
}

perks_status read_dev_error(perks_stencil *st, cudaStream_t s) {
    perks_context *ctx = st->ctx;
    PERKS_CUDA(ctx, cudaStreamSynchronize(s));
    if (!st->err) return PERKS_OK;
    DevError e{};
    PERKS_CUDA(ctx, cudaMemcpy(&e, st->err, sizeof(e), cudaMemcpyDeviceToHost));
    if (e.code != 0) {
        PERKS_CUDA(ctx, cudaMemset(st->err, 0, sizeof(DevError)));
        return fail(ctx, e.code, "persistent stencil: grid barrier wait timed out (block %d, barrier %d)",
                    e.block, e.epoch);
    }
    return PERKS_OK;
}

void fill_args(const perks_stencil *st, const Plan &pl, long long steps, PersistentArgs &a) {
    std::memset(&a, 0, sizeof(a));
    a.X = st->X; a.Y = st->Y; a.Z = st->Z;
    a.XY = (long long)st->X * st->Y;
    a.ntx = pl.ntx; a.nty = pl.nty; a.ntz = pl.ntz;
    a.txmax = pl.txmax; a.tymax = pl.tymax; a.tzmax = pl.tzmax;
    a.PW = pl.PW; a.plane = pl.plane; a.ncol = pl.ncol;
    a.zs = pl.zs;
    a.steps = steps;
    a.boundary = st->desc.boundary;
    a.boundary_f = (float)st->desc.boundary;
    for (int i = 0; i < kMaxKernelPoints; ++i) { a.w[i] = st->kw[i]; a.wf[i] = (float)st->kw[i]; }
    a.face_plane = (long long)pl.tzmax * pl.tymax;
    a.faces_cached_only = 1;
    a.lin_cols = pl.balanced ? pl.ntx * pl.nty : 0;
    a.iso = 0;
    if (st->shape_id == SH_3D7 && st->desc.dtype == PERKS_F64) {
        bool eq = true;
        for (int i = 2; i < 7; ++i) eq = eq && st->kw[i] == st->kw[1];
        a.iso = eq ? 1 : 0;
        a.wc = st->kw[0];
        a.wn = st->kw[1];
    }
}

perks_status run_persistent(perks_stencil *st, long long steps, cudaStream_t s, Plan &pl) {
    perks_context *ctx = st->ctx;
    perks_status rc = make_plan(st, pl);
    if (rc) return rc;
    if (pl.resident) return run_resident(st, steps, s, pl);
    rc = ensure_persistent_buffers(st, pl);
    if (rc) return rc;
    int per_sm = 0;
    PERKS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)pl.k->fn,
                                                                  pl.k->nt, pl.smem));
    if ((long long)per_sm * ctx->sm_count < pl.blocks)
        return fail(ctx, PERKS_ERR_LAUNCH_TOO_LARGE, "persistent grid of %d blocks is not co-resident",
                    pl.blocks);
    PersistentArgs a;
    fill_args(st, pl, steps, a);
    a.field[0] = st->field[st->cur];
    a.field[1] = st->field[st->cur ^ 1];
    a.faces[0] = st->faces[0];
    a.faces[1] = st->faces[1];
    a.bar = st->bar;
    a.err = st->err;
    a.timeout_ns = ctx->timeout_ns;
    if (st->trace && pl.blocks <= st->trace_blocks) {
        a.trace = st->trace;
        a.trace_steps = st->trace_steps;
        st->trace_grid = pl.blocks;
        PERKS_CUDA(ctx, cudaMemsetAsync(st->trace, 0, sizeof(unsigned long long) * 2 * (size_t)(st->trace_steps + 1) *
                                                          st->trace_blocks, s));
    }
    PERKS_CUDA(ctx, cudaMemsetAsync(st->bar, 0, sizeof(unsigned long long), s));
    PERKS_CUDA(ctx, cudaMemsetAsync(st->err, 0, sizeof(DevError), s));
    void *args[] = {&a};
    PERKS_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)pl.k->fn, dim3(pl.blocks),
                                                dim3(pl.k->nt), args, (size_t)pl.smem, s));
    if (steps & 1) st->cur ^= 1;
    return PERKS_OK;
}

// One launch per step of the vectorised kernel body with no caches and no
// grid barrier (the per-step baseline); false if no such kernel applies.
perks_status run_per_step_vec(perks_stencil *st, long long steps, cudaStream_t s, bool &used) {
    used = false;
    if (st->shape_id < 0) return PERKS_OK;
    if (!find_kernel(st->desc.dtype, st->shape_id, false, true, st->X, true)) return PERKS_OK;
    perks_context *ctx = st->ctx;
    Plan pl;
    perks_status rc = make_plan(st, pl, true);
    if (rc) return rc;
    PersistentArgs a;
    fill_args(st, pl, 1, a);
    a.timeout_ns = ctx->timeout_ns;
    for (long long k = 0; k < steps; ++k) {
        a.field[0] = st->field[st->cur];
        a.field[1] = st->field[st->cur ^ 1];
        pl.k->fn<<<pl.blocks, pl.k->nt, (size_t)pl.smem, s>>>(a);
        PERKS_CUDA(ctx, cudaGetLastError());
        st->cur ^= 1;
    }
    used = true;
    return PERKS_OK;
}

template <typename T>
perks_status launch_steps(perks_stencil *st, long long steps, cudaStream_t s) {
    perks_context *ctx = st->ctx;
    StepArgs a;
    std::memset(&a, 0, sizeof(a));
    a.X = st->uX; a.Y = st->uY; a.Z = st->uZ;
    a.XY = (long long)a.X * a.Y;
    a.npts = st->desc.npts;
    a.zchunk = a.Z >= 8 ? 8 : 1;
    a.boundary = st->desc.boundary;
    a.boundary_f = (float)st->desc.boundary;
    for (int i = 0; i < st->desc.npts; ++i) {
        for (int d = 0; d < 3; ++d) a.off[3 * i + d] = (short)st->desc.offsets[3 * i + d];
        a.w[i] = st->desc.weights[i];
        a.wf[i] = (float)st->desc.weights[i];
    }
    dim3 block(32, 8);
    dim3 grid((a.X + 31) / 32, (a.Y + 7) / 8, (a.Z + a.zchunk - 1) / a.zchunk);
    for (long long k = 0; k < steps; ++k) {
        const T *in = static_cast<const T *>(st->field[st->cur]);
        T *out = static_cast<T *>(st->field[st->cur ^ 1]);
        stencil_step_kernel<T><<<grid, block, 0, s>>>(in, out, a);
        PERKS_CUDA(ctx, cudaGetLastError());
        st->cur ^= 1;
    }
    return PERKS_OK;
}

}  // namespace

// ======================================================================= ABI

extern "C" perks_status perks_stencil_create(perks_context *ctx, const perks_stencil_desc *d,
                                             perks_stencil **out) {
    if (!ctx) return PERKS_ERR_INVALID_ARG;
    if (!d || !out) return fail(ctx, PERKS_ERR_INVALID_ARG, "stencil_create: NULL argument");
    *out = nullptr;
    if (d->ndim != 2 && d->ndim != 3)
        return fail(ctx, PERKS_ERR_INVALID_ARG, "stencil_create: ndim must be 2 or 3");
    if (d->nx < 1 || d->ny < 1 || d->nz < 1 || (d->ndim == 2 && d->nz != 1))
        return fail(ctx, PERKS_ERR_INVALID_ARG, "stencil_create: bad extents");
    if (d->nx > INT32_MAX / 2 || d->ny > INT32_MAX / 2 || d->nz > INT32_MAX / 2)
        return fail(ctx, PERKS_ERR_INVALID_ARG, "stencil_create: extent too large");
    if (d->radius < 1 || d->radius > 4)
        return fail(ctx, PERKS_ERR_INVALID_ARG, "stencil_create: radius must be 1..4");
    if (d->npts < 1 || d->npts > PERKS_MAX_POINTS)
        return fail(ctx, PERKS_ERR_INVALID_ARG, "stencil_create: npts out of range");
    for (int i = 0; i < d->npts; ++i)
        for (int a = 0; a < 3; ++a) {
            const int v = d->offsets[3 * i + a];
            if (v < -d->radius || v > d->radius || (a == 2 && d->ndim == 2 && v != 0))
                return fail(ctx, PERKS_ERR_INVALID_ARG, "stencil_create: offset %d outside the radius", i);
        }
    if (d->dtype != PERKS_F64 && d->dtype != PERKS_F32 && d->dtype != PERKS_BF16)
        return fail(ctx, PERKS_ERR_UNSUPPORTED, "stencil_create: unknown dtype %d", d->dtype);
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    perks_stencil *st = new perks_stencil();
    st->ctx = ctx;
    st->device = ctx->device;
    st->desc = *d;
    st->es = (int)dtype_size(d->dtype);
    st->uX = (int)d->nx; st->uY = (int)d->ny; st->uZ = (int)d->nz;
    if (d->ndim == 3) { st->X = (int)d->nx; st->Y = (int)d->ny; st->Z = (int)d->nz; }
    else { st->X = (int)d->nx; st->Y = 1; st->Z = (int)d->ny; }
    st->cells = (long long)d->nx * d->ny * d->nz;
    st->shape_id = match_shape(*d, st->kw);
    const size_t bytes = (size_t)st->cells * st->es;
    for (int i = 0; i < 2; ++i) {
        cudaError_t e = cudaMalloc(&st->field[i], bytes);
        if (e != cudaSuccess) {
            perks_stencil_destroy(st);
            return cuda_fail(ctx, e, "stencil_create: cudaMalloc");
        }
    }
    *out = st;
    return PERKS_OK;
}

extern "C" perks_status perks_stencil_destroy(perks_stencil *st) {
    if (!st) return PERKS_OK;
    cudaSetDevice(st->device);
    for (int i = 0; i < 2; ++i) {
        if (st->field[i]) cudaFree(st->field[i]);
        if (st->faces[i]) cudaFree(st->faces[i]);
    }
    for (int i = 0; i < 2; ++i)
        if (st->tfaces[i]) cudaFree(st->tfaces[i]);
    if (st->bar) cudaFree(st->bar);
    if (st->err) cudaFree(st->err);
    if (st->trace) cudaFree(st->trace);
    delete st;
    return PERKS_OK;
}

extern "C" perks_status perks_stencil_set_trace(perks_stencil *st, int32_t steps) {
    if (!st) return PERKS_ERR_INVALID_ARG;
    if (steps < 0) return fail(st->ctx, PERKS_ERR_INVALID_ARG, "stencil_set_trace: steps < 0");
    perks_status rc = use_device(st->ctx);
    if (rc) return rc;
    if (st->trace) cudaFree(st->trace);
    st->trace = nullptr;
    st->trace_steps = st->trace_blocks = st->trace_grid = 0;
    if (steps == 0) return PERKS_OK;
    const int blocks = 4 * st->ctx->sm_count;  // upper bound of any persistent grid
    PERKS_CUDA(st->ctx, cudaMalloc(&st->trace, sizeof(unsigned long long) * 2 * (size_t)(steps + 1) * blocks));
    st->trace_steps = steps;
    st->trace_blocks = blocks;
    return PERKS_OK;
}

extern "C" perks_status perks_stencil_get_trace(perks_stencil *st, uint64_t *host, int64_t capacity,
                                                int32_t *grid_blocks, int32_t *steps) {
    if (!st || !host || !grid_blocks || !steps) return PERKS_ERR_INVALID_ARG;
    if (!st->trace || st->trace_grid == 0)
        return fail(st->ctx, PERKS_ERR_INVALID_ARG, "stencil_get_trace: no traced persistent run");
    const long long need = 2LL * (st->trace_steps + 1) * st->trace_grid;
    if (capacity < need) return fail(st->ctx, PERKS_ERR_INVALID_ARG, "stencil_get_trace: need %lld entries", need);
    PERKS_CUDA(st->ctx, cudaMemcpy(host, st->trace, sizeof(uint64_t) * need, cudaMemcpyDeviceToHost));
    *grid_blocks = st->trace_grid;
    *steps = st->trace_steps;
    return PERKS_OK;
}

extern "C" perks_status perks_stencil_set_plan(perks_stencil *st, const perks_stencil_plan *plan) {
    if (!st) return PERKS_ERR_INVALID_ARG;
    if (!plan) { st->has_plan = false; return PERKS_OK; }
    if (plan->tiles_x < 0 || plan->tiles_y < 0 || plan->tiles_z < 0 || plan->smem_cache_planes < -1)
        return fail(st->ctx, PERKS_ERR_INVALID_ARG, "stencil_set_plan: negative field");
    if (plan->reserved[1] != 0 && plan->reserved[1] != 2 && plan->reserved[1] != 4)
        return fail(st->ctx, PERKS_ERR_INVALID_ARG, "stencil_set_plan: planes per barrier must be 0, 2 or 4");
    if (plan->reserved[2] < PERKS_KERNEL_AUTO || plan->reserved[2] > PERKS_KERNEL_STREAMING)
        return fail(st->ctx, PERKS_ERR_INVALID_ARG, "stencil_set_plan: kernel must be AUTO, RESIDENT or STREAMING");
    if (plan->reserved[3] != 0 && plan->reserved[3] != 256 && plan->reserved[3] != 512 && plan->reserved[3] != 1024)
        return fail(st->ctx, PERKS_ERR_INVALID_ARG, "stencil_set_plan: threads must be 0, 256, 512 or 1024");
    st->plan = *plan;
    st->has_plan = true;
    return PERKS_OK;
}

extern "C" perks_status perks_stencil_set_field(perks_stencil *st, const void *src, int src_on_device,
                                                perks_stream stream) {
    if (!st) return PERKS_ERR_INVALID_ARG;
    if (!src) return fail(st->ctx, PERKS_ERR_INVALID_ARG, "stencil_set_field: NULL src");
    perks_status rc = use_device(st->ctx);
    if (rc) return rc;
    const size_t bytes = (size_t)st->cells * st->es;
    PERKS_CUDA(st->ctx, cudaMemcpyAsync(st->field[st->cur], src, bytes,
                                        src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                        (cudaStream_t)stream));
    return PERKS_OK;
}

extern "C" perks_status perks_stencil_get_field(perks_stencil *st, void *dst, int dst_on_device,
                                                perks_stream stream) {
    if (!st) return PERKS_ERR_INVALID_ARG;
    if (!dst) return fail(st->ctx, PERKS_ERR_INVALID_ARG, "stencil_get_field: NULL dst");
    perks_status rc = use_device(st->ctx);
    if (rc) return rc;
    const size_t bytes = (size_t)st->cells * st->es;
    PERKS_CUDA(st->ctx, cudaMemcpyAsync(dst, st->field[st->cur], bytes,
                                        dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                        (cudaStream_t)stream));
    return PERKS_OK;
}

extern "C" perks_status perks_stencil_describe(perks_stencil *st, int64_t steps, int32_t variant,
                                               perks_run_stats *out) {
    if (!st) return PERKS_ERR_INVALID_ARG;
    if (!out || steps < 0) return fail(st->ctx, PERKS_ERR_INVALID_ARG, "stencil_describe: bad argument");
    if (variant == PERKS_PERSISTENT) {
        perks_status rc = use_device(st->ctx);
        if (rc) return rc;
        Plan pl;
        rc = make_plan(st, pl);
        if (rc) return rc;
        fill_stats(st, &pl, steps, variant, out);
    } else if (variant == PERKS_PER_STEP) {
        fill_stats(st, nullptr, steps, variant, out);
    } else {
        return fail(st->ctx, PERKS_ERR_INVALID_ARG, "stencil_describe: unknown variant");
    }
    return PERKS_OK;
}

extern "C" perks_status perks_stencil_run(perks_stencil *st, int64_t steps, int32_t variant,
                                          perks_stream stream, perks_run_stats *opt_out) {
    if (!st) return PERKS_ERR_INVALID_ARG;
    perks_context *ctx = st->ctx;
    if (steps < 0) return fail(ctx, PERKS_ERR_INVALID_ARG, "stencil_run: negative steps");
    if (variant != PERKS_PERSISTENT && variant != PERKS_PER_STEP)
        return fail(ctx, PERKS_ERR_INVALID_ARG, "stencil_run: unknown variant %d", variant);
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    Plan pl;
    bool planned = false;
    if (steps > 0) {
        if (variant == PERKS_PERSISTENT) {
            rc = run_persistent(st, steps, s, pl);
            planned = true;
        } else {
            bool used = false;
            rc = run_per_step_vec(st, steps, s, used);
            if (!rc && !used) {
                if (st->desc.dtype == PERKS_F64) rc = launch_steps<double>(st, steps, s);
                else if (st->desc.dtype == PERKS_F32) rc = launch_steps<float>(st, steps, s);
                else rc = launch_steps<__nv_bfloat16>(st, steps, s);
            }
        }
        if (rc) return rc;
    }
    if (opt_out) {
        if (variant == PERKS_PERSISTENT && !planned) {
            rc = make_plan(st, pl);
            if (rc) return rc;
        }
        fill_stats(st, variant == PERKS_PERSISTENT ? &pl : nullptr, steps, variant, opt_out);
        rc = read_dev_error(st, s);
        if (rc) return rc;
    }
    return PERKS_OK;
}

// ==================================================================== autotuner
//
// The tile decomposition that minimises halo traffic (make_plan's model) is
// not the fastest when a step is bound by the latency of each block's
// plane-by-plane walk rather than by HBM (small or fully cached domains): a
// thinner tile along z halves the walk at the price of more halo cells.  The
// autotuner times a handful of candidate plans on the stencil's own field
// (restored afterwards) and keeps the fastest: tilings ranked by
// tz * (1 + halo / volume) plus the model's choice, each with registers +
// shared memory, shared memory only or no cache (where the FP64 pipe, not HBM,
// bounds a step, caching only adds work), and with 2 or 4 planes per block
// barrier.

namespace {

struct TileCand {
    int ntx, nty, ntz;
    double score;
};

std::vector<TileCand> tile_candidates(perks_stencil *st, bool per_step, int max_cands) {
    std::vector<TileCand> all;
    const int sid = st->shape_id;
    if (sid < 0) return all;
    const ShapeInfo &sh = shape_by_id(sid);
    KernelEntry *kp = find_kernel(st->desc.dtype, sid, false, per_step, st->X, true);
    if (!kp) return all;
    const KernelEntry &k = *kp;
    const int R = sh.radius, RX = R, RY = sh.ndim == 3 ? R : 0, RZ = R;
    const int V = k.v;
    const int X = st->X, Y = st->Y, Z = st->Z, XU = X / V;
    const int maxG = st->ctx->sm_count;  // one block per SM
    for (int ntx = 1; ntx <= std::min(XU, 512); ++ntx) {
        const int txmax = ceil_div(XU, ntx) * V, txmin = (XU / ntx) * V;
        if (txmin < std::max(RX, 1) || (V > 1 && txmin < 2)) break;
        if (txmax / V > k.nt) continue;
        for (int nty = 1; nty <= std::min(Y, 512); ++nty) {
            const int tymax = ceil_div(Y, nty), tymin = Y / nty;
            if (tymin < std::max(RY, 1)) break;
            const long long threads = (long long)(txmax / V) * tymax;
            if (threads > k.nt || threads * 4 < k.nt) continue;
            const int ntz = std::min(Z / std::max(RZ, 1), maxG / (ntx * nty));
            if (ntz < 1 || Z / ntz < std::max(RZ, 1)) continue;
            if ((long long)ntx * nty * ntz * 4 < 3LL * maxG && ntz < Z / std::max(RZ, 1)) continue;  // idle SMs
            const int tzmax = ceil_div(Z, ntz);
            const double halo = 2.0 * RX / txmax + (RY ? 2.0 * RY / tymax : 0.0) + 2.0 * RZ / tzmax;
            all.push_back({ntx, nty, ntz, tzmax * (1.0 + halo) * (double)k.nt / (double)threads});
        }
    }
    std::sort(all.begin(), all.end(), [](const TileCand &a, const TileCand &b) { return a.score < b.score; });
    if ((int)all.size() > max_cands) all.resize(max_cands);
    return all;
}

}  // namespace

extern "C" perks_status perks_stencil_autotune(perks_stencil *st, int32_t variant, int32_t probe_steps,
                                               perks_stream stream, perks_stencil_plan *chosen,
                                               double *ms_per_step) {
    if (!st) return PERKS_ERR_INVALID_ARG;
    perks_context *ctx = st->ctx;
    if (variant != PERKS_PERSISTENT && variant != PERKS_PER_STEP)
        return fail(ctx, PERKS_ERR_INVALID_ARG, "stencil_autotune: unknown variant %d", variant);
    if (probe_steps < 2) return fail(ctx, PERKS_ERR_INVALID_ARG, "stencil_autotune: probe_steps >= 2");
    if (st->shape_id < 0) return fail(ctx, PERKS_ERR_UNSUPPORTED, "stencil_autotune: offsets match no compiled shape");
    perks_status rc = use_device(ctx);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const bool per_step = variant == PERKS_PER_STEP;
    const long long steps = probe_steps + (probe_steps & 1);  // even: the field buffer index is unchanged
    // candidate plans: the model's own tiling first, then the latency-ranked ones
    std::vector<perks_stencil_plan> plans;
    const bool had_plan = st->has_plan;
    const perks_stencil_plan saved_plan = st->plan;
    st->has_plan = false;
    Plan base;
    const bool had_no_resident = st->no_resident;
    st->no_resident = true;  // the plane-streaming kernel's own tiling
    rc = make_plan(st, base, per_step);
    st->no_resident = had_no_resident;
    if (rc) { st->has_plan = had_plan; st->plan = saved_plan; return rc; }
    // resident-tile candidates first (their tiling from the planner), one per thread count
    if (!per_step && !st->no_resident)
        for (int cand = 0; cand < 4; ++cand) {
            perks_stencil_plan p{};
            p.smem_cache_planes = -1;
            p.reg_cache = 1 + (cand & 1);  // rows per thread
            p.reserved[2] = PERKS_KERNEL_RESIDENT;
            p.reserved[3] = cand < 2 ? 256 : 512;
            st->plan = p;
            st->has_plan = true;
            Plan probe;
            const std::string saved_msg = ctx->last_error;
            if (make_plan(st, probe, false) == PERKS_OK) {
                p.tiles_x = probe.ntx; p.tiles_y = probe.nty; p.tiles_z = probe.ntz;
                plans.push_back(p);
            }
            ctx->last_error = saved_msg;
        }
    // plane-streaming kernels compiled with 256 threads (two blocks per SM): the model's tiling,
    // one tile per block and in balanced shares
    if (!per_step)
        for (int cand = 0; cand < 4; ++cand) {
            const int P = cand & 1 ? 4 : 2;
            perks_stencil_plan p{};
            p.smem_cache_planes = 0;
            p.reg_cache = 0;
            p.reserved[1] = P;
            p.reserved[3] = 256;
            p.balanced = cand >= 2;
            st->plan = p;
            st->has_plan = true;
            Plan probe;
            const std::string saved_msg = ctx->last_error;
            const bool had = st->no_resident;
            st->no_resident = true;
            if (make_plan(st, probe, false) == PERKS_OK && probe.k && probe.k->nt == 256) {
                p.tiles_x = probe.ntx; p.tiles_y = probe.nty; p.tiles_z = probe.ntz;
                plans.push_back(p);
            }
            st->no_resident = had;
            ctx->last_error = saved_msg;
        }
    st->has_plan = false;
    std::vector<std::array<int, 3>> tilings = {{base.ntx, base.nty, base.ntz}};
    for (const TileCand &c : tile_candidates(st, per_step, 6))
        if (!(c.ntx == base.ntx && c.nty == base.nty && c.ntz == base.ntz)) tilings.push_back({c.ntx, c.nty, c.ntz});
    for (const auto &t : tilings)
        for (int cache = per_step ? 0 : 2; cache >= -1; --cache)  // 2: registers + smem, 1: smem, 0: none,
            for (int P : {2, 4}) {                                  // -1: none, balanced shares
                perks_stencil_plan p{};
                p.tiles_x = t[0]; p.tiles_y = t[1]; p.tiles_z = cache < 0 ? 1 : t[2];
                p.smem_cache_planes = cache <= 0 ? 0 : -1;
                p.reg_cache = cache == 2 ? 1 : 0;
                p.reserved[1] = P;
                p.balanced = cache < 0;
                plans.push_back(p);
            }
    // save the field; every trial starts from it
    void *saved = nullptr;
    const size_t bytes = (size_t)st->cells * st->es;
    PERKS_CUDA(ctx, cudaMalloc(&saved, bytes));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best_ms = 1e300;
    perks_stencil_plan best = plans[0];
    perks_status out = PERKS_OK;
    cudaError_t ce = cudaMemcpyAsync(saved, st->field[st->cur], bytes, cudaMemcpyDeviceToDevice, s);
    for (size_t i = 0; i < plans.size() && ce == cudaSuccess && out == PERKS_OK; ++i) {
        st->plan = plans[i];
        st->has_plan = true;
        Plan probe;
        if (make_plan(st, probe, per_step) != PERKS_OK) continue;  // plan not hostable
        if (probe.ntx != plans[i].tiles_x || probe.nty != plans[i].tiles_y || probe.ntz != plans[i].tiles_z) continue;
        // time runs of `steps` and 3 `steps` steps: their difference is the cost of
        // 2 `steps` steps without the launch, prologue and epilogue of a run
        // (after one untimed run that allocates the plan's buffers)
        float ms_run[3] = {0.f, 0.f, 0.f};
        perks_status r = PERKS_OK;
        for (int rep = 0; rep < 3 && ce == cudaSuccess && r == PERKS_OK; ++rep) {
            ce = cudaMemcpyAsync(st->field[st->cur], saved, bytes, cudaMemcpyDeviceToDevice, s);
            if (ce != cudaSuccess) break;
            ce = cudaEventRecord(e0, s);
            r = perks_stencil_run(st, rep < 2 ? steps : 3 * steps, variant, stream, nullptr);
            if (r != PERKS_OK) break;
            ce = cudaEventRecord(e1, s);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            if (ce == cudaSuccess) cudaEventElapsedTime(&ms_run[rep], e0, e1);
        }
        ms_run[0] = ms_run[1];
        ms_run[1] = ms_run[2];
        if (r == PERKS_ERR_LAUNCH_TOO_LARGE || r == PERKS_ERR_UNSUPPORTED) continue;
        if (r != PERKS_OK) { out = r; break; }
        if (ce != cudaSuccess) break;
        const perks_status dev = read_dev_error(st, s);
        if (dev != PERKS_OK) { out = dev; break; }
        double per = (ms_run[1] - ms_run[0]) / (2.0 * (double)steps);
        if (!(per > 0.0)) per = ms_run[1] / (3.0 * (double)steps);
        if (per < best_ms) { best_ms = per; best = plans[i]; }
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(st->field[st->cur], saved, bytes, cudaMemcpyDeviceToDevice, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaFree(saved);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ce != cudaSuccess) { st->plan = saved_plan; st->has_plan = had_plan; return cuda_fail(ctx, ce, "stencil_autotune"); }
    if (out != PERKS_OK) { st->plan = saved_plan; st->has_plan = had_plan; return out; }
    if (best_ms >= 1e300) { st->plan = saved_plan; st->has_plan = had_plan; return fail(ctx, PERKS_ERR_UNSUPPORTED, "stencil_autotune: no candidate plan ran"); }
    st->plan = best;
    st->has_plan = true;
    if (chosen) *chosen = best;
    if (ms_per_step) *ms_per_step = best_ms;
    return PERKS_OK;
}

extern "C" perks_status perks_stencil_check(perks_stencil *st, perks_stream stream) {
    if (!st) return PERKS_ERR_INVALID_ARG;
    perks_status rc = use_device(st->ctx);
    if (rc) return rc;
    return read_dev_error(st, (cudaStream_t)stream);
}

// ============================================== allocation-free entry point
//
// For callers that must not allocate device memory (for example code that
// runs inside a memory-pool-managed runtime or a real-time loop where a
// cudaMalloc would block or is forbidden).  The caller supplies the input and
// output fields; everything else the persistent kernel needs -- the second
// ping-pong field, the transposed x-edge buffers, the grid-barrier counter
// and the device error record -- lives in one file-scope __device__ array.
// That array is part of the library image: every GPU on which the library is
// loaded keeps it (kNoallocScratchBytes, about 12 MiB) until the process
// exits.  All calls share it, so calls whose kernels overlap on the GPU
// (different streams, or several host threads) race and give wrong results;
// it keeps the last call's contents, and the counter and error record are
// cleared at the start of every call.

namespace {

constexpr long long kNoallocMaxCells = 1ll << 20;             // second field buffer
constexpr size_t kNoallocHeaderBytes = 256;                   // barrier counter + error record
constexpr size_t kNoallocFieldBytes = (size_t)kNoallocMaxCells * 8;
constexpr size_t kNoallocFaceBytes = (size_t)4 << 20;          // transposed x-edges, both parities
constexpr size_t kNoallocScratchBytes = kNoallocHeaderBytes + kNoallocFieldBytes + kNoallocFaceBytes;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kNoallocMaxDevices = 64;
std::atomic<unsigned char *> g_noalloc_addr[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, not a device address)
// and kept for the life of the process; several host threads may race to
// store it, which is harmless (they store the same address).
cudaError_t noalloc_scratch(int device, unsigned char **out) {
    if (device < 0 || device >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
    unsigned char *a = g_noalloc_addr[device].load(std::memory_order_acquire);
    if (!a) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        a = static_cast<unsigned char *>(p);
        g_noalloc_addr[device].store(a, std::memory_order_release);
    }
    *out = a;
    return cudaSuccess;
}

// Shape matching with a fixed-size table on the stack (no heap use).
int match_shape_noalloc(const perks_stencil_desc &d, double *kw) {
    for (int id = 0; id < kNumShapes; ++id) {
        const ShapeInfo &s = shape_by_id(id);
        if (s.ndim != d.ndim || s.npts != d.npts || s.radius != d.radius) continue;
        unsigned char used[PERKS_MAX_POINTS] = {};
        bool ok = true;
        for (int i = 0; i < s.npts && ok; ++i) {
            int found = -1;
            for (int j = 0; j < d.npts; ++j)
                if (!used[j] && d.offsets[3 * j] == shape_uoff(id, i, 0) &&
                    d.offsets[3 * j + 1] == shape_uoff(id, i, 1) && d.offsets[3 * j + 2] == shape_uoff(id, i, 2)) {
                    found = j;
                    break;
                }
            if (found < 0) ok = false;
            else { used[found] = 1; kw[i] = d.weights[found]; }
        }
        if (ok) return id;
    }
    return -1;
}

}  // namespace

extern "C" perks_status perks_stencil_run_noalloc(const perks_stencil_desc *desc, const void *in, void *out,
                                                  int64_t steps, perks_stream stream, int32_t sync) {
    if (!desc || !in || !out || steps < 0) return PERKS_ERR_INVALID_ARG;
    const perks_stencil_desc &d = *desc;
    if ((d.ndim != 2 && d.ndim != 3) || d.nx < 1 || d.ny < 1 || d.nz < 1 || (d.ndim == 2 && d.nz != 1))
        return PERKS_ERR_INVALID_ARG;
    if (d.radius < 1 || d.radius > 2 || d.npts < 1 || d.npts > PERKS_MAX_POINTS) return PERKS_ERR_INVALID_ARG;
    for (int i = 0; i < d.npts; ++i)
        for (int a = 0; a < 3; ++a) {
            const int v = d.offsets[3 * i + a];
            if (v < -d.radius || v > d.radius || (a == 2 && d.ndim == 2 && v != 0)) return PERKS_ERR_INVALID_ARG;
        }
    if (d.dtype != PERKS_F64 && d.dtype != PERKS_F32) return PERKS_ERR_UNSUPPORTED;
    // each extent is checked before the product is formed (no overflow)
    if (d.nx > kNoallocMaxCells || d.ny > kNoallocMaxCells || d.nz > kNoallocMaxCells) return PERKS_ERR_INVALID_ARG;
    const long long cells = d.nx * d.ny * d.nz;
    if (cells > kNoallocMaxCells) return PERKS_ERR_INVALID_ARG;  // beyond the scratch field's capacity
    cudaStream_t s = (cudaStream_t)stream;
    const size_t es = dtype_size(d.dtype);
    const size_t bytes = (size_t)cells * es;
    if (steps == 0) {
        if (in != out && cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return PERKS_ERR_CUDA;
        return PERKS_OK;
    }

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return PERKS_ERR_CUDA;
    unsigned char *scratch = nullptr;
    if (noalloc_scratch(device, &scratch) != cudaSuccess) return PERKS_ERR_CUDA;

    // device facts and a stencil description on the stack: nothing is allocated
    perks_context ctx;
    ctx.quiet = true;  // nothing is formatted or stored for a message
    ctx.device = device;
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return PERKS_ERR_CUDA;
    ctx.sm_count = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess)
        return PERKS_ERR_CUDA;
    ctx.smem_optin = v;
    perks_stencil st;
    st.ctx = &ctx;
    st.desc = d;
    st.es = (int)es;
    st.uX = (int)d.nx; st.uY = (int)d.ny; st.uZ = (int)d.nz;
    if (d.ndim == 3) { st.X = (int)d.nx; st.Y = (int)d.ny; st.Z = (int)d.nz; }
    else { st.X = (int)d.nx; st.Y = 1; st.Z = (int)d.ny; }
    st.cells = cells;
    st.shape_id = match_shape_noalloc(d, st.kw);
    if (st.shape_id < 0) return PERKS_ERR_UNSUPPORTED;
    st.no_resident = true;  // the scratch layout below is the plane-streaming kernel's
    Plan pl;
    perks_status rc = make_plan(&st, pl);
    if (rc) return rc;
    const int RX = shape_by_id(st.shape_id).radius;
    const int width = pl.k->v > 1 ? 2 : RX;
    const size_t face_bytes = (size_t)pl.blocks * 2 * width * pl.tzmax * pl.tymax * es;
    if (2 * face_bytes > kNoallocFaceBytes) return PERKS_ERR_INVALID_ARG;  // edges exceed the scratch

    unsigned long long *bar = reinterpret_cast<unsigned long long *>(scratch);
    DevError *err = reinterpret_cast<DevError *>(scratch + 64);
    void *field2 = scratch + kNoallocHeaderBytes;
    unsigned char *faces = scratch + kNoallocHeaderBytes + kNoallocFieldBytes;

    PersistentArgs a;
    fill_args(&st, pl, steps, a);
    a.field[0] = out;
    a.field[1] = field2;
    a.faces[0] = faces;
    a.faces[1] = faces + face_bytes;
    a.bar = bar;
    a.err = err;
    a.timeout_ns = ctx.timeout_ns;

    if (in != out && cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return PERKS_ERR_CUDA;
    if (cudaMemsetAsync(scratch, 0, kNoallocHeaderBytes, s) != cudaSuccess) return PERKS_ERR_CUDA;
    void *args[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)pl.k->fn, dim3(pl.blocks), dim3(pl.k->nt), args,
                                                (size_t)pl.smem, s);
    if (e == cudaErrorCooperativeLaunchTooLarge) return PERKS_ERR_LAUNCH_TOO_LARGE;
    if (e != cudaSuccess) return PERKS_ERR_CUDA;
    if (steps & 1) {  // the last step wrote the scratch field
        if (cudaMemcpyAsync(out, field2, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return PERKS_ERR_CUDA;
    }
    if (sync) {
        DevError he{};
        if (cudaMemcpyAsync(&he, err, sizeof(he), cudaMemcpyDeviceToHost, s) != cudaSuccess) return PERKS_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return PERKS_ERR_CUDA;
        if (he.code != 0) return he.code;
    }
    return PERKS_OK;
}
