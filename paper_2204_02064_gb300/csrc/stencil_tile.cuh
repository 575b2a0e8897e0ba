// Resident-tile persistent stencil kernel: the PERKS execution model (Sec. 3,
// Fig. 4) for domains whose every tile fits in one block's shared memory.
//
// The time loop runs inside one cooperative launch with a grid barrier per
// step (Listing 1's structure), and each block keeps its WHOLE tile of the
// field in shared memory for all steps (D_cache = D, D_uncache = 0 in the
// model of Sec. 5.2): the field in HBM is read once before the first step
// and written once after the last; between steps only the tile faces travel,
// through L2 (halo exchange, Sec. 4.2.2).
//
// Where the plane-streaming kernel (stencil_vec.cuh) walks a tile plane by
// plane with a block barrier per plane (or per 2-4 planes), this kernel
// splits the tile's z extent among G groups of threads that all work at the
// same time: a thread owns one 16-byte vector of cells (x0..x0+V-1, y) in
// every plane of its group's z segment.  A step is C chunks; in chunk c each
// thread computes M planes of its segment into registers (reading the old
// values from shared memory), the block synchronises once, and the new
// values overwrite the old ones.  Reads never see a new value:
//   * in-plane neighbours (x +-1 through warp shuffles -- a warp holds whole
//     rows of the tile -- and y +-1 from shared memory) lie in the plane being
//     computed, which nobody overwrites before the chunk's barrier;
//   * the z-1 / z+1 neighbours are the thread's own column: z-1 is carried in
//     a register from the previous plane, z+1 is read ahead;
//   * the first plane of each segment is the z+1 neighbour of the previous
//     segment's last plane, which another group computes in its LAST chunk,
//     so each thread holds its first plane's new values in registers and
//     stores them only after all chunks of the step.
//
// Halo exchange: faces of the tile are written to a per-tile global face
// buffer (double-buffered by step parity) as the new values are produced;
// after the grid barrier every block copies its neighbours' faces into the
// ghost cells of its shared-memory tile with 16-byte cp.async (bypassing L1).
// Ghost cells outside the domain hold the Dirichlet value and are written
// once.  x-faces are stored transposed ([z][y]) so they move as contiguous
// vectors (the paper's transposed vertical edges, Sec. 4.2.2).
//
// Shared memory (cells of T):
//   tile   (tzmax + 2) planes of PP = (tymax + 2 GY) * tx cells: plane zz holds
//          z = zz - 1 (planes 0 and tz + 1 are the z-ghosts), row yy holds
//          y = yy - GY (GY = 1 in 3-D: rows 0 and ty + 1 are the y-ghosts);
//   xg     two arrays of XGS cells, W and E x-ghost columns, [z][y] with
//          pitch tymax.
// Global face buffer per tile and parity (FS cells):
//   fxW, fxE [z][y] (XGS each) | fyS, fyN [z][x] (tzmax*tx each) |
//   fzB, fzT [y][x] (tymax*tx each).
//
// Scope: star stencils of radius 1 (2d5pt, 3d7pt), every storage type.
#pragma once

#include "stencil_vec.cuh"

namespace perks {

struct TileArgs {
    int X, Y, Z;            // internal interior extents (2-D: Y = 1)
    long long XY;
    int ntx, nty, ntz;      // tiles per axis; X = ntx * tx exactly
    int tx, tymax, tzmax;
    int PP;                 // shared-memory plane pitch (cells)
    int XGS;                // cells of one x-ghost array / one x-face (a multiple of V)
    long long FS;           // face cells per tile and parity
    int groups;             // z-groups of threads (each NT / groups threads = one plane)
    int chunks;             // chunks per step
    long long steps;
    double boundary;
    float boundary_f;
    double w[kMaxKernelPoints];
    float wf[kMaxKernelPoints];
    const void *in;         // field at step 0
    void *out;              // receives the field after `steps` steps
    void *faces[2];         // face buffers by step parity
    unsigned long long *bar;
    DevError *err;
    long long timeout_ns;
    unsigned long long *trace;  // optional step trace (as PersistentArgs::trace)
    int trace_steps;
};

__device__ __forceinline__ void tile_trace_mark(const TileArgs &a, long long k, int which) {
    if (a.trace != nullptr && threadIdx.x == 0 && k < a.trace_steps) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        a.trace[((k + 1) * gridDim.x + blockIdx.x) * 2 + which] = t;
    }
}

// Weights and boundary value in the accumulator / storage type.
template <typename T> __device__ __forceinline__ typename ScalarOps<T>::A tile_w(const TileArgs &a, int i) {
    if constexpr (std::is_same<T, double>::value) return a.w[i];
    else return a.wf[i];
}
template <typename T> __device__ __forceinline__ T tile_bnd(const TileArgs &a) {
    if constexpr (std::is_same<T, double>::value) return a.boundary;
    else if constexpr (std::is_same<T, float>::value) return a.boundary_f;
    else return __float2bfloat16_rn(a.boundary_f);
}

// Vector of V cells converted to the accumulator type.
template <typename T, int V>
__device__ __forceinline__ void to_acc_vec(const VecOf<T, V> &v, typename ScalarOps<T>::A (&o)[V]) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        const __nv_bfloat162 *c2 = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
        for (int j = 0; j < V / 2; ++j) {
            const float2 f = __bfloat1622float2(c2[j]);
            o[2 * j] = f.x;
            o[2 * j + 1] = f.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) o[j] = to_acc(v.v[j]);
    }
}

template <typename T, int V>
__device__ __forceinline__ VecOf<T, V> from_acc_vec(const typename ScalarOps<T>::A (&a)[V]) {
    VecOf<T, V> out;
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        __nv_bfloat162 *o2 = reinterpret_cast<__nv_bfloat162 *>(&out);
#pragma unroll
        for (int j = 0; j < V / 2; ++j) o2[j] = __floats2bfloat162_rn(a[2 * j], a[2 * j + 1]);
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) out.v[j] = from_acc<T>(a[j]);
    }
    return out;
}

// Per-thread geometry of the resident tile.
struct TileGeom {
    int ti, tj, tk;
    int x0, y0, z0, ty, tz;
    bool has_w, has_e, has_s, has_n, has_b, has_t;
    int nvx;        // vectors per row
    int ly, vx;     // the thread's row and vector position (row clamped to the tile)
    bool row_ok;    // the thread's row lies in the tile
    int s0, len;    // the thread's z segment [s0, s0 + len)
};

template <int V>
__device__ __forceinline__ TileGeom tile_geom(const TileArgs &a, int tile) {
    TileGeom g;
    g.ti = tile % a.ntx;
    g.tj = (tile / a.ntx) % a.nty;
    g.tk = tile / (a.ntx * a.nty);
    g.x0 = g.ti * a.tx;
    split_axis(a.Y, a.nty, g.tj, g.y0, g.ty);
    split_axis(a.Z, a.ntz, g.tk, g.z0, g.tz);
    g.has_w = g.ti > 0;
    g.has_e = g.ti + 1 < a.ntx;
    g.has_s = g.tj > 0;
    g.has_n = g.tj + 1 < a.nty;
    g.has_b = g.tk > 0;
    g.has_t = g.tk + 1 < a.ntz;
    g.nvx = a.tx / V;
    const int per_plane = g.nvx * a.tymax;
    const int grp = threadIdx.x / per_plane;
    const int p = threadIdx.x % per_plane;
    const int ly = p / g.nvx;
    g.vx = p % g.nvx;
    g.row_ok = ly < g.ty && grp < a.groups;
    g.ly = ly < g.ty ? ly : g.ty - 1;
    if (grp < a.groups) split_axis(g.tz, a.groups, grp, g.s0, g.len);
    else { g.s0 = 0; g.len = 0; }
    if (!g.row_ok) g.len = 0;
    return g;
}

template <typename T, class SH, int V>
struct TileSmem {
    static constexpr int GY = SH::RY;
    T *tile;
    T *xgw, *xge;
    int PP, tx;
    __device__ __forceinline__ int idx(int z, int y, int x) const { return (z + 1) * PP + (y + GY) * tx + x; }
};

// Faces of tile `t` in the face buffer `base`.
template <typename T>
struct TileFaces {
    T *fxw, *fxe, *fys, *fyn, *fzb, *fzt;
};

template <typename T>
__device__ __forceinline__ TileFaces<T> tile_faces(const TileArgs &a, void *buf, int t) {
    T *b = static_cast<T *>(buf) + (long long)t * a.FS;
    TileFaces<T> f;
    f.fxw = b;
    f.fxe = b + a.XGS;
    f.fys = b + 2 * a.XGS;
    f.fyn = f.fys + (long long)a.tzmax * a.tx;
    f.fzb = f.fyn + (long long)a.tzmax * a.tx;
    f.fzt = f.fzb + (long long)a.tymax * a.tx;
    return f;
}

// Writes the new vector of plane z (row ly, vector vx) to the faces the
// neighbours read at the next step.
template <typename T, class SH, int V>
__device__ __forceinline__ void tile_put_faces(const TileArgs &a, const TileGeom &g, const TileFaces<T> &f, int z,
                                               const VecOf<T, V> &v) {
    using VT = VecOf<T, V>;
    const int lx0 = g.vx * V;
    if (z == 0 && g.has_b) *reinterpret_cast<VT *>(f.fzb + g.ly * a.tx + lx0) = v;
    if (z == g.tz - 1 && g.has_t) *reinterpret_cast<VT *>(f.fzt + g.ly * a.tx + lx0) = v;
    if constexpr (SH::RY > 0) {
        if (g.ly == 0 && g.has_s) *reinterpret_cast<VT *>(f.fys + (long long)z * a.tx + lx0) = v;
        if (g.ly == g.ty - 1 && g.has_n) *reinterpret_cast<VT *>(f.fyn + (long long)z * a.tx + lx0) = v;
    }
    if (g.vx == 0 && g.has_w) f.fxw[z * a.tymax + g.ly] = v.v[0];
    if (g.vx == g.nvx - 1 && g.has_e) f.fxe[z * a.tymax + g.ly] = v.v[V - 1];
}

// Ghost cells outside the domain: the Dirichlet value, written once.
template <typename T, class SH, int V, int NT>
__device__ __forceinline__ void tile_fill_boundary(const TileArgs &a, const TileGeom &g, const TileSmem<T, SH, V> &s,
                                                   T bnd) {
    const int nv = g.nvx;
    // z-ghost planes: rows 0..ty-1
    for (int i = threadIdx.x; i < 2 * g.ty * nv; i += NT) {
        const int side = i / (g.ty * nv), r = i % (g.ty * nv);
        if (side == 0 ? g.has_b : g.has_t) continue;
        const int z = side == 0 ? -1 : g.tz;
        set_vec<T, V>(s.tile + s.idx(z, r / nv, (r % nv) * V), bnd);
    }
    if constexpr (SH::RY > 0) {
        for (int i = threadIdx.x; i < 2 * g.tz * nv; i += NT) {
            const int side = i / (g.tz * nv), r = i % (g.tz * nv);
            if (side == 0 ? g.has_s : g.has_n) continue;
            const int y = side == 0 ? -1 : g.ty;
            set_vec<T, V>(s.tile + s.idx(r / nv, y, (r % nv) * V), bnd);
        }
    }
    for (int i = threadIdx.x; i < 2 * a.XGS; i += NT) {
        const int side = i / a.XGS;
        if (side == 0 ? g.has_w : g.has_e) continue;
        (side == 0 ? s.xgw : s.xge)[i % a.XGS] = bnd;
    }
}

// Copies the neighbours' faces (step parity `par`) into the ghost cells.
template <typename T, class SH, int V, int NT>
__device__ __forceinline__ void tile_fill_ghosts(const TileArgs &a, const TileGeom &g, const TileSmem<T, SH, V> &s,
                                                 int par) {
    const int nv = g.nvx;
    const int t = blockIdx.x;
    const int sx = 1, sy = a.ntx, sz = a.ntx * a.nty;
    const int nzp = g.ty * nv;              // vectors of one z-ghost plane
    const int nyr = SH::RY > 0 ? g.tz * nv : 0;  // vectors of one y-ghost row set
    const int nxg = (g.tz * a.tymax + V - 1) / V;
    const int total = 2 * nzp + 2 * nyr + 2 * nxg;
    for (int i = threadIdx.x; i < total; i += NT) {
        int r = i;
        if (r < 2 * nzp) {
            const int side = r / nzp;
            r %= nzp;
            if (side == 0 ? !g.has_b : !g.has_t) continue;
            const TileFaces<T> f = tile_faces<T>(a, a.faces[par], side == 0 ? t - sz : t + sz);
            const int y = r / nv, x = (r % nv) * V;
            cp_async<16>(s.tile + s.idx(side == 0 ? -1 : g.tz, y, x), (side == 0 ? f.fzt : f.fzb) + y * a.tx + x);
            continue;
        }
        r -= 2 * nzp;
        if (r < 2 * nyr) {
            const int side = r / nyr;
            r %= nyr;
            if (side == 0 ? !g.has_s : !g.has_n) continue;
            const TileFaces<T> f = tile_faces<T>(a, a.faces[par], side == 0 ? t - sy : t + sy);
            const int z = r / nv, x = (r % nv) * V;
            cp_async<16>(s.tile + s.idx(z, side == 0 ? -1 : g.ty, x),
                         (side == 0 ? f.fyn : f.fys) + (long long)z * a.tx + x);
            continue;
        }
        r -= 2 * nyr;
        const int side = r / nxg;
        r %= nxg;
        if (side == 0 ? !g.has_w : !g.has_e) continue;
        const TileFaces<T> f = tile_faces<T>(a, a.faces[par], side == 0 ? t - sx : t + sx);
        cp_async<16>((side == 0 ? s.xgw : s.xge) + r * V, (side == 0 ? f.fxe : f.fxw) + r * V);
    }
    cp_async_wait_all();
}

template <typename T, class SH, int NT, int V, int M>
__global__ void __launch_bounds__(NT, 1) perks_stencil_tile_kernel(const __grid_constant__ TileArgs a) {
    static_assert(SH::R == 1 && !SH::BOX, "resident-tile kernel: radius-1 star stencils");
    static_assert(sizeof(T) * V == 16, "16-byte vectors");
    using A = typename ScalarOps<T>::A;
    using VT = VecOf<T, V>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<T, SH, V> s;
    s.tile = reinterpret_cast<T *>(smem_raw);
    s.PP = a.PP;
    s.tx = a.tx;
    s.xgw = s.tile + (long long)(a.tzmax + 2) * a.PP;
    s.xge = s.xgw + a.XGS;

    const TileGeom g = tile_geom<V>(a, blockIdx.x);
    const T bnd = tile_bnd<T>(a);
    const int lx0 = g.vx * V;
    unsigned long long epoch = 0;

    // ---- prologue: constant ghosts, the thread's own cells, faces of x^0
    tile_trace_mark(a, -1, 0);
    tile_fill_boundary<T, SH, V, NT>(a, g, s, bnd);
    {
        const T *in = static_cast<const T *>(a.in);
        const TileFaces<T> f0 = tile_faces<T>(a, a.faces[0], blockIdx.x);
        const long long base = (long long)g.z0 * a.XY + (long long)(g.y0 + g.ly) * a.X + g.x0 + lx0;
        for (int z = g.s0; z < g.s0 + g.len; ++z) {
            const VT v = *reinterpret_cast<const VT *>(in + base + (long long)z * a.XY);
            *reinterpret_cast<VT *>(s.tile + s.idx(z, g.ly, lx0)) = v;
            tile_put_faces<T, SH, V>(a, g, f0, z, v);
        }
    }
    tile_trace_mark(a, -1, 1);
    if (!grid_barrier(a.bar, gridDim.x, epoch, a.err, a.timeout_ns)) return;

    VT held;
    for (long long k = 0; k < a.steps; ++k) {
        const bool last = k + 1 == a.steps;
        tile_trace_mark(a, k, 0);
        tile_fill_ghosts<T, SH, V, NT>(a, g, s, (int)(k & 1));
        __syncthreads();
        const TileFaces<T> fo = tile_faces<T>(a, a.faces[(k + 1) & 1], blockIdx.x);
        // window of the thread's own column: prev = z-1, cur = z (old values)
        const int zs0 = g.len > 0 ? g.s0 : 0;
        VT prev = *reinterpret_cast<const VT *>(s.tile + s.idx(zs0 - 1, g.ly, lx0));
        VT cur = *reinterpret_cast<const VT *>(s.tile + s.idx(zs0, g.ly, lx0));
        for (int c = 0; c < a.chunks; ++c) {
            VT res[M];
            static_for<0, M>([&](auto JI) {
                constexpr int j = decltype(JI)::value;
                const int zo = c * M + j;                 // offset in the segment
                const bool valid = zo < g.len;
                int z = g.s0 + zo;
                z = z < g.tz ? z : g.tz - 1;              // clamped: dummy slots read valid cells
                const VT nxt = *reinterpret_cast<const VT *>(s.tile + s.idx(z + 1, g.ly, lx0));
                A cc[V], zl[V], zh[V], yl[V], yh[V];
                to_acc_vec<T, V>(cur, cc);
                to_acc_vec<T, V>(prev, zl);
                to_acc_vec<T, V>(nxt, zh);
                if constexpr (SH::RY > 0) {
                    to_acc_vec<T, V>(*reinterpret_cast<const VT *>(s.tile + s.idx(z, g.ly - 1, lx0)), yl);
                    to_acc_vec<T, V>(*reinterpret_cast<const VT *>(s.tile + s.idx(z, g.ly + 1, lx0)), yh);
                }
                // x neighbours: the adjacent lanes' vectors (a warp holds whole rows), the
                // x-ghost columns at the tile edges
                A xl = __shfl_up_sync(0xffffffffu, cc[V - 1], 1);
                A xr = __shfl_down_sync(0xffffffffu, cc[0], 1);
                if (g.vx == 0) xl = to_acc(s.xgw[z * a.tymax + g.ly]);
                if (g.vx == g.nvx - 1) xr = to_acc(s.xge[z * a.tymax + g.ly]);
                A acc[V];
                static_for<0, V>([&](auto QI) {
                    constexpr int q = decltype(QI)::value;
                    A sum = A(0);
                    static_for<0, SH::NPTS>([&](auto II) {
                        constexpr int i = decltype(II)::value;
                        constexpr int dx = SH::dx(i), dy = SH::dy(i), dz = SH::dz(i);
                        A v;
                        if constexpr (dz == -1) v = zl[q];
                        else if constexpr (dz == 1) v = zh[q];
                        else if constexpr (dy == -1) v = yl[q];
                        else if constexpr (dy == 1) v = yh[q];
                        else if constexpr (dx == -1) v = q > 0 ? cc[q > 0 ? q - 1 : 0] : xl;
                        else if constexpr (dx == 1) v = q < V - 1 ? cc[q < V - 1 ? q + 1 : 0] : xr;
                        else v = cc[q];
                        sum = fma(tile_w<T>(a, i), v, sum);
                    });
                    acc[q] = sum;
                });
                res[j] = from_acc_vec<T, V>(acc);
                if (valid) {
                    tile_put_faces<T, SH, V>(a, g, fo, z, res[j]);
                    prev = cur;
                    cur = nxt;
                }
            });
            __syncthreads();  // every read of this chunk's old values is done
            static_for<0, M>([&](auto JI) {
                constexpr int j = decltype(JI)::value;
                const int zo = c * M + j;
                if (zo < g.len) {
                    if (zo == 0) held = res[j];
                    else *reinterpret_cast<VT *>(s.tile + s.idx(g.s0 + zo, g.ly, lx0)) = res[j];
                }
            });
        }
        if (g.len > 0) *reinterpret_cast<VT *>(s.tile + s.idx(g.s0, g.ly, lx0)) = held;
        tile_trace_mark(a, k, 1);
        if (!last) {
            if (!grid_barrier(a.bar, gridDim.x, epoch, a.err, a.timeout_ns)) return;
        }
    }

    // ---- epilogue: the thread's own cells (its own shared-memory writes) to the output
    T *out = static_cast<T *>(a.out);
    const long long base = (long long)g.z0 * a.XY + (long long)(g.y0 + g.ly) * a.X + g.x0 + lx0;
    for (int z = g.s0; z < g.s0 + g.len; ++z)
        *reinterpret_cast<VT *>(out + base + (long long)z * a.XY) =
            *reinterpret_cast<const VT *>(s.tile + s.idx(z, g.ly, lx0));
}

using TileFn = void (*)(TileArgs);

// One compiled instantiation of the resident-tile kernel.
struct TileKernelEntry {
    int dtype = 0;   // PERKS_F64 / PERKS_F32 / PERKS_BF16
    int shape = 0;   // ShapeId
    TileFn fn = nullptr;
    int nt = 0;      // threads per block
    int v = 0;       // cells per 16-byte vector
    int m = 0;       // planes per chunk
};

template <typename T, class SH, int NT, int M>
TileKernelEntry tile_entry(int dtype, int shape) {
    TileKernelEntry e;
    e.dtype = dtype;
    e.shape = shape;
    e.fn = perks_stencil_tile_kernel<T, SH, NT, 16 / (int)sizeof(T), M>;
    e.nt = NT;
    e.v = 16 / (int)sizeof(T);
    e.m = M;
    return e;
}

}  // namespace perks
