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
// same time: a thread owns R rows of one 16-byte vector of cells
// (x0..x0+V-1; rows y0..y0+R-1) in every plane of its group's z segment.  A
// step is C chunks; in chunk c each thread computes M planes of its segment
// into registers (reading the old values from shared memory), the block
// synchronises once, and the new values overwrite the old ones.  Reads never
// see a new value:
//   * in-plane neighbours (x +-1 through warp shuffles -- a warp holds whole
//     rows of the tile -- and y +-1 from the thread's own rows or from shared
//     memory) lie in the plane being computed, which nobody overwrites before
//     the chunk's barrier;
//   * the z-1 / z+1 neighbours are the thread's own column: z-1 is carried in
//     registers from the previous plane, z+1 is read ahead;
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
    int lognv;              // log2(tx / V): a row is 2^lognv vectors
    int per_plane;          // threads per plane: (tx / V) * ceil(tymax / R)
    int PP;                 // shared-memory plane pitch (cells)
    int XGS;                // cells of one x-ghost array / one x-face (a multiple of V)
    long long FS;           // face cells per tile and parity
    int groups;             // z-groups of threads (each per_plane threads)
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

// 16-byte shared / global accesses, issued as single 128-bit loads / stores.
template <typename T, int V>
__device__ __forceinline__ VecOf<T, V> ld_vec(const T *p) {
    static_assert(sizeof(VecOf<T, V>) == 16, "16-byte vectors");
    union {
        uint4 u;
        VecOf<T, V> v;
    } x;
    x.u = *reinterpret_cast<const uint4 *>(p);
    return x.v;
}
template <typename T, int V>
__device__ __forceinline__ void st_vec(T *p, const VecOf<T, V> &v) {
    union {
        uint4 u;
        VecOf<T, V> v;
    } x;
    x.v = v;
    *reinterpret_cast<uint4 *>(p) = x.u;
}

// Weights of the stencil in registers: fp64 as they are; fp32 accumulation
// also as pairs {w, w} for the packed two-lane fused multiply-add.
template <typename T, class SH>
struct TileWeights {
    const TileArgs &a;  // scalar weights stay in the parameter bank (an fma operand)
    float2 w2[std::is_same<T, double>::value ? 1 : SH::NPTS];
    __device__ __forceinline__ explicit TileWeights(const TileArgs &args) : a(args) {
        if constexpr (!std::is_same<T, double>::value) {
#pragma unroll
            for (int i = 0; i < SH::NPTS; ++i) w2[i] = make_float2(a.wf[i], a.wf[i]);
        }
    }
    __device__ __forceinline__ typename ScalarOps<T>::A w(int i) const { return tile_w<T>(a, i); }
};

// New values of one row vector (V cells): y = sum_i w_i x(c + o_i), the
// terms added in table order from 0 by fused multiply-adds (Eq.
// iterativeStencil).  fp32 accumulation: terms whose offset has dx = 0
// update two cells with one packed fma (__ffma2_rn rounds each lane exactly
// as fmaf), the x-shifted terms one cell at a time -- every cell sees the
// same sequence of fmaf as the oracle's chain.
template <typename T, class SH, int V>
__device__ __forceinline__ VecOf<T, V> tile_update(const TileWeights<T, SH> &wt, const VecOf<T, V> &cur,
                                                   const VecOf<T, V> &prev, const VecOf<T, V> &nxt,
                                                   const VecOf<T, V> &yl, const VecOf<T, V> &yh,
                                                   typename ScalarOps<T>::A xl, typename ScalarOps<T>::A xr) {
    using A = typename ScalarOps<T>::A;
    A cc[V], zl[V], zh[V], ylo[V], yhi[V];
    to_acc_vec<T, V>(cur, cc);
    to_acc_vec<T, V>(prev, zl);
    to_acc_vec<T, V>(nxt, zh);
    if constexpr (SH::RY > 0) {
        to_acc_vec<T, V>(yl, ylo);
        to_acc_vec<T, V>(yh, yhi);
    }
    if constexpr (std::is_same<A, float>::value) {
        float2 acc[V / 2];
#pragma unroll
        for (int k = 0; k < V / 2; ++k) acc[k] = make_float2(0.f, 0.f);
        static_for<0, SH::NPTS>([&](auto II) {
            constexpr int i = decltype(II)::value;
            constexpr int dx = SH::dx(i), dy = SH::dy(i), dz = SH::dz(i);
            if constexpr (dx == 0) {
                const A *src = dz == -1 ? zl : dz == 1 ? zh : dy == -1 ? ylo : dy == 1 ? yhi : cc;
#pragma unroll
                for (int k = 0; k < V / 2; ++k)
                    acc[k] = __ffma2_rn(wt.w2[i], make_float2(src[2 * k], src[2 * k + 1]), acc[k]);
            } else {
#pragma unroll
                for (int q = 0; q < V; ++q) {
                    const A v = dx == -1 ? (q > 0 ? cc[q > 0 ? q - 1 : 0] : xl) : (q < V - 1 ? cc[q < V - 1 ? q + 1 : 0] : xr);
                    float &r = (q & 1) ? acc[q / 2].y : acc[q / 2].x;
                    r = fmaf(wt.w(i), v, r);
                }
            }
        });
        A out[V];
#pragma unroll
        for (int k = 0; k < V / 2; ++k) {
            out[2 * k] = acc[k].x;
            out[2 * k + 1] = acc[k].y;
        }
        return from_acc_vec<T, V>(out);
    } else {
        A out[V];
#pragma unroll
        for (int q = 0; q < V; ++q) {
            A sum = A(0);
            static_for<0, SH::NPTS>([&](auto II) {
                constexpr int i = decltype(II)::value;
                constexpr int dx = SH::dx(i), dy = SH::dy(i), dz = SH::dz(i);
                A v;
                if constexpr (dz == -1) v = zl[q];
                else if constexpr (dz == 1) v = zh[q];
                else if constexpr (dy == -1) v = ylo[q];
                else if constexpr (dy == 1) v = yhi[q];
                else if constexpr (dx == -1) v = q > 0 ? cc[q > 0 ? q - 1 : 0] : xl;
                else if constexpr (dx == 1) v = q < V - 1 ? cc[q < V - 1 ? q + 1 : 0] : xr;
                else v = cc[q];
                sum = fma(wt.w(i), v, sum);
            });
            out[q] = sum;
        }
        return from_acc_vec<T, V>(out);
    }
}

// Faces of tile `t` in the face buffer `buf`.
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

// Per-thread geometry of the resident tile.
template <int R>
struct TileThread {
    int ti, tj, tk;
    int x0, y0, z0, ty, tz;
    bool has_w, has_e, has_s, has_n, has_b, has_t;
    int nvx, vx, lx0;
    int ly0;          // first of the thread's R rows
    int s0, len;      // the thread's z segment [s0, s0 + len)
    unsigned rowv;    // bit r: row ly0 + r lies in the tile
    unsigned xwm, xem, ysm, ynm;  // bit r: row r writes the W / E / S / N face
};

template <int V, int R>
__device__ __forceinline__ TileThread<R> tile_thread(const TileArgs &a, int tile) {
    TileThread<R> g;
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
    g.nvx = 1 << a.lognv;
    const int grp = threadIdx.x / a.per_plane;
    const int p = threadIdx.x - grp * a.per_plane;
    g.vx = p & (g.nvx - 1);
    g.lx0 = g.vx * V;
    g.ly0 = (p >> a.lognv) * R;
    const bool act = grp < a.groups && g.ly0 < g.ty;
    if (act) split_axis(g.tz, a.groups, grp, g.s0, g.len);
    else { g.s0 = 0; g.len = 0; }
    if (g.ly0 >= g.ty) g.ly0 = g.ty - 1;  // idle threads read (and never write) a valid row
    g.rowv = g.xwm = g.xem = g.ysm = g.ynm = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (!act || g.ly0 + r >= g.ty) continue;
        g.rowv |= 1u << r;
        if (g.vx == 0 && g.has_w) g.xwm |= 1u << r;
        if (g.vx == g.nvx - 1 && g.has_e) g.xem |= 1u << r;
        if (g.ly0 + r == 0 && g.has_s) g.ysm |= 1u << r;
        if (g.ly0 + r == g.ty - 1 && g.has_n) g.ynm |= 1u << r;
    }
    return g;
}

// Where the thread's new values go in the face buffer of one step parity:
// per row r, the x-face cells (W lanes write the row's first cell, E lanes its
// last; a lane holding a whole row writes both), the y-face rows (rows 0 and
// ty - 1 of tiles with a neighbour there; a one-row tile writes both) and the
// z-faces (planes 0 and tz - 1), all addressed from per-thread pointers so
// that a plane slot issues a handful of predicated stores and little address
// arithmetic.
template <typename T, int V, int R>
struct TileFaceOut {
    T *xp[R];          // W x-face cell of row r at plane 0 (E: + xge; step z * tymax)
    T *yp;             // S y-face vector at plane 0 (N: + yne; step z * tx)
    T *zbp[R];         // bottom z-face vector of row r (top: + zte)
    int xge, yne, zte;
    unsigned xwm, xem, ysm, ynm, zbon, zton;  // bit r: row r writes that face
};

template <typename T, class SH, int V, int R>
__device__ __forceinline__ TileFaceOut<T, V, R> tile_face_out(const TileArgs &a, const TileThread<R> &g,
                                                               const TileFaces<T> &f) {
    TileFaceOut<T, V, R> o;
    o.xwm = g.xwm;
    o.xem = g.xem;
    o.ysm = SH::RY > 0 ? g.ysm : 0u;
    o.ynm = SH::RY > 0 ? g.ynm : 0u;
    o.zbon = g.has_b ? g.rowv : 0u;
    o.zton = g.has_t ? g.rowv : 0u;
    o.xge = (int)(f.fxe - f.fxw);
    o.yne = (int)(f.fyn - f.fys);
    o.zte = (int)(f.fzt - f.fzb);
    o.yp = f.fys + g.lx0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int ly = g.ly0 + r;
        o.xp[r] = f.fxw + ly;
        o.zbp[r] = f.fzb + ly * a.tx + g.lx0;
    }
    return o;
}

// Writes the new vector of row r, plane z, to the faces the neighbours read
// at the next step (zx = z * tymax, zy = z * tx, zt1 = tz - 1).
template <typename T, int V, int R>
__device__ __forceinline__ void tile_put_faces(const TileFaceOut<T, V, R> &o, int z, int zx, int zy, int zt1, int r,
                                               const VecOf<T, V> &v) {
    if ((o.xwm >> r) & 1u) o.xp[r][zx] = v.v[0];
    if ((o.xem >> r) & 1u) o.xp[r][zx + o.xge] = v.v[V - 1];
    if ((o.ysm >> r) & 1u) st_vec<T, V>(o.yp + zy, v);
    if ((o.ynm >> r) & 1u) st_vec<T, V>(o.yp + zy + o.yne, v);
    if (z == 0 && ((o.zbon >> r) & 1u)) st_vec<T, V>(o.zbp[r], v);
    if (z == zt1 && ((o.zton >> r) & 1u)) st_vec<T, V>(o.zbp[r] + o.zte, v);
}

// Shared-memory layout of the resident tile.
template <typename T, class SH>
struct TileSmem {
    static constexpr int GY = SH::RY > 0 ? 1 : 0;
    T *tile;
    T *xgw, *xge;
    int PP, tx;
    __device__ __forceinline__ int idx(int z, int y, int x) const { return (z + 1) * PP + (y + GY) * tx + x; }
};

// Ghost cells outside the domain: the Dirichlet value, written once.
template <typename T, class SH, int V, int NT, int R>
__device__ __forceinline__ void tile_fill_boundary(const TileArgs &a, const TileThread<R> &g,
                                                   const TileSmem<T, SH> &s, T bnd) {
    const int lnv = a.lognv, nv = g.nvx;
    const int nzp = g.ty << lnv;
    for (int i = threadIdx.x; i < 2 * nzp; i += NT) {
        const int side = i >= nzp, r = side ? i - nzp : i;
        if (side == 0 ? g.has_b : g.has_t) continue;
        set_vec<T, V>(s.tile + s.idx(side == 0 ? -1 : g.tz, r >> lnv, (r & (nv - 1)) * V), bnd);
    }
    if constexpr (SH::RY > 0) {
        const int nyr = g.tz << lnv;
        for (int i = threadIdx.x; i < 2 * nyr; i += NT) {
            const int side = i >= nyr, r = side ? i - nyr : i;
            if (side == 0 ? g.has_s : g.has_n) continue;
            set_vec<T, V>(s.tile + s.idx(r >> lnv, side == 0 ? -1 : g.ty, (r & (nv - 1)) * V), bnd);
        }
    }
    for (int i = threadIdx.x; i < 2 * a.XGS; i += NT) {
        const int side = i >= a.XGS;
        if (side == 0 ? g.has_w : g.has_e) continue;
        (side == 0 ? s.xgw : s.xge)[side ? i - a.XGS : i] = bnd;
    }
}

// Copies the neighbours' faces (step parity `par`) into the ghost cells.
template <typename T, class SH, int V, int NT, int R>
__device__ __forceinline__ void tile_fill_ghosts(const TileArgs &a, const TileThread<R> &g, const TileSmem<T, SH> &s,
                                                 int par) {
    const int lnv = a.lognv, nv = g.nvx;
    const int t = blockIdx.x;
    // z-ghost planes: the tile below's top face, the tile above's bottom face
    const int nzp = g.ty << lnv;
    const T *zb = g.has_b ? tile_faces<T>(a, a.faces[par], t - a.ntx * a.nty).fzt : nullptr;
    const T *zt = g.has_t ? tile_faces<T>(a, a.faces[par], t + a.ntx * a.nty).fzb : nullptr;
    for (int i = threadIdx.x; i < 2 * nzp; i += NT) {
        const int side = i >= nzp, r = side ? i - nzp : i;
        const T *src = side ? zt : zb;
        if (src == nullptr) continue;
        const int y = r >> lnv, x = (r & (nv - 1)) * V;
        cp_async<16>(s.tile + s.idx(side ? g.tz : -1, y, x), src + y * a.tx + x);
    }
    if constexpr (SH::RY > 0) {
        const int nyr = g.tz << lnv;
        const T *ys = g.has_s ? tile_faces<T>(a, a.faces[par], t - a.ntx).fyn : nullptr;
        const T *yn = g.has_n ? tile_faces<T>(a, a.faces[par], t + a.ntx).fys : nullptr;
        for (int i = threadIdx.x; i < 2 * nyr; i += NT) {
            const int side = i >= nyr, r = side ? i - nyr : i;
            const T *src = side ? yn : ys;
            if (src == nullptr) continue;
            const int z = r >> lnv, x = (r & (nv - 1)) * V;
            cp_async<16>(s.tile + s.idx(z, side ? g.ty : -1, x), src + z * a.tx + x);
        }
    }
    const int nxg = (g.tz * a.tymax + V - 1) / V;
    const T *xw = g.has_w ? tile_faces<T>(a, a.faces[par], t - 1).fxe : nullptr;
    const T *xe = g.has_e ? tile_faces<T>(a, a.faces[par], t + 1).fxw : nullptr;
    for (int i = threadIdx.x; i < 2 * nxg; i += NT) {
        const int side = i >= nxg, r = side ? i - nxg : i;
        const T *src = side ? xe : xw;
        if (src == nullptr) continue;
        cp_async<16>((side ? s.xge : s.xgw) + r * V, src + r * V);
    }
    cp_async_wait_all();
}

template <typename T, class SH, int NT, int V, int M, int R>
__global__ void __launch_bounds__(NT, 1) perks_stencil_tile_kernel(const __grid_constant__ TileArgs a) {
    static_assert(SH::R == 1 && !SH::BOX, "resident-tile kernel: radius-1 star stencils");
    static_assert(sizeof(T) * V == 16, "16-byte vectors");
    static_assert(R >= 1 && (SH::RY > 0 || R == 1), "rows per thread");
    using A = typename ScalarOps<T>::A;
    using VT = VecOf<T, V>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<T, SH> s;
    s.tile = reinterpret_cast<T *>(smem_raw);
    s.PP = a.PP;
    s.tx = a.tx;
    s.xgw = s.tile + (long long)(a.tzmax + 2) * a.PP;
    s.xge = s.xgw + a.XGS;
    constexpr int GY = TileSmem<T, SH>::GY;

    const TileThread<R> g = tile_thread<V, R>(a, blockIdx.x);
    const T bnd = tile_bnd<T>(a);
    const int PP = a.PP, tx = a.tx, tym = a.tymax;
    unsigned long long epoch = 0;

    // Per-thread addressing.  Row r loads row min(ly0 + r, ty) (a row past the
    // tile is the ghost row ty, the y+1 neighbour of the last valid row);
    // plane z of row r sits at col[r] + z * PP.
    T *col[R];
    const T *xgrow_w[R], *xgrow_e[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int yr = min(g.ly0 + r, g.ty);
        col[r] = s.tile + PP + (yr + GY) * tx + g.lx0;
        const int yx = min(g.ly0 + r, g.ty - 1);
        xgrow_w[r] = s.xgw + yx;
        xgrow_e[r] = s.xge + yx;
    }
    const T *ylo = s.tile + PP + (g.ly0 - 1 + GY) * tx + g.lx0;            // row ly0 - 1
    const T *yhi = s.tile + PP + (min(g.ly0 + R, g.ty) + GY) * tx + g.lx0;  // row ly0 + R
    const bool is_w = g.vx == 0, is_e = g.vx == g.nvx - 1;
    const TileWeights<T, SH> wt(a);

    // ---- prologue: constant ghosts, the thread's own cells, faces of x^0
    tile_trace_mark(a, -1, 0);
    tile_fill_boundary<T, SH, V, NT, R>(a, g, s, bnd);
    {
        const T *in = static_cast<const T *>(a.in);
        const TileFaceOut<T, V, R> f0 = tile_face_out<T, SH, V, R>(a, g, tile_faces<T>(a, a.faces[0], blockIdx.x));
        for (int z = g.s0; z < g.s0 + g.len; ++z) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (!(g.rowv >> r & 1u)) continue;
                const long long gi = (long long)(g.z0 + z) * a.XY + (long long)(g.y0 + g.ly0 + r) * a.X + g.x0 + g.lx0;
                const VT v = ld_vec<T, V>(in + gi);
                st_vec<T, V>(col[r] + z * PP, v);
                tile_put_faces<T, V, R>(f0, z, z * tym, z * tx, g.tz - 1, r, v);
            }
        }
    }
    tile_trace_mark(a, -1, 1);
    if (!grid_barrier(a.bar, gridDim.x, epoch, a.err, a.timeout_ns)) return;

    VT held[R];
    for (long long k = 0; k < a.steps; ++k) {
        const bool last = k + 1 == a.steps;
        tile_trace_mark(a, k, 0);
        tile_fill_ghosts<T, SH, V, NT, R>(a, g, s, (int)(k & 1));
        __syncthreads();
        const TileFaceOut<T, V, R> fo = tile_face_out<T, SH, V, R>(a, g, tile_faces<T>(a, a.faces[(k + 1) & 1], blockIdx.x));
        // window of the thread's own rows: prev = z-1, cur = z (old values)
        VT prev[R], cur[R];
        {
            const int zs0 = g.len > 0 ? g.s0 : 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                prev[r] = ld_vec<T, V>(col[r] + (zs0 - 1) * PP);
                cur[r] = ld_vec<T, V>(col[r] + zs0 * PP);
            }
        }
        for (int c = 0; c < a.chunks; ++c) {
            VT res[M][R];
            // one plane slot: z = s0 + c*M + j; FULL = every slot of the chunk is a plane of
            // the segment (no predicate); otherwise dummy slots read valid cells, write nothing
            auto slot = [&](auto JI, auto FULLC) {
                constexpr int j = decltype(JI)::value;
                constexpr bool FULL = decltype(FULLC)::value;
                const int zo = c * M + j;
                const bool valid = FULL || zo < g.len;
                int z = g.s0 + zo;
                if (!FULL) z = z < g.tz ? z : g.tz - 1;
                const int pz = z * PP, zx = z * tym;
                VT nxt[R];
#pragma unroll
                for (int r = 0; r < R; ++r) nxt[r] = ld_vec<T, V>(col[r] + pz + PP);
                VT yl, yh;
                if constexpr (SH::RY > 0) {
                    yl = ld_vec<T, V>(ylo + pz);
                    yh = ld_vec<T, V>(yhi + pz);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    // x neighbours: the adjacent lanes' vectors (a warp holds whole rows),
                    // the x-ghost columns at the tile edges
                    A xl = __shfl_up_sync(0xffffffffu, to_acc(cur[r].v[V - 1]), 1);
                    A xr = __shfl_down_sync(0xffffffffu, to_acc(cur[r].v[0]), 1);
                    if (is_w) xl = to_acc(xgrow_w[r][zx]);
                    if (is_e) xr = to_acc(xgrow_e[r][zx]);
                    res[j][r] = tile_update<T, SH, V>(wt, cur[r], prev[r], nxt[r], r == 0 ? yl : cur[r > 0 ? r - 1 : 0],
                                                      r == R - 1 ? yh : cur[r < R - 1 ? r + 1 : 0], xl, xr);
                }
                if (valid) {
#pragma unroll
                    for (int r = 0; r < R; ++r) tile_put_faces<T, V, R>(fo, z, zx, z * tx, g.tz - 1, r, res[j][r]);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        prev[r] = cur[r];
                        cur[r] = nxt[r];
                    }
                }
            };
            if (c * M + M <= g.len) {
                static_for<0, M>([&](auto JI) { slot(JI, std::true_type{}); });
            } else {
                static_for<0, M>([&](auto JI) { slot(JI, std::false_type{}); });
            }
            __syncthreads();  // every read of this chunk's old values is done
            static_for<0, M>([&](auto JI) {
                constexpr int j = decltype(JI)::value;
                const int zo = c * M + j;
                if (zo < g.len) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (!(g.rowv >> r & 1u)) continue;
                        if (zo == 0) held[r] = res[j][r];
                        else st_vec<T, V>(col[r] + (g.s0 + zo) * PP, res[j][r]);
                    }
                }
            });
        }
        if (g.len > 0) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (g.rowv >> r & 1u) st_vec<T, V>(col[r] + g.s0 * PP, held[r]);
        }
        tile_trace_mark(a, k, 1);
        if (!last) {
            if (!grid_barrier(a.bar, gridDim.x, epoch, a.err, a.timeout_ns)) return;
        }
    }

    // ---- epilogue: the thread's own cells (its own shared-memory writes) to the output
    T *out = static_cast<T *>(a.out);
    for (int z = g.s0; z < g.s0 + g.len; ++z) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!(g.rowv >> r & 1u)) continue;
            const long long gi = (long long)(g.z0 + z) * a.XY + (long long)(g.y0 + g.ly0 + r) * a.X + g.x0 + g.lx0;
            st_vec<T, V>(out + gi, ld_vec<T, V>(col[r] + z * PP));
        }
    }
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
    int r = 1;       // rows per thread
};

template <typename T, class SH, int NT, int M, int R>
TileKernelEntry tile_entry(int dtype, int shape) {
    TileKernelEntry e;
    e.dtype = dtype;
    e.shape = shape;
    e.fn = perks_stencil_tile_kernel<T, SH, NT, 16 / (int)sizeof(T), M, R>;
    e.nt = NT;
    e.v = 16 / (int)sizeof(T);
    e.m = M;
    e.r = R;
    return e;
}

}  // namespace perks
