// Vectorised persistent stencil kernel (the fast path).
//
// Same method and data flow as perks_stencil_kernel (Sec. 3 / Sec. 4.2:
// time loop inside one cooperative launch, grid barrier per step, each
// block's tile cached on chip between steps, halos through L2), laid out for
// GB300's issue rate:
//   * every thread owns V consecutive x-cells of a column (16-byte vectors),
//     so loads, stores and cp.async copies are 16 bytes wide and the
//     per-cell instruction count falls by ~V;
//   * all neighbour values are read from the shared-memory plane ring with
//     vector loads (the row a thread needs at offset (dy, dz) is its own
//     vector of that row plus R cells on either side);
//   * the transposed x-edges are stored as aligned PAIRS of cells
//     (x0, x0+1) and (x1-2, x1-1) per (z, y), so every element size,
//     including 2-byte bf16, moves them with one cp.async;
//   * the prefetch depth D is chosen per element size to keep ~40 KB of
//     loads in flight per SM (Little's law, Sec. 5.3).
// PER_STEP = true turns the same body into the one-launch-per-step baseline
// (the paper's SHM kernel that PERKS wraps): no caches, no grid barrier, and
// the x-halo pairs come straight from the field.
#pragma once

#include <type_traits>

#include "stencil_kernels.cuh"

namespace perks {

// Loop whose index is a constant expression in the body (so constexpr shape
// tables fold and per-thread arrays stay in registers).
template <int B, int E, class F> __device__ __forceinline__ void static_for(F &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

template <typename T, int V> struct alignas(sizeof(T) * V) VecOf { T v[V]; };
template <typename T> struct alignas(sizeof(T) * 2) PairOf { T v[2]; };

template <typename T> struct ScalarOps;
template <> struct ScalarOps<double> {
    using A = double;
    static __device__ __forceinline__ A w(const PersistentArgs &a, int i) { return a.w[i]; }
    static __device__ __forceinline__ double bnd(const PersistentArgs &a) { return a.boundary; }
};
template <> struct ScalarOps<float> {
    using A = float;
    static __device__ __forceinline__ A w(const PersistentArgs &a, int i) { return a.wf[i]; }
    static __device__ __forceinline__ float bnd(const PersistentArgs &a) { return a.boundary_f; }
};
template <> struct ScalarOps<__nv_bfloat16> {
    using A = float;
    static __device__ __forceinline__ A w(const PersistentArgs &a, int i) { return a.wf[i]; }
    static __device__ __forceinline__ __nv_bfloat16 bnd(const PersistentArgs &a) {
        return __float2bfloat16_rn(a.boundary_f);
    }
};

// Rows (dy, dz) of a shape with the extent of dx used in each.
template <class SH> struct RowsOf {
    static constexpr int MAXR = 25;
    __host__ __device__ static constexpr int count() {
        int n = 0;
        for (int i = 0; i < SH::NPTS; ++i) {
            bool seen = false;
            for (int k = 0; k < i; ++k)
                if (SH::dy(k) == SH::dy(i) && SH::dz(k) == SH::dz(i)) seen = true;
            if (!seen) ++n;
        }
        return n;
    }
    // index of the row of point i (rows numbered by first appearance)
    __host__ __device__ static constexpr int row_of(int i) {
        int n = 0;
        for (int j = 0; j <= i; ++j) {
            bool seen = false;
            int idx = -1;
            for (int k = 0; k < j; ++k)
                if (SH::dy(k) == SH::dy(j) && SH::dz(k) == SH::dz(j)) seen = true;
            if (!seen) { idx = n; ++n; }
            if (j == i) {
                if (idx >= 0) return idx;
                // row of an earlier point
                for (int k = 0; k < j; ++k)
                    if (SH::dy(k) == SH::dy(j) && SH::dz(k) == SH::dz(j)) return row_of(k);
            }
        }
        return 0;
    }
    __host__ __device__ static constexpr int first_point(int r) {
        for (int i = 0; i < SH::NPTS; ++i)
            if (row_of(i) == r) return i;
        return 0;
    }
    __host__ __device__ static constexpr int dy(int r) { return SH::dy(first_point(r)); }
    __host__ __device__ static constexpr int dz(int r) { return SH::dz(first_point(r)); }
    __host__ __device__ static constexpr int minx(int r) {
        int m = 0;
        for (int i = 0; i < SH::NPTS; ++i)
            if (row_of(i) == r && SH::dx(i) < m) m = SH::dx(i);
        return m;
    }
    __host__ __device__ static constexpr int maxx(int r) {
        int m = 0;
        for (int i = 0; i < SH::NPTS; ++i)
            if (row_of(i) == r && SH::dx(i) > m) m = SH::dx(i);
        return m;
    }
};

enum DutyKind : int { DUTY_NONE = 0, DUTY_BND_VEC, DUTY_BND_PAIR, DUTY_FIELD_VEC, DUTY_FIELD_PAIR, DUTY_XPAIR };

struct VecPlan {
    int tile, x0, y0, z0, tx, ty, tz;
    bool own;
    int rowpos, nvx;    // position of the thread's vector in its row, vectors per row
    unsigned own_mask;  // lanes of this warp that own cells
    int lx0, ly;
    long long gxy;      // field offset of the thread's first cell at z = 0
    int sidx;           // ring index of the thread's first cell
    bool field_shell;
    bool has_b, has_t;
    bool wface, eface;  // this thread writes the tile's W / E face pair
    int duty;
    int dsidx;          // ring index of the duty item
    long long dgxy;     // field offset (z = 0) of the duty item
    long long dface;    // face offset (z = 0) of an x-halo pair
    long long wface_off, eface_off;  // own face entries (z = 0)
};

// Element layout of a ring slot row: HX pad cells, tx cells, HX pad cells
// (HX a multiple of V, at least 2 and at least the radius).
template <int V, int R = 1> __host__ __device__ constexpr int vec_hx() {
    int hx = V >= 2 ? V : 2;
    while (hx < R) hx += V;
    return hx;
}
// Cells of one x-halo item (each side of a row): 2 up to radius 2, 4 beyond.
template <int R> __host__ __device__ constexpr int vec_xw() { return R <= 2 ? 2 : 4; }

template <class SH, int V, bool PER_STEP>
__device__ __forceinline__ VecPlan make_vec_plan(const PersistentArgs &a, int tile) {
    constexpr int RY = SH::RY;
    constexpr int HX = vec_hx<V, SH::R>();
    constexpr int XW = vec_xw<SH::R>();
    VecPlan p;
    p.tile = tile;
    const int ti = p.tile % a.ntx, tj = (p.tile / a.ntx) % a.nty, tk = p.tile / (a.ntx * a.nty);
    int xu0, txu;
    split_axis(a.X / V, a.ntx, ti, xu0, txu);  // x split in units of V cells
    p.x0 = xu0 * V;
    p.tx = txu * V;
    split_axis(a.Y, a.nty, tj, p.y0, p.ty);
    split_axis(a.Z, a.ntz, tk, p.z0, p.tz);
    const bool has_w = ti > 0, has_e = ti + 1 < a.ntx, has_s = tj > 0, has_n = tj + 1 < a.nty;
    p.has_b = tk > 0;
    p.has_t = tk + 1 < a.ntz;
    const int nvx = p.tx / V;
    const int c = threadIdx.x;
    p.own = c < nvx * p.ty;
    p.own_mask = __ballot_sync(0xffffffffu, p.own);
    p.rowpos = p.own ? c % nvx : 0;
    p.nvx = nvx;
    p.lx0 = p.own ? (c % nvx) * V : 0;
    p.ly = p.own ? c / nvx : 0;
    p.gxy = (long long)(p.x0 + p.lx0) + (long long)(p.y0 + p.ly) * a.X;
    p.sidx = (p.ly + RY) * a.PW + HX + p.lx0;
    p.field_shell = p.own && ((p.ly < RY && has_s) || (p.ly >= p.ty - RY && has_n));
    p.wface = !PER_STEP && p.own && p.lx0 == 0 && has_w;
    p.eface = !PER_STEP && p.own && p.lx0 + V == p.tx && has_e;
    // faces: [tile][side][z][y] pairs (face_plane = tzmax * tymax pairs per side)
    p.wface_off = ((long long)(p.tile * 2 + 0) * a.face_plane + p.ly) * 2;
    p.eface_off = ((long long)(p.tile * 2 + 1) * a.face_plane + p.ly) * 2;

    // duty items: y-row vectors, box corners (pairs), x-halo pairs
    const int n_yrow = 2 * RY * nvx;
    const int n_corner = SH::BOX ? 2 * RY * 2 : 0;
    const int n_xpair = 2 * p.ty;
    p.duty = DUTY_NONE;
    p.dsidx = 0;
    p.dgxy = 0;
    p.dface = 0;
    int lxr = 0, lyr = 0, kind = DUTY_NONE;
    if (c < n_yrow) {
        const int r = c / nvx;  // 0 .. 2RY-1
        lyr = r < RY ? r - RY : p.ty + (r - RY);
        lxr = (c % nvx) * V;
        kind = DUTY_FIELD_VEC;
    } else if (c < n_yrow + n_corner) {
        const int k = c - n_yrow;
        const int r = k / 2;
        lyr = r < RY ? r - RY : p.ty + (r - RY);
        lxr = (k % 2 == 0) ? -XW : p.tx;
        kind = DUTY_FIELD_PAIR;
    } else if (c < n_yrow + n_corner + n_xpair) {
        const int k = c - n_yrow - n_corner;
        const int side = k / p.ty;
        lyr = k % p.ty;
        lxr = side == 0 ? -XW : p.tx;
        kind = DUTY_XPAIR;
        if (!PER_STEP) {
            const int nb = side == 0 ? p.tile - 1 : p.tile + 1;
            const int nb_side = side == 0 ? 1 : 0;  // W strip = W neighbour's E face
            p.dface = ((long long)(nb * 2 + nb_side) * a.face_plane + lyr) * 2;
        }
    }
    if (kind != DUTY_NONE) {
        const int gx = p.x0 + lxr, gy = p.y0 + lyr;
        const int width = kind == DUTY_FIELD_VEC ? V : XW;
        p.dsidx = (lyr + RY) * a.PW + HX + lxr;
        if (gy < 0 || gy >= a.Y || gx < 0 || gx + width > a.X) {
            p.duty = kind == DUTY_FIELD_VEC ? DUTY_BND_VEC : DUTY_BND_PAIR;
        } else {
            p.duty = kind;
            p.dgxy = (long long)gx + (long long)gy * a.X;
        }
    }
    return p;
}

template <typename T, int V>
__device__ __forceinline__ void copy_vec(T *sdst, const T *gsrc) {
    cp_async<sizeof(T) * V>(sdst, gsrc);
}

template <typename T, int V>
__device__ __forceinline__ void set_vec(T *d, T v) {
    VecOf<T, V> x;
#pragma unroll
    for (int j = 0; j < V; ++j) x.v[j] = v;
    *reinterpret_cast<VecOf<T, V> *>(d) = x;
}

// Loads R cells (1 or 2) ending just left of / starting just right of a vector.
template <typename T, int N>
__device__ __forceinline__ void load_cells(const T *p, T (&out)[N > 0 ? N : 1]) {
    if constexpr (N == 1) {
        out[0] = *p;
    } else if constexpr (N == 2) {
        const PairOf<T> x = *reinterpret_cast<const PairOf<T> *>(p);
        out[0] = x.v[0];
        out[1] = x.v[1];
    }
}

// Ring slots of the vectorised kernel: an iteration over P planes reads
// planes z-RZ..z+P-1+RZ while P more are filled, D planes ahead.
template <int RZ, int D, int P = 2> __host__ __device__ constexpr int vec_slots() { return 2 * RZ + P + D; }

// Where a plane's own-column values come from (fill) or go to (store).
enum PlaneClass : int { PC_REG = 0, PC_SMEM = 1, PC_GLOBAL = 2, PC_HALO = 3, PC_NONE = 4 };

// Per-thread, per-step addressing kept in registers: pointers advance by one
// plane (XY elements) per iteration instead of being recomputed.
template <typename T> struct StepPtrs {
    const T *fill_own;   // field[src] at the thread's column, plane of the next fill
    const T *fill_duty;  // field[src] at the duty item, plane of the next fill
    const T *face_src;   // faces[src] at the duty pair, plane of the next fill
    T *store_own;        // field[dst] at the thread's column, plane being stored
    T *face_dst_w, *face_dst_e;
    double kz;           // fp64 3d7pt, equal neighbour weights: the pair sum carried to the next plane
};

template <typename T, class SH, int V, int ZR, bool PER_STEP, int FILL>
__device__ __forceinline__ void vfill_fast(const PersistentArgs &a, const VecPlan &tp, int q, T *sl,
                                           StepPtrs<T> &sp, const T *smc,
                                           const VecOf<T, V> (&regc)[ZR > 0 ? ZR : 1]) {
    using VT = VecOf<T, V>;
    using PT = PairOf<T>;
    if (FILL == PC_NONE) return;
    const T bnd = ScalarOps<T>::bnd(a);
    bool in_z = true;
    if (FILL == PC_HALO) {
        const int gz = tp.z0 + q;
        in_z = gz >= 0 && gz < a.Z;
    }
    if (tp.own) {
        T *d = sl + tp.sidx;
        if (FILL == PC_SMEM) {
            *reinterpret_cast<VT *>(d) = *reinterpret_cast<const VT *>(smc + ((q - ZR) * a.ncol + threadIdx.x * V));
        } else if (FILL == PC_REG) {
            if constexpr (ZR > 0) *reinterpret_cast<VT *>(d) = regc[q < 0 ? 0 : (q < ZR ? q : 0)];
        } else if (in_z) {
            copy_vec<T, V>(d, sp.fill_own);
        } else {
            set_vec<T, V>(d, bnd);
        }
    }
    const bool inside = FILL != PC_HALO;
    constexpr int XW = vec_xw<SH::R>();
    if (tp.duty != DUTY_NONE && (inside || SH::BOX)) {
        T *d = sl + tp.dsidx;
        if (!in_z || tp.duty == DUTY_BND_VEC || tp.duty == DUTY_BND_PAIR) {
            if (tp.duty == DUTY_FIELD_VEC || tp.duty == DUTY_BND_VEC) set_vec<T, V>(d, bnd);
            else
                static_for<0, XW>([&](auto JI) { d[decltype(JI)::value] = bnd; });
        } else if (tp.duty == DUTY_FIELD_VEC) {
            copy_vec<T, V>(d, sp.fill_duty);
        } else if (tp.duty == DUTY_XPAIR && inside && !PER_STEP && (FILL != PC_GLOBAL || !a.faces_cached_only)) {
            static_assert(XW == 2 || PER_STEP, "x-edge face buffers hold pairs: radius <= 2 for cached kernels");
            cp_async<sizeof(T) * 2>(d, sp.face_src);
        } else if constexpr (sizeof(T) * XW <= 16) {
            cp_async<sizeof(T) * XW>(d, sp.fill_duty);
        } else {  // fp64, 4 cells: two 16-byte copies
            cp_async<16>(d, sp.fill_duty);
            cp_async<16>(d + 16 / sizeof(T), sp.fill_duty + 16 / sizeof(T));
        }
    }
}

// Computes plane z (ring slot of plane z-RZ = slo) and stores it.
template <typename T, class SH, int V, int ZR, int D, bool PER_STEP, int STORE, int P>
__device__ __forceinline__ void vcompute_store(const PersistentArgs &a, const VecPlan &tp, int z, int slo, bool last,
                                               const T *ring, StepPtrs<T> &sp, T *smc,
                                               VecOf<T, V> (&regc)[ZR > 0 ? ZR : 1]) {
    using A = typename ScalarOps<T>::A;
    using VT = VecOf<T, V>;
    using PT = PairOf<T>;
    using RW = RowsOf<SH>;
    constexpr int RZ = SH::RZ;
    constexpr int R = SH::R;
    constexpr int S = vec_slots<RZ, D, P>();
    constexpr int NR = RW::count();
    if (tp.own) {
        A seg[NR][V + 2 * R];
        static_for<0, NR>([&](auto RI) {
            constexpr int r = decltype(RI)::value;
            constexpr int dzr = RW::dz(r), dyr = RW::dy(r);
            constexpr bool left = RW::minx(r) < 0, right = RW::maxx(r) > 0;
            int s = slo + RZ + dzr;
            s = s >= S ? s - S : s;
            const T *rp = ring + (s * a.plane + tp.sidx + dyr * a.PW);
            const VT c = *reinterpret_cast<const VT *>(rp);
            if constexpr (std::is_same<T, __nv_bfloat16>::value) {
                // two cells per conversion
                const __nv_bfloat162 *c2 = reinterpret_cast<const __nv_bfloat162 *>(&c);
                static_for<0, V / 2>([&](auto JI) {
                    constexpr int j = decltype(JI)::value;
                    const float2 f2 = __bfloat1622float2(c2[j]);
                    seg[r][R + 2 * j] = f2.x;
                    seg[r][R + 2 * j + 1] = f2.y;
                });
            } else {
                static_for<0, V>([&](auto JI) {
                    constexpr int j = decltype(JI)::value;
                    seg[r][R + j] = to_acc(c.v[j]);
                });
            }
            // x-neighbour cells: from the adjacent lanes' vectors of the same
            // row by warp shuffles; lanes at a row or warp edge read the ring.
            // fp64 reads them from the ring in every lane: one 8-byte load per
            // side instead of two 32-bit shuffles and a fallback load.
            const int lane = threadIdx.x & 31;
            if constexpr (std::is_same<T, double>::value) {
                if constexpr (left) static_for<0, R>([&](auto JI) {
                    constexpr int j = decltype(JI)::value;
                    seg[r][j] = rp[j - R];
                });
                if constexpr (right) static_for<0, R>([&](auto JI) {
                    constexpr int j = decltype(JI)::value;
                    seg[r][R + V + j] = rp[V + j];
                });
            } else {
            if constexpr (left) {
                static_for<0, R>([&](auto JI) {
                    constexpr int j = decltype(JI)::value;      // cell at offset j - R
                    constexpr int dist = R - j;                 // cells to the left
                    constexpr int back = (dist + V - 1) / V;    // lanes back
                    constexpr int el = V * back - dist;         // that lane's element
                    const A v = __shfl_up_sync(tp.own_mask, seg[r][R + el], back);
                    if (tp.rowpos >= back && lane >= back) seg[r][j] = v;
                    else seg[r][j] = to_acc(rp[j - R]);
                });
            }
            if constexpr (right) {
                static_for<0, R>([&](auto JI) {
                    constexpr int j = decltype(JI)::value;      // cell at offset V + j
                    constexpr int fwd = j / V + 1;              // lanes forward
                    constexpr int el = j - V * (fwd - 1);       // that lane's element
                    const A v = __shfl_down_sync(tp.own_mask, seg[r][R + el], fwd);
                    if (tp.rowpos + fwd < tp.nvx && lane + fwd < 32) seg[r][R + V + j] = v;
                    else seg[r][R + V + j] = to_acc(rp[V + j]);
                });
            }
            }
        });
        VT out;
        A accs[V];
        auto table_order = [&]() {
            if constexpr (std::is_same<A, float>::value && V % 2 == 0 && !SH::BOX && SH::R <= 2) {
                // fp32 accumulation (stars of radius <= 2): a term with dx = 0 updates two cells with
                // one packed fma (__ffma2_rn rounds each lane as fmaf does),
                // an x-shifted term one cell at a time; every cell still adds
                // its terms in table order from 0
                float2 acc2[V / 2];
#pragma unroll
                for (int k = 0; k < V / 2; ++k) acc2[k] = make_float2(0.f, 0.f);
                static_for<0, SH::NPTS>([&](auto II) {
                    constexpr int i = decltype(II)::value;
                    constexpr int r = RW::row_of(i);
                    constexpr int dx = SH::dx(i);
                    const float w = ScalarOps<T>::w(a, i);
                    if constexpr (dx == 0) {
                        const float2 w2 = make_float2(w, w);
#pragma unroll
                        for (int k = 0; k < V / 2; ++k)
                            acc2[k] = __ffma2_rn(w2, make_float2(seg[r][R + 2 * k], seg[r][R + 2 * k + 1]), acc2[k]);
                    } else {
                        static_for<0, V>([&](auto JI) {
                            constexpr int j = decltype(JI)::value;
                            if constexpr (j & 1) acc2[j / 2].y = fmaf(w, seg[r][R + j + dx], acc2[j / 2].y);
                            else acc2[j / 2].x = fmaf(w, seg[r][R + j + dx], acc2[j / 2].x);
                        });
                    }
                });
#pragma unroll
                for (int k = 0; k < V / 2; ++k) {
                    accs[2 * k] = acc2[k].x;
                    accs[2 * k + 1] = acc2[k].y;
                }
            } else {
                static_for<0, V>([&](auto JI) {
                    constexpr int j = decltype(JI)::value;
                    A acc = A(0);
                    static_for<0, SH::NPTS>([&](auto II) {
                        constexpr int i = decltype(II)::value;
                        constexpr int r = RW::row_of(i);
                        constexpr int col = R + j + SH::dx(i);
                        acc = fma(ScalarOps<T>::w(a, i), seg[r][col], acc);
                    });
                    accs[j] = acc;
                });
            }
        };
        if constexpr (std::is_same<T, double>::value && SH::NDIM == 3 && SH::R == 1 && !SH::BOX && V == 2 &&
                      PER_STEP) {
            if (a.iso) {
                // Equal neighbour weights: y = wc c + wn (sum of the six
                // neighbours).  The thread's cells are a (x0) and b (x0 + 1);
                // a's pair E + T = b(z) + a(z+1) is b's pair W + B on plane
                // z + 1 (a(z+1) + b(z)), so it is added once and carried:
                // 13 fp64 operations for the two cells instead of 14.  A
                // carried and a recomputed pair add the same two values, so
                // the result does not depend on where a block's planes start.
                constexpr int rc = RW::row_of(0), rS = RW::row_of(3), rN = RW::row_of(4);
                constexpr int rB = RW::row_of(5), rT = RW::row_of(6);
                const double av = seg[rc][1], bv = seg[rc][2];
                const double kn = bv + seg[rT][1];                       // E + T of a
                const double kp = z == 0 ? av + seg[rB][2] : sp.kz;      // W + B of b
                const double sa = ((kn + seg[rc][0]) + (seg[rS][1] + seg[rN][1])) + seg[rB][1];
                const double sb = ((kp + seg[rc][3]) + (seg[rS][2] + seg[rN][2])) + seg[rT][2];
                sp.kz = kn;
                accs[0] = fma(a.wn, sa, a.wc * av);
                accs[1] = fma(a.wn, sb, a.wc * bv);
            } else {
                table_order();
            }
        } else {
            table_order();
        }
        if constexpr (std::is_same<T, __nv_bfloat16>::value) {
            // round to nearest even, two cells per conversion
            __nv_bfloat162 *o2 = reinterpret_cast<__nv_bfloat162 *>(&out);
            static_for<0, V / 2>([&](auto JI) {
                constexpr int j = decltype(JI)::value;
                o2[j] = __floats2bfloat162_rn(accs[2 * j], accs[2 * j + 1]);
            });
        } else {
            static_for<0, V>([&](auto JI) {
                constexpr int j = decltype(JI)::value;
                out.v[j] = from_acc<T>(accs[j]);
            });
        }
        bool to_field;
        if (STORE == PC_REG) {
            if constexpr (ZR > 0) regc[z < ZR ? z : 0] = out;
            to_field = last || tp.field_shell || (z < RZ && tp.has_b) || (z >= tp.tz - RZ && tp.has_t);
        } else if (STORE == PC_SMEM) {
            *reinterpret_cast<VT *>(smc + ((z - ZR) * a.ncol + threadIdx.x * V)) = out;
            to_field = last || tp.field_shell || (z < RZ && tp.has_b) || (z >= tp.tz - RZ && tp.has_t);
        } else {
            to_field = true;
        }
        if (to_field) *reinterpret_cast<VT *>(sp.store_own) = out;
        if (!PER_STEP && (STORE != PC_GLOBAL || !a.faces_cached_only)) {
            if (tp.wface) {
                PT x; x.v[0] = out.v[0]; x.v[1] = out.v[V >= 2 ? 1 : 0];
                *reinterpret_cast<PT *>(sp.face_dst_w) = x;
            }
            if (tp.eface) {
                PT x; x.v[0] = out.v[V >= 2 ? V - 2 : 0]; x.v[1] = out.v[V - 1];
                *reinterpret_cast<PT *>(sp.face_dst_e) = x;
            }
        }
    }
    sp.store_own += a.XY;
    sp.face_dst_w += 2 * a.tymax;
    sp.face_dst_e += 2 * a.tymax;
}

// Starts the copy of plane q (= z + RZ + D) into its slot; one cp.async group.
template <typename T, class SH, int V, int ZR, int D, bool PER_STEP, int FILL, int P>
__device__ __forceinline__ void vfill_next(const PersistentArgs &a, const VecPlan &tp, int q, int slo_q, T *ring,
                                           StepPtrs<T> &sp, const T *smc,
                                           const VecOf<T, V> (&regc)[ZR > 0 ? ZR : 1]) {
    constexpr int S = vec_slots<SH::RZ, D, P>();
    int s = slo_q;
    s = s >= S ? s - S : s;
    vfill_fast<T, SH, V, ZR, PER_STEP, FILL>(a, tp, q, ring + s * a.plane, sp, smc, regc);
    sp.fill_own += a.XY;
    sp.fill_duty += a.XY;
    sp.face_src += 2 * a.tymax;
    cp_async_commit();
}

// One plane per barrier (the remainder of a segment).
template <typename T, class SH, int V, int ZR, int D, bool PER_STEP, int STORE, int FILL, int P>
__device__ __forceinline__ void vplane_fast(const PersistentArgs &a, const VecPlan &tp, int z, int &slo, bool last,
                                            T *ring, StepPtrs<T> &sp, T *smc,
                                            VecOf<T, V> (&regc)[ZR > 0 ? ZR : 1]) {
    constexpr int RZ = SH::RZ;
    constexpr int S = vec_slots<RZ, D, P>();
    cp_async_wait<D - 1>();
    __syncthreads();
    vcompute_store<T, SH, V, ZR, D, PER_STEP, STORE, P>(a, tp, z, slo, last, ring, sp, smc, regc);
    vfill_next<T, SH, V, ZR, D, PER_STEP, FILL, P>(a, tp, z + RZ + D, slo + 2 * RZ + D, ring, sp, smc, regc);
    slo = slo + 1 == S ? 0 : slo + 1;
}

// P planes per barrier (z .. z+P-1): the block synchronises once per P
// planes and every thread has P independent planes of loads and FMAs in
// flight between two barriers.  Slot safety: the iteration reads ring slots
// slo .. slo+2RZ+P-1 and fills slots slo+2RZ+D .. slo+2RZ+D+P-1; both ranges
// lie within one turn of the S = 2RZ+P+D slots, so they never overlap, and
// after wait_group<D-P> every plane up to z+P-1+RZ has landed.
template <typename T, class SH, int V, int ZR, int D, bool PER_STEP, int STORE, int FILL, int P>
__device__ __forceinline__ void vplane_multi(const PersistentArgs &a, const VecPlan &tp, int z, int &slo, bool last,
                                             T *ring, StepPtrs<T> &sp, T *smc,
                                             VecOf<T, V> (&regc)[ZR > 0 ? ZR : 1]) {
    constexpr int RZ = SH::RZ;
    constexpr int S = vec_slots<RZ, D, P>();
    static_assert(P >= 1 && P <= D, "planes per barrier");
    cp_async_wait<D - P>();
    __syncthreads();
    // each plane's fill follows its compute, spreading the copies over the
    // group: the filled slots (slo + 2RZ + D + p, i.e. the group's last P
    // slots before slo) are read by no plane of this group
    static_for<0, P>([&](auto PI) {
        constexpr int p = decltype(PI)::value;
        int s = slo + p;
        s = s >= S ? s - S : s;
        vcompute_store<T, SH, V, ZR, D, PER_STEP, STORE, P>(a, tp, z + p, s, last, ring, sp, smc, regc);
        vfill_next<T, SH, V, ZR, D, PER_STEP, FILL, P>(a, tp, z + p + RZ + D, slo + 2 * RZ + D + p, ring, sp, smc,
                                                      regc);
    });
    slo = slo + P >= S ? slo + P - S : slo + P;
}

template <typename T, class SH, int V, int ZR, int D, bool PER_STEP, int STORE, int FILL, int P>
__device__ __forceinline__ void vsegment(const PersistentArgs &a, const VecPlan &tp, int z0, int z1, int &slo,
                                         bool last, T *ring, StepPtrs<T> &sp, T *smc,
                                         VecOf<T, V> (&regc)[ZR > 0 ? ZR : 1]) {
    int z = z0;
    for (; z + P <= z1; z += P)
        vplane_multi<T, SH, V, ZR, D, PER_STEP, STORE, FILL, P>(a, tp, z, slo, last, ring, sp, smc, regc);
    for (; z < z1; ++z)
        vplane_fast<T, SH, V, ZR, D, PER_STEP, STORE, FILL, P>(a, tp, z, slo, last, ring, sp, smc, regc);
}

// One Jacobi step of one tile: fill the ring with planes -RZ.., then walk
// the tile's planes in segments where both the store class of plane z and
// the fill class of plane z+RZ+D are fixed.  `sb` is the ring slot of plane
// -RZ; returns the slot for the next step.
template <typename T, class SH, int V, int ZR, int D, bool PER_STEP, int P = 2>
__device__ __forceinline__ int vec_step(const PersistentArgs &a, const VecPlan &tp, long long k, bool last,
                                        int sb, T *ring, T *smc, VecOf<T, V> (&regc)[ZR > 0 ? ZR : 1]) {
    constexpr int RZ = SH::RZ;
    constexpr int S = vec_slots<RZ, D, P>();
    constexpr int LEAD = RZ + D;  // fill distance ahead of the plane being computed
    const int src = (int)(k & 1);
    const T *fs = static_cast<const T *>(a.field[src]);
    const T *hs = static_cast<const T *>(a.faces[src]);
    T *fd = static_cast<T *>(a.field[src ^ 1]);
    T *hd = static_cast<T *>(a.faces[src ^ 1]);
    const int tz = tp.tz;
    const int zc = PER_STEP ? 0 : min(tz, ZR + a.zs);  // cached planes
    StepPtrs<T> sp;
    // prologue fills: planes -RZ .. RZ+D-1
#pragma unroll
    for (int j = 0; j < 2 * RZ + D; ++j) {
        const int p = j - RZ;
        int s = sb + j;
        s = s >= S ? s - S : s;
        T *sl = ring + s * a.plane;
        sp.fill_own = fs + tp.gxy + (long long)(tp.z0 + p) * a.XY;
        sp.fill_duty = fs + tp.dgxy + (long long)(tp.z0 + p) * a.XY;
        sp.face_src = hs + tp.dface + (long long)p * a.tymax * 2;
        if (p >= tz + RZ) {
        } else if (p < 0 || p >= tz) {
            vfill_fast<T, SH, V, ZR, PER_STEP, PC_HALO>(a, tp, p, sl, sp, smc, regc);
        } else if (!PER_STEP && p < ZR) {
            vfill_fast<T, SH, V, ZR, PER_STEP, PC_REG>(a, tp, p, sl, sp, smc, regc);
        } else if (!PER_STEP && p < zc) {
            vfill_fast<T, SH, V, ZR, PER_STEP, PC_SMEM>(a, tp, p, sl, sp, smc, regc);
        } else {
            vfill_fast<T, SH, V, ZR, PER_STEP, PC_GLOBAL>(a, tp, p, sl, sp, smc, regc);
        }
        cp_async_commit();
    }
    sp.fill_own = fs + tp.gxy + (long long)(tp.z0 + LEAD) * a.XY;
    sp.fill_duty = fs + tp.dgxy + (long long)(tp.z0 + LEAD) * a.XY;
    sp.face_src = hs + tp.dface + (long long)LEAD * a.tymax * 2;
    sp.store_own = fd + tp.gxy + (long long)tp.z0 * a.XY;
    sp.face_dst_w = hd + tp.wface_off;
    sp.face_dst_e = hd + tp.eface_off;
    int slo = sb;
    // register-cached planes (compile-time index): fill class decided per plane
    if (!PER_STEP) {
#pragma unroll
        for (int z = 0; z < ZR; ++z) {
            if (z < tz) {
                const int q = z + LEAD;
                if (q >= tz + RZ) vplane_fast<T, SH, V, ZR, D, PER_STEP, PC_REG, PC_NONE, P>(a, tp, z, slo, last, ring, sp, smc, regc);
                else if (q >= tz) vplane_fast<T, SH, V, ZR, D, PER_STEP, PC_REG, PC_HALO, P>(a, tp, z, slo, last, ring, sp, smc, regc);
                else if (q < ZR) vplane_fast<T, SH, V, ZR, D, PER_STEP, PC_REG, PC_REG, P>(a, tp, z, slo, last, ring, sp, smc, regc);
                else if (q < zc) vplane_fast<T, SH, V, ZR, D, PER_STEP, PC_REG, PC_SMEM, P>(a, tp, z, slo, last, ring, sp, smc, regc);
                else vplane_fast<T, SH, V, ZR, D, PER_STEP, PC_REG, PC_GLOBAL, P>(a, tp, z, slo, last, ring, sp, smc, regc);
            }
        }
    }
    // runtime planes: [zr0, zc) shared-memory cached, [zc, tz) global
    const int zr0 = PER_STEP ? 0 : min(ZR, tz);
    auto bound = [&](int q_limit) { return max(zr0, min(tz, q_limit - LEAD)); };
    // fill class of plane z+LEAD changes at q = zc (smem->global), q = tz (->halo), q = tz+RZ (->none)
    const int b_sg = bound(zc), b_gh = bound(tz), b_hn = bound(tz + RZ);
    // z ranges: the store class changes at zc
    auto run = [&](int z0, int z1, auto STORE_C) {
        constexpr int STORE = decltype(STORE_C)::value;
        // sub-ranges by fill class
        const int e1 = min(z1, max(z0, b_sg));
        const int e2 = min(z1, max(z0, b_gh));
        const int e3 = min(z1, max(z0, b_hn));
        if (!PER_STEP) vsegment<T, SH, V, ZR, D, PER_STEP, STORE, PC_SMEM, P>(a, tp, z0, e1, slo, last, ring, sp, smc, regc);
        else vsegment<T, SH, V, ZR, D, PER_STEP, STORE, PC_GLOBAL, P>(a, tp, z0, e1, slo, last, ring, sp, smc, regc);
        vsegment<T, SH, V, ZR, D, PER_STEP, STORE, PC_GLOBAL, P>(a, tp, max(z0, e1), e2, slo, last, ring, sp, smc, regc);
        vsegment<T, SH, V, ZR, D, PER_STEP, STORE, PC_HALO, P>(a, tp, max(z0, e2), e3, slo, last, ring, sp, smc, regc);
        vsegment<T, SH, V, ZR, D, PER_STEP, STORE, PC_NONE, P>(a, tp, max(z0, e3), z1, slo, last, ring, sp, smc, regc);
    };
    if (!PER_STEP) run(zr0, max(zr0, zc), std::integral_constant<int, PC_SMEM>{});
    run(max(zr0, zc), tz, std::integral_constant<int, PC_GLOBAL>{});
    return (sb + tz + 2 * RZ) % S;
}

// Before step 0: load the tile's cached planes (registers and shared memory)
// from field[0] and publish its x-edge pairs into faces[0].
template <typename T, class SH, int V, int ZR>
__device__ __forceinline__ void vec_prologue(const PersistentArgs &a, const VecPlan &tp, T *smc,
                                             VecOf<T, V> (&regc)[ZR > 0 ? ZR : 1]) {
    using VT = VecOf<T, V>;
    using PT = PairOf<T>;
    const T *f0 = static_cast<const T *>(a.field[0]);
    T *h0 = static_cast<T *>(a.faces[0]);
    if (!tp.own) return;
#pragma unroll
    for (int p = 0; p < (ZR > 0 ? ZR : 1); ++p)
        if (ZR > 0 && p < tp.tz)
            regc[p] = *reinterpret_cast<const VT *>(f0 + (long long)(tp.z0 + p) * a.XY + tp.gxy);
    for (int p = 0; p < tp.tz; ++p) {
        const bool in_smem = p >= ZR && p < ZR + a.zs;
        if (!in_smem && !tp.wface && !tp.eface) {
            if (p >= ZR) break;
            continue;
        }
        const VT v = *reinterpret_cast<const VT *>(f0 + (long long)(tp.z0 + p) * a.XY + tp.gxy);
        if (in_smem) *reinterpret_cast<VT *>(smc + ((long long)(p - ZR) * a.ncol + threadIdx.x * V)) = v;
        const long long fz = (long long)p * a.tymax * 2;
        if (tp.wface) {
            PT x; x.v[0] = v.v[0]; x.v[1] = v.v[V >= 2 ? 1 : 0];
            *reinterpret_cast<PT *>(h0 + tp.wface_off + fz) = x;
        }
        if (tp.eface) {
            PT x; x.v[0] = v.v[V >= 2 ? V - 2 : 0]; x.v[1] = v.v[V - 1];
            *reinterpret_cast<PT *>(h0 + tp.eface_off + fz) = x;
        }
    }
}

template <typename T, class SH, int NT, int V, int ZR, int D, bool PER_STEP, int P, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB) perks_stencil_vec_kernel(const __grid_constant__ PersistentArgs a) {
    using VT = VecOf<T, V>;
    using PT = PairOf<T>;
    constexpr int RZ = SH::RZ;
    constexpr int S = vec_slots<RZ, D, P>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *ring = reinterpret_cast<T *>(smem_raw);
    T *smc = ring + (long long)S * a.plane;
    VT regc[ZR > 0 ? ZR : 1];

    const VecPlan tp = make_vec_plan<SH, V, PER_STEP>(a, blockIdx.x);
    unsigned long long epoch = 0;

    if (!PER_STEP) {
        trace_mark(a, -1, 0);
        vec_prologue<T, SH, V, ZR>(a, tp, smc, regc);
        trace_mark(a, -1, 1);
        if (!grid_barrier(a.bar, gridDim.x, epoch, a.err, a.timeout_ns)) return;
    }

    int sb = 0;
    for (long long k = 0; k < a.steps; ++k) {
        const bool last = (k + 1 == a.steps);
        if (!PER_STEP) trace_mark(a, k, 0);
        if (PER_STEP && a.lin_cols > 0) {
            // balanced shares: this block's run of column-planes [s0, s1), as
            // pieces of consecutive tile columns; halos come from the field,
            // so any piece of a column is computed like a tile of its own
            const long long L = (long long)a.lin_cols * a.Z;
            long long s0 = L * blockIdx.x / gridDim.x;
            const long long s1 = L * (blockIdx.x + 1) / gridDim.x;
            while (s0 < s1) {
                const int c = (int)(s0 / a.Z);
                const long long cz = (long long)c * a.Z;
                VecPlan sp = make_vec_plan<SH, V, PER_STEP>(a, c);
                sp.z0 = (int)(s0 - cz);
                sp.tz = (int)(min(s1, cz + a.Z) - s0);
                sb = vec_step<T, SH, V, ZR, D, PER_STEP, P>(a, sp, k, last, sb, ring, smc, regc);
                s0 = cz + a.Z;
                if (s0 < s1) {  // the next piece's prologue refills ring slots still being read
                    cp_async_wait_all();
                    __syncthreads();
                }
            }
        } else {
            sb = vec_step<T, SH, V, ZR, D, PER_STEP, P>(a, tp, k, last, sb, ring, smc, regc);
        }
        if (!PER_STEP) trace_mark(a, k, 1);
        if (!last) {
            if (!grid_barrier(a.bar, gridDim.x, epoch, a.err, a.timeout_ns)) break;
        }
    }
    cp_async_wait_all();
}

// Registry entry of one instantiation of the vectorised kernel (MINB: blocks
// per SM the register allocation must allow).
template <typename T, class SH, int NT, int V, int ZR, int D, bool PS, int P = 2, int MINB = 1>
KernelEntry vec_entry(int dtype, int shape) {
    KernelEntry e;
    e.dtype = dtype;
    e.shape = shape;
    e.per_step = PS;
    e.fn = perks_stencil_vec_kernel<T, SH, NT, V, ZR, D, PS, P, MINB>;
    e.nt = NT;
    e.zr = ZR;
    e.d = D;
    e.v = V;
    e.p = P;
    return e;
}

}  // namespace perks
