// Registry of compiled persistent-stencil kernels, filled by the
// translation units that instantiate them.
#pragma once

#include <vector>

#include "stencil_kernels.cuh"

namespace perks {

using S2d5 = Shape<2, 1, false>;
using S3d7 = Shape<3, 1, false>;
using S2d9 = Shape<2, 1, true>;
using S2d25 = Shape<2, 2, true>;
using S2ds9 = Shape<2, 2, false>;
using S3d27 = Shape<3, 1, true>;
using S3d13 = Shape<3, 2, false>;
using S3d19 = Shape<3, 1, 2>;  // "poisson": box without corners
using S2d13 = Shape<2, 3, 0>;  // high-order 2-D stars (cache-free body only)
using S2d17 = Shape<2, 4, 0>;

// shape ids (the order of the table in stencil.cu)
enum ShapeId : int { SH_2D5 = 0, SH_3D7, SH_2D9, SH_2D25, SH_2DS9, SH_3D27, SH_3D13, SH_3D19, SH_2D13, SH_2D17, SH_COUNT };

using PersistentFn = void (*)(PersistentArgs);

struct KernelEntry {
    int dtype = 0;          // PERKS_F64 / PERKS_F32 / PERKS_BF16
    int shape = 0;          // ShapeId
    bool per_step = false;  // one launch per step (no caches, no barrier)
    PersistentFn fn = nullptr;
    int nt = 0, zr = 0, d = 0;
    int v = 1;              // cells per thread along x (1: scalar kernel)
    int p = 2;              // planes per block barrier (vectorised kernel)
};

void register_vec_f64_core(std::vector<KernelEntry> &out);
void register_vec_f64_box2d(std::vector<KernelEntry> &out);
void register_vec_f64_box3d(std::vector<KernelEntry> &out);
void register_vec_f32_core(std::vector<KernelEntry> &out);
void register_vec_f32_box2d(std::vector<KernelEntry> &out);
void register_vec_f32_box3d(std::vector<KernelEntry> &out);
void register_vec_bf16_core(std::vector<KernelEntry> &out);
void register_vec_bf16_box2d(std::vector<KernelEntry> &out);
void register_vec_bf16_box3d(std::vector<KernelEntry> &out);
void register_vec_f64_poisson(std::vector<KernelEntry> &out);
void register_vec_f32_poisson(std::vector<KernelEntry> &out);
void register_vec_bf16_poisson(std::vector<KernelEntry> &out);
void register_vec_star2d_hi(std::vector<KernelEntry> &out);

struct TileKernelEntry;  // stencil_tile.cuh
void register_tile_kernels(std::vector<TileKernelEntry> &out);

}  // namespace perks
