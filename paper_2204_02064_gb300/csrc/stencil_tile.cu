// Instantiations of the resident-tile persistent stencil kernel (the whole
// tile in shared memory for all steps): 2d5pt and 3d7pt in fp64, fp32 and
// bf16 storage, with 256 or 512 threads per block, 2 or 4 planes per chunk
// and 1 or 2 rows per thread (tile_entry<T, shape, threads, planes, rows>).
#include "stencil_registry.h"
#include "stencil_tile.cuh"

namespace perks {

void register_tile_kernels(std::vector<TileKernelEntry> &out) {
    out.push_back(tile_entry<double, S3d7, 512, 4, 1>(PERKS_F64, SH_3D7));
    out.push_back(tile_entry<double, S3d7, 256, 2, 2>(PERKS_F64, SH_3D7));
    out.push_back(tile_entry<float, S3d7, 512, 4, 1>(PERKS_F32, SH_3D7));
    out.push_back(tile_entry<float, S3d7, 512, 2, 2>(PERKS_F32, SH_3D7));
    out.push_back(tile_entry<float, S3d7, 256, 4, 2>(PERKS_F32, SH_3D7));
    out.push_back(tile_entry<__nv_bfloat16, S3d7, 512, 4, 1>(PERKS_BF16, SH_3D7));
    out.push_back(tile_entry<__nv_bfloat16, S3d7, 512, 2, 2>(PERKS_BF16, SH_3D7));
    out.push_back(tile_entry<__nv_bfloat16, S3d7, 256, 4, 2>(PERKS_BF16, SH_3D7));
    out.push_back(tile_entry<double, S2d5, 512, 4, 1>(PERKS_F64, SH_2D5));
    out.push_back(tile_entry<double, S2d5, 256, 2, 1>(PERKS_F64, SH_2D5));
    out.push_back(tile_entry<float, S2d5, 512, 4, 1>(PERKS_F32, SH_2D5));
    out.push_back(tile_entry<float, S2d5, 256, 2, 1>(PERKS_F32, SH_2D5));
    out.push_back(tile_entry<__nv_bfloat16, S2d5, 512, 4, 1>(PERKS_BF16, SH_2D5));
    out.push_back(tile_entry<__nv_bfloat16, S2d5, 256, 2, 1>(PERKS_BF16, SH_2D5));
}

}  // namespace perks
