// Instantiations of the vectorised persistent stencil kernel: the 3d7pt and 2d5pt kernels,
// bf16 storage (2 bytes: V = 8 cells per thread, prefetch depth 16 planes; 16-byte vectors).
#include "stencil_registry.h"
#include "stencil_vec.cuh"

namespace perks {

void register_vec_bf16_core(std::vector<KernelEntry> &out) {
    out.push_back(vec_entry<__nv_bfloat16, S3d7, 512, 8, 0, 16, false>(PERKS_BF16, SH_3D7));
    out.push_back(vec_entry<__nv_bfloat16, S3d7, 512, 8, 0, 16, false, 4>(PERKS_BF16, SH_3D7));
    out.push_back(vec_entry<__nv_bfloat16, S3d7, 512, 8, 8, 16, false>(PERKS_BF16, SH_3D7));
    out.push_back(vec_entry<__nv_bfloat16, S3d7, 512, 8, 8, 16, false, 4>(PERKS_BF16, SH_3D7));
    out.push_back(vec_entry<__nv_bfloat16, S3d7, 512, 8, 0, 16, true>(PERKS_BF16, SH_3D7));
    out.push_back(vec_entry<__nv_bfloat16, S3d7, 512, 8, 0, 16, true, 4>(PERKS_BF16, SH_3D7));
    out.push_back(vec_entry<__nv_bfloat16, S2d5, 256, 8, 0, 16, false>(PERKS_BF16, SH_2D5));
    out.push_back(vec_entry<__nv_bfloat16, S2d5, 256, 8, 0, 16, false, 4>(PERKS_BF16, SH_2D5));
    out.push_back(vec_entry<__nv_bfloat16, S2d5, 256, 8, 16, 16, false>(PERKS_BF16, SH_2D5));
    out.push_back(vec_entry<__nv_bfloat16, S2d5, 256, 8, 16, 16, false, 4>(PERKS_BF16, SH_2D5));
    out.push_back(vec_entry<__nv_bfloat16, S2d5, 256, 8, 0, 16, true>(PERKS_BF16, SH_2D5));
    out.push_back(vec_entry<__nv_bfloat16, S2d5, 256, 8, 0, 16, true, 4>(PERKS_BF16, SH_2D5));
}

}  // namespace perks
