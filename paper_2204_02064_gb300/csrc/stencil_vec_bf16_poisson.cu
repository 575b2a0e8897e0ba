// Instantiations of the vectorised persistent stencil kernel: the 3-D 19-point
// "poisson" stencil (centre, faces, edges), bf16 storage (2 bytes: V = 8 cells per thread, prefetch depth 16 planes;
// 16-byte vectors).
#include "stencil_registry.h"
#include "stencil_vec.cuh"

namespace perks {

void register_vec_bf16_poisson(std::vector<KernelEntry> &out) {
    out.push_back(vec_entry<__nv_bfloat16, S3d19, 512, 8, 0, 16, false>(PERKS_BF16, SH_3D19));
    out.push_back(vec_entry<__nv_bfloat16, S3d19, 512, 8, 0, 16, true>(PERKS_BF16, SH_3D19));
}

}  // namespace perks
