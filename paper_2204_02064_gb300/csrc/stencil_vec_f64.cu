// Instantiations of the vectorised persistent stencil kernel for f64 storage
// (V = 2 cells per thread = 16 bytes, prefetch depth 8 planes).
#include "stencil_registry.h"
#include "stencil_vec.cuh"

namespace perks {

namespace {

template <class SH, int NT, int ZR, bool PS>
KernelEntry make(int shape) {
    KernelEntry e;
    e.dtype = PERKS_F64;
    e.shape = shape;
    e.per_step = PS;
    e.fn = perks_stencil_vec_kernel<double, SH, NT, 2, ZR, 8, PS>;
    e.nt = NT;
    e.zr = ZR;
    e.d = 8;
    e.v = 2;
    return e;
}

}  // namespace

void register_vec_f64(std::vector<KernelEntry> &out) {
    out.push_back(make<S3d7, 512, 0, false>(SH_3D7));
    out.push_back(make<S3d7, 512, 8, false>(SH_3D7));
    out.push_back(make<S3d7, 512, 0, true>(SH_3D7));
    out.push_back(make<S2d5, 256, 0, false>(SH_2D5));
    out.push_back(make<S2d5, 256, 16, false>(SH_2D5));
    out.push_back(make<S2d5, 256, 0, true>(SH_2D5));
    out.push_back(make<S2d9, 256, 0, false>(SH_2D9));
    out.push_back(make<S2d9, 256, 0, true>(SH_2D9));
    out.push_back(make<S2d25, 256, 0, false>(SH_2D25));
    out.push_back(make<S2d25, 256, 0, true>(SH_2D25));
    out.push_back(make<S2ds9, 256, 0, false>(SH_2DS9));
    out.push_back(make<S3d27, 512, 0, false>(SH_3D27));
    out.push_back(make<S3d13, 512, 0, false>(SH_3D13));
}

}  // namespace perks
