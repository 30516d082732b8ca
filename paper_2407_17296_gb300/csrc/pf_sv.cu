// pf_sv.cu -- particle-filter kernel instantiations for one model shape
// (family 1, d_x = 1, d_y = 1).  Split per model so the build compiles in parallel.
#include "pf_kernels.cuh"

namespace smc2 {

pf_launch_fn lookup_pf_sv(int P) {
    using Mdl = SV;
    switch (P) {
        case 1: return &launch_pf<Mdl, 1>;
        case 2: return &launch_pf<Mdl, 2>;
        case 4: return &launch_pf<Mdl, 4>;
        case 8: return &launch_pf<Mdl, 8>;
        default: return nullptr;
    }
}

}  // namespace smc2
