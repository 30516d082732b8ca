// pf_lg16_fwd.cu -- forward-pass kernel variants for the 16-dimensional linear-Gaussian
// model with H = I (LGSplit<16, 2>: each particle spread over 2 lanes).  One translation unit
// per model and pass so the build compiles in parallel.
#include "pf_kernels.cuh"

namespace smc2 {

pf_kernel_fn lookup_lg16_fwd(int P, int regs) {
    using Mdl = LGSplit<16, 2>;
#define SMC2_CASE(PP, RR) \
    if (P == PP && regs == RR) return &launch_forward<Mdl, PP, RR>;
    SMC2_PF_VARIANTS(SMC2_CASE)
#undef SMC2_CASE
    return nullptr;
}

pf_multi_fn lookup_lg16_fwd_multi(int P, int regs) {
    using Mdl = LGSplit<16, 2>;
#define SMC2_CASE(PP, RR) \
    if (P == PP && regs == RR) return &launch_forward_multi<Mdl, PP, RR>;
    SMC2_PF_VARIANTS(SMC2_CASE)
#undef SMC2_CASE
    return nullptr;
}

}  // namespace smc2
