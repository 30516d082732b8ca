// pf_opt_fwd.cu -- forward-pass kernel variants for one model shape
// (LGOpt).  One translation unit per model and pass so the build compiles in parallel; the
// _multi lookup gives the persistent multi-job kernel of the same variant.
#include "pf_kernels.cuh"

namespace smc2 {

pf_kernel_fn lookup_opt_fwd(int P, int regs) {
    using Mdl = LGOpt;
#define SMC2_CASE(PP, RR) \
    if (P == PP && regs == RR) return &launch_forward<Mdl, PP, RR>;
    SMC2_PF_VARIANTS(SMC2_CASE)
#undef SMC2_CASE
    return nullptr;
}

pf_multi_fn lookup_opt_fwd_multi(int P, int regs) {
    using Mdl = LGOpt;
#define SMC2_CASE(PP, RR) \
    if (P == PP && regs == RR) return &launch_forward_multi<Mdl, PP, RR>;
    SMC2_PF_VARIANTS(SMC2_CASE)
#undef SMC2_CASE
    return nullptr;
}

}  // namespace smc2
