// Rollout kernel instantiations for the double integrator (model 1).
#include "rollout_kernel.cuh"

namespace bss {

template <>
cudaError_t prepare_model<1>(const DevParams& dp, int P, bool comp, bool full, RollLaunch& L, const ConSet*)
{
    if (full) return plan_model<1, true, true>(dp, P, L);
    return comp ? plan_model<1, true, false>(dp, P, L) : plan_model<1, false, false>(dp, P, L);
}

template <>
cudaError_t launch_model_variant<1>(const DevParams& dp, const RollIO& io, const TailIO& tail, const ConSet& cs, int P,
                                     bool comp, bool full, const RollLaunch& L, cudaStream_t st)
{
    if (full) return launch_model<1, true, true>(dp, io, tail, cs, P, L, st);
    return comp ? launch_model<1, true, false>(dp, io, tail, cs, P, L, st)
                : launch_model<1, false, false>(dp, io, tail, cs, P, L, st);
}

}  // namespace bss
