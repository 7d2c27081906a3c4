// Rollout kernel instantiations for the 6-state bicycle (model 0).
#include "rollout_kernel.cuh"

namespace bss {

// The compensated racing-barrier variant has a second build for costs that weight only v_x, e_psi
// and e_y (the racing cost), used when nothing is recorded: it merges and costs those three means only.
static bool racing_cost_only(const DevParams& dp)
{
    return !dp.record && (dp.mean_mask & ~kRacingCostMask) == 0;
}

// The full-belief variant has a second build for a constraint set on the road plane (e_y and s only)
// with a cost on v_x, e_psi and e_y, without re-sampling or recording: it keeps those four means and
// the covariance of (e_y, s) only.
static bool plane_constraints_only(const DevParams& dp, const ConSet* cs)
{
    if (!cs || cs->n < 1 || dp.resample || dp.record || (dp.mean_mask & ~kPlaneMeanMask) != 0) return false;
    for (int q = 0; q < cs->n; ++q)
        for (int l = 0; l < kNxMax; ++l)
            if (!((kPlaneConMask >> l) & 1) && (cs->a[q][l] != 0.0f || cs->o[q][l] != 0.0f)) return false;
    return true;
}

template <>
cudaError_t prepare_model<0>(const DevParams& dp, int P, bool comp, bool full, RollLaunch& L, const ConSet* cs)
{
    if (full && comp && plane_constraints_only(dp, cs)) return plan_model<0, true, true, kPlaneMeanMask>(dp, P, L);
    if (full) return plan_model<0, true, true>(dp, P, L);
    if (comp && racing_cost_only(dp)) return plan_model<0, true, false, kRacingCostMask>(dp, P, L);
    return comp ? plan_model<0, true, false>(dp, P, L) : plan_model<0, false, false>(dp, P, L);
}

template <>
cudaError_t launch_model_variant<0>(const DevParams& dp, const RollIO& io, const TailIO& tail, const ConSet& cs, int P,
                                     bool comp, bool full, const RollLaunch& L, cudaStream_t st)
{
    if (full) {
        if (L.cost_mask == 0) return launch_model<0, true, true>(dp, io, tail, cs, P, L, st);
        if (!comp || L.cost_mask != kPlaneMeanMask || !plane_constraints_only(dp, &cs)) return cudaErrorInvalidValue;
        return launch_model<0, true, true, kPlaneMeanMask>(dp, io, tail, cs, P, L, st);
    }
    if (L.cost_mask != 0) {  // planned for the racing cost: valid only while the parameters still allow it
        if (!comp || L.cost_mask != kRacingCostMask || !racing_cost_only(dp)) return cudaErrorInvalidValue;
        return launch_model<0, true, false, kRacingCostMask>(dp, io, tail, cs, P, L, st);
    }
    return comp ? launch_model<0, true, false>(dp, io, tail, cs, P, L, st)
                : launch_model<0, false, false>(dp, io, tail, cs, P, L, st);
}

}  // namespace bss
