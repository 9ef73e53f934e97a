// lbm_fused_tma_f32_mrt.cu -- instances of the single-pass TMA step:
// FP32 storage, MRT collision.
#include "lbm_fused_tma.cuh"

namespace pplbm {

cudaError_t fused_tma_f32_mrt(int tx, int ty, int eos, const StepArgs& a, const CUtensorMap* map,
                             const LatDev* lat0, int grid, cudaStream_t st, bool q, int* occ) {
    return fused_tma_any<StoreF32, true>(tx, ty, eos, a, map, lat0, grid, st, q, occ);
}

}  // namespace pplbm
