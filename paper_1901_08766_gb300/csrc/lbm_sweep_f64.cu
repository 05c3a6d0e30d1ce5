// Sweep instantiations for LBM_F64 storage (cells per thread 1 and 2).
#include "lbm_sweep.cuh"

namespace lbm {

cudaError_t launch_sweep_f64(int vec, int grid, int warps, cudaStream_t st, const SweepArgs &a,
                               int s) {
  if (vec == 1) return launch_sweep_t<LBM_F64, 1>(grid, warps, st, a, s);
  if (vec == 2) return launch_sweep_t<LBM_F64, 2>(grid, warps, st, a, s);
  return cudaErrorInvalidValue;
}

int max_blocks_f64(int vec, int warps) {
  if (vec == 1) return max_blocks_t<LBM_F64, 1>(warps);
  if (vec == 2) return max_blocks_t<LBM_F64, 2>(warps);
  return 0;
}

}  // namespace lbm
