// Sweep instantiations for LBM_F16S storage (cells per thread 4 and 8; direct
// TMA-staged and register-prefetched row loads).
#include "lbm_sweep_tma.cuh"

namespace lbm {

cudaError_t launch_sweep_f16s(int vec, int pipe, int grid, int warps, cudaStream_t st,
                               const SweepArgs &a, int s, bool def) {
  if (pipe == 0 || pipe == 3 || pipe == 4) {  // the direct sweep at its register budgets
    if (vec == 4) return launch_sweep_t<LBM_F16S, 4>(grid, warps, st, a, s, def, pipe);
    if (vec == 8) return launch_sweep_t<LBM_F16S, 8>(grid, warps, st, a, s, def, pipe);
  } else if (pipe == 2) {
    if (vec == 4) return launch_sweep_pf_t<LBM_F16S, 4>(grid, warps, st, a, s);
    if (vec == 8) return launch_sweep_pf_t<LBM_F16S, 8>(grid, warps, st, a, s);
  } else {
    if (vec == 4) return launch_sweep_tma_t<LBM_F16S, 4>(grid, warps, st, a, s);
    if (vec == 8) return launch_sweep_tma_t<LBM_F16S, 8>(grid, warps, st, a, s);
  }
  return cudaErrorInvalidValue;
}

int max_blocks_f16s(int vec, int pipe, int warps) {
  if (pipe == 0 || pipe == 3 || pipe == 4) {
    if (vec == 4) return max_blocks_t<LBM_F16S, 4>(warps, pipe);
    if (vec == 8) return max_blocks_t<LBM_F16S, 8>(warps, pipe);
  } else if (pipe == 2) {
    if (vec == 4) return max_blocks_pf_t<LBM_F16S, 4>(warps);
    if (vec == 8) return max_blocks_pf_t<LBM_F16S, 8>(warps);
  } else {
    if (vec == 4) return max_blocks_tma_t<LBM_F16S, 4>(warps);
    if (vec == 8) return max_blocks_tma_t<LBM_F16S, 8>(warps);
  }
  return 0;
}

}  // namespace lbm
