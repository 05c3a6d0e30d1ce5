// The 3D sweep (lbm3d.cuh) instantiated for FP32 storage: the single-domain sweep
// (D3Q19 and D3Q15, rigid and pulsating bodies) and the batched sweep of fixed-geometry
// domains, one register budget (pipeline 0).
#include "lbm3d.cuh"

namespace lbm {
namespace d3 {

cudaError_t launch_sweep3_f32(int q, int pipe, bool deform, int grid, cudaStream_t st, const Dom3 &dom,
                               long long n, int par) {
  if (pipe != 0) return cudaErrorInvalidValue;
  return launch_sweep3_sp<LBM_F32, 0>(q, deform, grid, st, dom, n, par);
}

int sweep3_fits_f32(int q, int pipe) { return pipe == 0 ? sweep3_fits_sp<LBM_F32, 0>(q) : 0; }

cudaError_t launch_sweep3b_f32(int q, int pipe, int grid, cudaStream_t st, const Batch3Args &args) {
  if (pipe != 0) return cudaErrorInvalidValue;
  return launch_sweep3b_sp<LBM_F32, 0>(q, grid, st, args);
}

int sweep3b_fits_f32(int q, int pipe) { return pipe == 0 ? sweep3b_fits_sp<LBM_F32, 0>(q) : 0; }

}  // namespace d3
}  // namespace lbm
