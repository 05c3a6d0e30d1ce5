// The 3D sweep (lbm3d.cuh) instantiated for BF16-shifted storage: the single-domain sweep
// (D3Q19 and D3Q15, rigid and pulsating bodies) and the batched sweep of fixed-geometry
// domains, each for 16, 20 and 24 resident warps per SM (pipelines 0, 3, 4).
#include "lbm3d.cuh"

namespace lbm {
namespace d3 {

cudaError_t launch_sweep3_bf16s(int q, int pipe, bool deform, int grid, cudaStream_t st, const Dom3 &dom,
                               long long n, int par) {
  switch (pipe) {
    case 0: return launch_sweep3_sp<LBM_BF16S, 0>(q, deform, grid, st, dom, n, par);
    case 3: return launch_sweep3_sp<LBM_BF16S, 3>(q, deform, grid, st, dom, n, par);
    case 4: return launch_sweep3_sp<LBM_BF16S, 4>(q, deform, grid, st, dom, n, par);
  }
  return cudaErrorInvalidValue;
}

int sweep3_fits_bf16s(int q, int pipe) {
  switch (pipe) {
    case 0: return sweep3_fits_sp<LBM_BF16S, 0>(q);
    case 3: return sweep3_fits_sp<LBM_BF16S, 3>(q);
    case 4: return sweep3_fits_sp<LBM_BF16S, 4>(q);
  }
  return 0;
}

cudaError_t launch_sweep3b_bf16s(int q, int pipe, int grid, cudaStream_t st, const Batch3Args &args) {
  switch (pipe) {
    case 0: return launch_sweep3b_sp<LBM_BF16S, 0>(q, grid, st, args);
    case 3: return launch_sweep3b_sp<LBM_BF16S, 3>(q, grid, st, args);
    case 4: return launch_sweep3b_sp<LBM_BF16S, 4>(q, grid, st, args);
  }
  return cudaErrorInvalidValue;
}

int sweep3b_fits_bf16s(int q, int pipe) {
  switch (pipe) {
    case 0: return sweep3b_fits_sp<LBM_BF16S, 0>(q);
    case 3: return sweep3b_fits_sp<LBM_BF16S, 3>(q);
    case 4: return sweep3b_fits_sp<LBM_BF16S, 4>(q);
  }
  return 0;
}

}  // namespace d3
}  // namespace lbm
