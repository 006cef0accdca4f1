// 3-D instantiations: (N=3, K=3) -- the directional eutectic -- FP32 tile
// variants (fused and split) for the autotuner, and FP64.
#include "ms_launch.cuh"

namespace msgb {
void register_3d_n3(std::vector<StepKernel>& s, std::vector<DiagKernel>& d) {
  s.push_back(make_step_kernel<3, 3, 2, float, 32, 8>());
  s.push_back(make_step_kernel<3, 3, 2, float, 32, 4>());
  s.push_back(make_step_kernel<3, 3, 2, float, 64, 4>());
  s.push_back(make_step_kernel<3, 3, 2, float, 32, 16>());
  s.push_back(make_split_kernel<3, 2, 6>());
  s.push_back(make_step_kernel<3, 3, 2, double, 32, 8>());
  d.push_back(make_diag_kernel<3, 3, 2, float>());
  d.push_back(make_diag_kernel<3, 3, 2, double>());
}
}  // namespace msgb
