// 3-D instantiations: (N=8, K=2) -- seven grains and liquid -- FP32 tile
// variants for the autotuner, and FP64.
#include "ms_launch.cuh"

namespace msgb {
void register_3d_n8(std::vector<StepKernel>& s, std::vector<DiagKernel>& d) {
  s.push_back(make_step_kernel<3, 8, 1, float, 32, 8>());
  s.push_back(make_step_kernel<3, 8, 1, float, 32, 4>());
  s.push_back(make_split_kernel<8, 1, 6>());
  s.push_back(make_step_kernel<3, 8, 1, double, 32, 8>());
  d.push_back(make_diag_kernel<3, 8, 1, float>());
  d.push_back(make_diag_kernel<3, 8, 1, double>());
}
}  // namespace msgb
