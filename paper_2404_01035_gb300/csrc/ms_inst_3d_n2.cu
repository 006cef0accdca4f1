// 3-D instantiations: (N=2, K=2), FP32 and FP64.
#include "ms_launch.cuh"

namespace msgb {
void register_3d_n2(std::vector<StepKernel>& s, std::vector<DiagKernel>& d) {
  s.push_back(make_step_kernel<3, 2, 1, float, 32, 8>());
  s.push_back(make_split_kernel<2, 1, 6>());
  s.push_back(make_step_kernel<3, 2, 1, double, 32, 8>());
  d.push_back(make_diag_kernel<3, 2, 1, float>());
  d.push_back(make_diag_kernel<3, 2, 1, double>());
}
}  // namespace msgb
