// 2-D instantiations: (N=2, K=2) and (N=3, K=3), FP32 and FP64.
#include "ms_launch.cuh"

namespace msgb {
void register_2d(std::vector<StepKernel>& s, std::vector<DiagKernel>& d) {
  s.push_back(make_step_kernel<2, 2, 1, float, 32, 8>());
  s.push_back(make_step_kernel<2, 2, 1, float, 64, 4>());
  s.push_back(make_step_kernel<2, 2, 1, float, 32, 16>());
  s.push_back(make_step_kernel<2, 2, 1, double, 32, 8>());
  s.push_back(make_step_kernel<2, 3, 2, float, 32, 8>());
  s.push_back(make_step_kernel<2, 3, 2, double, 32, 8>());
  d.push_back(make_diag_kernel<2, 2, 1, float>());
  d.push_back(make_diag_kernel<2, 2, 1, double>());
  d.push_back(make_diag_kernel<2, 3, 2, float>());
  d.push_back(make_diag_kernel<2, 3, 2, double>());
}
}  // namespace msgb
