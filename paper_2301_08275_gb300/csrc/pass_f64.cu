// pass_f64.cu - double instantiations of the line-pass and on-chip 1D kernels.
#include "pass_kernels.cuh"

namespace gpe {

cudaError_t launch_pass_f64(bool rows, const PassArgs &a, cudaStream_t st) { return launch_pass_r<double>(rows, a, st); }
cudaError_t launch_line1d_f64(const Line1DArgs &a, cudaStream_t st) { return launch_line1d_r<double>(a, st); }
int lines_per_tile_f64(bool rows, int n) { return lines_per_tile_r<double>(rows, n); }

}  // namespace gpe
