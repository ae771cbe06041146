// pass_f32.cu - float instantiations of the line-pass and on-chip 1D kernels.
#include "pass_kernels.cuh"

namespace gpe {

cudaError_t launch_pass_f32(bool rows, const PassArgs &a, cudaStream_t st) { return launch_pass_r<float>(rows, a, st); }
cudaError_t launch_line1d_f32(const Line1DArgs &a, cudaStream_t st) { return launch_line1d_r<float>(a, st); }
int lines_per_tile_f32(bool rows, int n) { return lines_per_tile_r<float>(rows, n); }

}  // namespace gpe
