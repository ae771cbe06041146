// pass_f32_rows.cu - float instantiations of the x-axis (row) line-pass kernels.
#include "pass_kernels.cuh"

namespace gpe {

cudaError_t launch_pass_rows_f32(const PassArgs &a, cudaStream_t st) { return launch_pass_r<float, true>(a, st, nullptr); }

}  // namespace gpe
