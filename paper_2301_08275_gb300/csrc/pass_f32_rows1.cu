// pass_f32_rows1.cu - float instantiations of the x-axis (row) line-pass kernels, tile shape 1.
#include "pass_kernels.cuh"

namespace gpe {

cudaError_t launch_pass_rows1_f32(const PassArgs &a, cudaStream_t st)
{
    return launch_pass_r<float, true, 1>(a, st, nullptr);
}

}  // namespace gpe
