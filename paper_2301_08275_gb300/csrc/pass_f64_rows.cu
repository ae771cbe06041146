// pass_f64_rows.cu - double instantiations of the x-axis (row) line-pass kernels, tile shape 0.
#include "pass_kernels.cuh"

namespace gpe {

cudaError_t launch_pass_rows0_f64(const PassArgs &a, cudaStream_t st)
{
    return launch_pass_r<double, true, 0>(a, st, nullptr);
}

}  // namespace gpe
