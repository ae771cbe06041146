// pass_f64_rows1.cu - double instantiations of the x-axis (row) line-pass kernels, tile shape 1.
#include "pass_kernels.cuh"

namespace gpe {

cudaError_t launch_pass_rows1_f64(const PassArgs &a, cudaStream_t st)
{
    return launch_pass_r<double, true, 1>(a, st, nullptr);
}

}  // namespace gpe
