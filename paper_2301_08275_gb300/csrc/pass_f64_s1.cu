// pass_f64_s1.cu - double instantiations of the strided line-pass kernels, tile shape 1.
#include "pass_kernels.cuh"

namespace gpe {

cudaError_t launch_pass_s1_f64(const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap)
{
    return launch_pass_r<double, false, 1>(a, st, tmap);
}

}  // namespace gpe
