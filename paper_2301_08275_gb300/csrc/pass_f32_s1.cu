// pass_f32_s1.cu - float instantiations of the strided line-pass kernels, tile shape 1.
#include "pass_kernels.cuh"

namespace gpe {

cudaError_t launch_pass_s1_f32(const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap)
{
    return launch_pass_r<float, false, 1>(a, st, tmap);
}

}  // namespace gpe
