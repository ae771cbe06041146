// pass_f32_w256_0.cu - float instantiations of the strided line-pass kernels
// for 256-point lines, tile shape 0 (radix-32 plan).
#include "pass_kernels.cuh"

namespace gpe {

template <> cudaError_t launch_pass_wide_f32<256, 0>(const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap)
{
    return launch_pass_t<float, 256, false, 0>(a, st, tmap);
}

}  // namespace gpe
