// pass_f32_w512_1.cu - float instantiations of the strided line-pass kernels
// for 512-point lines, tile shape 1 (radix-32 plan).
#include "pass_kernels.cuh"

namespace gpe {

template <> cudaError_t launch_pass_wide_f32<512, 1>(const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap)
{
    return launch_pass_t<float, 512, false, 1>(a, st, tmap);
}

}  // namespace gpe
