// pass_f32.cu - float instantiations of the strided line-pass kernels (y, z
// axes, tile shape 0) and the on-chip 1D kernels, and the pass dispatcher; the
// other shapes are compiled in pass_f32_s1.cu, pass_f32_rows.cu and
// pass_f32_rows1.cu.
#include "pass_kernels.cuh"

namespace gpe {

cudaError_t launch_pass_s1_f32(const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap);
cudaError_t launch_pass_rows0_f32(const PassArgs &a, cudaStream_t st);
cudaError_t launch_pass_rows1_f32(const PassArgs &a, cudaStream_t st);

cudaError_t launch_pass_f32(bool rows, int var, const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap)
{
    if (rows) return var ? launch_pass_rows1_f32(a, st) : launch_pass_rows0_f32(a, st);
    return var ? launch_pass_s1_f32(a, st, tmap) : launch_pass_r<float, false, 0>(a, st, tmap);
}
cudaError_t launch_line1d_f32(const Line1DArgs &a, cudaStream_t st) { return launch_line1d_r<float>(a, st); }
int lines_per_tile_f32(bool rows, int n, int var) { return lines_per_tile_r<float>(rows, n, var); }

}  // namespace gpe
