// pass_f64.cu - double instantiations of the strided line-pass (y, z axes) and
// on-chip 1D kernels; the x-axis (row) passes are in pass_f64_rows.cu.
#include "pass_kernels.cuh"

namespace gpe {

cudaError_t launch_pass_rows_f64(const PassArgs &a, cudaStream_t st);

cudaError_t launch_pass_f64(bool rows, const PassArgs &a, cudaStream_t st, const CUtensorMap *tmap)
{
    return rows ? launch_pass_rows_f64(a, st) : launch_pass_r<double, false>(a, st, tmap);
}
cudaError_t launch_line1d_f64(const Line1DArgs &a, cudaStream_t st) { return launch_line1d_r<double>(a, st); }
int lines_per_tile_f64(bool rows, int n) { return lines_per_tile_r<double>(rows, n); }

}  // namespace gpe
