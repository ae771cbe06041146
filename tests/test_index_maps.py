"""Host checks of the shared-memory index shortcuts of the FFT tile engine.

The pass kernels address a thread's own points and the Stockham pass outputs
through closed forms (a per-thread base plus or XOR a constant) instead of the
swizzle function itself.  A host program built from the same header compares
both, for every point, line and pass of a set of tile shapes covering every
radix plan (first pass of radix 2, 4 or 8) and swizzle width.  No device work.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2301_08275_gb300", "csrc")

PROGRAM = r"""
#include "fft_tile.cuh"
#include <cstdio>
using namespace gpe;

template <typename T, int L> int own_points()
{
    int bad = 0;
    for (int tl = 0; tl < T::TPL; ++tl)
        for (int e = 0; e < T::E; ++e)
            for (int l = 0; l < L; ++l)
                bad += T::sidx_own(tl, e, l) != T::sidx(tl + T::TPL * e, l);
    return bad;
}
template <typename T, int N, int L, int p> int pass_outputs()
{
    if constexpr (p >= Radix<N>::P) {
        return 0;
    } else {
        constexpr int r = Radix<N>::radix(p), Ns = Radix<N>::ns(p);
        int bad = 0;
        for (int j = 0; j < N / r; ++j)
            for (int m = 0; m < r; ++m)
                for (int l = 0; l < L; ++l) {
                    const int base = (j / Ns) * Ns * r + (j & (Ns - 1));
                    bad += T::template sidx_out<Ns>(T::sraw(base), m, l) != T::sidx(base + m * Ns, l);
                }
        return bad + pass_outputs<T, N, L, p + 1>();
    }
}
template <typename R, int N, int L, bool SW, int E> void check()
{
    using T = GTile<R, N, L, 1, SW, E>;
    const int bad = own_points<T, L>() + pass_outputs<T, N, L, 0>();
    // every index in range and the map a bijection of the tile
    static int seen[1 << 16];
    for (int i = 0; i < N * L; ++i) seen[i] = 0;
    int range = 0;
    for (int i = 0; i < N; ++i)
        for (int l = 0; l < L; ++l) {
            const int s = T::sidx(i, l);
            if (s < 0 || s >= N * L) ++range; else ++seen[s];
        }
    for (int i = 0; i < N * L; ++i) range += seen[i] != 1;
    printf("%s N=%d L=%d SW=%d E=%d bad=%d range=%d\n", sizeof(R) == 4 ? "f32" : "f64", N, L, (int)SW, E, bad, range);
}
int main()
{
    check<float, 2, 4, true, 2>();    check<float, 4, 4, true, 4>();     check<float, 8, 8, true, 8>();
    check<float, 16, 4, true, 8>();   check<float, 32, 8, true, 8>();    check<float, 64, 4, true, 8>();
    check<float, 64, 8, true, 8>();   check<float, 128, 2, true, 8>();   check<float, 128, 4, true, 8>();
    check<float, 256, 2, true, 8>();  check<float, 256, 4, true, 8>();   check<float, 512, 1, true, 8>();
    check<float, 512, 4, true, 8>();  check<float, 1024, 1, true, 8>();  check<float, 1024, 4, true, 8>();
    check<float, 2048, 2, true, 8>(); check<float, 4096, 1, true, 8>();  check<float, 512, 1, true, 16>();
    check<float, 512, 16, false, 16>(); check<float, 512, 8, false, 16>(); check<float, 256, 16, false, 16>();
    check<double, 256, 2, true, 8>(); check<double, 512, 4, true, 8>();  check<double, 1024, 1, true, 8>();
    check<double, 64, 2, true, 8>();  check<double, 512, 4, false, 8>();
    return 0;
}
"""


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_index_shortcuts_match_the_swizzle(tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not found")
    src = tmp_path / "index_maps.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "index_maps"
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I" + CSRC, "-o", str(exe), str(src)], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    lines = out.strip().splitlines()
    assert len(lines) == 26
    for ln in lines:
        assert ln.endswith("bad=0 range=0"), ln
