"""Host checks of the pass-kernel configuration (no device work).

A host program built from the pass-kernel header checks, for every line
length, precision, axis kind and tile shape the library instantiates:
shared memory per CTA within the 227 KB an SM offers a block, the CTAs per SM
the launch bounds ask for fitting that memory, the optional third region only
on one-CTA kernels, and the sweep-program dispatch (each fixed program
recognised from its slots, the generic flag and unknown programs falling back
to the generic kernel).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2301_08275_gb300", "csrc")
INC = os.path.join(ROOT, "include")

PROGRAM = r"""
#include "pass_kernels.cuh"
#include <cstdio>
using namespace gpe;

static int bad = 0;
#define CHECK(c) do { if (!(c)) { printf("FAIL %s line %d (N=%d rows=%d var=%d)\n", #c, __LINE__, N, (int)ROWS, VAR); ++bad; } } while (0)

template <typename R, int N, bool ROWS, int VAR> void shape()
{
    constexpr size_t smem = pass_smem_bytes<R, N, ROWS, VAR>();
    constexpr int minb = pass_min_blocks<R, N, ROWS, VAR>();
    CHECK(smem <= 227 * 1024);
    CHECK(minb >= 1);
    CHECK((size_t)minb * (smem + 1024) <= 228 * 1024);
    constexpr bool ping = pass_ping<R, N, ROWS, VAR>();
    constexpr int nt = PassTile<R, N, ROWS, VAR>::NT;
    CHECK(!ping || minb == 1);
    CHECK(nt <= 1024);
}
template <typename R, bool ROWS, int VAR> void shapes()
{
    shape<R, 2, ROWS, VAR>(); shape<R, 4, ROWS, VAR>(); shape<R, 8, ROWS, VAR>(); shape<R, 16, ROWS, VAR>();
    shape<R, 32, ROWS, VAR>(); shape<R, 64, ROWS, VAR>(); shape<R, 128, ROWS, VAR>(); shape<R, 256, ROWS, VAR>();
    shape<R, 512, ROWS, VAR>(); shape<R, 1024, ROWS, VAR>(); shape<R, 2048, ROWS, VAR>(); shape<R, 4096, ROWS, VAR>();
}
int main()
{
    shapes<float, false, 0>(); shapes<float, false, 1>(); shapes<float, true, 0>(); shapes<float, true, 1>();
    shapes<double, false, 0>(); shapes<double, false, 1>(); shapes<double, true, 0>(); shapes<double, true, 1>();
    const int N = 0, VAR = 0;
    const bool ROWS = false;
    int seen = 0;
    for (int p = 1; p <= NUM_SWEEP_PROGS; ++p) {
        const SweepProg q = sweep_prog(p);
        if (q.op_pre < 0) continue;    // unused number
        ++seen;
        PassArgs a;
        memset(&a, 0, sizeof(a));
        a.op_pre = q.op_pre; a.fft1 = q.fft1; a.op_mid = q.op_mid; a.fft2 = q.fft2; a.op_post = q.op_post; a.red = q.red;
        CHECK(sweep_prog_of(a) == p);
        a.generic = 1;
        CHECK(sweep_prog_of(a) == 0);
        a.generic = 0;
        a.red = RED_DIAG_X;
        CHECK(sweep_prog_of(a) == 0);
        for (int p2 = 1; p2 < p; ++p2) {
            const SweepProg r = sweep_prog(p2);
            CHECK(!(r.op_pre == q.op_pre && r.fft1 == q.fft1 && r.op_mid == q.op_mid && r.fft2 == q.fft2 &&
                    r.op_post == q.op_post && r.red == q.red));
        }
    }
    CHECK(seen >= 4);
    PassArgs z;
    memset(&z, 0, sizeof(z));
    CHECK(sweep_prog_of(z) == 0);       // all slots empty: no fixed program
    printf("programs %d bad %d\n", seen, bad);
    return bad != 0;
}
"""


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_pass_shapes_fit_and_programs_dispatch(tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not found")
    src = tmp_path / "pass_layout.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "pass_layout"
    r = subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I" + CSRC, "-I" + INC,
                        "-o", str(exe), str(src), "-lcuda"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout[-2000:]
    assert "bad 0" in out.stdout
