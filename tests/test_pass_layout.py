"""Host checks of the pass-kernel configuration (no device work).

A host program built from the pass-kernel header checks, for every line
length, precision, axis kind and tile shape the library instantiates:
shared memory per CTA within the 227 KB an SM offers a block, the CTAs per SM
the launch bounds ask for fitting that memory, the optional third region only
on one-CTA kernels, and the sweep-program dispatch (each fixed program
recognised from its slots, the generic flag and unknown programs falling back
to the generic kernel).

For the shared layout of the transform exchanges it checks that every access
pattern of the passes addresses the slot the layout assigns (each point of
the tile at its own slot, all inside a buffer), that padded buffers keep the
copy engine's destinations aligned, and, with a model of the shared-memory
banks, that the strided tiles of 32 points per thread take the fewest
wavefronts their access width allows in the first pass's stores and the last
pass's loads; the same model finds the 4-way conflict of the unpadded 8-line
512-point layout.
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

// Shared-memory bank model: 32 banks of 4-byte words; a warp access of w
// bytes per lane runs in phases of 128/w lanes (one phase per 128 bytes), and
// a phase takes as many wavefronts as the most distinct words it touches in
// one bank.
static int wavefronts(const long long (&byte)[32], int w)
{
    const int lanes = 128 / w < 32 ? 128 / w : 32;
    int total = 0;
    for (int ph = 0; ph < 32; ph += lanes) {
        int worst = 1;
        for (int b = 0; b < 32; ++b) {
            long long words[64];
            int nw = 0;
            for (int l = ph; l < ph + lanes; ++l)
                for (int o = 0; o < w; o += 4) {
                    const long long wd = (byte[l] + o) / 4;
                    if (wd % 32 != b) continue;
                    bool seen = false;
                    for (int i = 0; i < nw; ++i) seen = seen || words[i] == wd;
                    if (!seen) words[nw++] = wd;
                }
            worst = nw > worst ? nw : worst;
        }
        total += worst;
    }
    return total;
}

// largest wavefront count of any warp access in the first pass's stores
// (Ns = 1) and in the loads of the pass after it, for tile T
template <typename T> void exchange_wavefronts(int &st, int &ld)
{
    using C = typename T::C;
    constexpr int r = T::PL::radix(0), B = T::E / r;
    st = ld = 0;
    for (int w0 = 0; w0 < T::NT; w0 += 32) {
        for (int q = 0; q < B; ++q)
            for (int m = 0; m < r; ++m) {
                long long byte[32];
                for (int l = 0; l < 32; ++l) {
                    const int t = w0 + l, l0 = (t % T::NP) * T::LPT_, tl = t / T::NP;
                    const int base = (tl + q * T::TPL) * r;
                    byte[l] = (long long)T::template sidx_out<1>(T::sbase(base), m, l0) * sizeof(C);
                }
                const int f = wavefronts(byte, (int)sizeof(C));
                st = f > st ? f : st;
            }
        for (int e = 0; e < T::E; ++e) {
            long long byte[32];
            for (int l = 0; l < 32; ++l) {
                const int t = w0 + l, l0 = (t % T::NP) * T::LPT_, tl = t / T::NP;
                byte[l] = (long long)T::sidx_own(tl, e, l0) * sizeof(C);
            }
            const int f = wavefronts(byte, (int)sizeof(C));
            ld = f > ld ? f : ld;
        }
    }
}

// Table of the modelled wavefronts of every exchange of every tile shape
// (worst warp access of the stores of each non-last pass and of the loads of
// each pass after the first, against the fewest the access width allows).
template <typename T, int p> void pass_table()
{
    using C = typename T::C;
    if constexpr (p < T::PL::P) {
        constexpr int r = T::PL::radix(p), Ns = T::PL::ns(p), B = T::E / r;
        int st = 0, ld = 0;
        for (int w0 = 0; w0 < T::NT; w0 += 32) {
            if (p + 1 < T::PL::P)
                for (int q = 0; q < B; ++q)
                    for (int m = 0; m < r; ++m) {
                        long long byte[32];
                        for (int l = 0; l < 32; ++l) {
                            const int t = (w0 + l) % T::NT, l0 = (t % T::NP) * T::LPT_, tl = t / T::NP;
                            const int j = tl + q * T::TPL, k = j & (Ns - 1);
                            byte[l] = (long long)T::template sidx_out<Ns>(T::sbase((j / Ns) * Ns * r + k), m, l0) *
                                      sizeof(C);
                        }
                        const int f = wavefronts(byte, (int)sizeof(C));
                        st = f > st ? f : st;
                    }
            if (p >= 1)
                for (int e = 0; e < T::E; ++e) {
                    long long byte[32];
                    for (int l = 0; l < 32; ++l) {
                        const int t = (w0 + l) % T::NT, l0 = (t % T::NP) * T::LPT_, tl = t / T::NP;
                        byte[l] = (long long)T::sidx_own(tl, e, l0) * sizeof(C);
                    }
                    const int f = wavefronts(byte, (int)sizeof(C));
                    ld = f > ld ? f : ld;
                }
        }
        printf("  p%d r%-2d st %2d ld %2d |", p, r, st, ld);
        pass_table<T, p + 1>();
    }
}
template <typename R, int N, bool ROWS, int VAR> void table_row()
{
    using T = PassTile<R, N, ROWS, VAR>;
    printf("%s %s N=%4d shape %d: %2d lines, %2d points/thread, %s, fewest %d:", sizeof(R) == 4 ? "c64 " : "c128",
           ROWS ? "rows   " : "strided", N, VAR, T::SMEM_POINTS / N, T::E,
           T::PADDED ? "padded " : pass_swizzle<R, N, ROWS, VAR>() ? "swizzled" : "plain  ", 32 * (int)sizeof(typename T::C) / 128);
    pass_table<T, 0>();
    printf("\n");
}
template <typename R, bool ROWS, int VAR> void table_rows()
{
    table_row<R, 16, ROWS, VAR>(); table_row<R, 32, ROWS, VAR>(); table_row<R, 64, ROWS, VAR>();
    table_row<R, 128, ROWS, VAR>(); table_row<R, 256, ROWS, VAR>(); table_row<R, 512, ROWS, VAR>();
    table_row<R, 1024, ROWS, VAR>(); table_row<R, 2048, ROWS, VAR>(); table_row<R, 4096, ROWS, VAR>();
}

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
    using T = PassTile<R, N, ROWS, VAR>;
    CHECK(T::layout_consistent());
    CHECK(T::BUF_POINTS >= T::SMEM_POINTS);
    // each point of each line at its own slot
    {
        static bool used[1 << 16];
        const int span = T::BUF_POINTS;
        bool fits = span <= (1 << 16);
        CHECK(fits);
        if (fits) {
            for (int i = 0; i < span; ++i) used[i] = false;
            bool dup = false;
            for (int i = 0; i < N; ++i)
                for (int l = 0; l < T::SMEM_POINTS / N; ++l) {
                    const int k = T::sidx(i, l);
                    if (k < 0 || k >= span || used[k]) dup = true;
                    else used[k] = true;
                }
            CHECK(!dup);
        }
    }
    if constexpr (T::PADDED) CHECK((sizeof(typename T::C) * T::BUF_POINTS) % 1024 == 0);
    if constexpr (pass_pad<R, N, ROWS>() && T::PL::P > 1) {
        int st = 0, ld = 0;
        exchange_wavefronts<T>(st, ld);
        const int fewest = 32 * (int)sizeof(typename T::C) / 128;
        CHECK(st == fewest);
        CHECK(ld == fewest);
    }
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
    {
        // the model against a known conflict: the 8-line 512-point tile in the
        // unpadded layout takes 4 wavefronts per first-pass warp store
        const int N = 512, VAR = 1;
        const bool ROWS = false;
        using Padded = PassTile<float, 512, false, 1>;
        using Plain = GTile<float, 512, 8, 1, false, 32, false>;
        CHECK(Padded::PADDED && Padded::SMEM_POINTS / 512 == 8);
        int st = 0, ld = 0;
        exchange_wavefronts<Plain>(st, ld);
        CHECK(st == 4);
        CHECK(ld == 2);
        exchange_wavefronts<Padded>(st, ld);
        CHECK(st == 2);
        printf("model: 8-line 512-point first-pass stores, plain 4 / padded %d wavefronts\n", st);
    }
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
    table_rows<float, false, 0>(); table_rows<float, false, 1>(); table_rows<double, false, 0>();
    table_rows<double, false, 1>(); table_rows<float, true, 0>(); table_rows<float, true, 1>();
    table_rows<double, true, 0>(); table_rows<double, true, 1>();
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
